"""The algebra of the runs' scaled and closing FTCS steps, checked on the CPU.

The 1D and 2D runs advance the field scaled by r^-m between closing steps
(include/hxc.h, hxc_heat1d_step_kinds / hxc_heat2d_step_kinds).  This file
restates that schedule from its documented definition in numpy FP64 (no
library arithmetic), runs it on small grids and compares the result with the
oracle's plain update u + r (s - 2d u): the reformulation must agree with the
FTCS step to rounding, through every group and interval boundary.  It also
checks that the restated schedule has the step counts the library reports,
which ties the restatement to the library's own schedule.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1810_11482_b300 import hxc, synth

GROWTH = 2.0 ** 96  # the documented bound on r^-m


@pytest.fixture(scope="module", autouse=True)
def _library():
    """The step-count queries need libhxc.so (host code only, no device)."""
    from paper_1810_11482_b300 import build
    build.build()


def max_scaled(dim, r):
    if not (0.0 < r <= 0.5 / dim):
        return 0
    m = 0
    while m < 96 and r ** (m + 1) >= 1.0 / GROWTH:
        m += 1
    return m


def kinds(dim, r, steps, interval):
    """Per step: ('canon',), ('scaled', k) or ('close', a, b)."""
    M = max_scaled(dim, r)
    c = 1.0 - 2.0 * dim * r
    out = []
    for g in range(steps):
        j = g % interval
        L = min(interval, steps - (g - j))
        if M == 0:
            out.append(("canon",))
            continue
        P = M + 1
        q = j % P
        end = min(L, j - q + P)
        if j + 1 < end:
            out.append(("scaled", c / r))
        else:
            out.append(("close", r ** (q + 1), c * r ** q))
    return out


def neighbour_sum(v):
    """Sum of the 2d neighbours: zero outside in 2D (Dirichlet), periodic in 1D."""
    if v.ndim == 1:
        return np.roll(v, 1) + np.roll(v, -1)
    p = np.pad(v, 1)
    return (p[:-2, 1:-1] + p[1:-1, :-2]) + (p[1:-1, 2:] + p[2:, 1:-1])


def run_scaled(u0, r, sched):
    dim = u0.ndim
    v = u0.copy()
    for k in sched:
        s = neighbour_sum(v)
        if k[0] == "scaled":
            v = k[1] * v + s
        elif k[0] == "close":
            v = k[1] * s + k[2] * v
        else:
            v = v + r * (s - 2 * dim * v)
    return v


def count(sched):
    return (sum(k[0] == "canon" for k in sched), sum(k[0] == "scaled" for k in sched),
            sum(k[0] == "close" for k in sched))


@pytest.mark.parametrize("r,steps,every", [(0.2, 130, 0), (0.25, 100, 0), (0.1, 60, 7),
                                           (0.01, 45, 0), (1e-30, 12, 0)])
def test_scaled_2d_schedule_matches_ftcs(r, steps, every):
    u0 = synth.bumps2d(40, 52, seed=700, nbumps=4, sigma=0.1)
    norms = np.zeros(max(1, steps // max(every, 1)))
    cfg = hxc.heat2d_cfg(40, 52, 1, 1, r, steps, every, "fused", norms if every else None, None)
    interval = every if every else min(steps, 100)
    sched = kinds(2, r, steps, interval)
    assert count(sched) == hxc.heat2d_step_kinds(cfg)
    got = run_scaled(u0, r, sched)
    want = oracle.heat2d(u0, r, steps)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("r,steps", [(0.25, 300), (0.5, 130), (0.2, 257), (1e-30, 10)])
def test_scaled_1d_schedule_matches_ftcs(r, steps):
    u0 = synth.heat1d_input(301, seed=701)
    sched = kinds(1, r, steps, min(steps, 128))
    assert count(sched) == hxc.heat1d_step_kinds(r, steps)
    got = run_scaled(u0, r, sched)
    want = oracle.heat1d(u0, r, steps)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_scaled_field_growth_bound():
    """Between closings the scaled field grows by at most 1/r per step, so by
    at most r^-M <= 2^96: a field of magnitude 2^900 stays finite."""
    r = 0.2
    M = max_scaled(2, r)
    assert r ** -M <= GROWTH < r ** -(M + 1)
    u0 = synth.bumps2d(24, 30, seed=702, nbumps=3, sigma=0.1) * 2.0 ** 900
    sched = kinds(2, r, 3 * (M + 1), min(3 * (M + 1), 100))
    v, peak = u0.copy(), 0.0
    for k in sched:
        s = neighbour_sum(v)
        v = k[1] * v + s if k[0] == "scaled" else k[1] * s + k[2] * v
        peak = max(peak, float(np.max(np.abs(v))))
    assert math.isfinite(peak) and peak <= np.max(np.abs(u0)) * GROWTH
    want = oracle.heat2d(u0, r, len(sched))
    assert np.max(np.abs(v - want)) <= 1e-12 * np.max(np.abs(want))
