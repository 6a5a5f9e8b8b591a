"""The 2D run streamed through the device every step (host-resident field,
Algorithm 1 per step): asynchronous and sequential forms against the
device-resident run (bit for bit) and the oracle."""
import time

import numpy as np
import pytest

import oracle
from paper_1810_11482_b300 import hxc, synth

from test_gpu_heat12 import run2d

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def dev():
    devs = hxc.get_all_devices(2, 0)
    assert devs
    return devs[0]


def streamed(dev, u0, tiles, r, steps, sequential, deps=()):
    a, b = hxc.host_empty(u0.shape), hxc.host_empty(u0.shape)
    a[:] = u0
    b[:] = np.nan
    f, st, res = hxc.heat2d_stream_run(dev, a, b, tiles, r, steps, sequential, deps)
    f.get()
    return np.array(res), st


@pytest.mark.parametrize("shape,tiles,steps", [((300, 302), (3, 4), 5), ((301, 257), (2, 3), 4),
                                               ((7, 9), (7, 3), 3), ((64, 64), (1, 1), 6),
                                               ((130, 98), (4, 4), 1), ((64, 66), (2, 2), 45)])
def test_streamed_matches_resident_and_oracle(dev, shape, tiles, steps):
    u0 = synth.bumps2d(*shape, seed=400 + shape[0], nbumps=6, sigma=0.1)
    want = run2d(dev, u0, (1, 1), 0.2, steps)[0]
    for seq in (False, True):
        got, st = streamed(dev, u0, tiles, 0.2, steps, seq)
        assert np.array_equal(got, want), (seq, tiles)
        assert st.kernel_launches == tiles[0] * tiles[1] * steps
        assert st.d2h_bytes == u0.nbytes * steps
    ora = oracle.heat2d(u0, 0.2, steps)
    assert np.max(np.abs(want - ora)) / np.max(np.abs(ora)) <= TOL


def test_zero_steps_leaves_the_field(dev):
    u0 = synth.bumps2d(40, 40, seed=410)
    got, st = streamed(dev, u0, (2, 2), 0.2, 0, False)
    assert np.array_equal(got, u0) and st.kernel_launches == 0


def test_streamed_waits_for_dependencies(dev):
    u0 = synth.bumps2d(128, 130, seed=411)
    a, b = hxc.host_empty(u0.shape), hxc.host_empty(u0.shape)
    a[:] = 0.0
    gate = hxc.promise()
    f, _, res = hxc.heat2d_stream_run(dev, a, b, (2, 2), 0.2, 3, False, deps=[gate])
    time.sleep(0.05)
    assert not f.is_ready()
    a[:] = u0  # the input is written before the gate opens
    hxc.promise_set(gate)
    f.get()
    want = run2d(dev, u0, (1, 1), 0.2, 3)[0]
    assert np.array_equal(res, want)


def test_full_size_two_steps(dev):
    """8192^2 in 64 tiles of 1024^2, two streamed steps, bit for bit equal to
    the device-resident run."""
    n = 8192
    u0 = synth.bumps2d(n, n, seed=2)
    want = run2d(dev, u0, (8, 8), 0.2, 2)[0]
    got, st = streamed(dev, u0, (8, 8), 0.2, 2, False)
    assert np.array_equal(got, want)
    assert st.h2d_bytes >= u0.nbytes * 2
