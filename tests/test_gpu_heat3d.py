"""GPU parity of the 3D FP32 temporally blocked path against the FP64 oracle.

The oracle runs in FP64 from the FP32-rounded initial field with
r = (double)0.15f, so the reported error is the kernel's FP32 arithmetic
error.  Bound: norm-wise relative error <= 1e-5 (FP32 rounding of the 7
operations of an update is <= ~4 ulp = 2.4e-7 per step and the FTCS operator
does not amplify errors for r <= 1/6, so 200 steps stay below ~5e-5 in the
worst case and far below it in practice; the test asserts 1e-5).
Every schedule (1..4 fused steps per launch, plain / graph / fused) must be
bit-identical."""
import math

import numpy as np
import pytest

import oracle
from paper_1810_11482_b300 import hxc, synth

pytestmark = pytest.mark.gpu
TOL32 = 1e-5
R = np.float32(0.15)


@pytest.fixture(scope="module")
def dev():
    devs = hxc.get_all_devices(2, 0)
    assert devs
    return devs[0]


def run3d(dev, u0, steps, mode="fused", spl=4):
    u0 = np.ascontiguousarray(u0, dtype=np.float32)
    u, t = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    u.write(u0).get()
    f, st = hxc.heat3d_run(dev, u, t, u0.shape, float(R), steps, mode, spl)
    f.get()
    out = np.empty_like(u0)
    u.read_sync(out)
    return out, st


def relerr(a, b, scale=None):
    scale = np.max(np.abs(b)) if scale is None else scale
    return float(np.max(np.abs(a.astype(np.float64) - b)) / scale)


@pytest.mark.parametrize("shape", [(16, 24, 40), (9, 70, 130), (33, 31, 17), (8, 8, 8),
                                   (1, 1, 1), (1, 2, 3), (2, 1, 5), (3, 65, 1), (1, 57, 129)])
def test_heat3d_vs_oracle_small(dev, shape):
    u0 = synth.heat3d_input(shape[2], seed=300 + shape[0], nz=shape[0], ny=shape[1])
    for steps in (1, 3, 4, 9):
        want = oracle.heat3d(u0.astype(np.float64), float(R), steps)
        for mode, spl in (("plain", 1), ("fused", 4), ("fused", 3), ("graph", 4)):
            got, _ = run3d(dev, u0, steps, mode, spl)
            assert relerr(got, want) <= TOL32, (shape, steps, mode, spl)


def test_heat3d_bitexact_across_blocking(dev):
    u0 = synth.heat3d_input(96, seed=310, nz=40, ny=72)
    ref, _ = run3d(dev, u0, 12, "plain", 1)
    for mode, spl in (("fused", 1), ("fused", 2), ("fused", 3), ("fused", 4), ("graph", 4),
                      ("graph", 2)):
        got, _ = run3d(dev, u0, 12, mode, spl)
        assert np.array_equal(got, ref), (mode, spl)
    # x <-> y swap symmetry is exact (((x-pair + y-pair) + z-below) + z-above is
    # symmetric in x and y)
    sw = np.ascontiguousarray(np.swapaxes(u0, 1, 2)[:, :72, :72])
    a, _ = run3d(dev, sw, 8, "fused", 4)
    b, _ = run3d(dev, np.ascontiguousarray(np.swapaxes(sw, 1, 2)), 8, "fused", 4)
    assert np.array_equal(a, np.swapaxes(b, 1, 2))


def test_heat3d_translation_and_reflection_exact(dev):
    """Periodic boundaries: a circular shift of the input along z, y and x
    (moving the data across region edges, the wrap and the z splits) gives
    the same shift of the output bit for bit, for every kernel form; the x and
    y pairs are symmetric sums, so reversing x or y reverses the output."""
    shape = (37, 150, 200)
    u0 = np.ascontiguousarray(synth.heat3d_input(shape[2], seed=350, nz=shape[0], ny=shape[1]),
                              dtype=np.float32)
    old = {k: hxc.tune_get(k) for k in ("heat3d.variant", "heat3d.variant1")}
    try:
        for variant in (2, 3, 4, 6, 7):
            hxc.tune_set("heat3d.variant", variant)
            hxc.tune_set("heat3d.variant1", variant)
            ref, _ = run3d(dev, u0, 8, "fused", 4)
            for sh in ((5, 0, 0), (0, 61, 0), (0, 0, 77), (19, 100, 3)):
                got, _ = run3d(dev, np.roll(u0, sh, axis=(0, 1, 2)), 8, "fused", 4)
                assert np.array_equal(got, np.roll(ref, sh, axis=(0, 1, 2))), (variant, sh)
            got, _ = run3d(dev, u0[:, ::-1, :].copy(), 8, "fused", 4)
            assert np.array_equal(got, ref[:, ::-1, :]), variant
            got, _ = run3d(dev, u0[:, :, ::-1].copy(), 8, "fused", 4)
            assert np.array_equal(got, ref[:, :, ::-1]), variant
    finally:
        for k, v in old.items():
            hxc.tune_set(k, v)


@pytest.mark.parametrize("shape", [(40, 72, 96), (9, 70, 131), (8, 8, 8), (21, 33, 64)])
def test_heat3d_kernel_variants_and_zchunks_bitexact(dev, shape):
    """Every form of the 3D kernel (three rotated plane registers per level on
    paired FP32 instructions, two planes per level with the z range split
    over the CTAs, the same with a cp.async plane ring, and with packed narrow
    tiles) and every z split give the bits of one plain step per launch
    of the default form; odd nx takes the scalar-load path, small nz the
    wrapped z index."""
    u0 = synth.heat3d_input(shape[2], seed=330 + shape[0], nz=shape[0], ny=shape[1])
    ref, _ = run3d(dev, u0, 9, "plain", 1)
    want = oracle.heat3d(u0.astype(np.float64), float(R), 9)
    old = {k: hxc.tune_get(k) for k in ("heat3d.variant", "heat3d.variant1", "heat3d.zchunks")}
    try:
        for variant in (2, 3, 4, 6, 7):
            hxc.tune_set("heat3d.variant", variant)
            hxc.tune_set("heat3d.variant1", variant)
            for nch in (0, 1, 3):
                hxc.tune_set("heat3d.zchunks", nch)
                for mode, spl in (("fused", 4), ("fused", 3), ("graph", 4)):
                    got, _ = run3d(dev, u0, 9, mode, spl)
                    assert np.array_equal(got, ref), (variant, nch, mode, spl)
        assert relerr(ref, want) <= TOL32
    finally:
        for k, v in old.items():
            hxc.tune_set(k, v)


@pytest.mark.parametrize("shape", [(40, 72, 96), (70, 33, 132), (8, 8, 8), (130, 17, 4),
                                   (3, 5, 128), (9, 70, 131)])
def test_heat3d_streaming_one_step_form(dev, shape):
    """The streaming one-step kernel (one-step form 5): z chunks with a ragged
    last chunk, rows not filling the last CTA, a partial last warp in x, tiny
    and degenerate shapes, and an odd nx (which takes another form) give the
    bits of the three-plane form, step after step."""
    u0 = np.ascontiguousarray(synth.heat3d_input(shape[2], seed=360 + shape[0], nz=shape[0],
                                                 ny=shape[1]), dtype=np.float32)
    old = hxc.tune_get("heat3d.variant1")
    try:
        hxc.tune_set("heat3d.variant1", 2)
        ref, _ = run3d(dev, u0, 7, "plain", 1)
        hxc.tune_set("heat3d.variant1", 5)
        for mode in ("plain", "graph", "fused"):
            got, _ = run3d(dev, u0, 7, mode, 1)
            assert np.array_equal(got, ref), mode
    finally:
        hxc.tune_set("heat3d.variant1", old)
    assert relerr(ref, oracle.heat3d(u0.astype(np.float64), float(R), 7)) <= TOL32


def test_heat3d_medium_vs_oracle_200_steps(dev):
    u0 = synth.heat3d_input(64, seed=320)
    want = oracle.heat3d(u0.astype(np.float64), float(R), 200)
    got, st = run3d(dev, u0, 200, "fused", 4)
    assert st.kernel_launches == 50
    assert relerr(got, want) <= TOL32
    # error against the exact-r FP64 solution is reported, not asserted tightly
    exact = oracle.heat3d(u0.astype(np.float64), 0.15, 200)
    assert relerr(got, exact) <= 1e-4


def test_heat3d_full_size_windows(dev):
    """512^3, r = 0.15f, 200 steps in 50 launches of 4 steps: the whole
    200-step field against the oracle, windows of a 20-step run against the
    oracle run on a periodic window of 20 steps' reach, plus the 200-step
    result's sum (conserved under periodic boundaries) and maximum
    principle."""
    n = 512
    u0 = synth.heat3d_input(n, seed=3)
    got20, _ = run3d(dev, u0, 20, "fused", 4)
    rng = np.random.default_rng(0)
    for _ in range(3):
        c = rng.integers(0, n, size=3)
        idx = [np.arange(ci - 28, ci + 28) % n for ci in c]
        w = u0[np.ix_(*idx)].astype(np.float64)
        want = oracle.heat3d(w, float(R), 20)[20:-20, 20:-20, 20:-20]
        mine = got20[np.ix_(*[ix[20:-20] for ix in idx])]
        assert relerr(mine, want, scale=1.0) <= TOL32
    got, st = run3d(dev, u0, 200, "fused", 4)
    assert st.kernel_launches == 50
    # the whole field against the oracle (its OpenMP build) from the FP32 input
    a = u0.astype(np.float64)
    b = np.zeros_like(a)
    want = oracle.heat3d_steps(a, b, float(R), 200, omp=True)
    assert relerr(got, want) <= TOL32
    del a, b, want
    s0 = math.fsum(u0.astype(np.float64).ravel())
    s1 = math.fsum(got.astype(np.float64).ravel())
    assert abs(s1 - s0) / s0 <= 1e-5
    assert got.max() <= u0.max() + 1e-6 and got.min() >= u0.min() - 1e-6
    ref, _ = run3d(dev, u0, 200, "graph", 4)
    assert np.array_equal(got, ref)
    # every two-plane form gives these bits at full size too
    old = hxc.tune_get("heat3d.variant")
    try:
        for variant in (3, 4, 6, 7):
            hxc.tune_set("heat3d.variant", variant)
            other, _ = run3d(dev, u0, 200, "fused", 4)
            assert np.array_equal(other, got), variant
    finally:
        hxc.tune_set("heat3d.variant", old)


def test_heat3d_product_mode_full_size(dev):
    n, steps = 512, 200
    k = np.arange(n, dtype=np.float64)
    a, b, c = 3, 5, 2
    u0 = (np.cos(2 * np.pi * a * k / n)[:, None, None] * np.cos(2 * np.pi * b * k / n)[None, :, None]
          * np.cos(2 * np.pi * c * k / n)[None, None, :]).astype(np.float32)
    r = float(R)
    g = 1.0 - 4.0 * r * sum(math.sin(math.pi * m / n) ** 2 for m in (a, b, c))
    got, _ = run3d(dev, u0, steps, "fused", 4)
    assert np.max(np.abs(got.astype(np.float64) - g ** steps * u0.astype(np.float64))) <= 2e-5


@pytest.mark.parametrize("shape", [(33, 200, 130), (5, 64, 64), (70, 57, 250)])
def test_heat3d_two_plane_form_any_grid(dev, shape):
    """The two-plane forms (variants 3, 4 and 6) split the (region, plane) pairs
    evenly over whatever grid they are launched with: one CTA, a few CTAs whose shares
    span several regions, and more CTAs than pairs (empty shares) all give the
    bits of the three-plane form (variant 2); 1..4 steps per launch."""
    u0 = np.ascontiguousarray(synth.heat3d_input(shape[2], seed=340 + shape[0], nz=shape[0],
                                                 ny=shape[1]), dtype=np.float32)
    old = {k: hxc.tune_get(k) for k in ("heat3d.variant", "heat3d.variant1")}
    a, b = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    try:
        for steps in (1, 2, 3, 4):
            want = None
            for variant, grid in ((2, None), (3, None), (3, 1), (3, 7), (3, 150), (3, 100000),
                                  (4, None), (4, 1), (4, 7), (4, 100000), (6, None), (6, 1),
                                  (6, 7), (6, 100000), (7, None), (7, 1), (7, 7),
                                  (7, 100000)):
                hxc.tune_set("heat3d.variant", variant)
                hxc.tune_set("heat3d.variant1", variant)
                a.write(u0).get()
                args = hxc.hxc_heat3d_args(a.h, b.h, shape[0], shape[1], shape[2], R, steps)
                cfg = None if grid is None else hxc.hxc_launch_cfg((grid, 1, 1), (512, 1, 1))
                dev.launch(hxc.HXC_K_HEAT3D, args, cfg=cfg).get()
                got = np.empty_like(u0)
                b.read_sync(got)
                if want is None:
                    want = got
                    ora = oracle.heat3d(u0.astype(np.float64), float(R), steps)
                    assert relerr(got, ora) <= TOL32
                else:
                    assert np.array_equal(got, want), (steps, variant, grid)
        # a block size other than 512 threads is rejected
        hxc.tune_set("heat3d.variant", 3)
        args = hxc.hxc_heat3d_args(a.h, b.h, shape[0], shape[1], shape[2], R, 4)
        with pytest.raises(hxc.HxcError):
            dev.launch(hxc.HXC_K_HEAT3D, args, cfg=hxc.hxc_launch_cfg((4, 1, 1), (256, 1, 1))).get()
    finally:
        for k, v in old.items():
            hxc.tune_set(k, v)


@pytest.mark.parametrize("shape", [(12, 200, 232), (5, 130, 176)])
def test_heat3d_tma_form(dev, shape):
    """Form 7 fetches the input planes of the regions inside the field with
    TMA tensor copies (4 steps per launch, nx % 4 == 0): on fields with
    several such regions in x and y, edge and narrow regions beside them and a
    z extent smaller than the launch's reach, every grid (fewer CTAs than
    tile kinds, a few, more CTAs than work) gives the bits of form 6 for 1..4
    steps per launch, and no bounded wait ran out."""
    u0 = np.ascontiguousarray(synth.heat3d_input(shape[2], seed=370 + shape[0], nz=shape[0],
                                                 ny=shape[1]), dtype=np.float32)
    old = {k: hxc.tune_get(k) for k in ("heat3d.variant", "heat3d.variant1")}
    a, b = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    hxc.debug_wait_errors(dev)
    try:
        for steps in (4, 3, 2, 1):
            want = None
            for variant, grid in ((6, None), (7, None), (7, 1), (7, 2), (7, 7), (7, 100000)):
                hxc.tune_set("heat3d.variant", variant)
                hxc.tune_set("heat3d.variant1", variant)
                a.write(u0).get()
                args = hxc.hxc_heat3d_args(a.h, b.h, shape[0], shape[1], shape[2], R, steps)
                cfg = None if grid is None else hxc.hxc_launch_cfg((grid, 1, 1), (512, 1, 1))
                dev.launch(hxc.HXC_K_HEAT3D, args, cfg=cfg).get()
                got = np.empty_like(u0)
                b.read_sync(got)
                if want is None:
                    want = got
                    ora = oracle.heat3d(u0.astype(np.float64), float(R), steps)
                    assert relerr(got, ora) <= TOL32
                else:
                    assert np.array_equal(got, want), (steps, variant, grid)
        # whole runs of several launches in every mode
        hxc.tune_set("heat3d.variant", 6)
        ref, _ = run3d(dev, u0, 13, "fused", 4)
        hxc.tune_set("heat3d.variant", 7)
        for mode in ("fused", "graph"):
            got, _ = run3d(dev, u0, 13, mode, 4)
            assert np.array_equal(got, ref), mode
        assert hxc.debug_wait_errors(dev) == 0
    finally:
        for k, v in old.items():
            hxc.tune_set(k, v)
