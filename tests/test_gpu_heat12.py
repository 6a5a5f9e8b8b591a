"""GPU parity of the 1D/2D path against the FP64 oracle, through the C ABI.

Tolerance: norm-wise relative error max|u_gpu - u_oracle| / max|u_oracle|
<= 1e-12.  The oracle rounds every operation separately (no FMA) while the
kernels use fused multiply-adds, so the two differ by rounding only: a few
ulps per step, well inside 1e-12 for the step counts used here.
Schedules of the GPU path (partition counts, tile grids, plain / graph /
fused launches) must agree bit for bit."""
import math

import numpy as np
import pytest

import oracle
from paper_1810_11482_b300 import hxc, synth

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def dev():
    devs = hxc.get_all_devices(2, 0)
    assert devs, "no CUDA device"
    return devs[0]


def upload(dev, a):
    a = np.ascontiguousarray(a)
    b = dev.buffer(a.nbytes)
    b.write(a).get()
    return b


def download(buf, shape, dtype=np.float64):
    out = np.empty(shape, dtype=dtype)
    buf.read_sync(out)
    return out


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ------------------------------------------------------------- Listing 2

def test_listing2_sum_workflow(dev):
    """Listing 2: buffers, async writes, wait_all, sum kernel with grid 1x1x1
    and block 32x1x1, synchronous read of the result."""
    n = 1000
    inp = np.ones(n, dtype=np.uint32)
    res = np.zeros(1, dtype=np.uint64)
    b_in, b_res = dev.buffer(n * 4), dev.buffer(8)
    futs = [b_in.write(inp), b_res.write(res)]
    assert hxc.wait_all(futs) == hxc.HXC_OK
    cfg = hxc.hxc_launch_cfg((1, 1, 1), (32, 1, 1))
    a = hxc.hxc_sum_args(b_in.h, b_res.h, n)
    dev.launch(hxc.HXC_K_SUM_U32, a, cfg=cfg).get()
    out = np.zeros(1, dtype=np.uint64)
    b_res.read_sync(out)
    assert int(out[0]) == 1000 == oracle.sum_u32(inp)
    # a larger ragged input, default launch shape
    x = (synth.splitmix64(9, 100003) >> np.uint64(40)).astype(np.uint32)
    b_x, b_r = upload(dev, x), upload(dev, np.zeros(1, dtype=np.uint64))
    dev.launch(hxc.HXC_K_SUM_U32, hxc.hxc_sum_args(b_x.h, b_r.h, x.size)).get()
    assert int(download(b_r, 1, np.uint64)[0]) == oracle.sum_u32(x)


def test_prk_stencil_bitexact(dev):
    x = synth.uniform(10, 4099, lo=-1, hi=1)
    bi, bo = upload(dev, x), dev.buffer(x.nbytes)
    dev.launch(hxc.HXC_K_PRK_STENCIL, hxc.hxc_prk_args(bi.h, bo.h, x.size)).get()
    assert np.array_equal(download(bo, x.size), oracle.prk_stencil(x))


def test_partition_kernel_is_one(dev):
    """Sec. 5.1.2: sqrt(sin^2 i + cos^2 i) = 1 within CUDA's sin/cos/sqrt error bounds."""
    n, off = 1 << 20, 333
    x = synth.partition_input(n + off) + 12345.0
    b = upload(dev, x)
    dev.launch(hxc.HXC_K_PARTITION, hxc.hxc_partition_args(b.h, n, off)).get()
    out = download(b, n + off)
    assert np.array_equal(out[:off], x[:off])  # outside [offset, offset+n) untouched
    assert np.max(np.abs(out[off:] - 1.0)) <= 8 * np.finfo(np.float64).eps
    assert np.max(np.abs(out[off:] - oracle.partition_k(x[off:]))) <= 8 * np.finfo(np.float64).eps


# ------------------------------------------------------------------ 1D

def run1d(dev, u0, parts, r, steps, mode="plain", spl=0):
    u, t = upload(dev, u0), dev.buffer(u0.nbytes)
    f, st = hxc.heat1d_run(dev, u, t, u0.size, parts, r, steps, mode, spl)
    f.get()
    return download(u, u0.size), st


@pytest.mark.parametrize("n,parts", [(1000, 3), (1023, 7), (17, 5), (4096, 1)])
@pytest.mark.parametrize("r", [0.25, 0.2])
def test_heat1d_vs_oracle_small(dev, n, parts, r):
    u0 = synth.heat1d_input(n, seed=100 + n)
    for steps in (1, 2, 37):
        want = oracle.heat1d(u0, r, steps)
        for mode, spl in (("plain", 0), ("fused", 0), ("fused", 5), ("graph", 0)):
            got, _ = run1d(dev, u0, parts, r, steps, mode, spl)
            assert relerr(got, want) <= TOL, (mode, spl, steps)


def test_heat1d_bitexact_across_schedules(dev):
    n, steps, r = 1 << 16, 37, 0.25
    u0 = synth.heat1d_input(n, seed=101)
    ref, _ = run1d(dev, u0, 1, r, steps, "plain")
    for parts in (2, 4, 8, 16):
        for mode, spl in (("plain", 0), ("graph", 0), ("fused", 0), ("fused", 1), ("fused", 7)):
            got, _ = run1d(dev, u0, parts, r, steps, mode, spl)
            assert np.array_equal(got, ref), (parts, mode, spl)


def test_heat1d_translation_and_reflection_exact(dev):
    """Periodic boundaries and a sum uL + uR that is symmetric: a circular
    shift of the input (across partition boundaries and the wrap) gives the
    same shift of the output, and the reversed input the reversed output,
    bit for bit, in every mode."""
    n, steps, r = 4099, 23, 0.25
    u0 = synth.uniform(102, n, lo=-1, hi=1)
    ref, _ = run1d(dev, u0, 5, r, steps, "fused")
    for k in (1, 37, n // 2, n - 3):
        for mode in ("plain", "fused"):
            got, _ = run1d(dev, np.roll(u0, k), 5, r, steps, mode)
            assert np.array_equal(got, np.roll(ref, k)), (k, mode)
    got, _ = run1d(dev, u0[::-1].copy(), 3, r, steps, "graph")
    assert np.array_equal(got, ref[::-1])


@pytest.mark.parametrize("r", [0.25, 0.5, 0.2, 0.01, 1e-30])
def test_heat1d_scaled_steps_vs_oracle(dev, r):
    """The 1D runs' scaled and closing steps (hxc_heat1d_step_kinds): 300
    steps are three intervals (128, 128, 44), so graph mode replays its
    graph twice and issues the rest; fused launches of 300, 50 and 7 steps
    straddle the intervals and groups.  Every mode, partition count and
    steps per launch gives the same bits, within the FP64 tolerance of the
    oracle; r = 1e-30 runs canonical steps only."""
    n, steps = 3001, 300
    u0 = synth.heat1d_input(n, seed=104)
    kinds = hxc.heat1d_step_kinds(r, steps)
    assert sum(kinds) == steps and (kinds[0] == steps) == (r == 1e-30)
    ref, _ = run1d(dev, u0, 1, r, steps, "plain")
    assert relerr(ref, oracle.heat1d(u0, r, steps)) <= TOL
    for parts in (1, 3, 8):
        for mode, spl in (("plain", 0), ("graph", 0), ("fused", 0), ("fused", 50), ("fused", 7)):
            got, _ = run1d(dev, u0, parts, r, steps, mode, spl)
            assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), (parts, mode, spl)


def test_heat1d_scaled_steps_large_magnitudes(dev):
    """A field of magnitude 2^900 at r = 1/4 (the scaled field grows by up
    to 4^48 = 2^96 before each closing step): finite, within the tolerance
    of the oracle."""
    u0 = synth.heat1d_input(2048, seed=105) * 2.0 ** 900
    want = oracle.heat1d(u0, 0.25, 120)
    for mode in ("plain", "fused"):
        got, _ = run1d(dev, u0, 4, 0.25, 120, mode)
        assert np.all(np.isfinite(got)) and relerr(got, want) <= TOL, mode


def test_heat1d_full_config_vs_oracle(dev):
    """2^20 points, 8 partitions, r = 1/4, 100 steps, every mode."""
    n, r, steps = 1 << 20, 0.25, 100
    u0 = synth.heat1d_input(n, seed=1)
    want = oracle.heat1d(u0, r, steps)
    outs = []
    for mode in ("plain", "graph", "fused"):
        got, st = run1d(dev, u0, 8, r, steps, mode)
        assert relerr(got, want) <= TOL, mode
        outs.append(got)
    assert all(np.array_equal(o, outs[0]) for o in outs)


def test_heat1d_fourier_mode_exact_decay(dev):
    n, r, steps = 1 << 20, 0.25, 100
    j = np.arange(n)
    u0 = np.sin(2 * np.pi * 3 * j / n)
    g = 1.0 - 2.0 * r * (1.0 - math.cos(2 * math.pi * 3 / n))
    got, _ = run1d(dev, u0, 8, r, steps, "fused")
    assert np.max(np.abs(got - g ** steps * u0)) <= 16 * steps * np.finfo(float).eps
    # Nyquist mode vanishes exactly after one step at r = 1/4
    got, _ = run1d(dev, np.where(j % 2 == 0, 1.0, -1.0), 8, 0.25, 1, "plain")
    assert np.all(got == 0.0)


def test_heat1d_zero_steps_and_args(dev):
    u0 = synth.heat1d_input(64, seed=3)
    got, _ = run1d(dev, u0, 4, 0.25, 0)
    assert np.array_equal(got, u0)
    u, t = upload(dev, u0), dev.buffer(u0.nbytes)
    with pytest.raises(hxc.HxcError):
        hxc.heat1d_run(dev, u, u, 64, 4, 0.25, 3)  # aliasing buffers rejected
    with pytest.raises(hxc.HxcError):
        hxc.heat1d_run(dev, u, t, 64, 65, 0.25, 3)  # more partitions than points


# ------------------------------------------------------------------ 2D

def run2d(dev, u0, tiles, r, steps, mode="plain", every=0):
    ny, nx = u0.shape
    u, t = upload(dev, u0), dev.buffer(u0.nbytes)
    nsnap = steps // every if every else 0
    T = tiles[0] * tiles[1]
    hn = np.full(max(1, nsnap * T), np.nan)
    gn = np.full(max(1, nsnap * T), np.nan)
    cfg = hxc.heat2d_cfg(ny, nx, tiles[0], tiles[1], r, steps, every, mode,
                         hn if nsnap else None, gn if nsnap else None)
    f, st = hxc.heat2d_run(dev, u, t, cfg)
    f.get()
    return download(u, (ny, nx)), hn[:nsnap * T].reshape(nsnap, T), gn[:nsnap * T].reshape(nsnap, T), st


@pytest.mark.parametrize("shape,tiles", [((100, 130), (3, 4)), ((77, 93), (2, 5)),
                                         ((64, 64), (1, 1)), ((33, 200), (4, 1))])
def test_heat2d_vs_oracle_small(dev, shape, tiles):
    u0 = synth.bumps2d(*shape, seed=200 + shape[0], nbumps=5, sigma=0.1)
    for r in (0.2, 0.25):
        for steps in (1, 2, 21):
            want = oracle.heat2d(u0, r, steps)
            for mode in ("plain", "graph", "fused"):
                got, _, _, _ = run2d(dev, u0, tiles, r, steps, mode)
                assert relerr(got, want) <= TOL, (mode, r, steps)


@pytest.mark.parametrize("shape,tiles", [((1, 1), (1, 1)), ((1, 7), (1, 3)), ((7, 1), (3, 1)),
                                         ((2, 3), (2, 1)), ((3, 64), (1, 2)), ((65, 2), (5, 1)),
                                         ((5, 130), (5, 2)), ((129, 3), (2, 3))])
def test_heat2d_degenerate_shapes(dev, shape, tiles):
    """Single rows and columns, fields narrower than a lane's two columns,
    widths just past a strip, one-row tiles: every mode against the oracle."""
    u0 = synth.uniform(250 + shape[0] * 7 + shape[1], shape[0] * shape[1], lo=-1, hi=1).reshape(shape)
    for steps in (1, 4):
        want = oracle.heat2d(u0, 0.2, steps)
        for mode in ("plain", "graph", "fused"):
            got, _, _, _ = run2d(dev, u0, tiles, 0.2, steps, mode)
            assert np.max(np.abs(got - want)) <= 1e-15, (mode, steps)


def test_heat2d_bitexact_across_tilings_and_modes(dev):
    u0 = synth.bumps2d(512, 384, seed=210, nbumps=8, sigma=0.05)
    ref, _, _, _ = run2d(dev, u0, (1, 1), 0.2, 25, "plain")
    for tiles in ((2, 2), (8, 8), (3, 5), (7, 1)):
        for mode in ("plain", "graph", "fused"):
            got, _, _, _ = run2d(dev, u0, tiles, 0.2, 25, mode)
            assert np.array_equal(got, ref), (tiles, mode)
    # the pair sums (uN + uW) + (uE + uS) are symmetric under a half turn and
    # under transposition: the turned or transposed input gives the turned or
    # transposed output bit for bit
    got, _, _, _ = run2d(dev, u0[::-1, ::-1].copy(), (2, 2), 0.2, 25, "fused")
    assert np.array_equal(got, ref[::-1, ::-1])
    got, _, _, _ = run2d(dev, u0.T.copy(), (3, 2), 0.2, 25, "fused")
    assert np.array_equal(got, ref.T)


@pytest.mark.parametrize("r", [0.2, 0.25, 0.1, 0.01, 1e-30])
def test_heat2d_scaled_steps_vs_oracle(dev, r):
    """The runs' scaled and closing steps (hxc_heat2d_step_kinds): 250 steps
    without snapshots are three intervals (100, 100, 50), each cut into
    groups that end in a closing step; r = 1e-30 runs canonical steps only.
    Every mode and tiling gives the same bits, within the FP64 tolerance of
    the oracle."""
    u0 = synth.bumps2d(96, 130, seed=235, nbumps=5, sigma=0.1)
    steps = 250
    kinds = hxc.heat2d_step_kinds(hxc.heat2d_cfg(96, 130, 2, 3, r, steps, 0, "plain", None, None))
    assert sum(kinds) == steps and (kinds[0] == steps) == (r == 1e-30)
    want = oracle.heat2d(u0, r, steps)
    ref, _, _, _ = run2d(dev, u0, (1, 1), r, steps, "fused")
    assert relerr(ref, want) <= TOL
    for tiles in ((2, 3), (4, 1)):
        for mode in ("plain", "graph", "fused"):
            got, _, _, _ = run2d(dev, u0, tiles, r, steps, mode)
            assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), (tiles, mode)


def test_heat2d_scaled_steps_large_magnitudes(dev):
    """A field of magnitude 2^900: the scaled field reaches about 2^995
    before each closing step (52 steps: groups of 42 and 10) and stays
    finite; the result is within the tolerance of the oracle."""
    u0 = synth.bumps2d(64, 72, seed=236, nbumps=4, sigma=0.1) * 2.0 ** 900
    want = oracle.heat2d(u0, 0.2, 52)
    for mode in ("plain", "fused"):
        got, _, _, _ = run2d(dev, u0, (2, 2), 0.2, 52, mode)
        assert np.all(np.isfinite(got)) and relerr(got, want) <= TOL, mode


def test_heat2d_kernel_launches_per_tile(dev):
    """HXC_K_HEAT2D through hxc_launch, the canonical step
    (t = fma(-4, u, s), u' = fma(r, t, u)): the tiles of a step launched on
    their own stream slots, each after every tile of the step before (the
    per-partition form of the paper's launch workflow); every tiling, odd
    tile origins included, gives the same bits, within the tolerance of the
    oracle."""
    u0 = synth.bumps2d(150, 174, seed=237, nbumps=5, sigma=0.1)
    ny, nx = u0.shape
    steps, r = 9, 0.2

    def run(tiles):
        a, b = upload(dev, u0), dev.buffer(u0.nbytes)
        rows = [p * ny // tiles[0] for p in range(tiles[0])] + [ny]
        cols = [q * nx // tiles[1] for q in range(tiles[1])] + [nx]
        prev = []
        for s in range(steps):
            src, dst = (a, b) if s % 2 == 0 else (b, a)
            cur = []
            for p in range(tiles[0]):
                for q in range(tiles[1]):
                    args = hxc.hxc_heat2d_args(src.h, dst.h, ny, nx, rows[p], cols[q],
                                               rows[p + 1] - rows[p], cols[q + 1] - cols[q], r)
                    cur.append(dev.launch(hxc.HXC_K_HEAT2D, args, slot=p * tiles[1] + q,
                                          deps=prev))
            prev = cur
        assert hxc.wait_all(prev) == hxc.HXC_OK
        return download(b if steps % 2 else a, (ny, nx))

    ref = run((1, 1))
    assert relerr(ref, oracle.heat2d(u0, r, steps)) <= TOL
    for tiles in ((3, 4), (5, 2), (2, 7)):
        got = run(tiles)
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), tiles


def test_heat2d_rows_and_occupancy_knobs_bitexact(dev):
    """The strip height (rows per warp, including heights that are not
    multiples of the 32-row groups in which the strip-edge pair sums are
    formed) and the compiled occupancy change speed only: every value gives
    the bits of the default, on an even width (two columns per lane) and an
    odd width (one column per lane), tiled and whole-field."""
    old = {k: hxc.tune_get(k) for k in ("heat2d.rows", "heat2d.occupancy")}
    try:
        for u0, tiles in ((synth.bumps2d(300, 386, seed=230, nbumps=6, sigma=0.05), (3, 2)),
                          (synth.uniform(231, 97 * 131, lo=-1, hi=1).reshape(97, 131), (1, 1))):
            ref, _, _, _ = run2d(dev, u0, tiles, 0.2, 9, "fused")
            assert relerr(ref, oracle.heat2d(u0, 0.2, 9)) <= TOL
            for rows in (1, 3, 16, 31, 32, 33, 64, 100, 4096):
                for occ in (4, 6):
                    hxc.tune_set("heat2d.rows", rows)
                    hxc.tune_set("heat2d.occupancy", occ)
                    got, _, _, _ = run2d(dev, u0, tiles, 0.2, 9, "fused")
                    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), (rows, occ)
    finally:
        for k, v in old.items():
            hxc.tune_set(k, v)


def test_heat2d_snapshot_norms(dev):
    """Host norms (then-continuations on device->host snapshots) and device
    norms (fixed-order reduction) against the oracle's tile norms."""
    u0 = synth.bumps2d(256, 320, seed=220, nbumps=6, sigma=0.05)
    tiles, every, steps, r = (4, 5), 7, 30, 0.2
    for mode in ("plain", "graph", "fused"):
        _, hn, gn, st = run2d(dev, u0, tiles, r, steps, mode, every)
        assert st.host_tasks == (steps // every) * 20
        for k in range(steps // every):
            state = oracle.heat2d(u0, r, (k + 1) * every)
            want = oracle.tile_norms(state[:, :], 64, 64).ravel()
            # host norms: long-double sums, within 1e-14 of the oracle's
            # long-double sum; device norms: FP64 fixed-order tree (about
            # 80 roundings deep, < 1e-14)
            assert np.max(np.abs(hn[k] - want) / want) <= 1e-14, (mode, k)
            assert np.max(np.abs(gn[k] - want) / want) <= 1e-14, (mode, k)
            assert np.max(np.abs(gn[k] - hn[k]) / hn[k]) <= 1e-14
    # device norms are bit-identical across modes (fixed reduction order)
    _, _, g1, _ = run2d(dev, u0, tiles, r, steps, "plain", every)
    _, _, g2, _ = run2d(dev, u0, tiles, r, steps, "graph", every)
    _, _, g3, _ = run2d(dev, u0, tiles, r, steps, "fused", every)
    assert np.array_equal(g1, g2) and np.array_equal(g1, g3)


def test_heat2d_device_norms_when_the_tile_count_changes(dev):
    """Fused runs share one reduction scratch whatever their tile grid:
    device norms stay right when the tile count goes down and up again."""
    u0 = synth.bumps2d(192, 240, seed=221, nbumps=5, sigma=0.06)
    for tiles in ((4, 5), (2, 3), (4, 5), (3, 4), (1, 1), (2, 3)):
        _, hn, gn, _ = run2d(dev, u0, tiles, 0.2, 12, "fused", 6)
        assert np.max(np.abs(gn - hn) / hn) <= 1e-14, tiles


def test_heat2d_full_config(dev):
    """8192^2, 64 tiles of 1024^2, r = 0.2, 1000 steps, snapshots every 100
    steps: every mode bit-identical; the whole field against the oracle, and
    a corner window against the oracle's windowed run (the dependence cone of
    a cell after 1000 steps is 1000 cells wide, so cells 1000 away from the
    window's cut edges are exact); device norms against host norms; the last
    snapshot's norms against norms of the downloaded final field."""
    n, steps, r, every = 8192, 1000, 0.2, 100
    u0 = synth.bumps2d(n, n, seed=2)
    outs = {}
    for mode in ("plain", "graph", "fused"):
        got, hn, gn, st = run2d(dev, u0, (8, 8), r, steps, mode, every)
        outs[mode] = got
        assert np.max(np.abs(gn - hn) / np.maximum(hn, 1e-300)) <= 1e-14
    assert np.array_equal(outs["plain"], outs["graph"])
    assert np.array_equal(outs["plain"], outs["fused"])
    got = outs["plain"]
    scale = np.max(np.abs(got))
    w = oracle.heat2d_window(u0, n - 1300, n - 1300, 1300, 1300, r, steps)
    assert np.max(np.abs(got[n - 300:, n - 300:] - w[1000:, 1000:])) <= TOL * scale
    # the whole field against the oracle (its OpenMP build: the same loop on
    # all host threads, bit-identical to the serial one)
    a, b = u0.copy(), np.zeros_like(u0)
    want = oracle.heat2d_steps(a, b, r, steps, omp=True)
    assert np.max(np.abs(got - want)) <= TOL * np.max(np.abs(want))
    del a, b, want
    fin = np.array([np.sqrt(np.sum(got[i * 1024:(i + 1) * 1024, j * 1024:(j + 1) * 1024]
                                   .astype(np.longdouble) ** 2))
                    for i in range(8) for j in range(8)], dtype=np.float64)
    assert np.max(np.abs(hn[-1] - fin) / fin) <= 1e-14
    # the end-to-end form the benchmark times: the field from pinned host
    # memory through the asynchronous host entry point, two calls in flight
    hu = hxc.host_empty((n, n))
    hu[:] = u0
    outs_h, keep = [], []
    for _ in range(2):
        ho = hxc.host_empty((n, n))
        hn2, gn2 = np.zeros(10 * 64), np.zeros(10 * 64)
        cfg = hxc.heat2d_cfg(n, n, 8, 8, r, steps, every, "fused", hn2, gn2)
        f, _ = hxc.heat2d_run_host_async(dev, hu.ctypes.data, ho.ctypes.data, cfg)
        outs_h.append((f, ho, hn2, gn2))
        keep.append(cfg)
    for f, ho, hn2, gn2 in outs_h:
        assert f.wait(600 * 10**9) == hxc.HXC_OK
        assert np.array_equal(np.array(ho), got)
        assert np.array_equal(hn2, hn.ravel()) and np.array_equal(gn2, gn.ravel())


def test_heat2d_full_size_window_at_peak(dev):
    """Full 8192^2 field, 150 steps, oracle window centred on the largest
    initial value (where the solution is significant)."""
    n, steps, r = 8192, 150, 0.2
    u0 = synth.bumps2d(n, n, seed=2)
    got, _, _, _ = run2d(dev, u0, (8, 8), r, steps, "plain")
    ci, cj = np.unravel_index(np.argmax(u0), u0.shape)
    half = steps + 64
    y0, x0 = max(0, ci - half), max(0, cj - half)
    wy, wx = min(n, ci + half) - y0, min(n, cj + half) - x0
    w = oracle.heat2d_window(u0, y0, x0, wy, wx, r, steps)
    ey0 = 0 if y0 == 0 else steps
    ex0 = 0 if x0 == 0 else steps
    ey1 = wy if y0 + wy == n else wy - steps
    ex1 = wx if x0 + wx == n else wx - steps
    exact = w[ey0:ey1, ex0:ex1]
    mine = got[y0 + ey0:y0 + ey1, x0 + ex0:x0 + ex1]
    assert exact.size > 0
    assert np.max(np.abs(mine - exact)) <= TOL * np.max(np.abs(got))


def test_heat2d_sine_mode_full_size(dev):
    """A Dirichlet sine mode on the full 8192^2 grid decays by exactly
    g^n, g = 1 - 4 r [sin^2(p pi h/2) + sin^2(q pi h/2)], up to rounding."""
    n, r, steps, p, q = 8192, 0.2, 200, 3, 5
    h = 1.0 / (n + 1)
    x = (np.arange(n) + 1) * h
    u0 = np.outer(np.sin(q * np.pi * x), np.sin(p * np.pi * x))
    g = 1.0 - 4.0 * r * (math.sin(p * math.pi * h / 2) ** 2 + math.sin(q * math.pi * h / 2) ** 2)
    got, _, _, _ = run2d(dev, u0, (8, 8), r, steps, "fused")
    assert np.max(np.abs(got - g ** steps * u0)) <= 64 * steps * np.finfo(float).eps


def test_heat2d_host_entry_point(dev):
    """hxc_heat2d_run_host: field in pinned host memory, per-tile copies."""
    ny, nx = 1024, 768
    u0 = synth.bumps2d(ny, nx, seed=230, nbumps=6, sigma=0.05)
    hu = hxc.host_empty((ny, nx))
    hu[:] = u0
    out = hxc.host_empty((ny, nx))
    hn = np.zeros(2 * 12)
    cfg = hxc.heat2d_cfg(ny, nx, 4, 3, 0.2, 40, 20, "plain", hn, None)
    st = hxc.heat2d_run_host(dev, hu.ctypes.data, out.ctypes.data, cfg)
    want = oracle.heat2d(u0, 0.2, 40)
    assert relerr(np.array(out), want) <= TOL
    assert st.h2d_bytes == u0.nbytes and st.d2h_bytes >= u0.nbytes


def test_heat2d_host_async_calls_overlap_and_match(dev):
    """hxc_heat2d_run_host_async: five calls issued back to back on different
    fields, two shapes (a device field pair grows while the other call is in
    flight), each result and each norm bit-identical to the synchronous entry
    point and the field within the oracle's tolerance."""
    shapes = [(512, 384), (512, 384), (640, 512), (512, 384), (640, 512)]
    fields = [synth.bumps2d(ny, nx, seed=600 + i, nbumps=5, sigma=0.06)
              for i, (ny, nx) in enumerate(shapes)]
    keep, futs = [], []
    for i, u0 in enumerate(fields):
        hu, ho = hxc.host_empty(u0.shape), hxc.host_empty(u0.shape)
        hu[:] = u0
        ho[:] = np.nan
        hn, gn = np.zeros(2 * 6), np.zeros(2 * 6)
        mode = ("fused", "plain", "graph")[i % 3]
        cfg = hxc.heat2d_cfg(u0.shape[0], u0.shape[1], 2, 3, 0.2, 30, 15, mode, hn, gn)
        f, st = hxc.heat2d_run_host_async(dev, hu.ctypes.data, ho.ctypes.data, cfg)
        assert st.h2d_bytes == u0.nbytes and st.d2h_bytes >= u0.nbytes
        keep.append((hu, ho, hn, gn, cfg))
        futs.append(f)
    for f in futs:
        assert f.wait(60 * 10**9) == hxc.HXC_OK
    for i, u0 in enumerate(fields):
        hu, ho, hn, gn, _ = keep[i]
        out = hxc.host_empty(u0.shape)
        hn2, gn2 = np.zeros(12), np.zeros(12)
        cfg = hxc.heat2d_cfg(u0.shape[0], u0.shape[1], 2, 3, 0.2, 30, 15, "fused", hn2, gn2)
        hxc.heat2d_run_host(dev, hu.ctypes.data, out.ctypes.data, cfg)
        assert np.array_equal(np.array(ho).view(np.uint64), np.array(out).view(np.uint64)), i
        assert np.array_equal(hn, hn2) and np.array_equal(gn, gn2), i
        assert relerr(np.array(ho), oracle.heat2d(u0, 0.2, 30)) <= TOL


def test_heat2d_host_async_dependencies_and_failure(dev):
    """The uploads of an asynchronous host call wait for its dependencies; a
    failed dependency fails that call only, and the next calls (which reuse
    its device field pair) run normally."""
    ny, nx = 256, 320
    u0 = synth.bumps2d(ny, nx, seed=610, nbumps=4, sigma=0.08)
    want = oracle.heat2d(u0, 0.2, 12)
    hu = hxc.host_empty((ny, nx))
    hu[:] = u0
    outs = [hxc.host_empty((ny, nx)) for _ in range(3)]
    hn = np.zeros(2 * 4)
    cfg = hxc.heat2d_cfg(ny, nx, 2, 2, 0.2, 12, 6, "fused", hn, None)
    gate = hxc.promise()
    f0, _ = hxc.heat2d_run_host_async(dev, hu.ctypes.data, outs[0].ctypes.data, cfg, deps=[gate])
    assert f0.wait(50 * 10**6) == hxc.HXC_E_TIMEOUT  # held by the gate
    hxc.promise_set(gate, hxc.HXC_OK)
    assert f0.wait(60 * 10**9) == hxc.HXC_OK
    assert relerr(np.array(outs[0]), want) <= TOL
    bad = hxc.promise()
    f1, _ = hxc.heat2d_run_host_async(dev, hu.ctypes.data, outs[1].ctypes.data, cfg, deps=[bad])
    hxc.promise_set(bad, hxc.HXC_E_CALLBACK)
    assert f1.wait(60 * 10**9) == hxc.HXC_E_DEP_FAILED
    for i in range(3):
        f, _ = hxc.heat2d_run_host_async(dev, hu.ctypes.data, outs[2].ctypes.data, cfg)
        assert f.wait(60 * 10**9) == hxc.HXC_OK, i
        assert np.array_equal(np.array(outs[2]), np.array(outs[0])), i


# ------------------------------------------- integer-pipe FP64 additions

def test_heat2d_integer_adder_splits_are_bit_identical(dev):
    """Every split of the 2D additions between the FP64 pipe and the
    integer-pipe IEEE adder gives the same bits: on smooth bumps, on random
    finite doubles spanning the whole exponent range (subnormals, mixed
    signs, huge magnitudes) and on an odd width (scalar path)."""
    old = hxc.tune_get("heat2d.emul")
    try:
        bits = synth.splitmix64(77, 300 * 258)
        raw = bits.view(np.float64).reshape(300, 258).copy()
        raw[~np.isfinite(raw)] = 0.0
        raw = np.where(np.abs(raw) > 1e300, raw * 1e-10, raw)
        fields = [synth.bumps2d(256, 320, seed=240, nbumps=6, sigma=0.05), raw,
                  synth.uniform(241, 97 * 131, lo=-1, hi=1).reshape(97, 131)]
        for u0 in fields:
            outs = []
            for em in range(5):
                hxc.tune_set("heat2d.emul", em)
                got, _, _, _ = run2d(dev, u0, (2, 3), 0.2, 7, "fused")
                outs.append(got)
            for em in range(1, 5):
                assert np.array_equal(outs[em].view(np.uint64), outs[0].view(np.uint64)), em
        want = oracle.heat2d(fields[0], 0.2, 7)
        assert relerr(outs[0], oracle.heat2d(fields[2], 0.2, 7)) <= TOL
        hxc.tune_set("heat2d.emul", 4)
        got, _, _, _ = run2d(dev, fields[0], (2, 3), 0.2, 7, "plain")
        assert relerr(got, want) <= TOL
    finally:
        hxc.tune_set("heat2d.emul", old)


def test_heat2d_integer_adder_full_size(dev):
    old = hxc.tune_get("heat2d.emul")
    try:
        u0 = synth.bumps2d(8192, 8192, seed=2)
        hxc.tune_set("heat2d.emul", 0)
        a, _, _, _ = run2d(dev, u0, (8, 8), 0.2, 1000, "fused")
        for em in (3, 4):
            hxc.tune_set("heat2d.emul", em)
            b, _, _, _ = run2d(dev, u0, (8, 8), 0.2, 1000, "fused")
            assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), em
    finally:
        hxc.tune_set("heat2d.emul", old)
