"""The allocation-free tile-norm entry point against the regular one.

hxc_tile_norms_noalloc serves callers that must not let the library
allocate device memory (a time-critical loop where cudaMalloc would stall
the device, memory owned by another allocator, no allocation after
start-up).  It keeps its reduction scratch in a fixed array inside the
library, so it is checked here against HXC_K_TILE_NORM2 (whose scratch comes
from the library's allocating cache) through the C ABI, on two calls in a
row: the second call must not see leftovers of the first.  This file runs
last so that a stop at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1810_11482_b300 import hxc, synth

pytestmark = pytest.mark.gpu
TOL = 1e-12  # the norm tolerance of the other GPU tests (the results are expected bit-equal)


@pytest.fixture(scope="module")
def dev():
    devs = hxc.get_all_devices(2, 0)
    assert devs
    return devs[0]


def tile_bounds(ny, nx, ty, tx):
    """The tile grid documented in include/hxc.h (that of hxc_heat2d_run)."""
    rows = [p * ny // ty for p in range(ty)] + [ny]
    if nx % 2 == 0:
        cols = [(q * (nx // 2) // tx) * 2 for q in range(tx)] + [nx]
    else:
        cols = [q * nx // tx for q in range(tx)] + [nx]
    return rows, cols


def reference_norms(dev, field, ny, nx, ty, tx):
    """Per-tile norms through the regular launch (HXC_K_TILE_NORM2)."""
    rows, cols = tile_bounds(ny, nx, ty, tx)
    sums = dev.buffer(ty * tx * 8)
    futs = []
    for p in range(ty):
        for q in range(tx):
            a = hxc.hxc_tile_norm2_args(field.h, None, sums.h, ny, nx, rows[p], cols[q],
                                        rows[p + 1] - rows[p], cols[q + 1] - cols[q], p * tx + q)
            futs.append(dev.launch(hxc.HXC_K_TILE_NORM2, a, slot=3))
    assert hxc.wait_all(futs) == hxc.HXC_OK
    out = np.empty(ty * tx)
    sums.read_sync(out)
    return out


def noalloc_norms(dev, field, ny, nx, ty, tx, out_buf, stream):
    L = hxc.lib()
    st = L.hxc_tile_norms_noalloc(ctypes.c_void_p(field.ptr), ny, nx, ty, tx,
                                  ctypes.c_void_p(out_buf.ptr), ctypes.c_void_p(stream))
    assert st == hxc.HXC_OK, L.hxc_last_error()
    dev.synchronize()
    out = np.empty(ty * tx)
    out_buf.read_sync(out)
    return out


def test_noalloc_tile_norms_match_regular_entry_point(dev):
    stream = dev.stream(7)
    cases = [((1000, 1002), (7, 9), 901), ((777, 501), (4, 5), 902)]
    out_buf = dev.buffer(256 * 8)
    for (ny, nx), (ty, tx), seed in cases:
        u = synth.bumps2d(ny, nx, seed=seed, nbumps=5, sigma=0.1)
        field = dev.buffer(u.nbytes)
        field.write(u).get()
        want = reference_norms(dev, field, ny, nx, ty, tx)
        for _ in range(2):  # two calls in a row share the scratch array
            got = noalloc_norms(dev, field, ny, nx, ty, tx, out_buf, stream)
            assert np.max(np.abs(got - want) / want) <= TOL
        # and against an independent host computation
        rows, cols = tile_bounds(ny, nx, ty, tx)
        host = np.array([np.sqrt(np.sum(u[rows[p]:rows[p + 1], cols[q]:cols[q + 1]]
                                        .astype(np.longdouble) ** 2))
                         for p in range(ty) for q in range(tx)], dtype=np.float64)
        assert np.max(np.abs(got - host) / host) <= TOL


def test_noalloc_rejects_grids_beyond_the_scratch(dev):
    L = hxc.lib()
    u = dev.buffer(64 * 64 * 8)
    out = dev.buffer(8 * 300)
    st = L.hxc_tile_norms_noalloc(ctypes.c_void_p(u.ptr), 64, 64, 16, 17,
                                  ctypes.c_void_p(out.ptr), None)
    assert st == hxc.HXC_E_INVALID
    assert b"exceed" in L.hxc_last_error()
