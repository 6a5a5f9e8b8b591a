"""The allocation-free tile-norm entry point against the regular one.

hxc_tile_norms_noalloc serves callers that must not let the library
allocate device memory (a time-critical loop where cudaMalloc would stall
the device, memory owned by another allocator, no allocation after
start-up).  It keeps its reduction scratch in a fixed array inside the
library and runs the same grid kernel as the 2D runs' device norms, so it is
checked here bit for bit against HXC_K_TILE_NORM2 (whose scratch comes from
the library's allocating cache) through the C ABI, on two calls in a row
(the second call must not see leftovers of the first), and against an
independent long-double host sum.  A fresh process checks that its first
call leaves the device's free memory unchanged.  This file runs last so that
a stop at the first failure has already run every other test.
"""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1810_11482_b300 import hxc, synth

pytestmark = pytest.mark.gpu
TOL = 1e-12  # the norm tolerance of the other GPU tests, for the host long-double sums
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dev():
    devs = hxc.get_all_devices(2, 0)
    assert devs
    return devs[0]


def cudart():
    return ctypes.CDLL("libcudart.so.13")


def tile_bounds(ny, nx, ty, tx):
    """The tile grid documented in include/hxc.h (that of hxc_heat2d_run)."""
    rows = [p * ny // ty for p in range(ty)] + [ny]
    if nx % 2 == 0:
        cols = [(q * (nx // 2) // tx) * 2 for q in range(tx)] + [nx]
    else:
        cols = [q * nx // tx for q in range(tx)] + [nx]
    return rows, cols


def reference_norms(dev, field, ny, nx, ty, tx):
    """Per-tile norms through the regular launch (HXC_K_TILE_NORM2); tiles of
    zero width are not launched and stay 0."""
    rows, cols = tile_bounds(ny, nx, ty, tx)
    sums = dev.buffer(ty * tx * 8)
    sums.write(np.zeros(ty * tx)).get()
    futs = []
    for p in range(ty):
        for q in range(tx):
            h, w = rows[p + 1] - rows[p], cols[q + 1] - cols[q]
            if h == 0 or w == 0:
                continue
            a = hxc.hxc_tile_norm2_args(field.h, None, sums.h, ny, nx, rows[p], cols[q], h, w,
                                        p * tx + q)
            futs.append(dev.launch(hxc.HXC_K_TILE_NORM2, a, slot=3))
    assert hxc.wait_all(futs) == hxc.HXC_OK
    out = np.empty(ty * tx)
    sums.read_sync(out)
    return out


def host_norms(u, ty, tx):
    ny, nx = u.shape
    rows, cols = tile_bounds(ny, nx, ty, tx)
    return np.array([np.sqrt(np.sum(u[rows[p]:rows[p + 1], cols[q]:cols[q + 1]]
                                    .astype(np.longdouble) ** 2))
                     for p in range(ty) for q in range(tx)], dtype=np.float64)


def noalloc_norms(field, ny, nx, ty, tx, out_buf, stream):
    L = hxc.lib()
    out_buf.write(np.full(ty * tx, np.nan)).get()
    st = L.hxc_tile_norms_noalloc(ctypes.c_void_p(field.ptr), ny, nx, ty, tx,
                                  ctypes.c_void_p(out_buf.ptr), ctypes.c_void_p(stream))
    assert st == hxc.HXC_OK, L.hxc_last_error()
    # the call runs on the caller's stream (the legacy stream for None)
    assert cudart().cudaDeviceSynchronize() == 0
    out = np.empty(ty * tx)
    out_buf.read_sync(out)
    return out


@pytest.mark.parametrize("shape,grid,seed", [
    ((1000, 1002), (7, 9), 901),   # even width, ragged tiles
    ((777, 501), (4, 5), 902),     # odd width
    ((64, 64), (16, 16), 903),     # exactly the largest grid (256 tiles)
    ((8, 8), (1, 6), 904),         # even width, more tiles than column pairs: empty tiles
])
def test_noalloc_tile_norms_match_regular_entry_point(dev, shape, grid, seed):
    (ny, nx), (ty, tx) = shape, grid
    u = synth.bumps2d(ny, nx, seed=seed, nbumps=5, sigma=0.1)
    field = dev.buffer(u.nbytes)
    field.write(u).get()
    want = reference_norms(dev, field, ny, nx, ty, tx)
    host = host_norms(u, ty, tx)
    out_buf = dev.buffer(256 * 8)
    for stream in (dev.stream(7), None):
        for _ in range(2):  # two calls in a row share the scratch array
            got = noalloc_norms(field, ny, nx, ty, tx, out_buf, stream)
            assert np.array_equal(got, want)
            empty = host == 0.0
            assert np.all(got[empty] == 0.0)
            assert np.max(np.abs(got[~empty] - host[~empty]) / host[~empty]) <= TOL
    if (ny, nx, ty, tx) == (8, 8, 1, 6):
        assert np.count_nonzero(host == 0.0) == 2  # tiles 0 and 3 have no columns


def test_noalloc_rejects_grids_beyond_the_scratch(dev):
    L = hxc.lib()
    u = dev.buffer(64 * 64 * 8)
    out = dev.buffer(8 * 300)
    st = L.hxc_tile_norms_noalloc(ctypes.c_void_p(u.ptr), 64, 64, 16, 17,
                                  ctypes.c_void_p(out.ptr), None)
    assert st == hxc.HXC_E_INVALID
    assert b"exceed" in L.hxc_last_error()


_FRESH = r"""
import ctypes, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1810_11482_b300 import hxc, synth
rt = ctypes.CDLL("libcudart.so.13")
dev = hxc.get_all_devices(2, 0)[0]
ny, nx, ty, tx = 1000, 1002, 7, 9
u = synth.bumps2d(ny, nx, seed=901, nbumps=5, sigma=0.1)
field, out = dev.buffer(u.nbytes), dev.buffer(ty * tx * 8)
field.write(u).get()
stream = dev.stream(2)
assert rt.cudaDeviceSynchronize() == 0
free0, free1, total = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
assert rt.cudaMemGetInfo(ctypes.byref(free0), ctypes.byref(total)) == 0
st = hxc.lib().hxc_tile_norms_noalloc(ctypes.c_void_p(field.ptr), ny, nx, ty, tx,
                                      ctypes.c_void_p(out.ptr), ctypes.c_void_p(stream))
assert rt.cudaDeviceSynchronize() == 0
assert rt.cudaMemGetInfo(ctypes.byref(free1), ctypes.byref(total)) == 0
got = np.empty(ty * tx)
out.read_sync(got)
print(json.dumps({"status": st, "free0": free0.value, "free1": free1.value,
                  "norms": got.tolist()}))
"""


def test_noalloc_first_call_in_fresh_process_allocates_nothing(dev):
    """The entry point's first call in a new process, before any other
    library operation that could allocate, leaves the device's free memory
    where it was (device code loaded eagerly at context creation, so module
    loading does not count), and its norms equal the regular launch's."""
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["status"] == hxc.HXC_OK
    assert res["free0"] - res["free1"] < (1 << 20), res
    ny, nx, ty, tx = 1000, 1002, 7, 9
    u = synth.bumps2d(ny, nx, seed=901, nbumps=5, sigma=0.1)
    field = dev.buffer(u.nbytes)
    field.write(u).get()
    assert np.array_equal(np.array(res["norms"]), reference_norms(dev, field, ny, nx, ty, tx))
