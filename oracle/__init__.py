"""FP64 CPU oracle for the heat-equation hot path (ctypes wrapper of oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports this package, and this package imports nothing from the
product library.

Each wrapper states the definition it evaluates; the C source holds the
plain loops.  All arrays are float64 numpy arrays in C order.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lib = None
_lib_omp = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.c_int64


def build():
    """Compile liboracle.so with -O2 -ffp-contract=off (no FMA contraction),
    and liboracle_omp.so, the same source with OpenMP enabled."""
    subprocess.check_call(["make", "-s", "-C", _HERE, "all"])


def _stale(path):
    src = os.path.join(_HERE, "oracle.c")
    return not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(src)


def _declare_batch(L):
    L.ora_varcoef2d_batch.argtypes = [_dp, _dp, _dp, ctypes.POINTER(_i64),
                                      ctypes.POINTER(_i64), _dp, _i64, ctypes.c_int]


def _declare_steps(L):
    L.ora_heat2d_steps.argtypes = [_dp, _dp, _i64, _i64, ctypes.c_double, ctypes.c_int]
    L.ora_heat2d_steps.restype = ctypes.c_void_p
    L.ora_heat3d_steps.argtypes = [_dp, _dp, _i64, _i64, _i64, ctypes.c_double, ctypes.c_int]
    L.ora_heat3d_steps.restype = ctypes.c_void_p
    L.ora_threads.restype = ctypes.c_int


def lib_omp():
    """The OpenMP build (liboracle_omp.so): only the row loop of the 2D
    stepping routine, the plane loop of the 3D one and the problem loop of
    the batch differ, and only in running on all threads."""
    global _lib_omp
    if _lib_omp is None:
        if _stale(_LIB_OMP):
            build()
        L = ctypes.CDLL(_LIB_OMP)
        _declare_steps(L)
        _declare_batch(L)
        _lib_omp = L
    return _lib_omp


def lib():
    global _lib
    if _lib is None:
        if _stale(_LIB):
            build()
        L = ctypes.CDLL(_LIB)
        _declare_steps(L)
        L.ora_prk_stencil.argtypes = [_dp, _dp, _i64]
        L.ora_sum_u32.argtypes = [ctypes.POINTER(ctypes.c_uint32), _i64]
        L.ora_sum_u32.restype = ctypes.c_uint64
        L.ora_heat1d.argtypes = [_dp, _dp, _i64, ctypes.c_double, ctypes.c_int]
        L.ora_heat2d.argtypes = [_dp, _dp, _i64, _i64, ctypes.c_double, ctypes.c_int]
        L.ora_heat2d_window.argtypes = [_dp, _dp, _i64, _i64, _i64, _i64, _i64, _i64,
                                        ctypes.c_double, ctypes.c_int]
        L.ora_tile_norms.argtypes = [_dp, _i64, _i64, _i64, _i64, _dp]
        L.ora_heat3d.argtypes = [_dp, _dp, _i64, _i64, _i64, ctypes.c_double, ctypes.c_int]
        L.ora_varcoef2d.argtypes = [_dp, _dp, _dp, _i64, _i64, ctypes.c_double, ctypes.c_int]
        L.ora_varcoef2d_transpose_step.argtypes = [_dp, _dp, _dp, _i64, _i64, ctypes.c_double]
        L.ora_varcoef2d_adjoint.argtypes = [_dp, _dp, _dp, _i64, _i64, ctypes.c_double,
                                            ctypes.c_int, _dp, _dp]
        L.ora_varcoef2d_adjoint.restype = ctypes.c_double
        _declare_batch(L)
        _fp = ctypes.POINTER(ctypes.c_float)
        L.ora_mandelbrot_counts.argtypes = [_fp, _fp, ctypes.POINTER(ctypes.c_int32), _i64,
                                            ctypes.c_int32]
        L.ora_mandelbrot_image.argtypes = [ctypes.POINTER(ctypes.c_uint8),
                                           ctypes.POINTER(ctypes.c_int32), _i64, _i64,
                                           ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                           ctypes.c_float, ctypes.c_int32]
        _lib = L
    return _lib


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _p(a):
    return a.ctypes.data_as(_dp)


def prk_stencil(x):
    """Sec. 5.1.1: s(x_i) = 0.5 x_{i-1} + x_i + 0.5 x_{i+1} (periodic ends)."""
    x = _f64(x)
    s = np.empty_like(x)
    lib().ora_prk_stencil(_p(x), _p(s), x.size)
    return s


def sum_u32(x):
    """Listing 2 (Sec. 4.2): the sum of n unsigned integers."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    return int(lib().ora_sum_u32(x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), x.size))


def partition_k(x):
    """Sec. 5.1.2: the partition kernel k(x) = sqrt(sin(x)^2 + cos(x)^2),
    elementwise, with the C library's sin, cos and sqrt."""
    x = _f64(x)
    return np.sqrt(np.sin(x) ** 2 + np.cos(x) ** 2)


def mandelbrot_counts(cr, ci, max_iter):
    """Sec. 5.1.3: escape counts of the points c = cr + i ci (binary32) under
    z <- z^2 + c from z = 0 (max_iter for points that do not escape)."""
    cr = np.ascontiguousarray(cr, dtype=np.float32)
    ci = np.ascontiguousarray(ci, dtype=np.float32)
    cnt = np.empty(cr.size, dtype=np.int32)
    fp = ctypes.POINTER(ctypes.c_float)
    lib().ora_mandelbrot_counts(cr.ctypes.data_as(fp), ci.ctypes.data_as(fp),
                                cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), cr.size, max_iter)
    return cnt


def mandelbrot_image(width, height, x0, y0, dx, dy, max_iter):
    """Sec. 5.1.3: the RGB8 image (height, width, 3) and escape counts
    (height, width) of pixel c = (x0 + i dx) + (y0 + j dy) i."""
    rgb = np.empty((height, width, 3), dtype=np.uint8)
    cnt = np.empty((height, width), dtype=np.int32)
    lib().ora_mandelbrot_image(rgb.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                               cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), width, height,
                               x0, y0, dx, dy, max_iter)
    return rgb, cnt


def heat1d(u0, r, steps):
    """Periodic 1D FTCS: u'_j = u_j + r (u_{j-1} - 2 u_j + u_{j+1})."""
    u0 = _f64(u0)
    out = np.empty_like(u0)
    lib().ora_heat1d(_p(u0), _p(out), u0.size, r, steps)
    return out


def heat2d(u0, r, steps):
    """2D FTCS, 5-point Laplacian, Dirichlet-zero ghost ring."""
    u0 = _f64(u0)
    out = np.empty_like(u0)
    lib().ora_heat2d(_p(u0), _p(out), u0.shape[0], u0.shape[1], r, steps)
    return out


def heat2d_steps(a, b, r, steps, omp=False):
    """2D FTCS as heat2d, stepping the caller's C-contiguous float64 arrays in
    place (a holds u^0, b is scratch; no allocation or copy inside).  Returns
    whichever of a, b holds u^steps.  omp=True runs the OpenMP build."""
    assert a.dtype == np.float64 and b.dtype == np.float64 and a.shape == b.shape
    assert a.flags.c_contiguous and b.flags.c_contiguous
    L = lib_omp() if omp else lib()
    res = L.ora_heat2d_steps(_p(a), _p(b), a.shape[0], a.shape[1], r, steps)
    return a if res == a.ctypes.data else b


def threads(omp=False):
    """Threads the 2D stepping routine runs on (1 for the serial build)."""
    return int((lib_omp() if omp else lib()).ora_threads())


def heat2d_window(u0, wy0, wx0, wny, wnx, r, steps):
    """2D FTCS on the window [wy0, wy0+wny) x [wx0, wx0+wnx) of u0, zero outside
    the window; cells at distance >= steps from every window edge that is not
    a domain edge are exact."""
    u0 = _f64(u0)
    out = np.empty((wny, wnx), dtype=np.float64)
    lib().ora_heat2d_window(_p(u0), _p(out), u0.shape[0], u0.shape[1],
                            wy0, wx0, wny, wnx, r, steps)
    return out


def tile_norms(u, ty, tx):
    """sqrt(sum u^2) per ty x tx tile (long-double accumulation)."""
    u = _f64(u)
    ny, nx = u.shape
    out = np.empty((ny // ty, nx // tx), dtype=np.float64)
    lib().ora_tile_norms(_p(u), ny, nx, ty, tx, _p(out))
    return out


def heat3d(u0, r, steps):
    """Periodic 3D FTCS, 7-point Laplacian, layout (z, y, x) x fastest, FP64."""
    u0 = _f64(u0)
    out = np.empty_like(u0)
    nz, ny, nx = u0.shape
    lib().ora_heat3d(_p(u0), _p(out), nz, ny, nx, r, steps)
    return out


def heat3d_steps(a, b, r, steps, omp=False):
    """3D FTCS as heat3d, stepping the caller's C-contiguous float64 arrays of
    shape (nz, ny, nx) in place (a holds u^0, b is scratch).  Returns whichever
    of a, b holds u^steps.  omp=True runs the OpenMP build."""
    assert a.dtype == np.float64 and b.dtype == np.float64 and a.shape == b.shape and a.ndim == 3
    assert a.flags.c_contiguous and b.flags.c_contiguous
    L = lib_omp() if omp else lib()
    nz, ny, nx = a.shape
    res = L.ora_heat3d_steps(_p(a), _p(b), nz, ny, nx, r, steps)
    return a if res == a.ctypes.data else b


def varcoef2d(u0, kappa, c, steps):
    """Variable-diffusivity FTCS, conservative flux form, arithmetic face mean,
    Dirichlet-zero ghosts whose diffusivity equals the facing interior cell."""
    u0 = _f64(u0)
    kappa = _f64(kappa)
    out = np.empty_like(u0)
    lib().ora_varcoef2d(_p(u0), _p(kappa), _p(out), u0.shape[0], u0.shape[1], c, steps)
    return out


def varcoef2d_transpose_step(lam, kappa, c):
    """Transpose of one variable-diffusivity step (scatter form)."""
    lam = _f64(lam)
    kappa = _f64(kappa)
    out = np.empty_like(lam)
    lib().ora_varcoef2d_transpose_step(_p(lam), _p(out), _p(kappa), lam.shape[0],
                                       lam.shape[1], c)
    return out


def varcoef2d_adjoint(u0, kappa, utgt, c, steps):
    """L = sum (u^T - u_tgt)^2 and (dL/dkappa, dL/du0) by reverse accumulation."""
    u0 = _f64(u0)
    kappa = _f64(kappa)
    utgt = _f64(utgt)
    gk = np.empty_like(u0)
    gu = np.empty_like(u0)
    loss = lib().ora_varcoef2d_adjoint(_p(u0), _p(kappa), _p(utgt), u0.shape[0],
                                       u0.shape[1], c, steps, _p(gk), _p(gu))
    return loss, gk, gu


def varcoef2d_batch(u0, kappa, sides, offsets, cs, steps, omp=False):
    """Independent square problems packed back to back; each stepped with its own c.
    omp=True runs the OpenMP build (problems spread over the host threads)."""
    u0 = _f64(u0)
    kappa = _f64(kappa)
    out = np.empty_like(u0)
    sides = np.ascontiguousarray(sides, dtype=np.int64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    cs = _f64(cs)
    P = ctypes.POINTER(_i64)
    L = lib_omp() if omp else lib()
    L.ora_varcoef2d_batch(_p(u0), _p(kappa), _p(out), sides.ctypes.data_as(P),
                          offsets.ctypes.data_as(P), _p(cs), sides.size, steps)
    return out
