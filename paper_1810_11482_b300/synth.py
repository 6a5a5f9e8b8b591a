"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds input recipes only: no step of the stencil method is
computed here, and it imports nothing else from this package, so the oracle
side and the CUDA side can both call it without depending on each other.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: the k-th output (k = 1, 2, ...) of the stream with state `seed` is
mix(seed + k * 0x9E3779B97F4A7C15), with the published finaliser
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
    z ^= z >> 27; z *= 0x94D049BB133111EB;
    z ^= z >> 31,
so element k can be generated without the k-1 before it.  A uniform double
in [0, 1) is (x >> 11) * 2^-53.
"""
import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def splitmix64(seed, n, start=0):
    """Outputs start+1 .. start+n of the SplitMix64 stream with state `seed`."""
    out = np.empty(n, dtype=np.uint64)
    seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for c0 in range(0, n, _CHUNK):
            c1 = min(n, c0 + _CHUNK)
            z = np.arange(start + c0 + 1, start + c1 + 1, dtype=np.uint64)
            z *= GAMMA
            z += seed
            z ^= z >> np.uint64(30)
            z *= _M1
            z ^= z >> np.uint64(27)
            z *= _M2
            z ^= z >> np.uint64(31)
            out[c0:c1] = z
    return out


def uniform(seed, n, start=0, lo=0.0, hi=1.0):
    """U[lo, hi): lo + (hi - lo) * ((x >> 11) * 2^-53), elementwise."""
    out = np.empty(n, dtype=np.float64)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        u = (splitmix64(seed, c1 - c0, start + c0) >> np.uint64(11)).astype(np.float64)
        u *= 2.0 ** -53
        if lo != 0.0 or hi != 1.0:
            u *= (hi - lo)
            u += lo
        out[c0:c1] = u
    return out


def normal(seed, n, start=0):
    """Standard normal deviates by Box-Muller from pairs of uniforms
    (u1 in (0, 1] as 1 - U, u2 in [0, 1)): sqrt(-2 ln u1) cos(2 pi u2)."""
    u = uniform(seed, 2 * n, 2 * start)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------
# Workload recipes (sizes and value distributions of the stencil runs)
# --------------------------------------------------------------------------

def heat1d_input(n=1 << 20, seed=1, mode=3, noise=1e-3):
    """Periodic grid x_j = j/n; u0 = sin(2 pi mode x_j) + U[-noise, noise)."""
    x = np.arange(n, dtype=np.float64) / n
    u = np.sin(2.0 * math.pi * mode * x)
    if noise:
        u += uniform(seed, n, lo=-noise, hi=noise)
    return u


def bumps2d(ny, nx, seed=2, nbumps=16, sigma=0.02):
    """Sum of `nbumps` unit Gaussians of width sigma on the Dirichlet grid
    x_j = (j+1)/(nx+1), y_i = (i+1)/(ny+1); centres U[0,1]^2 drawn as
    (cx_b, cy_b) = (U_{2b}, U_{2b+1}).  Each bump is evaluated in separable
    form exp(-(x-cx)^2/(2 s^2)) * exp(-(y-cy)^2/(2 s^2))."""
    cen = uniform(seed, 2 * nbumps)
    x = (np.arange(nx, dtype=np.float64) + 1.0) / (nx + 1)
    y = (np.arange(ny, dtype=np.float64) + 1.0) / (ny + 1)
    u = np.zeros((ny, nx), dtype=np.float64)
    two_s2 = 2.0 * sigma * sigma
    for b in range(nbumps):
        ex = np.exp(-((x - cen[2 * b]) ** 2) / two_s2)
        ey = np.exp(-((y - cen[2 * b + 1]) ** 2) / two_s2)
        rows = np.nonzero(ey)[0]
        if rows.size:
            u[rows] += ey[rows, None] * ex[None, :]
    return u


def heat3d_input(n=512, seed=3, passes=3, nz=None, ny=None):
    """U[0,1) on an nz x ny x n periodic grid (x fastest), smoothed by `passes`
    Jacobi sweeps (each cell <- mean of its 6 periodic neighbours) in FP64,
    then rounded to FP32."""
    nz = n if nz is None else nz
    ny = n if ny is None else ny
    u = uniform(seed, nz * ny * n).reshape(nz, ny, n)
    for _ in range(passes):
        v = np.roll(u, 1, 2)
        v += np.roll(u, -1, 2)
        v += np.roll(u, 1, 1)
        v += np.roll(u, -1, 1)
        v += np.roll(u, 1, 0)
        v += np.roll(u, -1, 0)
        v /= 6.0
        u = v
    return u.astype(np.float32)


def batch_sides(nprob=4096, seed=4, smin=32, smax=1024):
    """Side lengths s_p = clamp(round(exp(U(ln smin, ln smax))), smin, smax)."""
    u = uniform(seed, nprob)
    s = np.rint(np.exp(math.log(smin) + u * (math.log(smax) - math.log(smin))))
    return np.clip(s, smin, smax).astype(np.int64)


def batch_input(nprob=4096, seed=4, smin=32, smax=1024, sides=None):
    """Batch of independent square problems packed back to back (problem p is
    row-major s_p x s_p starting at offset[p]).  kappa ~ U[0.5, 1.5) from
    stream seed*10+1 and u0 ~ U[0, 1) from stream seed*10+2, both indexed by
    the packed position; c_p = 0.9 / (4 max kappa_p) (0.9 of the explicit
    stability limit).  Returns (sides, offsets, kappa, u0, c)."""
    if sides is None:
        sides = batch_sides(nprob, seed, smin, smax)
    sides = np.asarray(sides, dtype=np.int64)
    offsets = np.zeros(sides.size, dtype=np.int64)
    offsets[1:] = np.cumsum(sides * sides)[:-1]
    total = int(np.sum(sides * sides))
    kappa = uniform(seed * 10 + 1, total, lo=0.5, hi=1.5)
    u0 = uniform(seed * 10 + 2, total)
    c = np.empty(sides.size, dtype=np.float64)
    for p in range(sides.size):
        o, m = offsets[p], sides[p] * sides[p]
        c[p] = 0.9 / (4.0 * float(kappa[o:o + m].max()))
    return sides, offsets, kappa, u0, c


def adjoint_input(n=2048, seeds=(5, 6, 7), c=0.15):
    """kappa_ref ~ U[0.5,1.5) (seeds[0]), kappa ~ U[0.5,1.5) (seeds[1]) and
    u0 = 16 Gaussian bumps of width 0.02 (seeds[2]) on an n x n Dirichlet grid;
    c = 0.15 = 0.9 / (4 * 1.5), fixed.  Returns (kappa_ref, kappa, u0, c)."""
    kref = uniform(seeds[0], n * n, lo=0.5, hi=1.5).reshape(n, n)
    kap = uniform(seeds[1], n * n, lo=0.5, hi=1.5).reshape(n, n)
    u0 = bumps2d(n, n, seed=seeds[2])
    return kref, kap, u0, c


def fd_direction(k, n_kappa, n_u0, seed=8):
    """Direction k (k = 0, 1, ...) of the finite-difference check: a Gaussian
    vector over the joint (dkappa, du0), drawn from position k (n_kappa + n_u0)
    of the stream and normalised to unit 2-norm, so that one full-size
    direction at a time can be generated.  Returns (dk, du)."""
    m = n_kappa + n_u0
    d = normal(seed, m, start=k * m)
    d /= np.linalg.norm(d)
    return d[:n_kappa], d[n_kappa:]


def fd_directions(ndir, n_kappa, n_u0, seed=8):
    """Directions 0 .. ndir-1 of fd_direction stacked.
    Returns (dk [ndir, n_kappa], du [ndir, n_u0])."""
    rows = [fd_direction(k, n_kappa, n_u0, seed) for k in range(ndir)]
    return np.stack([r[0] for r in rows]), np.stack([r[1] for r in rows])


def partition_sizes(ms=range(1, 9), block=256, parts=4):
    """Vector lengths of the partition benchmark: n = 2^m * 1024 * block * parts."""
    return [(1 << m) * 1024 * block * parts for m in ms]


def partition_input(n, out=None):
    """The partition benchmark's vector: x_i = i (the kernel's argument is the
    element's index).  Filled into `out` (e.g. a page-locked array) if given."""
    if out is None:
        out = np.empty(n, dtype=np.float64)
    out[:] = np.arange(n, dtype=np.float64)
    return out
