"""Pins for the FP64 oracle: closed forms, exact rational brute force, dense
matrix constructions and invariants.  Nothing here is compared with the
oracle's own formula retyped; every check comes from a different route
(spectral closed form, matrix assembly, exact arithmetic, a different
differentiation mode, or an invariant of the method)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1810_11482_b300 import synth

EPS = np.finfo(np.float64).eps
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append([float(v) for v in line.split()])
    return out


# ---------------------------------------------------------------- generator

def test_splitmix64_published_vector():
    # First outputs of SplitMix64 seeded with 0 (reference implementation of
    # Steele, Lea & Flood 2014 / Vigna's splitmix64.c).
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
            0xF88BB8A8724C81EC, 0x1B39896A51A8749B]
    assert [int(v) for v in synth.splitmix64(0, 5)] == want
    # counter-based: a window of the stream equals the same slice of the whole
    full = synth.splitmix64(12345, 100)
    assert np.array_equal(synth.splitmix64(12345, 10, start=37), full[37:47])


# ---------------------------------------------------------- paper's formulas

def test_prk_stencil_golden():
    """Sec. 5.1.1 stencil against hand-evaluated values."""
    x = np.array([0, 1, 4, 9, 16, 25], dtype=np.float64)
    s = oracle.prk_stencil(x)
    for i, _, _, _, want in _rows("prk_stencil.txt"):
        assert s[int(i)] == want


def test_listing2_sum_golden():
    for n, fill, want in _rows("listing2_sum.txt"):
        x = np.full(int(n), int(fill), dtype=np.uint32)
        assert oracle.sum_u32(x) == int(want)


def test_ftcs_quarter_is_half_prk():
    """At r = 1/4 one FTCS step equals one half of the PRK stencil."""
    u = synth.heat1d_input(256, seed=11)
    a = oracle.heat1d(u, 0.25, 1)
    b = 0.5 * oracle.prk_stencil(u)
    assert np.max(np.abs(a - b)) <= 2 * EPS * np.max(np.abs(u))


# ----------------------------------------------------------------------- 1D

@pytest.mark.parametrize("n", [16, 64])
@pytest.mark.parametrize("r", [0.25, 0.2, 0.1])
def test_heat1d_fourier_decay(n, r):
    """Periodic sin/cos modes are eigenvectors: u^t = g^t u^0 with
    g = 1 - 2 r (1 - cos(2 pi m / n))."""
    j = np.arange(n)
    steps = 40
    for m in range(1, n // 2):
        for phase in (np.sin, np.cos):
            u0 = phase(2 * np.pi * m * j / n)
            g = 1.0 - 2.0 * r * (1.0 - math.cos(2 * math.pi * m / n))
            ut = oracle.heat1d(u0, r, steps)
            err = np.max(np.abs(ut - g ** steps * u0))
            assert err <= 16 * steps * EPS, (m, err)


def test_heat1d_nyquist_vanishes_exactly():
    """(-1)^j at r = 1/4 has g = 0: one step gives exact zeros."""
    u0 = np.where(np.arange(64) % 2 == 0, 1.0, -1.0)
    assert np.all(oracle.heat1d(u0, 0.25, 1) == 0.0)


def _exact_heat1d(u0, r, steps):
    n = len(u0)
    u = [Fraction(v) for v in u0]
    r = Fraction(r)
    for _ in range(steps):
        u = [u[j] + r * (u[(j - 1) % n] - 2 * u[j] + u[(j + 1) % n]) for j in range(n)]
    return u


@pytest.mark.parametrize("r", [Fraction(1, 4), Fraction(1, 5), Fraction(3, 20)])
def test_heat1d_bruteforce_rational(r):
    """Exact rational evolution of a 16-point grid (dyadic inputs are exact
    Fractions); the oracle stays within a few ulps per step."""
    u0 = synth.uniform(21, 16, lo=-1.0, hi=1.0)
    for steps in range(1, 9):
        exact = _exact_heat1d(u0, r, steps)
        got = oracle.heat1d(u0, float(r), steps)
        err = max(abs(Fraction(g) - e) for g, e in zip(got, exact))
        assert err <= 8 * steps * EPS, (steps, float(err))


def test_heat1d_conservation_and_max_principle():
    u0 = synth.heat1d_input(4096, seed=12)
    for r in (0.25, 0.5, 0.1):
        ut = oracle.heat1d(u0, r, 50)
        assert abs(math.fsum(ut) - math.fsum(u0)) <= 50 * 4096 * EPS * np.max(np.abs(u0))
        assert ut.max() <= u0.max() and ut.min() >= u0.min()


# ----------------------------------------------------------------------- 2D

def test_heat2d_dirichlet_sine_modes():
    """sin(p pi x) sin(q pi y) on the grid x_j = (j+1) h, h = 1/(n+1) decays by
    g = 1 - 4 r [sin^2(p pi h / 2) + sin^2(q pi h / 2)] per step."""
    ny, nx = 24, 17            # unequal sides catch an x/y mix-up
    steps = 30
    for r in (0.25, 0.2):
        for p, q in [(1, 1), (3, 2), (nx, 1), (5, ny)]:
            hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
            x = (np.arange(nx) + 1) * hx
            y = (np.arange(ny) + 1) * hy
            u0 = np.outer(np.sin(q * np.pi * y), np.sin(p * np.pi * x))
            g = 1.0 - 4.0 * r * (math.sin(p * math.pi * hx / 2) ** 2
                                 + math.sin(q * math.pi * hy / 2) ** 2)
            ut = oracle.heat2d(u0, r, steps)
            assert np.max(np.abs(ut - g ** steps * u0)) <= 32 * steps * EPS, (p, q)


def _dirichlet2d_matrix(ny, nx, r):
    """Dense FTCS matrix I + r (L_y (x) I + I (x) L_x), L = tridiag(1,-2,1)."""
    def lap(n):
        return -2 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    return np.eye(ny * nx) + r * (np.kron(lap(ny), np.eye(nx)) + np.kron(np.eye(ny), lap(nx)))


def test_heat2d_dense_kron_matrix():
    ny, nx, r, steps = 7, 5, 0.2, 6
    u0 = synth.uniform(31, ny * nx).reshape(ny, nx)
    A = _dirichlet2d_matrix(ny, nx, r)
    want = np.linalg.matrix_power(A, steps) @ u0.ravel()
    got = oracle.heat2d(u0, r, steps).ravel()
    assert np.max(np.abs(got - want)) <= 64 * EPS


def test_heat2d_bruteforce_rational():
    n, r, steps = 16, Fraction(1, 5), 4
    u0 = synth.uniform(32, n * n).reshape(n, n)
    u = [[Fraction(v) for v in row] for row in u0]

    def g(a, i, j):
        return a[i][j] if 0 <= i < n and 0 <= j < n else Fraction(0)

    for _ in range(steps):
        u = [[u[i][j] + r * (g(u, i, j - 1) + g(u, i, j + 1) + g(u, i - 1, j)
                             + g(u, i + 1, j) - 4 * u[i][j]) for j in range(n)]
             for i in range(n)]
    got = oracle.heat2d(u0, float(r), steps)
    err = max(abs(Fraction(got[i, j]) - u[i][j]) for i in range(n) for j in range(n))
    assert err <= 8 * steps * EPS


def test_heat2d_window_matches_full():
    u0 = synth.bumps2d(64, 48, seed=33, nbumps=4, sigma=0.1)
    steps = 5
    full = oracle.heat2d(u0, 0.2, steps)
    # interior window: exact at distance >= steps from the window edges
    w = oracle.heat2d_window(u0, 20, 10, 30, 25, 0.2, steps)
    assert np.array_equal(w[steps:-steps, steps:-steps], full[20 + steps:50 - steps, 10 + steps:35 - steps])
    # corner window: the domain edges are real edges
    w = oracle.heat2d_window(u0, 0, 0, 20, 20, 0.2, steps)
    assert np.array_equal(w[:-steps, :-steps], full[:20 - steps, :20 - steps])


@pytest.mark.parametrize("ny,nx,steps", [(1, 1, 3), (3, 500, 5), (257, 130, 6), (600, 77, 1)])
def test_heat2d_stepping_builds_agree(ny, nx, steps):
    """The caller-buffer stepping routine equals heat2d, and its OpenMP build
    (rows on all threads) equals the serial build bit for bit, on ragged
    shapes with odd and even step counts (the result may end in either
    array)."""
    u0 = synth.uniform(77 + nx, ny * nx, lo=-1.0, hi=1.0).reshape(ny, nx)
    want = oracle.heat2d(u0, 0.2, steps)
    for omp in (False, True):
        a, b = u0.copy(), np.full_like(u0, np.nan)
        got = oracle.heat2d_steps(a, b, 0.2, steps, omp=omp)
        assert got is (a if steps % 2 == 0 else b)
        assert np.array_equal(got, want), omp
    assert oracle.threads(False) == 1 and oracle.threads(True) >= 1


@pytest.mark.parametrize("shape,steps", [((1, 1, 1), 3), ((7, 3, 130), 4), ((33, 21, 40), 5)])
def test_heat3d_stepping_builds_agree(shape, steps):
    """The caller-buffer 3D stepping routine equals heat3d, and its OpenMP
    build (planes on all threads) equals the serial build bit for bit."""
    nz, ny, nx = shape
    u0 = synth.uniform(91 + nx, nz * ny * nx, lo=-1.0, hi=1.0).reshape(shape)
    want = oracle.heat3d(u0, 0.15, steps)
    for omp in (False, True):
        a, b = u0.copy(), np.full_like(u0, np.nan)
        got = oracle.heat3d_steps(a, b, 0.15, steps, omp=omp)
        assert got is (a if steps % 2 == 0 else b)
        assert np.array_equal(got, want), omp


def test_batch_builds_agree():
    """The OpenMP build of the batch (problems on all threads) equals the
    serial build bit for bit, on ragged problem sizes."""
    sides, offs, kap, u0, cs = synth.batch_input(nprob=23, seed=413, smin=1, smax=40)
    want = oracle.varcoef2d_batch(u0, kap, sides, offs, cs, 6)
    assert np.array_equal(oracle.varcoef2d_batch(u0, kap, sides, offs, cs, 6, omp=True), want)


def test_heat2d_max_principle():
    u0 = synth.bumps2d(40, 40, seed=34, nbumps=3, sigma=0.1)
    ut = oracle.heat2d(u0, 0.25, 100)
    assert ut.max() <= u0.max() and ut.min() >= 0.0


def test_tile_norms_against_fsum():
    u = synth.uniform(35, 64 * 96, lo=-1, hi=1).reshape(64, 96)
    got = oracle.tile_norms(u, 32, 32)
    assert got.shape == (2, 3)
    for p in range(2):
        for q in range(3):
            t = u[32 * p:32 * (p + 1), 32 * q:32 * (q + 1)].ravel()
            want = math.sqrt(math.fsum(float(v) * float(v) for v in t))
            assert abs(got[p, q] - want) <= 1e-14 * want
    # closed form: a constant tile of value a has norm |a| sqrt(ty tx)
    assert oracle.tile_norms(np.full((16, 16), -3.0), 16, 16)[0, 0] == 48.0


# ----------------------------------------------------------------------- 3D

def test_heat3d_product_modes():
    nz, ny, nx = 8, 6, 10
    steps, r = 20, 0.15
    k = np.arange(nz)[:, None, None]
    i = np.arange(ny)[None, :, None]
    j = np.arange(nx)[None, None, :]
    for a, b, c in [(1, 1, 1), (2, 3, 4), (4, 0, 5), (0, 2, 1)]:
        u0 = np.cos(2 * np.pi * a * k / nz) * np.sin(2 * np.pi * b * i / ny + 0.3) \
            * np.cos(2 * np.pi * c * j / nx)
        g = 1.0 - 4.0 * r * (math.sin(math.pi * a / nz) ** 2 + math.sin(math.pi * b / ny) ** 2
                             + math.sin(math.pi * c / nx) ** 2)
        ut = oracle.heat3d(u0, r, steps)
        assert np.max(np.abs(ut - g ** steps * u0)) <= 64 * steps * EPS, (a, b, c)


def test_heat3d_dense_kron_matrix_and_conservation():
    nz, ny, nx, r, steps = 5, 4, 6, 0.15, 7

    def plap(n):
        m = -2 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
        m[0, -1] += 1
        m[-1, 0] += 1
        return m
    Iz, Iy, Ix = np.eye(nz), np.eye(ny), np.eye(nx)
    L = (np.kron(np.kron(plap(nz), Iy), Ix) + np.kron(np.kron(Iz, plap(ny)), Ix)
         + np.kron(np.kron(Iz, Iy), plap(nx)))
    A = np.eye(nz * ny * nx) + r * L
    u0 = synth.uniform(41, nz * ny * nx).reshape(nz, ny, nx)
    want = np.linalg.matrix_power(A, steps) @ u0.ravel()
    got = oracle.heat3d(u0, r, steps)
    assert np.max(np.abs(got.ravel() - want)) <= 64 * EPS
    assert abs(math.fsum(got.ravel()) - math.fsum(u0.ravel())) <= steps * u0.size * EPS


def test_heat3d_input_recipe_properties():
    u = synth.heat3d_input(16, seed=42)
    assert u.dtype == np.float32 and u.shape == (16, 16, 16)
    # Jacobi smoothing preserves the mean (periodic averaging) up to rounding
    raw = synth.uniform(42, 16 ** 3)
    assert abs(float(u.astype(np.float64).mean()) - raw.mean()) < 1e-6


# ------------------------------------------------------------ variable kappa

def _varcoef_matrix_exact(kap, c):
    """Step matrix A = I - c L_k assembled from the list of faces: every
    interior face (a, b) with conductance (k_a + k_b)/2 couples a and b, and
    every boundary face of cell a removes c k_a from the diagonal (Dirichlet
    ghost of value 0 with the interior cell's diffusivity)."""
    ny, nx = len(kap), len(kap[0])
    n = ny * nx
    A = [[Fraction(0)] * n for _ in range(n)]
    for a in range(n):
        A[a][a] = Fraction(1)
    for i in range(ny):
        for j in range(nx):
            a = i * nx + j
            for di, dj in ((0, -1), (0, 1), (-1, 0), (1, 0)):
                i2, j2 = i + di, j + dj
                if 0 <= i2 < ny and 0 <= j2 < nx:
                    b = i2 * nx + j2
                    kf = (kap[i][j] + kap[i2][j2]) * Fraction(1, 2)
                    A[a][b] += c * kf
                    A[a][a] -= c * kf
                else:
                    A[a][a] -= c * kap[i][j]
    return A


def _matvec(A, x):
    return [sum(Aij * xj for Aij, xj in zip(row, x)) for row in A]


def test_varcoef_bruteforce_matrix():
    ny, nx, steps = 5, 4, 4
    kap = synth.uniform(51, ny * nx, lo=0.5, hi=1.5).reshape(ny, nx)
    c = 0.9 / (4 * kap.max())
    u0 = synth.uniform(52, ny * nx).reshape(ny, nx)
    A = _varcoef_matrix_exact([[Fraction(v) for v in row] for row in kap], Fraction(c))
    u = [Fraction(v) for v in u0.ravel()]
    for _ in range(steps):
        u = _matvec(A, u)
    got = oracle.varcoef2d(u0, kap, c, steps).ravel()
    err = max(abs(Fraction(g) - e) for g, e in zip(got, u))
    assert err <= 16 * steps * EPS


def test_varcoef_constant_kappa_is_5pt():
    u0 = synth.bumps2d(20, 30, seed=53, nbumps=3, sigma=0.1)
    kap = np.full_like(u0, 0.75)
    c = 0.2 / 0.75
    a = oracle.varcoef2d(u0, kap, c, 10)
    b = oracle.heat2d(u0, 0.75 * c, 10)
    assert np.max(np.abs(a - b)) <= 64 * EPS * np.max(np.abs(u0))


def test_varcoef_constant_field_rowsums():
    """A constant field stays exactly constant at cells with no boundary face;
    a boundary cell loses c * kappa_a * (number of its boundary faces)."""
    ny, nx = 6, 7
    kap = synth.uniform(54, ny * nx, lo=0.5, hi=1.5).reshape(ny, nx)
    c = 0.125
    u1 = oracle.varcoef2d(np.ones((ny, nx)), kap, c, 1)
    for i in range(ny):
        for j in range(nx):
            nb = (i == 0) + (i == ny - 1) + (j == 0) + (j == nx - 1)
            want = 1.0 - c * kap[i, j] * nb
            assert abs(u1[i, j] - want) <= 4 * EPS


def test_varcoef_step_symmetric_and_transpose():
    """<A x, y> = <x, A y> (the step matrix is symmetric) and the scatter-form
    transpose agrees: <A x, y> = <x, A^T y>."""
    ny, nx = 9, 11
    kap = synth.uniform(55, ny * nx, lo=0.5, hi=1.5).reshape(ny, nx)
    c = 0.9 / (4 * kap.max())
    x = synth.uniform(56, ny * nx, lo=-1, hi=1).reshape(ny, nx)
    y = synth.uniform(57, ny * nx, lo=-1, hi=1).reshape(ny, nx)
    Ax = oracle.varcoef2d(x, kap, c, 1)
    Ay = oracle.varcoef2d(y, kap, c, 1)
    ATy = oracle.varcoef2d_transpose_step(y, kap, c)
    lhs = math.fsum((Ax * y).ravel())
    assert abs(lhs - math.fsum((x * Ay).ravel())) <= 1e-13
    assert abs(lhs - math.fsum((x * ATy).ravel())) <= 1e-13
    assert np.max(np.abs(ATy - Ay)) <= 8 * EPS


def test_varcoef_max_principle():
    sides, offsets, kap, u0, c = synth.batch_input(nprob=3, seed=58, smin=8, smax=20)
    out = oracle.varcoef2d_batch(u0, kap, sides, offsets, c, 30)
    for p in range(3):
        o, m = offsets[p], sides[p] ** 2
        assert out[o:o + m].max() <= u0[o:o + m].max() and out[o:o + m].min() >= 0.0
        single = oracle.varcoef2d(u0[o:o + m].reshape(sides[p], sides[p]),
                                  kap[o:o + m].reshape(sides[p], sides[p]), c[p], 30)
        assert np.array_equal(single.ravel(), out[o:o + m])


# ------------------------------------------------------------------ adjoint

class _Dual:
    """Exact forward-mode dual number over Fractions: value + eps * deriv."""
    __slots__ = ("v", "d")

    def __init__(self, v, d=Fraction(0)):
        self.v, self.d = v, d

    def __add__(self, o):
        o = o if isinstance(o, _Dual) else _Dual(o)
        return _Dual(self.v + o.v, self.d + o.d)

    __radd__ = __add__

    def __sub__(self, o):
        o = o if isinstance(o, _Dual) else _Dual(o)
        return _Dual(self.v - o.v, self.d - o.d)

    def __rsub__(self, o):
        return _Dual(o) - self

    def __mul__(self, o):
        o = o if isinstance(o, _Dual) else _Dual(o)
        return _Dual(self.v * o.v, self.v * o.d + self.d * o.v)

    __rmul__ = __mul__


def _loss_forward_mode(u0, kap, utgt, c, steps):
    """L(u0, kappa) evaluated with the face-assembled step matrix on dual
    numbers: returns the exact dL along the seeded direction."""
    ny, nx = len(kap), len(kap[0])
    n = ny * nx
    u = list(u0)
    for _ in range(steps):
        A = _varcoef_matrix_exact(kap, c)
        u = [sum((A[a][b] * u[b] for b in range(n)), _Dual(Fraction(0))) for a in range(n)]
    L = _Dual(Fraction(0))
    for a in range(n):
        d = u[a] - utgt[a]
        L = L + d * d
    return L


def test_adjoint_against_exact_forward_mode():
    """Reverse-mode gradients equal exact forward-mode derivatives (dual
    numbers over Fractions) on a 3 x 4 grid, 3 steps."""
    ny, nx, steps = 3, 4, 3
    kap = synth.uniform(61, ny * nx, lo=0.5, hi=1.5).reshape(ny, nx)
    u0 = synth.uniform(62, ny * nx).reshape(ny, nx)
    utgt = synth.uniform(63, ny * nx).reshape(ny, nx)
    c = 0.15
    loss, gk, gu = oracle.varcoef2d_adjoint(u0, kap, utgt, c, steps)
    n = ny * nx
    tg = [Fraction(v) for v in utgt.ravel()]
    cF = Fraction(c)
    for a in range(n):
        # d/dkappa_a
        kd = [[_Dual(Fraction(kap[i, j]), Fraction(int(i * nx + j == a))) for j in range(nx)]
              for i in range(ny)]
        L = _loss_forward_mode([_Dual(Fraction(v)) for v in u0.ravel()], kd, tg, cF, steps)
        assert abs(gk.ravel()[a] - float(L.d)) <= 1e-13 * max(1.0, abs(float(L.d))), a
        # d/du0_a
        ud = [_Dual(Fraction(v), Fraction(int(b == a))) for b, v in enumerate(u0.ravel())]
        kk = [[_Dual(Fraction(kap[i, j])) for j in range(nx)] for i in range(ny)]
        L = _loss_forward_mode(ud, kk, tg, cF, steps)
        assert abs(gu.ravel()[a] - float(L.d)) <= 1e-13 * max(1.0, abs(float(L.d))), a
    assert abs(loss - float(L.v)) <= 1e-14 * max(1.0, float(L.v))


def test_adjoint_central_differences():
    n, steps, c = 24, 20, 0.15
    kref, kap, _, _ = synth.adjoint_input(n)
    u0 = synth.bumps2d(n, n, seed=7, nbumps=4, sigma=0.15)
    utgt = oracle.varcoef2d(u0, kref, c, steps)
    loss, gk, gu = oracle.varcoef2d_adjoint(u0, kap, utgt, c, steps)
    dk, du = synth.fd_directions(4, n * n, n * n, seed=8)
    for d in range(4):
        ek = 1e-4 * np.abs(kap).max()
        kp = kap + ek * dk[d].reshape(n, n)
        km = kap - ek * dk[d].reshape(n, n)
        fd = (oracle.varcoef2d_adjoint(u0, kp, utgt, c, steps)[0]
              - oracle.varcoef2d_adjoint(u0, km, utgt, c, steps)[0]) / (2 * ek)
        an = float(np.dot(gk.ravel(), dk[d]))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * np.linalg.norm(gk)), (d, fd, an)
        eu = 1e-3
        up = u0 + eu * du[d].reshape(n, n)
        um = u0 - eu * du[d].reshape(n, n)
        fd = (oracle.varcoef2d_adjoint(up, kap, utgt, c, steps)[0]
              - oracle.varcoef2d_adjoint(um, kap, utgt, c, steps)[0]) / (2 * eu)
        an = float(np.dot(gu.ravel(), du[d]))
        assert abs(fd - an) <= 1e-9 * max(abs(an), np.linalg.norm(gu)), (d, fd, an)


def test_adjoint_u0_gradient_is_forward_of_residual():
    """A is symmetric, so dL/du0 = A^T..A^T 2(u^T - u_tgt) = A^steps 2(u^T - u_tgt)."""
    n, steps, c = 12, 7, 0.15
    kap = synth.uniform(64, n * n, lo=0.5, hi=1.5).reshape(n, n)
    u0 = synth.uniform(65, n * n).reshape(n, n)
    utgt = synth.uniform(66, n * n).reshape(n, n)
    _, _, gu = oracle.varcoef2d_adjoint(u0, kap, utgt, c, steps)
    uT = oracle.varcoef2d(u0, kap, c, steps)
    want = oracle.varcoef2d(2 * (uT - utgt), kap, c, steps)
    assert np.max(np.abs(gu - want)) <= 64 * EPS * np.max(np.abs(want))


def test_partition_kernel_is_one_and_sizes():
    """Sec. 5.1.2: k(x) = sqrt(sin^2 x + cos^2 x) is identically 1 (up to the
    rounding of sin, cos, the squares, the sum and the root), and the vector
    lengths are 2^m * 1024 * 256 * 4 for m = 1..8, i.e. 2^21 .. 2^28."""
    x = np.concatenate([np.arange(4096, dtype=np.float64),
                        np.arange((1 << 28) - 4096, 1 << 28, dtype=np.float64),
                        synth.uniform(11, 4096, lo=0.0, hi=float(1 << 28)).round()])
    k = oracle.partition_k(x)
    assert np.max(np.abs(k - 1.0)) <= 4 * np.finfo(np.float64).eps
    assert k[0] == 1.0  # sin 0 = 0, cos 0 = 1 exactly
    # a sign slip (sin^2 - cos^2 = -cos 2x) or a squared-sum mix-up is far from 1
    assert np.max(np.abs(np.sqrt(np.abs(np.sin(x) ** 2 - np.cos(x) ** 2)) - 1.0)) > 0.5
    assert synth.partition_sizes() == [1 << e for e in range(21, 29)]
    assert np.array_equal(synth.partition_input(5), [0.0, 1.0, 2.0, 3.0, 4.0])


def test_mandelbrot_exact_orbits():
    """Sec. 5.1.3, points with orbits exact in binary32: 0, -1, -2, i, 1/4 and
    -3/4 stay bounded (members); c = 1 runs 0, 1, 2, 5 and escapes at k = 3;
    c = 2i runs 0, 2i, -4 + 2i and escapes at k = 2 (|2i|^2 = 4 is not > 4);
    c = 3 and c = 5/2 escape at k = 1 (z_0 = 0 is inside, z_1 = c is not)."""
    cr = [0.0, -1.0, -2.0, 0.0, 0.25, -0.75, 1.0, 0.0, 3.0, 2.5]
    ci = [0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 2.0, 0.0, 0.0]
    got = oracle.mandelbrot_counts(cr, ci, 300)
    assert got.tolist() == [300, 300, 300, 300, 300, 300, 3, 2, 1, 1]


def _exact_count(cr, ci, max_iter):
    """Escape count in exact rational arithmetic; also the smallest distance
    of |z_k|^2 from 4 seen before the decision."""
    c = (Fraction(float(cr)), Fraction(float(ci)))
    x = y = Fraction(0)
    margin = Fraction(10)
    for k in range(max_iter):
        m = x * x + y * y
        margin = min(margin, abs(m - 4))
        if m > 4:
            return k, margin
        x, y = x * x - y * y + c[0], 2 * x * y + c[1]
    return max_iter, margin


def test_mandelbrot_against_exact_arithmetic_and_symmetry():
    """Brute force: short orbits in exact rational arithmetic decide the same
    count as the binary32 oracle wherever |z_k|^2 stays clear of 4 (the
    rounding of a few float steps cannot cross the threshold there); and
    conjugate points escape together (every step is odd in Im z)."""
    cr = synth.uniform(21, 3000, lo=-2.5, hi=1.5).astype(np.float32)
    ci = synth.uniform(22, 3000, lo=-1.6, hi=1.6).astype(np.float32)
    max_iter = 6
    got = oracle.mandelbrot_counts(cr, ci, max_iter)
    checked = 0
    for a, b, g in zip(cr, ci, got):
        want, margin = _exact_count(a, b, max_iter)
        if margin > Fraction(1, 20):
            assert g == want, (a, b, g, want)
            checked += 1
    assert checked > 2000
    assert np.array_equal(oracle.mandelbrot_counts(cr, -ci, 200), oracle.mandelbrot_counts(cr, ci, 200))


def test_mandelbrot_area_and_image():
    """The members of an 800 x 800 grid over [-2, 1] x [-1.5, 1.5] (500
    iterations) cover about the set's area, 1.5066; the image colours follow
    the counts (members black, else (9k, 5k, 13k) mod 256)."""
    n, it = 800, 500
    h = np.float32(3.0 / n)
    rgb, cnt = oracle.mandelbrot_image(n, n, np.float32(-2.0), np.float32(-1.5), h, h, it)
    area = (cnt == it).mean() * 9.0
    assert abs(area - 1.5066) < 0.02
    k = cnt.astype(np.uint32)
    want = np.stack([(9 * k) & 255, (5 * k) & 255, (13 * k) & 255], axis=-1).astype(np.uint8)
    want[cnt == it] = 0
    assert np.array_equal(rgb, want)
    # pixel (i, j) is the point (x0 + i dx, y0 + j dy)
    j, i = 123, 456
    assert cnt[j, i] == oracle.mandelbrot_counts([np.float32(-2.0) + np.float32(i) * h],
                                                 [np.float32(-1.5) + np.float32(j) * h], it)[0]
