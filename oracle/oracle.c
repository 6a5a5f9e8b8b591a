/*
 * Plain FP64 CPU oracle for the heat-equation hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * with the CUDA path.
 *
 * Every routine is the textbook definition written out with one loop per
 * index, separate source and destination arrays, FP64 throughout, compiled
 * with -O2 -ffp-contract=off (no fused multiply-add, no fast-math) so that
 * each arithmetic operation is one IEEE-754 double operation in source order.
 *
 * Method sources.
 *  - The paper's only stencil is the 3-point PRK stencil of Sec. 5.1.1,
 *    s(x_i) = 0.5 x_{i-1} + x_i + 0.5 x_{i+1}.  The explicit heat update
 *    u' = u + r (u_{i-1} - 2 u_i + u_{i+1}) is the forward-time
 *    centred-space (FTCS) discretisation of u_t = u_xx with r = dt/h^2; at
 *    r = 1/4 it equals one half of the PRK stencil.
 *  - 2D/3D: the same FTCS scheme with the 5- and 7-point Laplacians.
 *  - Variable diffusivity: conservative flux form, face conductance equal
 *    to the arithmetic mean of the two cell diffusivities; a Dirichlet-zero
 *    ghost takes the diffusivity of the interior cell it faces.
 *  - Adjoint: reverse-mode derivative of L = sum (u^T - u_tgt)^2 through
 *    the explicit steps, written as the transpose (scatter) of each step.
 *  - Partitioning (Algorithm 1) does not change the mathematics: the oracle
 *    works on whole domains.
 *
 *  - Mandelbrot (Sec. 5.1.3): escape-time iteration in binary32 with a
 *    fixed rounding sequence (see the routine); the only non-FP64 routine.
 *
 * Parity status: every routine here is pinned by the CPU test-suite against
 * closed forms, exact rational brute force, dense-matrix constructions or
 * (Mandelbrot) exactly known orbits and the set's area.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

static i64 wrap(i64 i, i64 n) { i64 m = i % n; return m < 0 ? m + n : m; }

/* Sec. 5.1.1: the PRK 3-point stencil s(x_i) = 0.5 x_{i-1} + x_i + 0.5 x_{i+1},
 * periodic indexing (the paper leaves the ends unstated; periodic is the
 * reading used here). */
void ora_prk_stencil(const double *x, double *s, i64 n) {
    for (i64 i = 0; i < n; i++) {
        double xl = x[wrap(i - 1, n)], xr = x[wrap(i + 1, n)];
        s[i] = 0.5 * xl + x[i] + 0.5 * xr;
    }
}

/* Listing 2 (Sec. 4.2): the sum of n unsigned integers into one result. */
uint64_t ora_sum_u32(const uint32_t *x, i64 n) {
    uint64_t acc = 0;
    for (i64 i = 0; i < n; i++) acc += x[i];
    return acc;
}

/* 1D FTCS, periodic: u'_j = u_j + r (u_{j-1} - 2 u_j + u_{j+1}). */
void ora_heat1d(const double *u0, double *out, i64 n, double r, int steps) {
    double *a = (double *)malloc(sizeof(double) * n);
    double *b = (double *)malloc(sizeof(double) * n);
    memcpy(a, u0, sizeof(double) * n);
    for (int t = 0; t < steps; t++) {
        for (i64 j = 0; j < n; j++) {
            double lap = a[wrap(j - 1, n)] - 2.0 * a[j] + a[wrap(j + 1, n)];
            b[j] = a[j] + r * lap;
        }
        double *tmp = a; a = b; b = tmp;
    }
    memcpy(out, a, sizeof(double) * n);
    free(a); free(b);
}

/* Value of a row-major ny x nx field with a Dirichlet-zero ghost ring. */
static double at2(const double *u, i64 ny, i64 nx, i64 i, i64 j) {
    if (i < 0 || i >= ny || j < 0 || j >= nx) return 0.0;
    return u[i * nx + j];
}

/* 2D FTCS, 5-point Laplacian, Dirichlet-zero ghosts:
 * u' = u + r (u_W + u_E + u_S + u_N - 4u).  Row-major, index (i, j) = (y, x).
 * Steps caller-owned ping-pong arrays: a holds u^0 on entry, b is scratch;
 * returns the array that holds u^steps (a for an even count, else b).
 * Within a step every cell reads only the previous state, so the rows are
 * independent: the OpenMP build of this file (liboracle_omp.so) runs the
 * row loop on all threads, the serial build runs it in order, and both
 * perform exactly the same operations on every cell. */
double *ora_heat2d_steps(double *a, double *b, i64 ny, i64 nx, double r, int steps) {
    for (int t = 0; t < steps; t++) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (i64 i = 0; i < ny; i++)
            for (i64 j = 0; j < nx; j++) {
                double c = a[i * nx + j];
                double lap = at2(a, ny, nx, i, j - 1) + at2(a, ny, nx, i, j + 1)
                           + at2(a, ny, nx, i - 1, j) + at2(a, ny, nx, i + 1, j)
                           - 4.0 * c;
                b[i * nx + j] = c + r * lap;
            }
        double *tmp = a; a = b; b = tmp;
    }
    return a;
}

/* The same run on a copy: out = u^steps from u0 (u0 is not modified). */
void ora_heat2d(const double *u0, double *out, i64 ny, i64 nx, double r, int steps) {
    i64 n = ny * nx;
    double *a = (double *)malloc(sizeof(double) * n);
    double *b = (double *)malloc(sizeof(double) * n);
    memcpy(a, u0, sizeof(double) * n);
    double *res = ora_heat2d_steps(a, b, ny, nx, r, steps);
    memcpy(out, res, sizeof(double) * n);
    free(a); free(b);
}

/* Number of threads the row loop of ora_heat2d_steps uses (1 in the serial
 * build). */
int ora_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* 2D FTCS restricted to a window of a larger domain.  The window
 * [wy0, wy0+wny) x [wx0, wx0+wnx) is cut out of the full ny x nx field u0 and
 * stepped with zero outside the window; ghosts of the true domain are zero
 * as in ora_heat2d.  A cell at distance >= steps from every window edge that
 * is not a domain edge is exact (each step widens the dependence cone by one
 * cell), which lets full-size runs be checked on samples. */
void ora_heat2d_window(const double *u0, double *out, i64 ny, i64 nx,
                       i64 wy0, i64 wx0, i64 wny, i64 wnx, double r, int steps) {
    double *w = (double *)malloc(sizeof(double) * wny * wnx);
    for (i64 i = 0; i < wny; i++)
        for (i64 j = 0; j < wnx; j++)
            w[i * wnx + j] = at2(u0, ny, nx, wy0 + i, wx0 + j);
    ora_heat2d(w, out, wny, wnx, r, steps);
    free(w);
}

/* Per-tile L2 norm sqrt(sum u^2) of a row-major ny x nx field cut into
 * tiles of ty x tx (tile (p, q) covers rows p*ty.. and columns q*tx..),
 * accumulated in long double.  norms has (ny/ty) * (nx/tx) entries,
 * tile-row-major. */
void ora_tile_norms(const double *u, i64 ny, i64 nx, i64 ty, i64 tx, double *norms) {
    i64 py = ny / ty, px = nx / tx;
    for (i64 p = 0; p < py; p++)
        for (i64 q = 0; q < px; q++) {
            long double acc = 0.0L;
            for (i64 i = p * ty; i < (p + 1) * ty; i++)
                for (i64 j = q * tx; j < (q + 1) * tx; j++) {
                    long double v = (long double)u[i * nx + j];
                    acc += v * v;
                }
            norms[p * px + q] = (double)sqrtl(acc);
        }
}

/* 3D FTCS, 7-point Laplacian, periodic in all three directions, FP64.
 * Layout x fastest: index (k, i, j) = (z, y, x) -> (k*ny + i)*nx + j.
 * Steps caller-owned ping-pong arrays like ora_heat2d_steps (a holds u^0;
 * returns the array holding u^steps); the planes of a step are independent,
 * so the OpenMP build runs the plane loop on all threads with the same
 * operations on every cell. */
double *ora_heat3d_steps(double *a, double *b, i64 nz, i64 ny, i64 nx, double r, int steps) {
#define IDX3(k, i, j) ((wrap((k), nz) * ny + wrap((i), ny)) * nx + wrap((j), nx))
    for (int t = 0; t < steps; t++) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (i64 k = 0; k < nz; k++)
            for (i64 i = 0; i < ny; i++)
                for (i64 j = 0; j < nx; j++) {
                    double c = a[IDX3(k, i, j)];
                    double lap = a[IDX3(k, i, j - 1)] + a[IDX3(k, i, j + 1)]
                               + a[IDX3(k, i - 1, j)] + a[IDX3(k, i + 1, j)]
                               + a[IDX3(k - 1, i, j)] + a[IDX3(k + 1, i, j)]
                               - 6.0 * c;
                    b[IDX3(k, i, j)] = c + r * lap;
                }
        double *tmp = a; a = b; b = tmp;
    }
#undef IDX3
    return a;
}

void ora_heat3d(const double *u0, double *out, i64 nz, i64 ny, i64 nx, double r, int steps) {
    i64 n = nz * ny * nx;
    double *a = (double *)malloc(sizeof(double) * n);
    double *b = (double *)malloc(sizeof(double) * n);
    memcpy(a, u0, sizeof(double) * n);
    double *res = ora_heat3d_steps(a, b, nz, ny, nx, r, steps);
    memcpy(out, res, sizeof(double) * n);
    free(a); free(b);
}

/* Face conductance between cell a and its neighbour b: the arithmetic mean
 * of their diffusivities.  Across the Dirichlet boundary the ghost takes the
 * interior cell's diffusivity, so the face value is kappa_a. */
static double face_k(const double *kap, i64 ny, i64 nx, i64 i, i64 j, i64 i2, i64 j2) {
    double ka = kap[i * nx + j];
    if (i2 < 0 || i2 >= ny || j2 < 0 || j2 >= nx) return ka;
    return 0.5 * (ka + kap[i2 * nx + j2]);
}

/* One variable-diffusivity FTCS step (conservative flux form):
 * u'_a = u_a + c * sum_{f in W,E,S,N} k_f (u_b - u_a), Dirichlet-zero ghosts. */
static void varcoef_step(const double *a, double *b, const double *kap, i64 ny, i64 nx, double c) {
    static const int di[4] = {0, 0, -1, 1}, dj[4] = {-1, 1, 0, 0};
    for (i64 i = 0; i < ny; i++)
        for (i64 j = 0; j < nx; j++) {
            double ua = a[i * nx + j], flux = 0.0;
            for (int f = 0; f < 4; f++) {
                i64 i2 = i + di[f], j2 = j + dj[f];
                double kf = face_k(kap, ny, nx, i, j, i2, j2);
                flux += kf * (at2(a, ny, nx, i2, j2) - ua);
            }
            b[i * nx + j] = ua + c * flux;
        }
}

void ora_varcoef2d(const double *u0, const double *kap, double *out, i64 ny, i64 nx,
                   double c, int steps) {
    i64 n = ny * nx;
    double *a = (double *)malloc(sizeof(double) * n);
    double *b = (double *)malloc(sizeof(double) * n);
    memcpy(a, u0, sizeof(double) * n);
    for (int t = 0; t < steps; t++) {
        varcoef_step(a, b, kap, ny, nx, c);
        double *tmp = a; a = b; b = tmp;
    }
    memcpy(out, a, sizeof(double) * n);
    free(a); free(b);
}

/* Transpose of one variable-diffusivity step applied to lam (scatter form:
 * every contribution of the forward step is sent back along its own edge,
 * so the symmetry of the step matrix is not assumed). */
static void varcoef_step_transpose(const double *lam, double *out, const double *kap,
                                   i64 ny, i64 nx, double c) {
    static const int di[4] = {0, 0, -1, 1}, dj[4] = {-1, 1, 0, 0};
    i64 n = ny * nx;
    for (i64 q = 0; q < n; q++) out[q] = 0.0;
    for (i64 i = 0; i < ny; i++)
        for (i64 j = 0; j < nx; j++) {
            double la = lam[i * nx + j];
            /* forward: b_a = u_a + c sum_f k_f u_b - c (sum_f k_f) u_a */
            out[i * nx + j] += la;
            for (int f = 0; f < 4; f++) {
                i64 i2 = i + di[f], j2 = j + dj[f];
                double kf = face_k(kap, ny, nx, i, j, i2, j2);
                out[i * nx + j] -= c * kf * la;
                if (i2 >= 0 && i2 < ny && j2 >= 0 && j2 < nx)
                    out[i2 * nx + j2] += c * kf * la;
            }
        }
}

/* Gradient contribution of one step to dL/dkappa, given the forward state u
 * entering the step and the adjoint lam of the state leaving it.  Each face
 * f of cell a contributes c*(u_b - u_a)*lam_a to dL/dk_f; an interior face
 * conductance is 0.5*(kappa_a + kappa_b) and a boundary face is kappa_a. */
static void varcoef_kappa_grad(const double *u, const double *lam, double *gk,
                               i64 ny, i64 nx, double c) {
    static const int di[4] = {0, 0, -1, 1}, dj[4] = {-1, 1, 0, 0};
    for (i64 i = 0; i < ny; i++)
        for (i64 j = 0; j < nx; j++) {
            double ua = u[i * nx + j], la = lam[i * nx + j];
            for (int f = 0; f < 4; f++) {
                i64 i2 = i + di[f], j2 = j + dj[f];
                double dkf = c * (at2(u, ny, nx, i2, j2) - ua) * la;  /* dL/dk_f from row a */
                if (i2 >= 0 && i2 < ny && j2 >= 0 && j2 < nx) {
                    gk[i * nx + j] += 0.5 * dkf;
                    gk[i2 * nx + j2] += 0.5 * dkf;
                } else {
                    gk[i * nx + j] += dkf;
                }
            }
        }
}

/* Loss L = sum (u^T - u_tgt)^2 after `steps` variable-diffusivity steps, and
 * its gradients with respect to kappa (gk) and the initial field (gu0) by
 * reverse accumulation: lam^T = 2 (u^T - u_tgt), lam^n = A^T lam^{n+1},
 * gk += dA/dkappa contraction at every step, gu0 = lam^0.  All forward
 * states are stored.  Returns L. */
double ora_varcoef2d_adjoint(const double *u0, const double *kap, const double *utgt,
                             i64 ny, i64 nx, double c, int steps,
                             double *gk, double *gu0) {
    i64 n = ny * nx;
    double *states = (double *)malloc(sizeof(double) * n * (size_t)(steps + 1));
    memcpy(states, u0, sizeof(double) * n);
    for (int t = 0; t < steps; t++)
        varcoef_step(states + (size_t)t * n, states + (size_t)(t + 1) * n, kap, ny, nx, c);
    const double *uT = states + (size_t)steps * n;
    double loss = 0.0;
    double *lam = (double *)malloc(sizeof(double) * n);
    double *nxt = (double *)malloc(sizeof(double) * n);
    for (i64 q = 0; q < n; q++) {
        double d = uT[q] - utgt[q];
        loss += d * d;
        lam[q] = 2.0 * d;
    }
    for (i64 q = 0; q < n; q++) gk[q] = 0.0;
    for (int t = steps - 1; t >= 0; t--) {
        varcoef_kappa_grad(states + (size_t)t * n, lam, gk, ny, nx, c);
        varcoef_step_transpose(lam, nxt, kap, ny, nx, c);
        double *tmp = lam; lam = nxt; nxt = tmp;
    }
    memcpy(gu0, lam, sizeof(double) * n);
    free(states); free(lam); free(nxt);
    return loss;
}

/* Transpose step exported for the dot-product test <A x, y> = <x, A^T y>. */
void ora_varcoef2d_transpose_step(const double *lam, double *out, const double *kap,
                                  i64 ny, i64 nx, double c) {
    varcoef_step_transpose(lam, out, kap, ny, nx, c);
}

/* A batch of independent variable-diffusivity problems (square sides
 * side[p], packed one after another, problem p starting at offset[p]),
 * each stepped `steps` times with its own c[p].  The oracle simply loops;
 * the problems share nothing, so the OpenMP build hands them to its threads
 * (each problem computed by one thread, exactly as in the serial loop). */
void ora_varcoef2d_batch(const double *u0, const double *kap, double *out,
                         const i64 *side, const i64 *offset, const double *c,
                         i64 nprob, int steps) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (i64 p = 0; p < nprob; p++)
        ora_varcoef2d(u0 + offset[p], kap + offset[p], out + offset[p],
                      side[p], side[p], c[p], steps);
}

/* ------------------------------------------------------------------------
 * Sec. 5.1.3 Mandelbrot set, escape-time form, in binary32 (the paper does
 * not fix the precision; this reading takes single precision and this
 * exact rounding sequence, which the device kernel follows too).
 *   z_0 = 0;  for k = 0, 1, ..., max_iter-1:
 *       if |z_k|^2 > 4 the count is k;  z_{k+1} = z_k^2 + c.
 *   The count is max_iter if no z_k escapes (c taken as a member).
 * One iteration, with x = Re z, y = Im z, each operation rounded to float:
 *   xx = x*x, yy = y*y, escape test xx + yy > 4,
 *   Im z' = fma(x + x, y, Im c)   (2xy + Im c, one rounding; x + x is exact),
 *   Re z' = (xx - yy) + Re c.
 * Pixel (i, j) of a width x height image is c = (x0 + i*dx) + (y0 + j*dy) i,
 * each product and sum rounded to float.
 * Colour: members black; otherwise (R, G, B) = (9k, 5k, 13k) mod 256.
 * ---------------------------------------------------------------------- */
static int32_t mandel_count(float cr, float ci, int32_t max_iter) {
    float x = 0.0f, y = 0.0f;
    for (int32_t k = 0; k < max_iter; k++) {
        float xx = x * x, yy = y * y;
        if (xx + yy > 4.0f) return k;
        float ny = fmaf(x + x, y, ci);
        x = (xx - yy) + cr;
        y = ny;
    }
    return max_iter;
}

void ora_mandelbrot_counts(const float *cr, const float *ci, int32_t *cnt, i64 n,
                           int32_t max_iter) {
    for (i64 p = 0; p < n; p++) cnt[p] = mandel_count(cr[p], ci[p], max_iter);
}

void ora_mandelbrot_image(uint8_t *rgb, int32_t *cnt, i64 width, i64 height, float x0,
                          float y0, float dx, float dy, int32_t max_iter) {
    for (i64 j = 0; j < height; j++) {
        float ci = y0 + (float)j * dy;
        for (i64 i = 0; i < width; i++) {
            float cr = x0 + (float)i * dx;
            int32_t k = mandel_count(cr, ci, max_iter);
            i64 p = j * width + i;
            if (cnt) cnt[p] = k;
            uint8_t *o = rgb + 3 * p;
            if (k == max_iter) {
                o[0] = o[1] = o[2] = 0;
            } else {
                o[0] = (uint8_t)((9 * (uint32_t)k) & 255u);
                o[1] = (uint8_t)((5 * (uint32_t)k) & 255u);
                o[2] = (uint8_t)((13 * (uint32_t)k) & 255u);
            }
        }
    }
}
