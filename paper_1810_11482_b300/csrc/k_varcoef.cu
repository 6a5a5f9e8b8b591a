// Variable-diffusivity 2D FTCS (conservative flux form) and its adjoint.
//
// Method: u'_a = u_a + c * sum_{f in W,E,N,S} k_f (u_b - u_a) with face
// conductance k_f = (kappa_a + kappa_b) / 2, Dirichlet-zero ghosts whose
// diffusivity equals the facing interior cell (k_f = kappa_a on a boundary
// face).  Algebraically u' = m_a u_a + sum_f w_f u_b with w_f = c k_f and
// m_a = 1 - sum_f w_f (boundary faces included in m, their u_b = 0), which
// is how the kernels evaluate it: the coefficients are computed once per
// problem and every step costs 5 FP64 operations.
//
// Canonical coefficients (bit-identical wherever computed):
//   h = 0.5 * kappa;  k_E = h_a + h_{a+1} (interior) or kappa_a (boundary)
//   w_f = c * k_f;    m = 1 - ((w_W + w_E) + (w_N + w_S))
//   stored: wE[a] = w_E (0 on the east boundary), wS[a] = w_S (0 on the south
//   boundary), m[a]; the west/north weights of a are wE[a-1] / wS[a-nx].
// Canonical step (also the adjoint step: the step matrix is symmetric):
//   u' = fma(wE, uE, fma(wW, uW, fma(wN, uN, fma(wS, uS, m * u))))
// (products and differences issued as fused multiply-adds that round
// identically, see Fk below).
// with zero neighbours (and zero weights) outside the field.
// Canonical kappa-gradient, dL/dkappa_a = sum_n sum_f dk_f/dkappa_a *
// c (u_b - u_a)(l_a - l_b) with u = u^n, l = lambda^{n+1} (u_b = l_b = 0
// outside; dk_f/dkappa_a = 1/2 on an interior face, 1 on a boundary face).
// The face product p_f = (u_b - u_a)(l_a - l_b) is the same seen from either
// cell of the face, so it is formed once per face and step and summed over
// the steps per face:
//   GE[a] += p(a, east face), GS[a] += p(a, south face)   (every cell; the
//     east/south face of the last column/row is a boundary face, ghost 0),
//   GW0[i] += p((i,0), west face), GN0[j] += p((0,j), north face),
// each as fma(fma(u_a, -1, u_b), fma(l_b, -1, l_a), G).  After the last step
//   gk_a = (c/2) * ((W + E) + (N + S)),
// E = GE[a] (x2 on the east boundary), W = GE[a-1] (x2 GW0[i] on the west
// boundary), S = GS[a] (x2 on the south boundary), N = GS[a-nx] (x2 GN0[j]
// on the north boundary).  Per cell and step: 6 FP64 operations.
#include "kernels.cuh"
#include "pdl.cuh"
#include "tune.hpp"

#include <algorithm>

namespace hxc {
namespace k {

struct VcCoef {
    double wE, wS, m;
};

__device__ __forceinline__ VcCoef vc_coef_at(const double *__restrict__ kap, double c, int64_t ny,
                                            int64_t nx, int64_t i, int64_t j) {
    const int64_t a = i * nx + j;
    const double ka = __ldg(kap + a);
    const double ha = __dmul_rn(0.5, ka);
    const double kW = j > 0 ? __dadd_rn(ha, __dmul_rn(0.5, __ldg(kap + a - 1))) : ka;
    const double kE = j + 1 < nx ? __dadd_rn(ha, __dmul_rn(0.5, __ldg(kap + a + 1))) : ka;
    const double kN = i > 0 ? __dadd_rn(ha, __dmul_rn(0.5, __ldg(kap + a - nx))) : ka;
    const double kS = i + 1 < ny ? __dadd_rn(ha, __dmul_rn(0.5, __ldg(kap + a + nx))) : ka;
    const double wW = __dmul_rn(c, kW), wE = __dmul_rn(c, kE), wN = __dmul_rn(c, kN),
                 wS = __dmul_rn(c, kS);
    VcCoef r;
    r.m = __dsub_rn(1.0, __dadd_rn(__dadd_rn(wW, wE), __dadd_rn(wN, wS)));
    r.wE = j + 1 < nx ? wE : 0.0;
    r.wS = i + 1 < ny ? wS : 0.0;
    return r;
}

// Run-time constants (kernel arguments, so that the compiler cannot fold
// them): products and differences are issued as fused multiply-adds, which
// round identically -- fma(a, b, -0) == a*b, fma(b, -1, a) == a - b -- but
// issue faster than DMUL/DADD on B300.
struct Fk {
    double nz;    // -0.0
    double mone;  // -1.0
};

__device__ __forceinline__ double vc_update(double u, double uW, double uE, double uN, double uS,
                                            double wW, double wE, double wN, double wS, double m,
                                            Fk f) {
    return __fma_rn(wE, uE, __fma_rn(wW, uW, __fma_rn(wN, uN, __fma_rn(wS, uS, __fma_rn(m, u, f.nz)))));
}

// One step of one problem at cell (i, j) with stored coefficients.
__device__ __forceinline__ double vc_step_at(const double *__restrict__ u,
                                             const double *__restrict__ wE,
                                             const double *__restrict__ wS,
                                             const double *__restrict__ m, int64_t ny, int64_t nx,
                                             int64_t i, int64_t j, Fk f) {
    const int64_t a = i * nx + j;
    const double uW = j > 0 ? u[a - 1] : 0.0, uE = j + 1 < nx ? u[a + 1] : 0.0;
    const double uN = i > 0 ? u[a - nx] : 0.0, uS = i + 1 < ny ? u[a + nx] : 0.0;
    const double wW = j > 0 ? wE[a - 1] : 0.0, wN = i > 0 ? wS[a - nx] : 0.0;
    return vc_update(u[a], uW, uE, uN, uS, wW, wE[a], wN, wS[a], m[a], f);
}

// ------------------------------------------------------------ one problem
__global__ void k_vc_coef(const double *__restrict__ kap, double c, int64_t ny, int64_t nx,
                          double *__restrict__ wE, double *__restrict__ wS, double *__restrict__ m) {
    const int64_t n = ny * nx;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x) {
        const VcCoef q = vc_coef_at(kap, c, ny, nx, a / nx, a % nx);
        wE[a] = q.wE;
        wS[a] = q.wS;
        m[a] = q.m;
    }
}

__global__ void k_vc_step(const double *__restrict__ u, double *__restrict__ un,
                          const double *__restrict__ wE, const double *__restrict__ wS,
                          const double *__restrict__ m, int64_t ny, int64_t nx, Fk f) {
    pdl_prologue();
    // warps walk rows: lanes cover consecutive columns (coalesced)
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t segs = (nx + 31) / 32;
    for (int64_t w = blockIdx.x * wpb + (threadIdx.x >> 5); w < ny * segs;
         w += (int64_t)gridDim.x * wpb) {
        const int64_t i = w / segs, j = (w % segs) * 32 + lane;
        if (j < nx) un[i * nx + j] = vc_step_at(u, wE, wS, m, ny, nx, i, j, f);
    }
}

// The same step with two adjacent cells per thread (even nx): 16-byte loads
// of u, its north/south rows and the coefficients halve the load
// instructions; warps walk rows, a lane covering columns 2l, 2l+1 of a
// 64-column segment.  Same canonical update as vc_step_at.
__global__ void k_vc_step2(const double *__restrict__ u, double *__restrict__ un,
                           const double *__restrict__ wE, const double *__restrict__ wS,
                           const double *__restrict__ m, int64_t ny, int64_t nx, Fk f) {
    pdl_prologue();
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t segs = (nx + 63) / 64;
    const double2 z2 = make_double2(0.0, 0.0);
    for (int64_t w = blockIdx.x * wpb + (threadIdx.x >> 5); w < ny * segs;
         w += (int64_t)gridDim.x * wpb) {
        const int64_t i = w / segs, j = (w % segs) * 64 + 2 * lane;
        if (j >= nx) continue;
        const int64_t a = i * nx + j;
        const double2 c = __ldg(reinterpret_cast<const double2 *>(u + a));
        const double2 no = i > 0 ? __ldg(reinterpret_cast<const double2 *>(u + a - nx)) : z2;
        const double2 so = i + 1 < ny ? __ldg(reinterpret_cast<const double2 *>(u + a + nx)) : z2;
        const double uw = j > 0 ? __ldg(u + a - 1) : 0.0;
        const double ue = j + 2 < nx ? __ldg(u + a + 2) : 0.0;
        const double2 e = __ldg(reinterpret_cast<const double2 *>(wE + a));
        const double ww = j > 0 ? __ldg(wE + a - 1) : 0.0;
        const double2 ss = __ldg(reinterpret_cast<const double2 *>(wS + a));
        const double2 sn = i > 0 ? __ldg(reinterpret_cast<const double2 *>(wS + a - nx)) : z2;
        const double2 mm = __ldg(reinterpret_cast<const double2 *>(m + a));
        double2 o;
        o.x = vc_update(c.x, uw, c.y, no.x, so.x, ww, e.x, sn.x, ss.x, mm.x, f);
        o.y = vc_update(c.y, c.x, ue, no.y, so.y, e.x, e.y, sn.y, ss.y, mm.y, f);
        *reinterpret_cast<double2 *>(un + a) = o;
    }
}

// Coefficients computed on the fly (the hxc_launch kernel): same bits.
__global__ void k_vc_step_otf(const double *__restrict__ u, double *__restrict__ un,
                              const double *__restrict__ kap, double c, int64_t ny, int64_t nx,
                              Fk f) {
    const int64_t n = ny * nx;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = a / nx, j = a % nx;
        const VcCoef q = vc_coef_at(kap, c, ny, nx, i, j);
        const double wW = j > 0 ? vc_coef_at(kap, c, ny, nx, i, j - 1).wE : 0.0;
        const double wN = i > 0 ? vc_coef_at(kap, c, ny, nx, i - 1, j).wS : 0.0;
        const double uW = j > 0 ? u[a - 1] : 0.0, uE = j + 1 < nx ? u[a + 1] : 0.0;
        const double uN = i > 0 ? u[a - nx] : 0.0, uS = i + 1 < ny ? u[a + nx] : 0.0;
        un[a] = vc_update(u[a], uW, uE, uN, uS, wW, q.wE, wN, q.wS, q.m, f);
    }
}

// Face product (u_b - u_a)(l_a - l_b) accumulated into g (see above).
__device__ __forceinline__ double face_acc(double ua, double la, double ub, double lb, double g,
                                           Fk f) {
    return __fma_rn(__fma_rn(ua, f.mone, ub), __fma_rn(lb, f.mone, la), g);
}

// Face-sum arrays of the kappa-gradient: GE (n), GS (n), GW0 (ny), GN0 (nx).
struct FaceSums {
    double *GE, *GS, *GW0, *GN0;
};

__device__ __forceinline__ FaceSums face_sums(double *face, int64_t ny, int64_t nx) {
    const int64_t n = ny * nx;
    return FaceSums{face, face + n, face + 2 * n, face + 2 * n + ny};
}

// Per-face kappa-gradient accumulation of one step at cell (i, j): its east
// and south faces.
__device__ __forceinline__ void vc_face_step(const double *__restrict__ u,
                                             const double *__restrict__ lam, FaceSums g,
                                             int64_t ny, int64_t nx, int64_t i, int64_t j, Fk f) {
    const int64_t a = i * nx + j;
    const double ua = u[a], la = lam[a];
    const bool e = j + 1 < nx, so = i + 1 < ny;
    const double uE = e ? u[a + 1] : 0.0, lE = e ? lam[a + 1] : 0.0;
    const double uS = so ? u[a + nx] : 0.0, lS = so ? lam[a + nx] : 0.0;
    g.GE[a] = face_acc(ua, la, uE, lE, g.GE[a], f);
    g.GS[a] = face_acc(ua, la, uS, lS, g.GS[a], f);
}

// The west boundary face of a cell of column 0 and the north boundary face
// of a cell of row 0.  Kept out of line and entered only by the warps that
// hold such cells: inlined, the compiler predicates it into every warp,
// where its FP64 operations still take the (narrow) FP64 pipe's cycles.
__device__ __noinline__ void vc_face_edges(const double *__restrict__ u,
                                           const double *__restrict__ lam, FaceSums g,
                                           int64_t nx, int64_t i, int64_t j, Fk f) {
    const int64_t a = i * nx + j;
    const double ua = u[a], la = lam[a];
    if (j == 0) g.GW0[i] = face_acc(ua, la, 0.0, 0.0, g.GW0[i], f);
    if (i == 0) g.GN0[j] = face_acc(ua, la, 0.0, 0.0, g.GN0[j], f);
}

// Adjoint step fused with the per-face kappa-gradient accumulation (either
// part can be switched off to launch them separately).
__global__ void k_vc_adjoint(const double *__restrict__ lam, double *__restrict__ lam_out,
                             const double *__restrict__ u, const double *__restrict__ wE,
                             const double *__restrict__ wS, const double *__restrict__ m,
                             double *face, int64_t ny, int64_t nx, int do_lam, int do_grad,
                             Fk f) {
    pdl_prologue();
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t segs = (nx + 31) / 32;
    const FaceSums g = face_sums(face, ny, nx);
    for (int64_t w = blockIdx.x * wpb + (threadIdx.x >> 5); w < ny * segs;
         w += (int64_t)gridDim.x * wpb) {
        const int64_t i = w / segs, seg = w % segs, j = seg * 32 + lane;
        if (j >= nx) continue;
        if (do_lam) lam_out[i * nx + j] = vc_step_at(lam, wE, wS, m, ny, nx, i, j, f);
        if (do_grad) {
            vc_face_step(u, lam, g, ny, nx, i, j, f);
            if (seg == 0 || i == 0) vc_face_edges(u, lam, g, nx, i, j, f);  // warp-uniform
        }
    }
}

// gk from the face sums after the last step (see above).
__global__ void k_vc_face_combine(const double *face, double *__restrict__ gk, double ch,
                                  int64_t ny, int64_t nx) {
    const int64_t n = ny * nx;
    const FaceSums g = face_sums(const_cast<double *>(face), ny, nx);
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = a / nx, j = a % nx;
        const double E = j + 1 < nx ? g.GE[a] : __dmul_rn(2.0, g.GE[a]);
        const double W = j > 0 ? g.GE[a - 1] : __dmul_rn(2.0, g.GW0[i]);
        const double S = i + 1 < ny ? g.GS[a] : __dmul_rn(2.0, g.GS[a]);
        const double N = i > 0 ? g.GS[a - nx] : __dmul_rn(2.0, g.GN0[j]);
        gk[a] = __dmul_rn(ch, __dadd_rn(__dadd_rn(W, E), __dadd_rn(N, S)));
    }
}

// Adjoint step with on-the-fly coefficients (the hxc_launch kernel): one
// step's face products, doubled on boundary faces, combined and accumulated
// per step, gk_a = fma(c/2, (W + E) + (N + S), gk_a) -- from gk = 0 the same
// bits as a one-step adjoint run.
__global__ void k_vc_adjoint_otf(const double *__restrict__ lam, double *__restrict__ lam_out,
                                 const double *__restrict__ u, const double *__restrict__ kap,
                                 double *__restrict__ gk, double c, int64_t ny, int64_t nx,
                                 Fk f) {
    const int64_t n = ny * nx;
    const double ch = __dmul_rn(0.5, c);
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = a / nx, j = a % nx;
        const VcCoef q = vc_coef_at(kap, c, ny, nx, i, j);
        const double wW = j > 0 ? vc_coef_at(kap, c, ny, nx, i, j - 1).wE : 0.0;
        const double wN = i > 0 ? vc_coef_at(kap, c, ny, nx, i - 1, j).wS : 0.0;
        const double la = lam[a], ua = u[a];
        const double lW = j > 0 ? lam[a - 1] : 0.0, lE = j + 1 < nx ? lam[a + 1] : 0.0;
        const double lN = i > 0 ? lam[a - nx] : 0.0, lS = i + 1 < ny ? lam[a + nx] : 0.0;
        const double uW = j > 0 ? u[a - 1] : 0.0, uE = j + 1 < nx ? u[a + 1] : 0.0;
        const double uN = i > 0 ? u[a - nx] : 0.0, uS = i + 1 < ny ? u[a + nx] : 0.0;
        lam_out[a] = vc_update(la, lW, lE, lN, lS, wW, q.wE, wN, q.wS, q.m, f);
        // each face product as the face's own cells form it (the west and
        // north faces from the neighbour's side: both factors change sign,
        // the rounded product does not)
        const double pE = face_acc(ua, la, uE, lE, 0.0, f);
        const double pS = face_acc(ua, la, uS, lS, 0.0, f);
        const double pW = j > 0 ? face_acc(uW, lW, ua, la, 0.0, f) : face_acc(ua, la, 0.0, 0.0, 0.0, f);
        const double pN = i > 0 ? face_acc(uN, lN, ua, la, 0.0, f) : face_acc(ua, la, 0.0, 0.0, 0.0, f);
        const double E = j + 1 < nx ? pE : __dmul_rn(2.0, pE);
        const double W = j > 0 ? pW : __dmul_rn(2.0, pW);
        const double S = i + 1 < ny ? pS : __dmul_rn(2.0, pS);
        const double N = i > 0 ? pN : __dmul_rn(2.0, pN);
        gk[a] = __fma_rn(ch, __dadd_rn(__dadd_rn(W, E), __dadd_rn(N, S)), gk[a]);
    }
}

// Squared error and adjoint seed: lam = 2 (u - t); partial sums of (u - t)^2
// in a fixed order (grid of kSqBlocks CTAs, element k to thread k mod
// (kSqBlocks*256) accumulated in increasing k, then a fixed tree), the last
// CTA adds the partials in order and stores the loss.
constexpr int kSqBlocks = 256;
__global__ void __launch_bounds__(256) k_sqerr_seed(const double *__restrict__ u,
                                                    const double *__restrict__ t,
                                                    double *__restrict__ lam, int64_t n,
                                                    double *partials, unsigned *counter,
                                                    double *loss) {
    const int64_t stride = (int64_t)kSqBlocks * 256;
    double acc = 0.0;
    for (int64_t k = blockIdx.x * 256 + threadIdx.x; k < n; k += stride) {
        const double d = __dsub_rn(u[k], t[k]);
        if (lam) lam[k] = __dmul_rn(2.0, d);
        acc = __fma_rn(d, d, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    __shared__ double ws[8];
    __shared__ bool is_last;
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double s = __dadd_rn(__dadd_rn(__dadd_rn(ws[0], ws[1]), __dadd_rn(ws[2], ws[3])),
                                   __dadd_rn(__dadd_rn(ws[4], ws[5]), __dadd_rn(ws[6], ws[7])));
        partials[blockIdx.x] = s;
        __threadfence();
        is_last = atomicAdd(counter, 1u) == kSqBlocks - 1;
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (int q = 0; q < kSqBlocks; q++) s = __dadd_rn(s, __ldcg(partials + q));
        *loss = s;
        *counter = 0u;  // leave the scratch ready for the next launch
    }
}

// --------------------------------------------------------------- batches
// Problem descriptor of a batch (problems packed back to back).
struct VcProblem {
    int64_t off;
    int32_t side;
    int32_t pad;
    double c;
};

// Persistent batch kernel: every CTA takes whole problems from a work queue
// (largest first) and runs all `steps` steps of a problem before taking the
// next one, so the batch is a single launch with no device-wide barrier.
// The CTA computes the problem's coefficients into wE/wS/m first.  A problem
// of side <= smem_side keeps both of its fields in shared memory for all its
// steps (2 side^2 doubles of dynamic shared memory; the coefficients stay in
// global memory, where their few KB remain in L1/L2), so u is read and
// written in global memory once per run; larger problems ping-pong between u
// and tmp in global memory and an odd step count ends with a copy into u.
// Both paths evaluate the same canonical update in the same order.
// All steps of one problem with both fields in shared memory (the CTA's
// dynamic shared memory, 2 s^2 doubles).  Out of line, so that the code of
// the global-memory path of the batch kernel stays as it is without it.
__device__ __noinline__ void vc_resident_problem(double *pu, const double *pe, const double *ps,
                                                 const double *pm, int64_t s, int steps, Fk f) {
    extern __shared__ double vc_sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t n = s * s;
    double *sa = vc_sm, *sb = vc_sm + n;
    for (int64_t a = threadIdx.x; a < n; a += blockDim.x) sa[a] = pu[a];
    __syncthreads();
    for (int st = 0; st < steps; st++) {
        const double *src = (st & 1) ? sb : sa;
        double *dst = (st & 1) ? sa : sb;
        for (int64_t i = warp; i < s; i += nw)
            for (int64_t j = lane; j < s; j += 32)
                dst[i * s + j] = vc_step_at(src, pe, ps, pm, s, s, i, j, f);
        __syncthreads();
    }
    const double *fin = (steps & 1) ? sb : sa;
    for (int64_t a = threadIdx.x; a < n; a += blockDim.x) pu[a] = fin[a];
    __syncthreads();
}

__global__ void __launch_bounds__(1024) k_vc_batch(const VcProblem *__restrict__ probs, int nprob,
                                                  unsigned *queue, double *u, double *tmp,
                                                  const double *__restrict__ kap, double *wE,
                                                  double *wS, double *m, int steps, int smem_side,
                                                  Fk f) {
    __shared__ int item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) item = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int p = item;
        __syncthreads();
        if (p >= nprob) break;
        const VcProblem pr = probs[p];
        const int64_t s = pr.side, n = s * s, off = pr.off;
        double *pu = u + off, *pt = tmp + off, *pe = wE + off, *ps = wS + off, *pm = m + off;
        const double *pk = kap + off;
        for (int64_t a = threadIdx.x; a < n; a += blockDim.x) {
            const VcCoef q = vc_coef_at(pk, pr.c, s, s, a / s, a % s);
            pe[a] = q.wE;
            ps[a] = q.wS;
            pm[a] = q.m;
        }
        if (s <= smem_side) {
            vc_resident_problem(pu, pe, ps, pm, s, steps, f);
            continue;
        }
        __syncthreads();
        for (int st = 0; st < steps; st++) {
            const double *src = (st & 1) ? pt : pu;
            double *dst = (st & 1) ? pu : pt;
            for (int64_t i = warp; i < s; i += nw)
                for (int64_t j = lane; j < s; j += 32)
                    dst[i * s + j] = vc_step_at(src, pe, ps, pm, s, s, i, j, f);
            __syncthreads();
        }
        if (steps & 1) {
            for (int64_t a = threadIdx.x; a < n; a += blockDim.x) pu[a] = pt[a];
            __syncthreads();
        }
    }
}

// Batched coefficient and step kernels for the per-step schedule: the work
// is the list of rows of all problems; row r belongs to the problem whose
// row range [rows[p], rows[p+1]) contains it.
__device__ __forceinline__ int find_problem(const int64_t *__restrict__ rows, int nprob, int64_t r) {
    int lo = 0, hi = nprob;  // rows[lo] <= r < rows[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(rows + mid) <= r)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__global__ void k_vc_batch_coef(const VcProblem *__restrict__ probs, const int64_t *__restrict__ rows,
                                int nprob, const double *__restrict__ kap, double *wE, double *wS,
                                double *m) {
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5, total = rows[nprob];
    for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < total; r += (int64_t)gridDim.x * wpb) {
        const int p = find_problem(rows, nprob, r);
        const VcProblem pr = probs[p];
        const int64_t s = pr.side, i = r - rows[p];
        for (int64_t j = lane; j < s; j += 32) {
            const VcCoef q = vc_coef_at(kap + pr.off, pr.c, s, s, i, j);
            const int64_t a = pr.off + i * s + j;
            wE[a] = q.wE;
            wS[a] = q.wS;
            m[a] = q.m;
        }
    }
}

__global__ void k_vc_batch_step(const VcProblem *__restrict__ probs, const int64_t *__restrict__ rows,
                                int nprob, const double *__restrict__ u, double *__restrict__ un,
                                const double *__restrict__ wE, const double *__restrict__ wS,
                                const double *__restrict__ m, Fk f) {
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5, total = rows[nprob];
    for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < total; r += (int64_t)gridDim.x * wpb) {
        const int p = find_problem(rows, nprob, r);
        const VcProblem pr = probs[p];
        const int64_t s = pr.side, i = r - rows[p], o = pr.off;
        for (int64_t j = lane; j < s; j += 32)
            un[o + i * s + j] = vc_step_at(u + o, wE + o, wS + o, m + o, s, s, i, j, f);
    }
}

// ---------------------------------------------------------------- launchers
static const Fk kF{-0.0, -1.0};
// largest shared-memory-resident problem side (2 fields fill 226.6 KB)
constexpr int kBatchSmemMaxSide = 119;

static unsigned grid_for(int64_t work, unsigned per_block, const hxc_launch_cfg *cfg) {
    if (cfg) return cfg->grid[0] * cfg->grid[1] * cfg->grid[2];
    int64_t g = (work + per_block - 1) / per_block;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sm_count() * 16));
}

cudaError_t vc_coef(const double *kap, double c, int64_t ny, int64_t nx, double *wE, double *wS,
                    double *m, cudaStream_t s) {
    k_vc_coef<<<grid_for(ny * nx, 256, nullptr), 256, 0, s>>>(kap, c, ny, nx, wE, wS, m);
    return cudaGetLastError();
}

cudaError_t vc_step(const double *u, double *un, const double *wE, const double *wS,
                    const double *m, int64_t ny, int64_t nx, cudaStream_t s, bool pdl) {
    const bool vec = nx % 2 == 0 && reinterpret_cast<uintptr_t>(u) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(un) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(wE) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(wS) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(m) % 16 == 0;
    if (vec) {
        const int64_t work2 = ny * ((nx + 63) / 64);
        return launch_pdl(k_vc_step2, grid_for(work2, 8, nullptr), 256, s, pdl, u, un, wE, wS, m,
                          ny, nx, kF);
    }
    const int64_t work = ny * ((nx + 31) / 32);
    return launch_pdl(k_vc_step, grid_for(work, 8, nullptr), 256, s, pdl, u, un, wE, wS, m, ny, nx,
                      kF);
}

cudaError_t vc_step_otf(const double *u, double *un, const double *kap, double c, int64_t ny,
                        int64_t nx, const hxc_launch_cfg *cfg, cudaStream_t s) {
    unsigned b = cfg ? cfg->block[0] * cfg->block[1] * cfg->block[2] : 256;
    k_vc_step_otf<<<grid_for(ny * nx, b, cfg), b, 0, s>>>(u, un, kap, c, ny, nx, kF);
    return cudaGetLastError();
}

cudaError_t vc_adjoint(const double *lam, double *lam_out, const double *u, const double *wE,
                       const double *wS, const double *m, double *face, int64_t ny, int64_t nx,
                       bool do_lam, bool do_grad, cudaStream_t s, bool pdl) {
    const int64_t work = ny * ((nx + 31) / 32);
    return launch_pdl(k_vc_adjoint, grid_for(work, 8, nullptr), 256, s, pdl, lam, lam_out, u, wE,
                      wS, m, face, ny, nx, (int)do_lam, (int)do_grad, kF);
}

size_t vc_face_doubles(int64_t ny, int64_t nx) { return (size_t)(2 * ny * nx + ny + nx); }

cudaError_t vc_face_combine(const double *face, double *gk, double c, int64_t ny, int64_t nx,
                            cudaStream_t s) {
    k_vc_face_combine<<<grid_for(ny * nx, 256, nullptr), 256, 0, s>>>(face, gk, 0.5 * c, ny, nx);
    return cudaGetLastError();
}

cudaError_t vc_adjoint_otf(const double *lam, double *lam_out, const double *u, const double *kap,
                           double *gk, double c, int64_t ny, int64_t nx, const hxc_launch_cfg *cfg,
                           cudaStream_t s) {
    unsigned b = cfg ? cfg->block[0] * cfg->block[1] * cfg->block[2] : 256;
    k_vc_adjoint_otf<<<grid_for(ny * nx, b, cfg), b, 0, s>>>(lam, lam_out, u, kap, gk, c, ny, nx, kF);
    return cudaGetLastError();
}

cudaError_t sqerr_seed(const double *u, const double *t, double *lam, int64_t n, void *scratch,
                       double *loss, cudaStream_t s) {
    double *partials = static_cast<double *>(scratch);
    unsigned *counter = reinterpret_cast<unsigned *>(partials + kSqBlocks);
    k_sqerr_seed<<<kSqBlocks, 256, 0, s>>>(u, t, lam, n, partials, counter, loss);
    return cudaGetLastError();
}

size_t sqerr_scratch_bytes() { return kSqBlocks * sizeof(double) + 16; }

cudaError_t vc_batch_persistent(const void *probs, int nprob, unsigned *queue, double *u,
                                double *tmp, const double *kap, double *wE, double *wS, double *m,
                                int steps, int ctas_per_sm, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const int g = sm_count() * (ctas_per_sm > 0 ? ctas_per_sm : (int)tune::get("batch.ctas_per_sm"));
    const int b = (int)tune::get("batch.block") / 32 * 32;  // whole warps
    const int side = (int)tune::get("batch.smem_side");
    const size_t smem = (size_t)2 * side * side * sizeof(double);
    static std::atomic<uint64_t> attr{0};
    if (smem > 48 * 1024) {
        // the largest accepted side needs all of a CTA's shared memory
        e = smem_optin(k_vc_batch, 2 * kBatchSmemMaxSide * kBatchSmemMaxSide * (int)sizeof(double),
                       attr);
        if (e != cudaSuccess) return e;
    }
    k_vc_batch<<<g, b, smem, s>>>(static_cast<const VcProblem *>(probs), nprob, queue, u, tmp, kap,
                                  wE, wS, m, steps, side, kF);
    return cudaGetLastError();
}

cudaError_t vc_batch_coef(const void *probs, const int64_t *rows, int nprob, int64_t total_rows,
                          const double *kap, double *wE, double *wS, double *m, cudaStream_t s) {
    k_vc_batch_coef<<<grid_for(total_rows, 8, nullptr), 256, 0, s>>>(
        static_cast<const VcProblem *>(probs), rows, nprob, kap, wE, wS, m);
    return cudaGetLastError();
}

cudaError_t vc_batch_step(const void *probs, const int64_t *rows, int nprob, int64_t total_rows,
                          const double *u, double *un, const double *wE, const double *wS,
                          const double *m, cudaStream_t s) {
    k_vc_batch_step<<<grid_for(total_rows, 8, nullptr), 256, 0, s>>>(
        static_cast<const VcProblem *>(probs), rows, nprob, u, un, wE, wS, m, kF);
    return cudaGetLastError();
}

size_t vc_problem_bytes() { return sizeof(VcProblem); }

void vc_pack_problem(void *dst, int64_t off, int32_t side, double c) {
    VcProblem p{off, side, 0, c};
    *static_cast<VcProblem *>(dst) = p;
}

}  // namespace k
}  // namespace hxc
