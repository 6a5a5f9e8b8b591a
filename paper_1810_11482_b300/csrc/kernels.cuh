// Launchers of the sm_103a kernels.  Arguments are raw device pointers;
// the C ABI layer validates sizes and handles before calling these.
#pragma once

#include <atomic>
#include <cstdint>

#include <cuda_runtime.h>

#include "hxc.h"

namespace hxc {
namespace k {

// Number of row bands of the tile-norm reduction; fixed so that the
// reduction order (and therefore every bit of the result) does not depend
// on how tiles are grouped into launches.
constexpr int kNormBands = 64;
// Scratch of one tile-norm launch: kNormBands partial sums + a counter.
constexpr size_t kNormScratchBytes = kNormBands * sizeof(double) + 16;

int sm_count();

// Raises `kernel`'s dynamic shared-memory limit to `bytes` once per device
// (the attribute belongs to the function as loaded on each device); `done`
// is the caller's static mask of the devices already set.
template <typename Kernel>
cudaError_t smem_optin(Kernel *kernel, int bytes, std::atomic<uint64_t> &done) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (d & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
    return e;
}

cudaError_t sum_u32(const uint32_t *in, unsigned long long *result, int64_t n,
                    const hxc_launch_cfg *cfg, cudaStream_t s);
cudaError_t prk(const double *in, double *out, int64_t n, const hxc_launch_cfg *cfg,
                cudaStream_t s);
cudaError_t partition(double *x, int64_t n, const hxc_launch_cfg *cfg, cudaStream_t s);
// Sec. 5.1.3: RGB8 image (and optional int32 escape counts) of the
// Mandelbrot set; pixel (i, j) is c = (x0 + i dx) + (y0 + j dy) i.
cudaError_t mandelbrot(uint8_t *rgb, int32_t *counts, int64_t width, int64_t height, float x0,
                       float y0, float dx, float dy, int32_t max_iter, const hxc_launch_cfg *cfg,
                       cudaStream_t s);

// Kinds of FTCS step in d dimensions (d = 1, 2).  With s the sum of the 2d
// neighbours of the values read ((uN + uW) + (uE + uS) in 2D, ul + ur in 1D):
//   kFtcsCanon  (c0 = r):             t = fma(-2d, u, s); u' = fma(r, t, u)
//   kFtcsScaled (c0 = (1 - 2d r)/r):  u' = fma(c0, u, s)
//   kFtcsClose  (c0, c1):             u' = fma(c0, s, c1 * u)
// A scaled step maps v = u_n / r^m to u_{n+1} / r^(m+1); a closing step
// with c0 = r^(m+1), c1 = (1 - 2d r) r^m maps v = u_n / r^m to u_{n+1}.
enum : int { kFtcsCanon = 0, kFtcsScaled = 1, kFtcsClose = 2 };
struct FtcsStep {
    int kind;
    double c0, c1;
};

// The step kinds of a whole run, for kernels that advance several steps per
// launch.  Run step g (0-based, of `total`) is step j = g mod I of its
// interval (I steps, the last interval shorter); an interval is cut into
// groups of P steps (the last shorter) whose last step closes; the others
// are scaled.  P = 0: every step canonical with r.  The closing step after q
// scaled steps uses a[q], b[q].
constexpr int kFtcsMaxGroup = 97;
struct FtcsPlan {
    double r, k;
    int P, I;
    int64_t total;
    double a[kFtcsMaxGroup], b[kFtcsMaxGroup];
};

#ifdef __CUDACC__
#define HXC_HD __host__ __device__
#else
#define HXC_HD
#endif
// Kind and coefficients of run step g under plan p (the one rule, for the
// host and the device).
HXC_HD inline FtcsStep ftcs_plan_step(const FtcsPlan &p, int64_t g) {
    if (p.P == 0) return {kFtcsCanon, p.r, 0.0};
    const int64_t j = g % p.I, s0 = g - j;
    const int64_t L = p.total - s0 < p.I ? p.total - s0 : (int64_t)p.I;
    const int64_t q = j % p.P, end = L < j - q + p.P ? L : j - q + p.P;
    if (j + 1 < end) return {kFtcsScaled, p.k, 0.0};
    return {kFtcsClose, p.a[q], p.b[q]};
}
#undef HXC_HD

// dst[lo, lo+count) <- `steps` periodic FTCS steps of src (period n),
// canonical arithmetic.
cudaError_t heat1d(const double *src, double *dst, int64_t n, int64_t lo, int64_t count,
                   double r, int steps, const hxc_launch_cfg *cfg, cudaStream_t s);
// The same, run steps g0 .. g0+steps-1 of a run whose kinds `plan` gives.
cudaError_t heat1d_plan(const double *src, double *dst, int64_t n, int64_t lo, int64_t count,
                        const FtcsPlan &plan, int64_t g0, int steps, const hxc_launch_cfg *cfg,
                        cudaStream_t s);
// Largest `steps` a single temporally blocked 1D launch accepts.
constexpr int kHeat1dMaxSteps = 1024;

// One 2D FTCS step of the tile [y0, y0+ty) x [x0, x0+tx); rows_per_warp <= 0
// picks the default.  Canonical arithmetic (true values in and out).
cudaError_t heat2d(const double *src, double *dst, int64_t ny, int64_t nx, int64_t y0,
                   int64_t x0, int64_t ty, int64_t tx, double r, int rows_per_warp,
                   const hxc_launch_cfg *cfg, cudaStream_t s);
// One 2D step of kind `step`; `pdl`: launched with programmatic dependent
// launch, for a launch that directly follows another step kernel on `s`.
cudaError_t heat2d_step(const double *src, double *dst, int64_t ny, int64_t nx, int64_t y0,
                        int64_t x0, int64_t ty, int64_t tx, const FtcsStep &step,
                        int rows_per_warp, cudaStream_t s, bool pdl = false);

// 2D kernel knobs (tuning registry): share of the additions run on the
// integer pipe (half-additions per point, 0..6), rows per warp, compiled
// occupancy.  Results are bit-identical for every value.
int heat2d_emul();
void set_heat2d_emul(int v);
int heat2d_rows();
void set_heat2d_rows(int v);
int heat2d_occupancy();
void set_heat2d_occupancy(int v);

// Snapshot + L2 norm of a tile: snap (optional, compact ty x tx) <- tile of
// src; norms[index] <- sqrt(sum u^2) in a fixed order.  scratch holds
// kNormScratchBytes, zero on first use, returned to zero by the kernel;
// launches that may run concurrently need distinct scratch.
cudaError_t tile_norm(const double *src, double *snap, double *norms, void *scratch,
                      int64_t ny, int64_t nx, int64_t y0, int64_t x0, int64_t ty, int64_t tx,
                      int64_t index, cudaStream_t s);

// Snapshot + norms of every tile of a TY x TX tile grid (the split of the
// whole-run entry points) in one launch; same bits as tile_norm per tile.
// scratch: tile_norm_grid_scratch_bytes(TY*TX), zero on first use.
cudaError_t tile_norm_grid(const double *src, double *snap, int64_t snap_stride, double *norms,
                           void *scratch, int64_t ny, int64_t nx, int64_t TY, int64_t TX,
                           cudaStream_t s);
size_t tile_norm_grid_scratch_bytes(int64_t tiles);

// 3D FTCS, FP32, periodic: `steps` (1..4) fused steps per launch.  zchunk
// <= 0 picks the z-chunk length that fills whole waves.
cudaError_t heat3d(const float *src, float *dst, int nz, int ny, int nx, float r, int steps,
                   int zchunk, const hxc_launch_cfg *cfg, cudaStream_t s);
int heat3d_default_zchunk(int nz, int ny, int nx, int T);
// Reads and clears the record of 3D launches whose bounded waits ran out
// (form 7's TMA barriers); synchronous.
cudaError_t heat3d_wait_errors(unsigned *flags);

// Variable-diffusivity step (coefficients precomputed by vc_coef or on the
// fly), adjoint step with kappa-gradient, squared-error seed, batches.
cudaError_t vc_coef(const double *kap, double c, int64_t ny, int64_t nx, double *wE, double *wS,
                    double *m, cudaStream_t s);
// `pdl`: launched with programmatic dependent launch, for a launch that
// directly follows another step kernel on `s` (pdl.cuh).
cudaError_t vc_step(const double *u, double *un, const double *wE, const double *wS,
                    const double *m, int64_t ny, int64_t nx, cudaStream_t s, bool pdl = false);
cudaError_t vc_step_otf(const double *u, double *un, const double *kap, double c, int64_t ny,
                        int64_t nx, const hxc_launch_cfg *cfg, cudaStream_t s);
// Adjoint step (do_lam) and per-face kappa-gradient accumulation (do_grad)
// into face = [GE (n) | GS (n) | GW0 (ny) | GN0 (nx)] (vc_face_doubles(ny,
// nx) doubles, zero before the first step); vc_face_combine turns the face
// sums into gk after the last step.
cudaError_t vc_adjoint(const double *lam, double *lam_out, const double *u, const double *wE,
                       const double *wS, const double *m, double *face, int64_t ny, int64_t nx,
                       bool do_lam, bool do_grad, cudaStream_t s, bool pdl = false);
size_t vc_face_doubles(int64_t ny, int64_t nx);
cudaError_t vc_face_combine(const double *face, double *gk, double c, int64_t ny, int64_t nx,
                            cudaStream_t s);
cudaError_t vc_adjoint_otf(const double *lam, double *lam_out, const double *u, const double *kap,
                           double *gk, double c, int64_t ny, int64_t nx, const hxc_launch_cfg *cfg,
                           cudaStream_t s);
cudaError_t sqerr_seed(const double *u, const double *t, double *lam, int64_t n, void *scratch,
                       double *loss, cudaStream_t s);
size_t sqerr_scratch_bytes();
cudaError_t vc_batch_persistent(const void *probs, int nprob, unsigned *queue, double *u,
                                double *tmp, const double *kap, double *wE, double *wS, double *m,
                                int steps, int ctas_per_sm, cudaStream_t s);
cudaError_t vc_batch_coef(const void *probs, const int64_t *rows, int nprob, int64_t total_rows,
                          const double *kap, double *wE, double *wS, double *m, cudaStream_t s);
cudaError_t vc_batch_step(const void *probs, const int64_t *rows, int nprob, int64_t total_rows,
                          const double *u, double *un, const double *wE, const double *wS,
                          const double *m, cudaStream_t s);
size_t vc_problem_bytes();
void vc_pack_problem(void *dst, int64_t off, int32_t side, double c);

}  // namespace k
}  // namespace hxc
