// Core kernels: Listing 2 sum, PRK stencil, partition kernel, 1D and 2D
// FTCS steps and the tile snapshot/norm reduction.
//
// Fixed arithmetic.  Every kernel variant (per-step, temporally blocked,
// any tile shape, any launch order) evaluates one update with exactly the
// same sequence of correctly rounded FP64 operations, so results are
// bit-identical across partition counts, schedules and graph replay:
//   1D: s = ul + ur;                 t = fma(-2, u, s); u' = fma(r, t, u)
//   2D: s = (uN + uW) + (uE + uS);   t = fma(-4, u, s); u' = fma(r, t, u)
// (the additions are issued as fma(a, 1, b), which rounds identically).
// The 2D neighbours are paired along the anti-diagonal: uE + uS of a point
// is also uN + uW of the point below and to the right, so each pair sum is
// computed once and used by two points (4 FP64 operations per point).  The
// sums are symmetric under transposition and under a half turn, so
// transposed or reversed inputs give transposed or reversed bits.
//
// The 1D and 2D runs use two more step kinds of the same sums (kernels.cuh):
// FTCS is linear, so u_{n+1} = r ((1 - 2d r)/r u_n + s(u_n)) in d dimensions,
// and the field scaled by r^-m after m steps advances by one FMA after the
// sum (2 operations per point in 1D, 3 in 2D); a closing step takes the
// scaled field back to true values.  Which step of a run is which kind
// depends only on the step's index, so the bit-identity across partitions,
// schedules, steps per launch and graph replay holds for them too.
#include "fp64_int.cuh"
#include "kernels.cuh"
#include "pdl.cuh"
#include "tune.hpp"

#include <algorithm>
#include <cstdlib>

namespace hxc {
namespace k {

// SM count of the current device (cached per device ordinal).
int sm_count() {
    static std::atomic<int> cache[64];
    int d = 0;
    cudaGetDevice(&d);
    std::atomic<int> &c = cache[d & 63];
    int n = c.load(std::memory_order_relaxed);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || n <= 0)
            n = 148;
        c.store(n, std::memory_order_relaxed);
    }
    return n;
}

static inline unsigned grid_from(const hxc_launch_cfg *cfg, int64_t want) {
    if (cfg) return cfg->grid[0] * cfg->grid[1] * cfg->grid[2];
    if (want < 1) want = 1;
    return (unsigned)std::min<int64_t>(want, 1 << 20);
}
static inline unsigned block_from(const hxc_launch_cfg *cfg, unsigned dflt) {
    if (cfg) return cfg->block[0] * cfg->block[1] * cfg->block[2];
    return dflt;
}

// An FP64 addition issued as a fused multiply-add with a run-time 1.0:
// fma(a, 1, b) rounds a*1 + b = a + b once, so the result is bit-identical
// to a + b, but B300 issues DFMA faster than DADD (598 vs 504 Gop/s
// measured).  `one` must be a kernel argument so that the compiler cannot
// fold the multiplication away.
__device__ __forceinline__ double addf(double a, double b, double one) {
    return __fma_rn(a, one, b);
}

// The 1D update of kind M (kFtcsCanon / Scaled / Close, kernels.cuh).
template <int M>
__device__ __forceinline__ double ftcs3(double ul, double u, double ur, double c0, double c1,
                                        double one) {
    const double s = addf(ul, ur, one);
    if constexpr (M == kFtcsScaled) {
        return __fma_rn(c0, u, s);
    } else if constexpr (M == kFtcsClose) {
        return __fma_rn(c0, s, __dmul_rn(c1, u));
    } else {
        const double t = __fma_rn(-2.0, u, s);
        return __fma_rn(c0, t, u);
    }
}

// One 2D pair sum (uE + uS of a point, = uN + uW of the point below and to
// the right), on the integer-pipe adder when E >= 1.
template <int E>
__device__ __forceinline__ double pair2(double a, double b, double one) {
    return E >= 1 ? dadd_int(a, b) : addf(a, b, one);
}

// The 2D update from the point's two pair sums, pNW = uN + uW and
// pSE = uE + uS; their sum on the integer-pipe adder when E >= 2.  Every E
// gives the same bits; the split balances the FP64 pipe against the
// integer pipe.  M is the step kind (kFtcsCanon / Scaled / Close): the
// scaled step is one FMA after the sum, so a scaled run costs 3 FP64
// operations per point instead of 4.
template <int E, int M>
__device__ __forceinline__ double ftcs5p(double u, double pNW, double pSE, double c0, double c1,
                                         double one) {
    const double s = E >= 2 ? dadd_int(pNW, pSE) : addf(pNW, pSE, one);
    if constexpr (M == kFtcsScaled) {
        return __fma_rn(c0, u, s);
    } else if constexpr (M == kFtcsClose) {
        return __fma_rn(c0, s, __dmul_rn(c1, u));
    } else {
        const double t = __fma_rn(-4.0, u, s);
        return __fma_rn(c0, t, u);
    }
}

// ------------------------------------------------------------ Listing 2 sum
__global__ void k_sum_u32(const uint32_t *__restrict__ in, unsigned long long *result,
                          int64_t n) {
    unsigned long long acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc += in[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(result, acc);
}

cudaError_t sum_u32(const uint32_t *in, unsigned long long *result, int64_t n,
                    const hxc_launch_cfg *cfg, cudaStream_t s) {
    unsigned b = block_from(cfg, 256), g = grid_from(cfg, std::min<int64_t>((n + b - 1) / b, sm_count() * 4));
    k_sum_u32<<<g, b, 0, s>>>(in, result, n);
    return cudaGetLastError();
}

// ------------------------------------------------------- Sec. 5.1.1 PRK
__global__ void k_prk(const double *__restrict__ in, double *__restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double xl = in[i == 0 ? n - 1 : i - 1], xr = in[i == n - 1 ? 0 : i + 1];
        out[i] = __dadd_rn(__dadd_rn(__dmul_rn(0.5, xl), in[i]), __dmul_rn(0.5, xr));
    }
}

cudaError_t prk(const double *in, double *out, int64_t n, const hxc_launch_cfg *cfg,
                cudaStream_t s) {
    unsigned b = block_from(cfg, 256), g = grid_from(cfg, std::min<int64_t>((n + b - 1) / b, sm_count() * 8));
    k_prk<<<g, b, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

// ------------------------------------------------- Sec. 5.1.2 partition k
// In place: x_i <- sqrt(sin(x_i)^2 + cos(x_i)^2), one sincos per element.
__global__ void k_partition(double *__restrict__ x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double sv, cv;
        sincos(x[i], &sv, &cv);
        x[i] = sqrt(sv * sv + cv * cv);
    }
}

cudaError_t partition(double *x, int64_t n, const hxc_launch_cfg *cfg, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    unsigned b = block_from(cfg, 256), g = grid_from(cfg, std::min<int64_t>((n + b - 1) / b, sm_count() * 8));
    k_partition<<<g, b, 0, s>>>(x, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------ 1D FTCS
template <int M>
__global__ void k_heat1d_step(const double *__restrict__ src, double *__restrict__ dst,
                              int64_t n, int64_t lo, int64_t count, double c0, double c1,
                              double one) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = lo + t;
        int64_t jl = j == 0 ? n - 1 : j - 1, jr = j == n - 1 ? 0 : j + 1;
        dst[j] = ftcs3<M>(src[jl], src[j], src[jr], c0, c1, one);
    }
}

// Temporally blocked 1D FTCS: a CTA loads its chunk of C points plus a halo of
// T points on each side (wrapping periodically) into shared memory, advances
// T steps there (the valid window shrinks by one point per side per step)
// and writes its C points.  Chunks are visited grid-stride.
__global__ void k_heat1d_tb(const double *__restrict__ src, double *__restrict__ dst, int64_t n,
                            int64_t lo, int64_t count, const __grid_constant__ FtcsPlan plan,
                            int64_t g0, int T, int C, double one) {
    extern __shared__ double sm[];
    const int W = C + 2 * T;
    double *a = sm, *b = sm + W;
    for (int64_t c0 = (int64_t)blockIdx.x * C; c0 < count; c0 += (int64_t)gridDim.x * C) {
        int64_t base = lo + c0 - T;
        bool wraps = base < 0 || base + W > n;
        for (int i = threadIdx.x; i < W; i += blockDim.x) {
            int64_t g = base + i;
            if (wraps) {
                g %= n;
                if (g < 0) g += n;
            }
            a[i] = src[g];
        }
        __syncthreads();
        double *pa = a, *pb = b;
        for (int s = 1; s <= T; s++) {
            const FtcsStep st = ftcs_plan_step(plan, g0 + s - 1);  // uniform per level
            if (st.kind == kFtcsScaled) {
                for (int i = s + threadIdx.x; i < W - s; i += blockDim.x)
                    pb[i] = ftcs3<kFtcsScaled>(pa[i - 1], pa[i], pa[i + 1], st.c0, st.c1, one);
            } else if (st.kind == kFtcsClose) {
                for (int i = s + threadIdx.x; i < W - s; i += blockDim.x)
                    pb[i] = ftcs3<kFtcsClose>(pa[i - 1], pa[i], pa[i + 1], st.c0, st.c1, one);
            } else {
                for (int i = s + threadIdx.x; i < W - s; i += blockDim.x)
                    pb[i] = ftcs3<kFtcsCanon>(pa[i - 1], pa[i], pa[i + 1], st.c0, st.c1, one);
            }
            __syncthreads();
            double *t = pa;
            pa = pb;
            pb = t;
        }
        int cnt = (int)(count - c0 < (int64_t)C ? count - c0 : (int64_t)C);
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) dst[lo + c0 + i] = pa[T + i];
        __syncthreads();
    }
}

cudaError_t heat1d_plan(const double *src, double *dst, int64_t n, int64_t lo, int64_t count,
                        const FtcsPlan &plan, int64_t g0, int steps, const hxc_launch_cfg *cfg,
                        cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (steps == 1) {
        unsigned b = block_from(cfg, 256);
        unsigned g = grid_from(cfg, std::min<int64_t>((count + b - 1) / b, sm_count() * 8));
        const FtcsStep st = ftcs_plan_step(plan, g0);  // decided on the host
        switch (st.kind) {
            case kFtcsScaled:
                k_heat1d_step<kFtcsScaled><<<g, b, 0, s>>>(src, dst, n, lo, count, st.c0, st.c1, 1.0);
                break;
            case kFtcsClose:
                k_heat1d_step<kFtcsClose><<<g, b, 0, s>>>(src, dst, n, lo, count, st.c0, st.c1, 1.0);
                break;
            default:
                k_heat1d_step<kFtcsCanon><<<g, b, 0, s>>>(src, dst, n, lo, count, st.c0, st.c1, 1.0);
        }
        return cudaGetLastError();
    }
    unsigned b = block_from(cfg, 512);
    unsigned g = grid_from(cfg, sm_count());
    // chunk per CTA: spread `count` over the grid, bounded by shared memory
    const int64_t max_w = (200 * 1024) / (2 * sizeof(double));
    int64_t C = (count + g - 1) / g;
    C = (C + 15) / 16 * 16;
    if (C + 2 * steps > max_w) C = std::max<int64_t>(16, (max_w - 2 * steps) / 16 * 16);
    if (C + 2 * steps > max_w) return cudaErrorInvalidValue;
    size_t smem = 2 * (size_t)(C + 2 * steps) * sizeof(double);
    static std::atomic<uint64_t> attr{0};
    cudaError_t e = smem_optin(k_heat1d_tb, 227 * 1024, attr);
    if (e != cudaSuccess) return e;
    k_heat1d_tb<<<g, b, smem, s>>>(src, dst, n, lo, count, plan, g0, steps, (int)C, 1.0);
    return cudaGetLastError();
}

cudaError_t heat1d(const double *src, double *dst, int64_t n, int64_t lo, int64_t count,
                   double r, int steps, const hxc_launch_cfg *cfg, cudaStream_t s) {
    FtcsPlan p{};
    p.r = r;
    p.P = 0;
    p.I = 1;
    p.total = steps;
    return heat1d_plan(src, dst, n, lo, count, p, 0, steps, cfg, s);
}

// ------------------------------------------------------------ 2D FTCS
// A warp owns a strip of 32*V columns (V consecutive columns per lane) and
// `H` rows and walks the rows keeping rows y and y+1 in registers.  Walking
// row y it forms the pair sums P(y, x) = u[y][x+1] + u[y+1][x] of its
// columns (the right neighbour of its last column from the next lane by a
// shuffle, or from memory at the strip's right end) and updates row y with
// S(y, x) = P(y-1, x-1) + P(y, x): P(y-1, x-1) is the previous row's pair
// sum of the column to the left (own register, or the left lane's by a
// shuffle).  Lane 0's P(y-1, xs-1) straddles the strip's left edge; those
// are formed for 32 rows at a time, one row per lane, and handed to lane 0
// by a shuffle.  The row above the strip seeds P(ys-1, .).  Values outside
// the field are zero.
template <int V>
struct Vec;
template <>
struct Vec<1> {
    double a;
};
template <>
struct Vec<2> {
    double a, b;
};

template <int V>
__device__ __forceinline__ void load_row(Vec<V> &v, const double *__restrict__ src, int64_t ny,
                                         int64_t nx, int64_t y, int64_t x, bool active) {
    if (active && y >= 0 && y < ny) {
        if constexpr (V == 2) {
            double2 q = __ldg(reinterpret_cast<const double2 *>(src + y * nx + x));
            v.a = q.x;
            v.b = q.y;
        } else {
            v.a = __ldg(src + y * nx + x);
        }
    } else {
        v.a = 0.0;
        if constexpr (V == 2) v.b = 0.0;
    }
}

__device__ __forceinline__ double at2(const double *__restrict__ src, int64_t ny, int64_t nx,
                                      int64_t y, int64_t x) {
    return (y >= 0 && y < ny && x >= 0 && x < nx) ? __ldg(src + y * nx + x) : 0.0;
}

template <int V, int EA, int EB, int MINB, int M>
__global__ void __launch_bounds__(256, MINB) k_heat2d(const double *__restrict__ src,
                                                double *__restrict__ dst, int64_t ny, int64_t nx,
                                                int64_t y0, int64_t x0, int64_t ty, int64_t tx,
                                                double c0, double c1, int H, double one) {
    pdl_prologue();  // launched back to back with programmatic dependent launch
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t SW = 32 * V;
    const int64_t nsx = (tx + SW - 1) / SW, nsy = (ty + H - 1) / H;
    const int64_t nwork = nsx * nsy;
    for (int64_t w = blockIdx.x * wpb + (threadIdx.x >> 5); w < nwork; w += (int64_t)gridDim.x * wpb) {
        const int64_t sx = w % nsx, sy = w / nsx;
        const int64_t xs = x0 + sx * SW, xe = min(x0 + tx, xs + SW);
        const int64_t ys = y0 + sy * H, ye = min(y0 + ty, ys + H);
        const int64_t xl = xs + (int64_t)lane * V;
        const bool active = xl < xe;
        const bool last = active && xl + V >= xe;  // owns the strip's last column
        Vec<V> cur, nxt;
        // pair sums of row ys-1: P(ys-1, x) = u[ys-1][x+1] + u[ys][x]
        double pp0, pp1 = 0.0;  // P(y-1, xl), P(y-1, xl+1)
        {
            Vec<V> prv;
            load_row<V>(prv, src, ny, nx, ys - 1, xl, active);
            load_row<V>(cur, src, ny, nx, ys, xl, active);
            double rgt = __shfl_down_sync(0xffffffffu, prv.a, 1);
            if (last) rgt = at2(src, ny, nx, ys - 1, xl + V);
            if constexpr (V == 2) {
                pp0 = pair2<EA>(prv.b, cur.a, one);
                pp1 = pair2<EB>(rgt, cur.b, one);
            } else {
                pp0 = pair2<EA>(rgt, cur.a, one);
            }
        }
        // right neighbour of the strip's last column; the next row and its
        // right neighbour are loaded two rows ahead of their use (measured
        // 0.6% faster than one row ahead, same bits)
        double eR = last ? at2(src, ny, nx, ys, xl + V) : 0.0;
        load_row<V>(nxt, src, ny, nx, ys + 1, xl, active);
        double eRn = last && ys + 1 < ye ? at2(src, ny, nx, ys + 1, xl + V) : 0.0;
        for (int64_t yb = ys; yb < ye; yb += 32) {
            const int64_t yn = min(ye, yb + 32);
            // lane k: P(yb+k-1, xs-1) = u[yb+k-1][xs] + u[yb+k][xs-1]
            double pe = 0.0;
            if (yb + lane < yn)
                pe = pair2<EA>(at2(src, ny, nx, yb + lane - 1, xs), at2(src, ny, nx, yb + lane, xs - 1),
                               one);
            for (int64_t y = yb; y < yn; y++) {
                Vec<V> nx2;
                load_row<V>(nx2, src, ny, nx, y + 2, xl, active);
                const double eR2 = last && y + 2 < ye ? at2(src, ny, nx, y + 2, xl + V) : 0.0;
                double rgt = __shfl_down_sync(0xffffffffu, cur.a, 1);
                if (last) rgt = eR;
                double pnw = __shfl_up_sync(0xffffffffu, V == 2 ? pp1 : pp0, 1);
                const double pel = __shfl_sync(0xffffffffu, pe, (int)(y - yb));
                if (lane == 0) pnw = pel;
                if constexpr (V == 2) {
                    const double q0 = pair2<EA>(cur.b, nxt.a, one);
                    const double q1 = pair2<EB>(rgt, nxt.b, one);
                    if (active) {
                        double2 o;
                        o.x = ftcs5p<EA, M>(cur.a, pnw, q0, c0, c1, one);
                        o.y = ftcs5p<EB, M>(cur.b, pp0, q1, c0, c1, one);
                        *reinterpret_cast<double2 *>(dst + y * nx + xl) = o;
                    }
                    pp0 = q0;
                    pp1 = q1;
                } else {
                    const double q0 = pair2<EA>(rgt, nxt.a, one);
                    if (active) dst[y * nx + xl] = ftcs5p<EA, M>(cur.a, pnw, q0, c0, c1, one);
                    pp0 = q0;
                }
                eR = eRn;
                eRn = eR2;
                cur = nxt;
                nxt = nx2;
            }
        }
    }
}

// 2D knobs live in the tuning registry (speed only, never results).
int heat2d_emul() { return (int)tune::get("heat2d.emul"); }
void set_heat2d_emul(int v) { tune::set("heat2d.emul", v); }
int heat2d_rows() { return (int)tune::get("heat2d.rows"); }
void set_heat2d_rows(int v) { tune::set("heat2d.rows", v); }
int heat2d_occupancy() { return (int)tune::get("heat2d.occupancy"); }
void set_heat2d_occupancy(int v) { tune::set("heat2d.occupancy", v); }

namespace {

template <int M>
cudaError_t heat2d_launch(const double *src, double *dst, int64_t ny, int64_t nx, int64_t y0,
                          int64_t x0, int64_t ty, int64_t tx, double c0, double c1,
                          int rows_per_warp, const hxc_launch_cfg *cfg, cudaStream_t s,
                          bool pdl = false) {
    if (ty <= 0 || tx <= 0) return cudaSuccess;
    const int H = rows_per_warp > 0 ? rows_per_warp : heat2d_rows();
    const bool vec = (nx % 2 == 0) && (x0 % 2 == 0) && (tx % 2 == 0) &&
                     (reinterpret_cast<uintptr_t>(src) % 16 == 0) &&
                     (reinterpret_cast<uintptr_t>(dst) % 16 == 0);
    const int V = vec ? 2 : 1;
    const int64_t nwork = ((tx + 32 * V - 1) / (32 * V)) * ((ty + H - 1) / H);
    unsigned b = block_from(cfg, 256);
    unsigned g = grid_from(cfg, std::min<int64_t>((nwork + b / 32 - 1) / (b / 32), (int64_t)sm_count() * 64));
    // integer-pipe share of the additions, in half-additions per point
    // (0..4: points a and b of a lane take floor/ceil of half of it), and
    // the minimum resident CTAs per SM the kernel is compiled for (4..6)
    const int em = heat2d_emul(), occ = heat2d_occupancy();
#define HXC_L2D(VV, A, B, MB)                                                                 \
    return launch_pdl(k_heat2d<VV, A, B, MB, M>, g, b, s, pdl, src, dst, ny, nx, y0, x0, ty, tx, \
                      c0, c1, H, 1.0)
    if (!vec) {
        switch (em / 2) {
            case 0: HXC_L2D(1, 0, 0, 4);
            case 1: HXC_L2D(1, 1, 1, 4);
            default: HXC_L2D(1, 2, 2, 4);
        }
    }
    if (em == 0) {
        switch (occ) {
            case 5: HXC_L2D(2, 0, 0, 5);
            case 6: HXC_L2D(2, 0, 0, 6);
            default: HXC_L2D(2, 0, 0, 4);
        }
    }
    switch (em) {
        case 1: HXC_L2D(2, 0, 1, 4);
        case 2: HXC_L2D(2, 1, 1, 4);
        case 3: HXC_L2D(2, 1, 2, 4);
        default: HXC_L2D(2, 2, 2, 4);
    }
#undef HXC_L2D
}

}  // namespace

cudaError_t heat2d(const double *src, double *dst, int64_t ny, int64_t nx, int64_t y0,
                   int64_t x0, int64_t ty, int64_t tx, double r, int rows_per_warp,
                   const hxc_launch_cfg *cfg, cudaStream_t s) {
    return heat2d_launch<kFtcsCanon>(src, dst, ny, nx, y0, x0, ty, tx, r, 0.0, rows_per_warp,
                                      cfg, s);
}

cudaError_t heat2d_step(const double *src, double *dst, int64_t ny, int64_t nx, int64_t y0,
                        int64_t x0, int64_t ty, int64_t tx, const FtcsStep &step,
                        int rows_per_warp, cudaStream_t s, bool pdl) {
    switch (step.kind) {
        case kFtcsScaled:
            return heat2d_launch<kFtcsScaled>(src, dst, ny, nx, y0, x0, ty, tx, step.c0, step.c1,
                                               rows_per_warp, nullptr, s, pdl);
        case kFtcsClose:
            return heat2d_launch<kFtcsClose>(src, dst, ny, nx, y0, x0, ty, tx, step.c0, step.c1,
                                              rows_per_warp, nullptr, s, pdl);
        default:
            return heat2d_launch<kFtcsCanon>(src, dst, ny, nx, y0, x0, ty, tx, step.c0, step.c1,
                                              rows_per_warp, nullptr, s, pdl);
    }
}

// ------------------------------------------------------ tile snapshot/norm
// Fixed reduction order: the tile's rows are cut into kNormBands bands
// (band g = rows [g*ty/B, (g+1)*ty/B)); thread t of band g accumulates, in
// increasing order, the squares of the band's elements whose row-major index
// within the band is congruent to t mod 256 (acc = fma(v, v, acc)); the 256
// partials are combined by a butterfly over lanes and a fixed tree over the
// 8 warps; the last band to finish adds the band sums in order g = 0..B-1
// and stores the square root.
__global__ void __launch_bounds__(256) k_tile_norm(const double *__restrict__ src,
                                                   double *__restrict__ snap, double *norms,
                                                   double *partials, unsigned *counter,
                                                   int64_t nx, int64_t y0, int64_t x0, int64_t ty,
                                                   int64_t tx, int64_t index) {
    const int g = blockIdx.x;
    const int64_t r0 = (int64_t)g * ty / kNormBands, r1 = (int64_t)(g + 1) * ty / kNormBands;
    const int64_t m = (r1 - r0) * tx;
    double acc = 0.0;
    int64_t i = r0 + threadIdx.x / tx, j = threadIdx.x % tx;  // element k = threadIdx.x
    for (int64_t k = threadIdx.x; k < m; k += 256) {
        const double v = __ldg(src + (y0 + i) * nx + x0 + j);
        if (snap) snap[i * tx + j] = v;
        acc = __fma_rn(v, v, acc);
        j += 256;  // advance to element k + 256 of the band
        if (j >= tx) {
            i += j / tx;
            j %= tx;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    __shared__ double ws[8];
    __shared__ bool is_last;
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = __dadd_rn(__dadd_rn(__dadd_rn(ws[0], ws[1]), __dadd_rn(ws[2], ws[3])),
                             __dadd_rn(__dadd_rn(ws[4], ws[5]), __dadd_rn(ws[6], ws[7])));
        partials[g] = s;
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        is_last = (prev == kNormBands - 1);
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (int q = 0; q < kNormBands; q++) s = __dadd_rn(s, __ldcg(partials + q));
        norms[index] = __dsqrt_rn(s);
        *counter = 0u;  // leave the scratch ready for the next launch
    }
}

// All tiles of a tile grid in one launch (blockIdx.y = tile): the same
// per-tile reduction order as k_tile_norm, so the same bits.  Tile bounds:
// rows at p*ny/TY, columns at 2*(q*(nx/2)/TX) when nx is even, else q*nx/TX.
// The snapshot of tile t goes to snap + t*snap_stride (compact ty x tx).
__global__ void __launch_bounds__(256) k_tile_norm_grid(const double *__restrict__ src,
                                                        double *__restrict__ snap,
                                                        int64_t snap_stride, double *norms,
                                                        double *partials, unsigned *counters,
                                                        int64_t ny, int64_t nx, int64_t TY,
                                                        int64_t TX) {
    const int g = blockIdx.x;
    const int64_t tile = blockIdx.y, p = tile / TX, q = tile % TX;
    const int64_t y0 = p * ny / TY, y1 = (p + 1) * ny / TY;
    int64_t x0, x1;
    if (nx % 2 == 0) {
        x0 = (q * (nx / 2) / TX) * 2;
        x1 = q + 1 == TX ? nx : ((q + 1) * (nx / 2) / TX) * 2;
    } else {
        x0 = q * nx / TX;
        x1 = (q + 1) * nx / TX;
    }
    const int64_t ty = y1 - y0, tx = x1 - x0;
    double *part = partials + tile * kNormBands;
    unsigned *counter = counters + tile;
    double *sn = snap ? snap + tile * snap_stride : nullptr;
    const int64_t r0 = (int64_t)g * ty / kNormBands, r1 = (int64_t)(g + 1) * ty / kNormBands;
    const int64_t m = (r1 - r0) * tx;
    double acc = 0.0;
    if (tx > 0) {
        int64_t i = r0 + threadIdx.x / tx, j = threadIdx.x % tx;
        for (int64_t k = threadIdx.x; k < m; k += 256) {
            const double v = __ldg(src + (y0 + i) * nx + x0 + j);
            if (sn) sn[i * tx + j] = v;
            acc = __fma_rn(v, v, acc);
            j += 256;
            if (j >= tx) {
                i += j / tx;
                j %= tx;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    __shared__ double ws[8];
    __shared__ bool is_last;
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sm = __dadd_rn(__dadd_rn(__dadd_rn(ws[0], ws[1]), __dadd_rn(ws[2], ws[3])),
                              __dadd_rn(__dadd_rn(ws[4], ws[5]), __dadd_rn(ws[6], ws[7])));
        part[g] = sm;
        __threadfence();
        is_last = atomicAdd(counter, 1u) == kNormBands - 1;
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
        __threadfence();
        double sm = 0.0;
        for (int b = 0; b < kNormBands; b++) sm = __dadd_rn(sm, __ldcg(part + b));
        norms[tile] = __dsqrt_rn(sm);
    }
}

cudaError_t tile_norm_grid(const double *src, double *snap, int64_t snap_stride, double *norms,
                           void *scratch, int64_t ny, int64_t nx, int64_t TY, int64_t TX,
                           cudaStream_t s) {
    double *partials = static_cast<double *>(scratch);
    unsigned *counters = reinterpret_cast<unsigned *>(partials + TY * TX * kNormBands);
    // the counters sit behind the partials, so their place moves with the
    // tile count: clear them for every launch (the scratch is shared by runs
    // of any tile grid)
    cudaError_t e = cudaMemsetAsync(counters, 0, (size_t)TY * TX * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    dim3 grid(kNormBands, (unsigned)(TY * TX));
    k_tile_norm_grid<<<grid, 256, 0, s>>>(src, snap, snap_stride, norms, partials, counters, ny,
                                          nx, TY, TX);
    return cudaGetLastError();
}

size_t tile_norm_grid_scratch_bytes(int64_t tiles) {
    return (size_t)tiles * (kNormBands * sizeof(double) + sizeof(unsigned)) + 16;
}

cudaError_t tile_norm(const double *src, double *snap, double *norms, void *scratch,
                      int64_t ny, int64_t nx, int64_t y0, int64_t x0, int64_t ty, int64_t tx,
                      int64_t index, cudaStream_t s) {
    (void)ny;
    double *partials = static_cast<double *>(scratch);
    unsigned *counter = reinterpret_cast<unsigned *>(partials + kNormBands);
    k_tile_norm<<<kNormBands, 256, 0, s>>>(src, snap, norms, partials, counter, nx, y0, x0, ty,
                                           tx, index);
    return cudaGetLastError();
}

}  // namespace k
}  // namespace hxc
