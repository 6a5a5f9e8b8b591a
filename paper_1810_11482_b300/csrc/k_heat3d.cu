// 3D 7-point FTCS, FP32, periodic, T (1..4) fused steps per launch.
//
// Canonical arithmetic (every form, every T):
//   s  = (((u[x-1] + u[x+1]) + (u[y-1] + u[y+1])) + u[z-1]) + u[z+1]
//   t  = fma(-6, u, s);   u' = fma(r, t, u)            (FP32, round-to-nearest)
// so T fused steps give the same bits as T single-step launches.
//
// Temporal blocking.  A CTA owns an x-y region (its output tile plus a halo
// of T columns on every side) and streams it along z.  Level t (the field
// after t steps) is kept per thread in registers for the columns the thread
// owns; x-neighbours come from the adjacent lanes by shuffles and
// y-neighbours from the thread's own rows or from shared memory.  In every
// iteration a new level-0 plane arrives and each level t < T produces one
// plane of level t+1.  Cells within distance t of the region edge are wrong
// at level t and are never written: only the central columns of level T are
// stored.  Forms: 2 (three plane registers per level, 64 x 32 regions, z cut
// into chunks), 3 (two registers per level, 64 x 64 regions, the (region,
// plane) pairs split evenly over one CTA per SM), 4 (form 3 fed by a
// cp.async ring of input planes), 6 (form 4 with packed narrow tiles), and
// for one-step launches 5 (a streaming kernel).
#include <algorithm>
#include <cstring>
#include <mutex>

#include <cuda.h>  // CUtensorMap: the TMA descriptor passed to form 7
#include <cudaTypedefs.h>

#include "f32x2.cuh"
#include "kernels.cuh"
#include "tune.hpp"

namespace hxc {
namespace k {

namespace {
constexpr int RX = 64, RY = 32, NT = 512;

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}
}  // namespace

// ---------------------------------------------------------------------------
// Global offsets of a thread's 2 x 2 cells (form 2).
namespace {

struct Cols {
    size_t o00, o01, o10, o11;
    bool pair;  // columns 0/1 (and 2/3) adjacent and 8-byte aligned
};

}  // namespace

// ---------------------------------------------------------------------------
// Form 2.  A CTA owns a 64 x 32 region, a thread 2 x 2 cells: the two
// x-adjacent cells of each of its rows held as one 64-bit pair (the low half
// the lower x) and updated with the paired FP32 instructions (f32x2.cuh).
// Each level keeps three plane slots (oldest, middle, newest) whose roles
// rotate by one each iteration (the z loop is unrolled by three, so every
// register index is a compile-time constant); levels are computed top-down,
// level t writing its output plane straight into the oldest slot of level
// t+1, so level t runs 3t-1 planes behind level 0.  y-neighbours outside the
// thread's two rows come from a shared-memory copy of each level's middle
// plane.
namespace {

// ftcs7 on two cells at once (same operation order and rounding)
__device__ __forceinline__ f2 ftcs7x2(f2 u, f2 xm, f2 xp, f2 ym, f2 yp, f2 zm, f2 zp, f2 r2,
                                      f2 m6) {
    const f2 s = add2(add2(add2(add2(xm, xp), add2(ym, yp)), zm), zp);
    return fma2(r2, fma2(m6, u, s), u);
}

__device__ __forceinline__ void load2x2(f2 (&v)[2], const float *__restrict__ src, size_t zo,
                                        const Cols &c) {
    if (c.pair) {
        v[0] = __ldg(reinterpret_cast<const unsigned long long *>(src + zo + c.o00));
        v[1] = __ldg(reinterpret_cast<const unsigned long long *>(src + zo + c.o10));
    } else {
        v[0] = pk(__ldg(src + zo + c.o00), __ldg(src + zo + c.o01));
        v[1] = pk(__ldg(src + zo + c.o10), __ldg(src + zo + c.o11));
    }
}

template <int T, int R>
__device__ __forceinline__ void h3p_iter(f2 (&L)[T][3][2], f2 (&nxt)[2], f2 (*S)[RY][RX / 2],
                                         const float *__restrict__ src, float *__restrict__ dst,
                                         const Cols &c, int lane, int wr, int wru, int wrd, int &zl,
                                         int nz, size_t plane, bool more, int zout, int z0, int z1,
                                         bool ox0, bool ox1, bool oy0, bool oy1, f2 r2, f2 m6) {
    constexpr int P = R % 3, M = (R + 1) % 3, N = (R + 2) % 3;
    L[0][P][0] = nxt[0];
    L[0][P][1] = nxt[1];
    if (more) {
        zl = zl + 1 < nz ? zl + 1 : zl + 1 - nz;
        load2x2(nxt, src, (size_t)zl * plane, c);
    }
    S[0][wr][lane] = L[0][N][0];
    S[0][wr + 1][lane] = L[0][N][1];
    __syncthreads();
    f2 out[2];
#pragma unroll
    for (int t = T - 1; t >= 0; t--) {
        const int a = t == 0 ? M : P, b = t == 0 ? N : M, d = t == 0 ? P : N;
        const f2 A = L[t][b][0], B = L[t][b][1];  // rows ry and ry+1 of the middle plane
        const f2 up = S[t][wru][lane], dn = S[t][wrd][lane];
        const float l0 = __shfl_up_sync(0xffffffffu, hi_of(A), 1);
        const float r0 = __shfl_down_sync(0xffffffffu, lo_of(A), 1);
        const float l1 = __shfl_up_sync(0xffffffffu, hi_of(B), 1);
        const float r1 = __shfl_down_sync(0xffffffffu, lo_of(B), 1);
        const f2 vA = ftcs7x2(A, pk(l0, lo_of(A)), pk(hi_of(A), r0), up, B, L[t][a][0],
                              L[t][d][0], r2, m6);
        const f2 vB = ftcs7x2(B, pk(l1, lo_of(B)), pk(hi_of(B), r1), A, dn, L[t][a][1],
                              L[t][d][1], r2, m6);
        if (t == T - 1) {
            out[0] = vA;
            out[1] = vB;
        } else {
            L[t + 1][P][0] = vA;
            L[t + 1][P][1] = vB;
        }
    }
    __syncthreads();
#pragma unroll
    for (int t = 1; t < T; t++) {
        S[t][wr][lane] = L[t][N][0];
        S[t][wr + 1][lane] = L[t][N][1];
    }
    if (zout >= z0 && zout < z1) {
        float *d = dst + (size_t)zout * plane;
        if (c.pair && ox0 && ox1) {
            if (oy0) *reinterpret_cast<f2 *>(d + c.o00) = out[0];
            if (oy1) *reinterpret_cast<f2 *>(d + c.o10) = out[1];
        } else {
            if (oy0 && ox0) d[c.o00] = lo_of(out[0]);
            if (oy0 && ox1) d[c.o01] = hi_of(out[0]);
            if (oy1 && ox0) d[c.o10] = lo_of(out[1]);
            if (oy1 && ox1) d[c.o11] = hi_of(out[1]);
        }
    }
}

}  // namespace

template <int T>
__global__ void __launch_bounds__(NT, 1)
    k_heat3d_pk(const float *__restrict__ src, float *__restrict__ dst, int nz, int ny, int nx,
                float r, int zchunk) {
    constexpr int BX = RX - 2 * T, BY = RY - 2 * T;
    __shared__ __align__(16) f2 S[T][RY][RX / 2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tiles_x = (nx + BX - 1) / BX, tiles_y = (ny + BY - 1) / BY;
    const int nchunks = (nz + zchunk - 1) / zchunk;
    const int nblk = tiles_x * tiles_y * nchunks;
    const int rx = 2 * lane, ry = 2 * warp;
    const int ryu = ry > 0 ? ry - 1 : 0, ryd = ry + 2 < RY ? ry + 2 : RY - 1;
    const size_t plane = (size_t)ny * nx;
    const f2 r2 = pk(r, r), m6 = pk(-6.0f, -6.0f);

    for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
        const int tx = b % tiles_x, ty = (b / tiles_x) % tiles_y, ch = b / (tiles_x * tiles_y);
        const int x0 = tx * BX - T, y0 = ty * BY - T;
        const int z0 = ch * zchunk, z1 = min(nz, z0 + zchunk);
        const int gx0 = wrapi(x0 + rx, nx), gx1 = wrapi(x0 + rx + 1, nx);
        const int gy0 = wrapi(y0 + ry, ny), gy1 = wrapi(y0 + ry + 1, ny);
        const bool ox0 = rx >= T && rx < RX - T && x0 + rx < nx;
        const bool ox1 = rx + 1 >= T && rx + 1 < RX - T && x0 + rx + 1 < nx;
        const bool oy0 = ry >= T && ry < RY - T && y0 + ry < ny;
        const bool oy1 = ry + 1 >= T && ry + 1 < RY - T && y0 + ry + 1 < ny;
        Cols c;
        c.o00 = (size_t)gy0 * nx + gx0;
        c.o01 = (size_t)gy0 * nx + gx1;
        c.o10 = (size_t)gy1 * nx + gx0;
        c.o11 = (size_t)gy1 * nx + gx1;
        c.pair = gx1 == gx0 + 1 && (gx0 & 1) == 0 && (nx & 1) == 0;

        f2 L[T][3][2];
#pragma unroll
        for (int t = 0; t < T; t++)
#pragma unroll
            for (int s = 0; s < 3; s++) L[t][s][0] = L[t][s][1] = 0ull;

        const int iters = (z1 - z0) + 3 * T - 1;
        int zl = wrapi(z0 - T, nz);
        f2 nxt[2];
        load2x2(nxt, src, (size_t)zl * plane, c);
        const int zout = z0 - 3 * T + 1;
        for (int i = 0; i < iters; i += 3) {
            h3p_iter<T, 0>(L, nxt, S, src, dst, c, lane, ry, ryu, ryd, zl, nz, plane,
                           i + 1 < iters, zout + i, z0, z1, ox0, ox1, oy0, oy1, r2, m6);
            if (i + 1 >= iters) break;
            h3p_iter<T, 1>(L, nxt, S, src, dst, c, lane, ry, ryu, ryd, zl, nz, plane,
                           i + 2 < iters, zout + i + 1, z0, z1, ox0, ox1, oy0, oy1, r2, m6);
            if (i + 2 >= iters) break;
            h3p_iter<T, 2>(L, nxt, S, src, dst, c, lane, ry, ryu, ryd, zl, nz, plane,
                           i + 3 < iters, zout + i + 2, z0, z1, ox0, ox1, oy0, oy1, r2, m6);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Variant 3: two values per cell and level instead of three, 2 x 4 cells per
// thread, and the z range split evenly over the CTAs.
//
// A level keeps, per cell, its centre plane c and the partial sum
// p = (x-pair + y-pair) + (plane below c), formed as soon as c arrives; when
// the plane above arrives the update is u' = fma(r, fma(-6, c, p + above), c).
// So a level needs two planes of registers, and the levels chain through
// registers within one z iteration: the plane level t produces is the plane
// level t+1 receives in the same iteration (level t+1 lags one plane).
//
// A warp covers the 64 columns of its region row band as 32 lanes x 2
// adjacent columns (one paired-FP32 register per row) and 4 rows, so 16
// warps cover a 64 x 64 region.  x-neighbours outside the thread's pair come
// from the adjacent lanes by shuffles, y-neighbours inside its 4 rows from its
// own registers, and only the band's first and last rows go through shared
// memory (double-buffered, one barrier per z iteration).
//
// Work: the (region, output plane) pairs are numbered region-major and every
// CTA takes an equal contiguous share, so the CTAs finish together; each
// region segment of a share costs 2T extra iterations to fill the level chain.
namespace {

constexpr int V3_NW = 16, V3_H = 4 * V3_NW;  // warps per CTA, region rows

// the thread's two columns of one row (one 8-byte load when adjacent and aligned)
__device__ __forceinline__ f2 ld_pair(const float *__restrict__ p, unsigned a0, unsigned a1,
                                      bool pair) {
    if (pair) return __ldg(reinterpret_cast<const unsigned long long *>(p + a0));
    return pk(__ldg(p + a0), __ldg(p + a1));
}

// One z iteration.  Q selects which of X / Y holds the centre planes (the
// other receives the incoming planes and becomes the centre).
template <int T, int Q>
__device__ __forceinline__ void v3_iter(f2 (&X)[T][4], f2 (&Y)[T][4], f2 (&Pp)[T][4],
                                        f2 (&nxt)[4], f2 *__restrict__ Sb,
                                        const float *__restrict__ src, float *__restrict__ dst,
                                        const unsigned (&row)[4], unsigned gx0, unsigned gx1,
                                        bool pair, int &zl, int nz, size_t plane, bool more,
                                        bool store, int zout, unsigned omask, int lane, int warp,
                                        int wu, int wd, f2 r2, f2 m6) {
    f2(&C)[T][4] = Q ? Y : X;
    f2(&N)[T][4] = Q ? X : Y;
    // level 0 receives the prefetched plane; fetch the next one
#pragma unroll
    for (int k = 0; k < 4; k++) N[0][k] = nxt[k];
    if (more) {
        zl = zl + 1 < nz ? zl + 1 : 0;
        const float *p = src + (size_t)zl * plane;
#pragma unroll
        for (int k = 0; k < 4; k++) nxt[k] = ld_pair(p, row[k] + gx0, row[k] + gx1, pair);
    }
    // step 1: every level finishes the cells of its centre plane; the result
    // is the incoming plane of the next level (level T's is stored)
#pragma unroll
    for (int t = 0; t < T; t++) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const f2 v = fma2(r2, fma2(m6, C[t][k], add2(Pp[t][k], N[t][k])), C[t][k]);
            if (t + 1 < T) N[t + 1][k] = v;
            if (t + 1 == T && store) {
                float *d = dst + (size_t)zout * plane;
                const unsigned m = omask >> (2 * k);
                if (pair && (m & 3u) == 3u) {
                    *reinterpret_cast<f2 *>(d + row[k] + gx0) = v;
                } else {
                    if (m & 1u) d[row[k] + gx0] = lo_of(v);
                    if (m & 2u) d[row[k] + gx1] = hi_of(v);
                }
            }
        }
    }
    // step 2: publish the band edge rows of every incoming plane, then form
    // the partial sums of the new centre planes
#pragma unroll
    for (int t = 0; t < T; t++) {
        Sb[((t * V3_NW + warp) * 2 + 0) * 32 + lane] = N[t][0];
        Sb[((t * V3_NW + warp) * 2 + 1) * 32 + lane] = N[t][3];
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < T; t++) {
        const f2 up = Sb[((t * V3_NW + wu) * 2 + 1) * 32 + lane];
        const f2 dn = Sb[((t * V3_NW + wd) * 2 + 0) * 32 + lane];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const f2 v = N[t][k];
            const float lft = __shfl_up_sync(0xffffffffu, hi_of(v), 1);
            const float rgt = __shfl_down_sync(0xffffffffu, lo_of(v), 1);
            // left cell: (left lane's high) + own high; right cell: own low + (right lane's low)
            const f2 xs = pk(__fadd_rn(lft, hi_of(v)), __fadd_rn(lo_of(v), rgt));
            const f2 ys = add2(k == 0 ? up : N[t][k - 1], k == 3 ? dn : N[t][k + 1]);
            Pp[t][k] = add2(add2(xs, ys), C[t][k]);
        }
    }
}
}  // namespace

template <int T>
__global__ void __launch_bounds__(V3_NW * 32, 1)
    k_heat3d_v3(const float *__restrict__ src, float *__restrict__ dst, int nz, int ny, int nx,
                float r) {
    constexpr int BX = 64 - 2 * T, BY = V3_H - 2 * T;
    extern __shared__ __align__(16) f2 v3_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wu = warp > 0 ? warp - 1 : 0, wd = warp + 1 < V3_NW ? warp + 1 : V3_NW - 1;
    const int tiles_x = (nx + BX - 1) / BX, tiles_y = (ny + BY - 1) / BY;
    const int64_t work = (int64_t)tiles_x * tiles_y * nz;
    const int64_t w_end = work * (blockIdx.x + 1) / gridDim.x;
    const size_t plane = (size_t)ny * nx;
    const f2 r2 = pk(r, r), m6 = pk(-6.0f, -6.0f);
    constexpr int SB = T * V3_NW * 2 * 32;  // f2 per shared buffer
    int buf = 0;

    for (int64_t w = work * blockIdx.x / gridDim.x; w < w_end;) {
        const int64_t reg = w / nz;
        const int za = (int)(w - reg * nz);
        const int zb = (int)min((int64_t)nz, za + (w_end - w));
        w += zb - za;
        const int tx = (int)(reg % tiles_x), ty = (int)(reg / tiles_x);
        const int x0 = tx * BX - T, y0 = ty * BY - T;
        const int c0 = 2 * lane;
        const unsigned gx0 = wrapi(x0 + c0, nx), gx1 = wrapi(x0 + c0 + 1, nx);
        const bool pair = gx1 == gx0 + 1 && (gx0 & 1u) == 0 && (nx & 1) == 0;
        const bool ox0 = c0 >= T && c0 < 64 - T && x0 + c0 < nx;
        const bool ox1 = c0 + 1 >= T && c0 + 1 < 64 - T && x0 + c0 + 1 < nx;
        unsigned row[4], omask = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int q = 4 * warp + k;
            row[k] = (unsigned)wrapi(y0 + q, ny) * (unsigned)nx;
            const bool oy = q >= T && q < V3_H - T && y0 + q < ny;
            omask |= (oy && ox0 ? 1u : 0u) << (2 * k);
            omask |= (oy && ox1 ? 2u : 0u) << (2 * k);
        }

        f2 X[T][4], Y[T][4], Pp[T][4];
#pragma unroll
        for (int t = 0; t < T; t++)
#pragma unroll
            for (int k = 0; k < 4; k++) X[t][k] = Y[t][k] = Pp[t][k] = 0ull;
        // iteration j receives level-0 plane za - T + j and emits level-T
        // plane za - 2T + j (stored for j >= 2T)
        const int iters = (zb - za) + 2 * T;
        int zl = wrapi(za - T, nz);
        f2 nxt[4];
        {
            const float *p = src + (size_t)zl * plane;
#pragma unroll
            for (int k = 0; k < 4; k++) nxt[k] = ld_pair(p, row[k] + gx0, row[k] + gx1, pair);
        }
        for (int j = 0; j < iters; j += 2) {
            v3_iter<T, 0>(X, Y, Pp, nxt, v3_smem + buf * SB, src, dst, row, gx0, gx1, pair, zl, nz,
                          plane, j + 1 < iters, j >= 2 * T, za - 2 * T + j, omask, lane, warp, wu,
                          wd, r2, m6);
            buf ^= 1;
            if (j + 1 >= iters) break;
            v3_iter<T, 1>(X, Y, Pp, nxt, v3_smem + buf * SB, src, dst, row, gx0, gx1, pair, zl, nz,
                          plane, j + 2 < iters, j + 1 >= 2 * T, za - 2 * T + j + 1, omask, lane,
                          warp, wu, wd, r2, m6);
            buf ^= 1;
        }
    }
}

template <int T>
cudaError_t v3_launch(unsigned g, const float *src, float *dst, int nz, int ny, int nx, float r,
                      cudaStream_t s) {
    constexpr size_t smem = sizeof(f2) * 2 * T * V3_NW * 2 * 32;
    static std::atomic<uint64_t> attr{0};
    cudaError_t e = smem_optin(k_heat3d_v3<T>, (int)smem, attr);
    if (e != cudaSuccess) return e;
    k_heat3d_v3<T><<<g, V3_NW * 32, smem, s>>>(src, dst, nz, ny, nx, r);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Variant 4: variant 3 with the level-0 planes copied into a shared-memory
// ring by cp.async, V4_D planes ahead, instead of loaded into registers one
// plane ahead.  The ring holds the region's whole plane, so level 0's band
// edge rows are read from it directly; levels 1..T-1 publish theirs as in
// variant 3.  A ring slot is refilled two iterations after its last read
// (V4_D + 2 slots), which the per-iteration barrier orders.
namespace {

constexpr int V4_D = 2, V4_RS = V4_D + 2;

__device__ __forceinline__ void cp8(void *sdst, const void *gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp4(void *sdst, const void *gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// copy the thread's 4 x 2 cells of plane zq into ring slot `slot`
__device__ __forceinline__ void v4_fetch(f2 *__restrict__ ring, int slot, const float *__restrict__ p,
                                         const unsigned (&row)[4], unsigned gx0, unsigned gx1,
                                         bool pair, int lane, int warp) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
        f2 *d = ring + ((size_t)slot * V3_H + 4 * warp + k) * 32 + lane;
        if (pair) {
            cp8(d, p + row[k] + gx0);
        } else {
            cp4(d, p + row[k] + gx0);
            cp4(reinterpret_cast<float *>(d) + 1, p + row[k] + gx1);
        }
    }
    cp_commit();
}

// How the level-0 planes reach the ring: each thread copies its own cells
// with cp.async (any region), waiting for its own copies.
struct CpFetch {
    f2 *ring;
    const float *src;
    size_t plane;
    const unsigned *row;
    unsigned gx0, gx1;
    bool pair;
    int lane, warp;
    __device__ __forceinline__ void issue(int slot, int z) {
        const unsigned r4[4] = {row[0], row[1], row[2], row[3]};
        v4_fetch(ring, slot, src + (size_t)z * plane, r4, gx0, gx1, pair, lane, warp);
    }
    __device__ __forceinline__ void wait(int) { cp_wait<V4_D>(); }
    __device__ __forceinline__ void drain() { cp_wait<0>(); }
    __device__ __forceinline__ void sync() { __syncthreads(); }
    static constexpr bool failed = false;
};

// Form 7: one thread copies a region's whole 64 x 64 input plane into the
// ring slot with a TMA tensor copy (cp.async.bulk.tensor, completion on the
// slot's mbarrier); every thread waits on the barrier's phase before reading
// the slot.  Only regions that lie inside the field are fetched this way (a
// TMA tile does not wrap around the periodic edges).  Waits are bounded: a
// wait that runs out records it in g_heat3d_wait_errors, the CTA agrees on
// the failure at its next barrier, stops issuing copies, waits (again
// bounded) for the copies still in flight and leaves.
__device__ unsigned g_heat3d_wait_errors;

constexpr unsigned kTmaTileBytes = 64 * 64 * sizeof(float);
constexpr int kTmaMaxTries = 1 << 22;

struct TmaFetch {
    f2 *ring;
    const CUtensorMap *map;
    unsigned bars;      // shared-space address of V4_RS mbarriers, 8 bytes each
    int x0, y0;         // the region's origin (inside the field)
    unsigned phase;     // per slot: parity of the barrier phase to wait for next
    unsigned inflight;  // per slot: a copy issued and not yet waited for
    int failed;
    __device__ __forceinline__ void issue(int slot, int z) {
        if (failed) return;
        if (threadIdx.x == 0) {
            const unsigned bar = bars + 8u * (unsigned)slot;
            const unsigned dst = (unsigned)__cvta_generic_to_shared(ring + (size_t)slot * V3_H * 32);
            // the slot's previous contents were read through the generic
            // proxy (ordered by the last CTA barrier); order those reads
            // before the async-proxy write
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         :: "r"(bar), "r"(kTmaTileBytes) : "memory");
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4}], [%5];"
                :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x0), "r"(y0), "r"(z),
                   "r"(bar)
                : "memory");
        }
        inflight |= 1u << slot;
    }
    __device__ __forceinline__ bool wait_slot(int slot) {
        const unsigned bar = bars + 8u * (unsigned)slot, par = (phase >> slot) & 1u;
        unsigned done = 0;
        for (int it = 0; it < kTmaMaxTries && !done; ++it)
            asm volatile(
                "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;"
                " selp.u32 %0, 1, 0, p; }"
                : "=r"(done) : "r"(bar), "r"(par) : "memory");
        if (!done) {
            atomicOr(&g_heat3d_wait_errors, 1u);
            return false;
        }
        phase ^= 1u << slot;
        inflight &= ~(1u << slot);
        return true;
    }
    __device__ __forceinline__ void wait(int slot) {
        if (!failed && !wait_slot(slot)) failed = 1;
    }
    __device__ __forceinline__ void drain() {
        for (int sl = 0; sl < V4_RS; sl++)
            if (inflight & (1u << sl)) wait_slot(sl);
    }
    // the per-iteration CTA barrier, which also makes a failure CTA-uniform
    __device__ __forceinline__ void sync() { failed = __syncthreads_or(failed); }
};

template <int T, int Q, int SW, class F>
__device__ __forceinline__ void v4_iter(f2 (&X)[T][4], f2 (&Y)[T][4], f2 (&Pp)[T][4],
                                        f2 *__restrict__ ring, int slot, int fslot,
                                        f2 *__restrict__ Sb, F &fetch,
                                        float *__restrict__ dst, const unsigned (&row)[4],
                                        unsigned gx0, unsigned gx1, bool pair, int &zf, int nz,
                                        size_t plane, bool store, int zout, unsigned omask,
                                        int lane, int warp, int ru, int rd, int wu, int wd, f2 r2,
                                        f2 m6) {
    f2(&C)[T][4] = Q ? Y : X;
    f2(&N)[T][4] = Q ? X : Y;
    // fetch plane V4_D ahead, then wait for this iteration's plane
    zf = zf + 1 < nz ? zf + 1 : 0;
    fetch.issue(fslot, zf);
    fetch.wait(slot);
    const f2 *rs = ring + (size_t)slot * V3_H * 32;
#pragma unroll
    for (int k = 0; k < 4; k++) N[0][k] = rs[(4 * warp + k) * 32 + lane];
#pragma unroll
    for (int t = 0; t < T; t++) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const f2 v = fma2(r2, fma2(m6, C[t][k], add2(Pp[t][k], N[t][k])), C[t][k]);
            if (t + 1 < T) N[t + 1][k] = v;
            if (t + 1 == T && store) {
                float *d = dst + (size_t)zout * plane;
                const unsigned m = omask >> (2 * k);
                if (pair && (m & 3u) == 3u) {
                    *reinterpret_cast<f2 *>(d + row[k] + gx0) = v;
                } else {
                    if (m & 1u) d[row[k] + gx0] = lo_of(v);
                    if (m & 2u) d[row[k] + gx1] = hi_of(v);
                }
            }
        }
    }
#pragma unroll
    for (int t = 1; t < T; t++) {
        Sb[(((t - 1) * V3_NW + warp) * 2 + 0) * 32 + lane] = N[t][0];
        Sb[(((t - 1) * V3_NW + warp) * 2 + 1) * 32 + lane] = N[t][3];
    }
    fetch.sync();
#pragma unroll
    for (int t = 0; t < T; t++) {
        const f2 up = t == 0 ? rs[ru * 32 + lane] : Sb[(((t - 1) * V3_NW + wu) * 2 + 1) * 32 + lane];
        const f2 dn = t == 0 ? rs[rd * 32 + lane] : Sb[(((t - 1) * V3_NW + wd) * 2 + 0) * 32 + lane];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const f2 v = N[t][k];
            // lanes exchange within segments of SW lanes (one region each)
            const float lft = __shfl_up_sync(0xffffffffu, hi_of(v), 1, SW);
            const float rgt = __shfl_down_sync(0xffffffffu, lo_of(v), 1, SW);
            // left cell: (left lane's high) + own high; right cell: own low + (right lane's low)
            const f2 xs = pk(__fadd_rn(lft, hi_of(v)), __fadd_rn(lo_of(v), rgt));
            const f2 ys = add2(k == 0 ? up : N[t][k - 1], k == 3 ? dn : N[t][k + 1]);
            Pp[t][k] = add2(add2(xs, ys), C[t][k]);
        }
    }
}

template <int T>
constexpr size_t v4_smem_bytes() {
    return sizeof(f2) * ((size_t)V4_RS * V3_H * 32 + 2 * (T > 1 ? T - 1 : 1) * V3_NW * 2 * 32);
}

}  // namespace

template <int T>
__global__ void __launch_bounds__(V3_NW * 32, 1)
    k_heat3d_v4(const float *__restrict__ src, float *__restrict__ dst, int nz, int ny, int nx,
                float r) {
    constexpr int BX = 64 - 2 * T, BY = V3_H - 2 * T;
    extern __shared__ __align__(128) f2 v4_smem[];
    f2 *ring = v4_smem;
    f2 *sbase = v4_smem + (size_t)V4_RS * V3_H * 32;
    constexpr int SB = (T > 1 ? T - 1 : 1) * V3_NW * 2 * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wu = warp > 0 ? warp - 1 : 0, wd = warp + 1 < V3_NW ? warp + 1 : V3_NW - 1;
    const int ru = warp > 0 ? 4 * warp - 1 : 0, rd = warp + 1 < V3_NW ? 4 * warp + 4 : V3_H - 1;
    const int tiles_x = (nx + BX - 1) / BX, tiles_y = (ny + BY - 1) / BY;
    const int64_t work = (int64_t)tiles_x * tiles_y * nz;
    const int64_t w_end = work * (blockIdx.x + 1) / gridDim.x;
    const size_t plane = (size_t)ny * nx;
    const f2 r2 = pk(r, r), m6 = pk(-6.0f, -6.0f);
    int buf = 0;

    for (int64_t w = work * blockIdx.x / gridDim.x; w < w_end;) {
        const int64_t reg = w / nz;
        const int za = (int)(w - reg * nz);
        const int zb = (int)min((int64_t)nz, za + (w_end - w));
        w += zb - za;
        const int tx = (int)(reg % tiles_x), ty = (int)(reg / tiles_x);
        const int x0 = tx * BX - T, y0 = ty * BY - T;
        const int c0 = 2 * lane;
        const unsigned gx0 = wrapi(x0 + c0, nx), gx1 = wrapi(x0 + c0 + 1, nx);
        const bool pair = gx1 == gx0 + 1 && (gx0 & 1u) == 0 && (nx & 1) == 0;
        const bool ox0 = c0 >= T && c0 < 64 - T && x0 + c0 < nx;
        const bool ox1 = c0 + 1 >= T && c0 + 1 < 64 - T && x0 + c0 + 1 < nx;
        unsigned row[4], omask = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int q = 4 * warp + k;
            row[k] = (unsigned)wrapi(y0 + q, ny) * (unsigned)nx;
            const bool oy = q >= T && q < V3_H - T && y0 + q < ny;
            omask |= (oy && ox0 ? 1u : 0u) << (2 * k);
            omask |= (oy && ox1 ? 2u : 0u) << (2 * k);
        }

        f2 X[T][4], Y[T][4], Pp[T][4];
#pragma unroll
        for (int t = 0; t < T; t++)
#pragma unroll
            for (int k = 0; k < 4; k++) X[t][k] = Y[t][k] = Pp[t][k] = 0ull;
        // iteration j receives level-0 plane za - T + j (ring slot j % V4_RS)
        // and emits level-T plane za - 2T + j (stored for j >= 2T)
        const int iters = (zb - za) + 2 * T;
        CpFetch fetch{ring, src, plane, row, gx0, gx1, pair, lane, warp};
        int zf = wrapi(za - T, nz);
        fetch.issue(0, zf);
#pragma unroll
        for (int q = 1; q < V4_D; q++) {
            zf = zf + 1 < nz ? zf + 1 : 0;
            fetch.issue(q, zf);
        }
        int slot = 0;
        for (int j = 0; j < iters; j += 2) {
            int fs = slot + V4_D < V4_RS ? slot + V4_D : slot + V4_D - V4_RS;
            v4_iter<T, 0, 32>(X, Y, Pp, ring, slot, fs, sbase + buf * SB, fetch, dst, row, gx0, gx1, pair,
                          zf, nz, plane, j >= 2 * T, za - 2 * T + j, omask, lane, warp, ru, rd, wu,
                          wd, r2, m6);
            buf ^= 1;
            slot = slot + 1 < V4_RS ? slot + 1 : 0;
            if (j + 1 >= iters) break;
            fs = slot + V4_D < V4_RS ? slot + V4_D : slot + V4_D - V4_RS;
            v4_iter<T, 1, 32>(X, Y, Pp, ring, slot, fs, sbase + buf * SB, fetch, dst, row, gx0, gx1, pair,
                          zf, nz, plane, j + 1 >= 2 * T, za - 2 * T + j + 1, omask, lane, warp, ru,
                          rd, wu, wd, r2, m6);
            buf ^= 1;
            slot = slot + 1 < V4_RS ? slot + 1 : 0;
        }
        // the copies fetched past the segment land before the ring is reused
        fetch.drain();
        __syncthreads();
    }
}

template <int T>
cudaError_t v4_launch(unsigned g, const float *src, float *dst, int nz, int ny, int nx, float r,
                      cudaStream_t s) {
    constexpr size_t smem = v4_smem_bytes<T>();
    static std::atomic<uint64_t> attr{0};
    cudaError_t e = smem_optin(k_heat3d_v4<T>, (int)smem, attr);
    if (e != cudaSuccess) return e;
    k_heat3d_v4<T><<<g, V3_NW * 32, smem, s>>>(src, dst, nz, ny, nx, r);
    return cudaGetLastError();
}

// Form 6: form 4 with packed narrow tiles.  Along each axis, full regions
// are 64 cells wide (a warp's 32 lanes x 2 columns, or 16 warps x 4 rows)
// and store their 64 - 2T central cells; the axis holds floor(n / (64 - 2T))
// of them and the remainder goes to narrow regions 16 cells wide (8 lanes,
// or 4 warps) that store 16 - 2T.  A CTA runs narrow regions four (narrow in
// both axes: sixteen) at a time side by side in its lane segments and warp
// groups, so no CTA computes a whole region for a few remaining columns:
// 512 = 9 x 56 + 8 at T = 4 gives 88 region-sized units per plane instead
// of the 100 of form 4.  Units: full x full (one region); narrow-x x full-y
// (one narrow x tile, four y tiles in the four lane segments); full-x x
// narrow-y (four x tiles in the four warp groups, one narrow y tile);
// narrow x narrow (four x tiles by segment, four y tiles by group).
//
// The tiling of a launch, computed on the host and passed by value (kernel
// parameters stay in the constant bank, so they cost no registers in the
// register-bound level chain).  The units whose regions are 64 columns wide
// take the CTAs [0, ctas_wide) and exchange x neighbours across all 32
// lanes; the narrow-x units take the remaining CTAs, their lanes split into
// segments of 8.  Each group splits its (unit, plane) pairs evenly over its
// CTAs.
struct Tiling3 {
    int fx, fy, nxn, nyn;       // full and narrow tiles per axis
    int fx4, fy4, nxn4, nyn4;   // the same in blocks of four (rounded up)
    int ff, fn, nf, nn;         // units of each kind per plane
    int ctas_wide;
    // form 7: full x full tiles whose regions lie inside the field (no
    // periodic wrap), x tiles [ia, ia + nix) by y tiles [ja, ja + niy),
    // fetched by TMA in CTAs [0, ctas_tma); the other ne = ff - nix*niy full
    // tiles and the full-x narrow-y units in CTAs [ctas_tma, ctas_wide)
    int ia, nix, ja, niy, ne, ctas_tma;
};

inline Tiling3 tiling3(int ny, int nx, int T) {
    const int fw = 64 - 2 * T, nw = 16 - 2 * T;
    Tiling3 t;
    t.fx = nx / fw;
    t.fy = ny / fw;
    t.nxn = (nx - t.fx * fw + nw - 1) / nw;
    t.nyn = (ny - t.fy * fw + nw - 1) / nw;
    t.fx4 = (t.fx + 3) / 4;
    t.fy4 = (t.fy + 3) / 4;
    t.nxn4 = (t.nxn + 3) / 4;
    t.nyn4 = (t.nyn + 3) / 4;
    t.ff = t.fx * t.fy;
    t.fn = t.fx4 * t.nyn;
    t.nf = t.nxn * t.fy4;
    t.nn = t.nxn4 * t.nyn4;
    t.ctas_wide = 0;
    t.ia = t.nix = t.ja = t.niy = 0;
    t.ne = t.ff;
    t.ctas_tma = 0;
    return t;
}

// Interior tiles of an axis of n cells: those whose 64-cell region starts
// at or after 0 and ends at or before n.
inline void interior3(int n, int full, int T, int *lo, int *cnt) {
    const int fw = 64 - 2 * T;
    const int a = (T + fw - 1) / fw;                 // first i with i*fw - T >= 0
    const int b = n + T - 64 >= 0 ? (n + T - 64) / fw : -1;  // last i ending inside
    const int hi = std::min(b, full - 1);
    *lo = a;
    *cnt = hi >= a ? hi - a + 1 : 0;
}

// Region of unit u for this thread: output origin (ox, oy), stored extent
// wx x hy, gw warps per region, and whether the thread's slot holds a region
// at all, packed as (ox, oy, wx | hy << 8, gw | valid << 8).  An empty slot
// gets an origin inside the field and stores nothing.
template <int T, int SW>
__device__ __forceinline__ int4 v6_decode(int u, int ny, int nx, const Tiling3 &tl, int lane,
                                          int warp) {
    constexpr int FW = 64 - 2 * T, NWD = 16 - 2 * T;
    int i, j, ox, oy, gw;
    bool valid;
    if (SW == 32) {
        if (u < tl.ff) {
            i = u % tl.fx;
            j = u / tl.fx;
            valid = true;
            oy = j * FW;
            gw = V3_NW;
        } else {
            u -= tl.ff;
            i = 4 * (u % tl.fx4) + warp / 4;
            j = u / tl.fx4;
            valid = i < tl.fx;
            oy = tl.fy * FW + j * NWD;
            gw = 4;
        }
        ox = i * FW;
    } else {
        if (u < tl.nf) {
            i = u % tl.nxn;
            j = 4 * (u / tl.nxn) + lane / 8;
            valid = j < tl.fy;
            oy = j * FW;
            gw = V3_NW;
        } else {
            u -= tl.nf;
            i = 4 * (u % tl.nxn4) + lane / 8;
            j = 4 * (u / tl.nxn4) + warp / 4;
            valid = i < tl.nxn && j < tl.nyn;
            oy = tl.fy * FW + j * NWD;
            gw = 4;
        }
        ox = tl.fx * FW + i * NWD;
    }
    const int wx = valid ? min(SW == 32 ? FW : NWD, nx - ox) : 0;
    const int hy = valid ? min(gw == V3_NW ? FW : NWD, ny - oy) : 0;
    if (!valid) ox = oy = T;
    return make_int4(ox, oy, wx | (hy << 8), gw | ((valid ? 1 : 0) << 8));
}

// All iterations of one unit over planes [za, zb) with the ring filled by
// `fetch`.  Returns false when the fetch failed (form 7's bounded waits).
template <int T, int SW, class F>
__device__ __forceinline__ bool unit_loop(F &fetch, f2 *__restrict__ ring, f2 *__restrict__ sbase,
                                          int &buf, float *__restrict__ dst,
                                          const unsigned (&row)[4], unsigned gx0, unsigned gx1,
                                          bool pair, int nz, size_t plane, int za, int zb,
                                          unsigned omask, int lane, int warp, int ru, int rd,
                                          int wu, int wd, f2 r2, f2 m6) {
    constexpr int SB = (T > 1 ? T - 1 : 1) * V3_NW * 2 * 32;
    f2 X[T][4], Y[T][4], Pp[T][4];
#pragma unroll
    for (int t = 0; t < T; t++)
#pragma unroll
        for (int k = 0; k < 4; k++) X[t][k] = Y[t][k] = Pp[t][k] = 0ull;
    // iteration j receives level-0 plane za - T + j (ring slot j % V4_RS)
    // and emits level-T plane za - 2T + j (stored for j >= 2T)
    const int iters = (zb - za) + 2 * T;
    int zf = wrapi(za - T, nz);
    fetch.issue(0, zf);
#pragma unroll
    for (int q = 1; q < V4_D; q++) {
        zf = zf + 1 < nz ? zf + 1 : 0;
        fetch.issue(q, zf);
    }
    int slot = 0;
    for (int j = 0; j < iters; j += 2) {
        int fs = slot + V4_D < V4_RS ? slot + V4_D : slot + V4_D - V4_RS;
        v4_iter<T, 0, SW>(X, Y, Pp, ring, slot, fs, sbase + buf * SB, fetch, dst, row, gx0, gx1,
                          pair, zf, nz, plane, j >= 2 * T, za - 2 * T + j, omask, lane, warp, ru,
                          rd, wu, wd, r2, m6);
        buf ^= 1;
        slot = slot + 1 < V4_RS ? slot + 1 : 0;
        if (j + 1 >= iters || fetch.failed) break;
        fs = slot + V4_D < V4_RS ? slot + V4_D : slot + V4_D - V4_RS;
        v4_iter<T, 1, SW>(X, Y, Pp, ring, slot, fs, sbase + buf * SB, fetch, dst, row, gx0, gx1,
                          pair, zf, nz, plane, j + 1 >= 2 * T, za - 2 * T + j + 1, omask, lane,
                          warp, ru, rd, wu, wd, r2, m6);
        buf ^= 1;
        slot = slot + 1 < V4_RS ? slot + 1 : 0;
        if (fetch.failed) break;
    }
    // the copies fetched past the segment land before the ring is reused
    fetch.drain();
    __syncthreads();
    return !fetch.failed;
}

// Form 7's decodes.  G = 2: interior full x full tiles (i, j) in
// [ia, ia + nix) x [ja, ja + niy).  G = 3: the other full x full tiles (the
// rows of tiles outside [ja, ja + niy), then the columns outside
// [ia, ia + nix) of the rows inside), then the full-x narrow-y units.
template <int T, int G>
__device__ __forceinline__ int4 v7_decode(int u, int ny, int nx, const Tiling3 &tl, int lane,
                                          int warp) {
    constexpr int FW = 64 - 2 * T;
    if (G == 2) {
        const int ox = (tl.ia + u % tl.nix) * FW, oy = (tl.ja + u / tl.nix) * FW;
        return make_int4(ox, oy, min(FW, nx - ox) | (min(FW, ny - oy) << 8), V3_NW | (1 << 8));
    }
    if (u >= tl.ne) return v6_decode<T, 32>(u - tl.ne + tl.ff, ny, nx, tl, lane, warp);
    int i, j;
    const int rows_out = (tl.fy - tl.niy) * tl.fx;
    if (u < rows_out) {
        const int jj = u / tl.fx;
        j = jj < tl.ja ? jj : jj + tl.niy;
        i = u % tl.fx;
    } else {
        const int k = u - rows_out, ncol = tl.fx - tl.nix;
        j = tl.ja + k / ncol;
        const int ii = k % ncol;
        i = ii < tl.ia ? ii : ii + tl.nix;
    }
    const int ox = i * FW, oy = j * FW;
    return make_int4(ox, oy, min(FW, nx - ox) | (min(FW, ny - oy) << 8), V3_NW | (1 << 8));
}

// The (unit, plane) pairs [w0, w1) of one group of CTAs.  G = 0: form 6's
// wide units, 1: the narrow-x units (both forms), 2: form 7's interior
// tiles (TMA), 3: form 7's other wide units.  SW = lanes per region in x.
template <int T, int SW, int G>
__device__ __forceinline__ void units_run(const float *__restrict__ src, float *__restrict__ dst,
                                          int nz, int ny, int nx, float r, const Tiling3 &tl,
                                          int64_t w0, int64_t w1, const CUtensorMap *map) {
    extern __shared__ __align__(128) f2 v4_smem[];
    __shared__ __align__(8) unsigned long long tma_bar[V4_RS];
    f2 *ring = v4_smem;
    f2 *sbase = v4_smem + (size_t)V4_RS * V3_H * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t plane = (size_t)ny * nx;
    const f2 r2 = pk(r, r), m6 = pk(-6.0f, -6.0f);
    int buf = 0;
    unsigned tma_bars = 0, tma_phase = 0;
    if constexpr (G == 2) {
        tma_bars = (unsigned)__cvta_generic_to_shared(tma_bar);
        if (threadIdx.x == 0) {
            for (int sl = 0; sl < V4_RS; sl++)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tma_bars + 8u * sl)
                             : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }

    for (int64_t w = w0; w < w1;) {
        int64_t u = w / nz;
        const int za = (int)(w - u * nz);
        const int zb = (int)min((int64_t)nz, za + (w1 - w));
        w += zb - za;
        // this thread's region of the unit
        int4 geo;
        if constexpr (G == 0 || G == 1)
            geo = v6_decode<T, SW>((int)u, ny, nx, tl, lane, warp);
        else
            geo = v7_decode<T, G>((int)u, ny, nx, tl, lane, warp);
        const int ox = geo.x, oy = geo.y, wx = geo.z & 0xff, hy = geo.z >> 8, gw = geo.w & 0xff;
        const bool valid = (geo.w >> 8) != 0;
        const int x0 = ox - T, y0 = oy - T;
        const int ll = lane % SW, lw = warp % gw;
        const int wu = lw > 0 ? warp - 1 : warp, wd = lw + 1 < gw ? warp + 1 : warp;
        const int ru = lw > 0 ? 4 * warp - 1 : 4 * warp, rd = lw + 1 < gw ? 4 * warp + 4 : 4 * warp + 3;
        const int c0 = 2 * ll;
        const unsigned gx0 = wrapi(x0 + c0, nx), gx1 = wrapi(x0 + c0 + 1, nx);
        const bool pair = gx1 == gx0 + 1 && (gx0 & 1u) == 0 && (nx & 1) == 0;
        const bool ox0 = valid && c0 >= T && c0 < T + wx;
        const bool ox1 = valid && c0 + 1 >= T && c0 + 1 < T + wx;
        unsigned row[4], omask = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int q = 4 * lw + k;
            row[k] = (unsigned)wrapi(y0 + q, ny) * (unsigned)nx;
            const bool oy_ = q >= T && q < T + hy;
            omask |= (oy_ && ox0 ? 1u : 0u) << (2 * k);
            omask |= (oy_ && ox1 ? 2u : 0u) << (2 * k);
        }

        if constexpr (G == 2) {
            TmaFetch fetch{ring, map, tma_bars, x0, y0, tma_phase, 0u, 0};
            const bool ok = unit_loop<T, SW>(fetch, ring, sbase, buf, dst, row, gx0, gx1, pair, nz,
                                             plane, za, zb, omask, lane, warp, ru, rd, wu, wd, r2,
                                             m6);
            tma_phase = fetch.phase;
            if (!ok) return;  // a bounded wait ran out (recorded): leave
        } else {
            CpFetch fetch{ring, src, plane, row, gx0, gx1, pair, lane, warp};
            unit_loop<T, SW>(fetch, ring, sbase, buf, dst, row, gx0, gx1, pair, nz, plane, za, zb,
                             omask, lane, warp, ru, rd, wu, wd, r2, m6);
        }
    }
}

template <int T>
__global__ void __launch_bounds__(V3_NW * 32, 1)
    k_heat3d_v6(const float *__restrict__ src, float *__restrict__ dst, int nz, int ny, int nx,
                float r, const Tiling3 tl) {
    const int64_t work_wide = (int64_t)(tl.ff + tl.fn) * nz;
    const int64_t work_narrow = (int64_t)(tl.nf + tl.nn) * nz;
    const int64_t b = blockIdx.x;
    if (b < tl.ctas_wide) {
        const int64_t g = tl.ctas_wide;
        units_run<T, 32, 0>(src, dst, nz, ny, nx, r, tl, work_wide * b / g,
                            work_wide * (b + 1) / g, nullptr);
    } else {
        const int64_t g = gridDim.x - tl.ctas_wide, c = b - tl.ctas_wide;
        units_run<T, 8, 1>(src, dst, nz, ny, nx, r, tl, work_narrow * c / g,
                           work_narrow * (c + 1) / g, nullptr);
    }
}

// Form 7: form 6 with the interior full tiles' planes fetched by TMA
// (CTAs [0, ctas_tma)), the other wide units in [ctas_tma, ctas_wide) and the
// narrow-x units in the rest, each group splitting its (unit, plane) pairs
// evenly over its CTAs.
template <int T>
__global__ void __launch_bounds__(V3_NW * 32, 1)
    k_heat3d_v7(const float *__restrict__ src, float *__restrict__ dst, int nz, int ny, int nx,
                float r, const Tiling3 tl, const __grid_constant__ CUtensorMap map) {
    const int64_t wt = (int64_t)tl.nix * tl.niy * nz;
    const int64_t we = (int64_t)(tl.ne + tl.fn) * nz;
    const int64_t wn = (int64_t)(tl.nf + tl.nn) * nz;
    const int64_t b = blockIdx.x;
    if (b < tl.ctas_tma) {
        const int64_t g = tl.ctas_tma;
        units_run<T, 32, 2>(src, dst, nz, ny, nx, r, tl, wt * b / g, wt * (b + 1) / g, &map);
    } else if (b < tl.ctas_wide) {
        const int64_t g = tl.ctas_wide - tl.ctas_tma, c = b - tl.ctas_tma;
        units_run<T, 32, 3>(src, dst, nz, ny, nx, r, tl, we * c / g, we * (c + 1) / g, nullptr);
    } else {
        const int64_t g = gridDim.x - tl.ctas_wide, c = b - tl.ctas_wide;
        units_run<T, 8, 1>(src, dst, nz, ny, nx, r, tl, wn * c / g, wn * (c + 1) / g, nullptr);
    }
}

template <int T>
cudaError_t v6_launch(unsigned g, const float *src, float *dst, int nz, int ny, int nx, float r,
                      cudaStream_t s) {
    constexpr size_t smem = v4_smem_bytes<T>();
    static std::atomic<uint64_t> attr{0};
    cudaError_t e = smem_optin(k_heat3d_v6<T>, (int)smem, attr);
    if (e != cudaSuccess) return e;
    Tiling3 tl = tiling3(ny, nx, T);
    // CTAs in proportion to the work of the two groups (each group with
    // work gets at least one CTA)
    const int64_t wide = tl.ff + tl.fn, narrow = tl.nf + tl.nn;
    if (narrow == 0) {
        tl.ctas_wide = (int)g;
    } else if (wide == 0) {
        tl.ctas_wide = 0;
    } else {
        if (g < 2) g = 2;
        const int64_t cw = (int64_t)g * wide / (wide + narrow);
        tl.ctas_wide = (int)std::max<int64_t>(1, std::min<int64_t>(g - 1, cw));
    }
    k_heat3d_v6<T><<<g, V3_NW * 32, smem, s>>>(src, dst, nz, ny, nx, r, tl);
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link to
// the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Splits g CTAs over groups with the given work in proportion (a group with
// work gets at least one CTA; g is raised to the number of such groups).
void split_ctas(unsigned &g, const int64_t (&work)[3], int (&ctas)[3]) {
    int need = 0;
    for (int64_t w : work) need += w > 0;
    if ((int)g < need) g = (unsigned)need;
    int64_t total = work[0] + work[1] + work[2];
    int left = (int)g;
    for (int k = 0; k < 3; k++) {
        if (work[k] == 0) {
            ctas[k] = 0;
            continue;
        }
        int later = 0;  // groups after this one that still need a CTA
        for (int q = k + 1; q < 3; q++) later += work[q] > 0;
        int c = (int)std::max<int64_t>(1, (int64_t)g * work[k] / std::max<int64_t>(1, total));
        c = std::min(c, left - later);
        if (later == 0) c = left;
        ctas[k] = c;
        left -= c;
    }
}

template <int T>
cudaError_t v7_launch(unsigned g, const float *src, float *dst, int nz, int ny, int nx, float r,
                      cudaStream_t s) {
    constexpr size_t smem = v4_smem_bytes<T>();
    static std::atomic<uint64_t> attr{0};
    cudaError_t e = smem_optin(k_heat3d_v7<T>, (int)smem, attr);
    if (e != cudaSuccess) return e;
    Tiling3 tl = tiling3(ny, nx, T);
    CUtensorMap map;
    memset(&map, 0, sizeof map);
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    // TMA needs 16-byte row strides and base, and every tile's x origin
    // i*(64 - 2T) - T a multiple of 4 floats (16 bytes): T = 4 only; the tile
    // must lie inside the field
    constexpr bool aligned_origins = (64 - 2 * T) % 4 == 0 && T % 4 == 0;
    if (aligned_origins && enc && nx % 4 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0) {
        interior3(nx, tl.fx, T, &tl.ia, &tl.nix);
        interior3(ny, tl.fy, T, &tl.ja, &tl.niy);
        if (tl.nix > 0 && tl.niy > 0) {
            const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
            const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
            const cuuint32_t box[3] = {64, 64, 1}, estr[3] = {1, 1, 1};
            if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(src), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                tl.nix = tl.niy = 0;
        } else {
            tl.nix = tl.niy = 0;
        }
    }
    tl.ne = tl.ff - tl.nix * tl.niy;
    const int64_t work[3] = {(int64_t)tl.nix * tl.niy, (int64_t)tl.ne + tl.fn,
                             (int64_t)tl.nf + tl.nn};
    int ctas[3];
    split_ctas(g, work, ctas);
    tl.ctas_tma = ctas[0];
    tl.ctas_wide = ctas[0] + ctas[1];
    k_heat3d_v7<T><<<g, V3_NW * 32, smem, s>>>(src, dst, nz, ny, nx, r, tl, map);
    return cudaGetLastError();
}

// Units of work per plane of form 6.
int64_t v6_units(int ny, int nx, int T) {
    const Tiling3 t = tiling3(ny, nx, T);
    return (int64_t)t.ff + t.fn + t.nf + t.nn;
}

int heat3d_blocks(int nz, int ny, int nx, int T, int zchunk) {
    const int BX = RX - 2 * T, BY = RY - 2 * T;
    return ((nx + BX - 1) / BX) * ((ny + BY - 1) / BY) * ((nz + zchunk - 1) / zchunk);
}

// ---------------------------------------------------------------------------
// Form 5, one step per launch: a streaming kernel.  A thread owns 4 adjacent
// x cells of one row (16-byte loads and stores; nx % 4 == 0) and walks a
// chunk of S1_ZC planes with the planes z-1, z and z+1 of its cells in
// registers.  The x neighbours beyond its 4 cells come from the adjacent
// lanes by shuffles (a lane at the warp's or the field's x end loads its
// own, wrapped), the y neighbours are 16-byte loads of the rows above and
// below (wrapped), which the warps holding those rows load as their own, so
// they are mostly L1 and L2 hits.  Arithmetic on paired FP32 instructions in
// the canonical order.  Grid: (nx / 128 rounded up, ny / S1_ROWS rounded up,
// nz / S1_ZC rounded up) CTAs of 32 x S1_ROWS threads.
namespace {
constexpr int S1_ROWS = 8, S1_ZC = 64;

__device__ __forceinline__ ulonglong2 ld16(const float *p) {
    return __ldg(reinterpret_cast<const ulonglong2 *>(p));
}
}  // namespace

__global__ void __launch_bounds__(32 * S1_ROWS) k_heat3d_s1(const float *__restrict__ src,
                                                           float *__restrict__ dst, int nz, int ny,
                                                           int nx, float r) {
    const int lane = threadIdx.x & 31;
    const int x = (blockIdx.x * 32 + lane) * 4;
    const int y = blockIdx.y * S1_ROWS + (threadIdx.x >> 5);
    const int z0 = blockIdx.z * S1_ZC, z1 = min(nz, z0 + S1_ZC);
    const bool active = x < nx && y < ny;
    const int yy = active ? y : 0, xx = active ? x : 0;
    const int ym = yy == 0 ? ny - 1 : yy - 1, yp = yy + 1 == ny ? 0 : yy + 1;
    const size_t plane = (size_t)ny * nx;
    const size_t oc = (size_t)yy * nx + xx, om = (size_t)ym * nx + xx, op = (size_t)yp * nx + xx;
    // x neighbours: shuffled from the adjacent lane when it holds them, else loaded
    const bool own_l = lane == 0, own_r = lane == 31 || x + 4 >= nx;
    const size_t ol = (size_t)yy * nx + (xx == 0 ? nx - 1 : xx - 1);
    const size_t orr = (size_t)yy * nx + (xx + 4 >= nx ? 0 : xx + 4);
    const f2 r2 = pk(r, r), m6 = pk(-6.0f, -6.0f);
    auto wz = [nz](int z) { return z >= nz ? z - nz : (z < 0 ? z + nz : z); };
    // planes z-1, z, z+1 of the thread's cells, the rows above and below and
    // the loaded x neighbours of plane z; every load is issued one plane ahead
    ulonglong2 zm = {0ull, 0ull}, u = {0ull, 0ull}, zp = {0ull, 0ull}, a = {0ull, 0ull},
               b = {0ull, 0ull};
    float xl = 0.0f, xr = 0.0f;
    if (active) {
        const float *pz = src + plane * (size_t)z0;
        zm = ld16(src + plane * (size_t)wz(z0 - 1) + oc);
        u = ld16(pz + oc);
        zp = ld16(src + plane * (size_t)wz(z0 + 1) + oc);
        a = ld16(pz + om);
        b = ld16(pz + op);
        if (own_l) xl = __ldg(pz + ol);
        if (own_r) xr = __ldg(pz + orr);
    }
    for (int z = z0; z < z1; z++) {
        ulonglong2 pre = {0ull, 0ull}, na = {0ull, 0ull}, nb = {0ull, 0ull};
        float nxl = 0.0f, nxr = 0.0f;
        if (active && z + 1 < z1) {
            const float *pn = src + plane * (size_t)wz(z + 1);
            pre = ld16(src + plane * (size_t)wz(z + 2) + oc);
            na = ld16(pn + om);
            nb = ld16(pn + op);
            if (own_l) nxl = __ldg(pn + ol);
            if (own_r) nxr = __ldg(pn + orr);
        }
        const float sl = __shfl_up_sync(0xffffffffu, hi_of(u.y), 1);
        const float sr = __shfl_down_sync(0xffffffffu, lo_of(u.x), 1);
        // cells (c0, c1) = u.x, (c2, c3) = u.y
        const f2 xmA = pk(own_l ? xl : sl, lo_of(u.x)), xpA = pk(hi_of(u.x), lo_of(u.y));
        const f2 xpB = pk(hi_of(u.y), own_r ? xr : sr);
        const f2 sA = add2(add2(add2(add2(xmA, xpA), add2(a.x, b.x)), zm.x), zp.x);
        const f2 sB = add2(add2(add2(add2(xpA, xpB), add2(a.y, b.y)), zm.y), zp.y);
        ulonglong2 o;
        o.x = fma2(r2, fma2(m6, u.x, sA), u.x);
        o.y = fma2(r2, fma2(m6, u.y, sB), u.y);
        if (active) *reinterpret_cast<ulonglong2 *>(dst + plane * (size_t)z + oc) = o;
        zm = u;
        u = zp;
        zp = pre;
        a = na;
        b = nb;
        xl = nxl;
        xr = nxr;
    }
}

// z chunk length: split z so that the CTA count fills whole waves of one
// CTA per SM (each extra chunk re-reads 3T-1 planes).
int heat3d_default_zchunk(int nz, int ny, int nx, int T) {
    const int sms = sm_count();
    int best = nz;
    double best_eff = 0;
    for (int nch = 1; nch <= 16 && nch <= nz; nch++) {
        const int zc = (nz + nch - 1) / nch;
        const int blocks = heat3d_blocks(nz, ny, nx, T, zc);
        const int waves = (blocks + sms - 1) / sms;
        const double fill = (double)blocks / ((double)waves * sms);
        const double halo = (double)zc / (zc + 3 * T - 1);
        const double eff = fill * halo;
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = zc;
        }
    }
    return best;
}

cudaError_t heat3d(const float *src, float *dst, int nz, int ny, int nx, float r, int steps,
                   int zchunk, const hxc_launch_cfg *cfg, cudaStream_t s) {
    if (steps < 1 || steps > 4) return cudaErrorInvalidValue;
    if (zchunk <= 0) {
        const int nch = (int)tune::get("heat3d.zchunks");
        zchunk = nch > 0 ? (nz + nch - 1) / nch : heat3d_default_zchunk(nz, ny, nx, steps);
    }
    const int blocks = heat3d_blocks(nz, ny, nx, steps, zchunk);
    unsigned g = cfg ? cfg->grid[0] * cfg->grid[1] * cfg->grid[2] : (unsigned)blocks;
    // variant 3 keeps in-plane offsets in 32 bits; larger planes take variant 2 (same bits)
    // one-step launches have a knob of their own: with a single level the
    // copied-plane form streams faster than the two-plane forms
    const int64_t variant = tune::get(steps == 1 ? "heat3d.variant1" : "heat3d.variant");
    if (variant == 5 && steps == 1 && !cfg && nx % 4 == 0 && (ny + S1_ROWS - 1) / S1_ROWS <= 65535 &&
        (nz + S1_ZC - 1) / S1_ZC <= 65535 && reinterpret_cast<uintptr_t>(src) % 16 == 0 &&
        reinterpret_cast<uintptr_t>(dst) % 16 == 0) {
        dim3 grid((unsigned)((nx + 127) / 128), (unsigned)((ny + S1_ROWS - 1) / S1_ROWS),
                  (unsigned)((nz + S1_ZC - 1) / S1_ZC));
        k_heat3d_s1<<<grid, 32 * S1_ROWS, 0, s>>>(src, dst, nz, ny, nx, r);
        return cudaGetLastError();
    }
    if (variant >= 3 && (uint64_t)ny * (uint64_t)nx <= 0xffffffffull) {
        if (cfg && cfg->block[0] * cfg->block[1] * cfg->block[2] != V3_NW * 32)
            return cudaErrorInvalidValue;
        const int BX = 64 - 2 * steps, BY = V3_H - 2 * steps;
        int64_t work = (int64_t)((nx + BX - 1) / BX) * ((ny + BY - 1) / BY) * nz;
        if (variant >= 6) work = v6_units(ny, nx, steps) * nz;
        const unsigned g3 = cfg ? g : (unsigned)std::min<int64_t>(sm_count(), work);
        if (variant == 7) {
            switch (steps) {
                case 1: return v7_launch<1>(g3, src, dst, nz, ny, nx, r, s);
                case 2: return v7_launch<2>(g3, src, dst, nz, ny, nx, r, s);
                case 3: return v7_launch<3>(g3, src, dst, nz, ny, nx, r, s);
                case 4: return v7_launch<4>(g3, src, dst, nz, ny, nx, r, s);
            }
        }
        if (variant == 6) {
            switch (steps) {
                case 1: return v6_launch<1>(g3, src, dst, nz, ny, nx, r, s);
                case 2: return v6_launch<2>(g3, src, dst, nz, ny, nx, r, s);
                case 3: return v6_launch<3>(g3, src, dst, nz, ny, nx, r, s);
                case 4: return v6_launch<4>(g3, src, dst, nz, ny, nx, r, s);
            }
        }
        if (variant == 4) {
            switch (steps) {
                case 1: return v4_launch<1>(g3, src, dst, nz, ny, nx, r, s);
                case 2: return v4_launch<2>(g3, src, dst, nz, ny, nx, r, s);
                case 3: return v4_launch<3>(g3, src, dst, nz, ny, nx, r, s);
                case 4: return v4_launch<4>(g3, src, dst, nz, ny, nx, r, s);
            }
        }
        switch (steps) {
            case 1: return v3_launch<1>(g3, src, dst, nz, ny, nx, r, s);
            case 2: return v3_launch<2>(g3, src, dst, nz, ny, nx, r, s);
            case 3: return v3_launch<3>(g3, src, dst, nz, ny, nx, r, s);
            case 4: return v3_launch<4>(g3, src, dst, nz, ny, nx, r, s);
        }
    }
    if (cfg && cfg->block[0] * cfg->block[1] * cfg->block[2] != NT) return cudaErrorInvalidValue;
    switch (steps) {
        case 1: k_heat3d_pk<1><<<g, NT, 0, s>>>(src, dst, nz, ny, nx, r, zchunk); break;
        case 2: k_heat3d_pk<2><<<g, NT, 0, s>>>(src, dst, nz, ny, nx, r, zchunk); break;
        case 3: k_heat3d_pk<3><<<g, NT, 0, s>>>(src, dst, nz, ny, nx, r, zchunk); break;
        case 4: k_heat3d_pk<4><<<g, NT, 0, s>>>(src, dst, nz, ny, nx, r, zchunk); break;
    }
    return cudaGetLastError();
}

cudaError_t heat3d_wait_errors(unsigned *flags) {
    unsigned v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_heat3d_wait_errors, sizeof v);
    if (e == cudaSuccess && v) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbol(g_heat3d_wait_errors, &zero, sizeof zero);
    }
    if (flags) *flags = v;
    return e;
}

}  // namespace k
}  // namespace hxc
