// 3D 7-point FTCS, FP32, periodic, T (1..4) fused steps per launch.
//
// Canonical arithmetic (every variant, every T):
//   s  = ((u[x-1] + u[x+1]) + (u[y-1] + u[y+1])) + (u[z-1] + u[z+1])
//   t  = fma(-6, u, s);   u' = fma(r, t, u)            (FP32, round-to-nearest)
// so T fused steps give the same bits as T single-step launches.
//
// Temporal blocking.  A CTA owns an x-y region of RX x RY = 64 x 32 columns
// (its output tile plus a halo of T columns on every side) and streams it
// along z.  Level t (the field after t steps) is kept per thread in
// registers for three consecutive planes (z-1, z, z+1) of the 2 x 2 columns
// the thread owns; x-neighbours come from the adjacent lanes by shuffles and
// y-neighbours from a shared-memory copy of the level's middle plane.  In
// every iteration a new level-0 plane is loaded and each level t < T
// produces one plane of level t+1; the levels advance together (their
// inputs are the registers and shared planes at the start of the
// iteration), so level t runs 2t planes behind level 0; the shared planes
// are double-buffered so that one barrier per plane suffices.  Cells within
// distance t of the region edge are wrong at level t and are never written:
// only the central (RX-2T) x (RY-2T) columns of level T are stored.
#include "kernels.cuh"

namespace hxc {
namespace k {

namespace {
constexpr int RX = 64, RY = 32, NT = 512;

__device__ __forceinline__ float ftcs7(float u, float xm, float xp, float ym, float yp, float zm,
                                       float zp, float r) {
    float s = __fadd_rn(__fadd_rn(__fadd_rn(xm, xp), __fadd_rn(ym, yp)), __fadd_rn(zm, zp));
    float t = __fmaf_rn(-6.0f, u, s);
    return __fmaf_rn(r, t, u);
}

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}
}  // namespace

// Register ring: R[t][slot][c] holds level t at the plane whose sequence
// number is congruent to `slot` mod 3 (4 columns c of the thread).  The
// main loop is unrolled by three so that every slot index is a compile-time
// constant and no register is ever copied.
//
// Iteration i (phase ph = i mod 3): level 0 holds planes i-2, i-1, i of its
// sequence (slots ph+1, ph+2, ph); every level t >= 1 holds planes i-3, i-2,
// i-1 of its own sequence (slots ph, ph+1, ph+2).  The middle planes go to
// shared memory (double-buffered by iteration parity, so one barrier per
// iteration suffices), then the levels advance from the top down: level
// t+1's new plane goes into its slot ph, which level t+1 has just read.
template <int T, int PH>
__device__ __forceinline__ void heat3d_iter(float (&R)[T][3][4], float (*S)[T][RY][RX],
                                            const float *__restrict__ src, float *__restrict__ dst,
                                            size_t plane, size_t o00, size_t o01, size_t o10,
                                            size_t o11, int i, int iters, int &zload, int nz,
                                            int zout0, int z0, int z1, bool ox0, bool ox1, bool oy0,
                                            bool oy1, float r, int rx, int ry, int ryu, int ryd) {
    constexpr int P0 = (PH + 1) % 3, M0 = (PH + 2) % 3, N0 = PH;   // level 0
    constexpr int PT = PH, MT = (PH + 1) % 3, NT_ = (PH + 2) % 3;  // levels >= 1
    const int b = i & 1;
    *reinterpret_cast<float2 *>(&S[b][0][ry][rx]) = make_float2(R[0][M0][0], R[0][M0][1]);
    *reinterpret_cast<float2 *>(&S[b][0][ry + 1][rx]) = make_float2(R[0][M0][2], R[0][M0][3]);
#pragma unroll
    for (int t = 1; t < T; t++) {
        *reinterpret_cast<float2 *>(&S[b][t][ry][rx]) = make_float2(R[t][MT][0], R[t][MT][1]);
        *reinterpret_cast<float2 *>(&S[b][t][ry + 1][rx]) = make_float2(R[t][MT][2], R[t][MT][3]);
    }
    __syncthreads();
    // prefetch level 0's next plane (stored into the ring at the end)
    float nxt[4];
    const bool more = i + 1 < iters;
    if (more) {
        const size_t zo = (size_t)zload * plane;
        nxt[0] = __ldg(src + zo + o00);
        nxt[1] = __ldg(src + zo + o01);
        nxt[2] = __ldg(src + zo + o10);
        nxt[3] = __ldg(src + zo + o11);
        if (++zload == nz) zload = 0;
    }
#pragma unroll
    for (int t = T - 1; t >= 0; t--) {
        const int Pt = t == 0 ? P0 : PT, Mt = t == 0 ? M0 : MT, Nt = t == 0 ? N0 : NT_;
        const float2 up = *reinterpret_cast<const float2 *>(&S[b][t][ryu][rx]);
        const float2 dn = *reinterpret_cast<const float2 *>(&S[b][t][ryd][rx]);
        const float m0 = R[t][Mt][0], m1 = R[t][Mt][1], m2 = R[t][Mt][2], m3 = R[t][Mt][3];
        const float l0 = __shfl_up_sync(0xffffffffu, m1, 1);
        const float r0 = __shfl_down_sync(0xffffffffu, m0, 1);
        const float l1 = __shfl_up_sync(0xffffffffu, m3, 1);
        const float r1 = __shfl_down_sync(0xffffffffu, m2, 1);
        const float v0 = ftcs7(m0, l0, m1, up.x, m2, R[t][Pt][0], R[t][Nt][0], r);
        const float v1 = ftcs7(m1, m0, r0, up.y, m3, R[t][Pt][1], R[t][Nt][1], r);
        const float v2 = ftcs7(m2, l1, m3, m0, dn.x, R[t][Pt][2], R[t][Nt][2], r);
        const float v3 = ftcs7(m3, m2, r1, m1, dn.y, R[t][Pt][3], R[t][Nt][3], r);
        if (t + 1 < T) {
            R[t + 1][PH][0] = v0;
            R[t + 1][PH][1] = v1;
            R[t + 1][PH][2] = v2;
            R[t + 1][PH][3] = v3;
        } else {
            // level T: the output plane
            const int zout = zout0 + i;
            if (zout >= z0 && zout < z1) {
                float *d = dst + (size_t)zout * plane;
                if (oy0 && ox0) d[o00] = v0;
                if (oy0 && ox1) d[o01] = v1;
                if (oy1 && ox0) d[o10] = v2;
                if (oy1 && ox1) d[o11] = v3;
            }
        }
    }
    if (more) {
        constexpr int NX = (PH + 1) % 3;  // the slot the next phase calls N0
        R[0][NX][0] = nxt[0];
        R[0][NX][1] = nxt[1];
        R[0][NX][2] = nxt[2];
        R[0][NX][3] = nxt[3];
    }
}

template <int T>
__global__ void __launch_bounds__(NT, 1)
    k_heat3d_tb(const float *__restrict__ src, float *__restrict__ dst, int nz, int ny, int nx,
                float r, int zchunk) {
    constexpr int BX = RX - 2 * T, BY = RY - 2 * T;
    // two buffers of the T middle planes (dynamic: 64 KB for T = 4)
    extern __shared__ __align__(16) float sm3[];
    float(*S)[T][RY][RX] = reinterpret_cast<float(*)[T][RY][RX]>(sm3);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tiles_x = (nx + BX - 1) / BX, tiles_y = (ny + BY - 1) / BY;
    const int nchunks = (nz + zchunk - 1) / zchunk;
    const int nblk = tiles_x * tiles_y * nchunks;
    const int rx = 2 * lane, ry = 2 * warp;
    // rows of the neighbouring warps (clamped inside the region: the clamped
    // rows only feed cells that are never stored)
    const int ryu = ry > 0 ? ry - 1 : 0, ryd = ry + 2 < RY ? ry + 2 : RY - 1;

    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const int tx = blk % tiles_x, ty = (blk / tiles_x) % tiles_y, ch = blk / (tiles_x * tiles_y);
        const int x0 = tx * BX - T, y0 = ty * BY - T;
        const int z0 = ch * zchunk, z1 = min(nz, z0 + zchunk);
        const int gx0 = wrapi(x0 + rx, nx), gx1 = wrapi(x0 + rx + 1, nx);
        const int gy0 = wrapi(y0 + ry, ny), gy1 = wrapi(y0 + ry + 1, ny);
        // output columns of this thread (inside the tile and the field)
        const bool ox0 = rx >= T && rx < RX - T && x0 + rx < nx;
        const bool ox1 = rx + 1 >= T && rx + 1 < RX - T && x0 + rx + 1 < nx;
        const bool oy0 = ry >= T && ry < RY - T && y0 + ry < ny;
        const bool oy1 = ry + 1 >= T && ry + 1 < RY - T && y0 + ry + 1 < ny;
        const size_t o00 = (size_t)gy0 * nx + gx0, o01 = (size_t)gy0 * nx + gx1;
        const size_t o10 = (size_t)gy1 * nx + gx0, o11 = (size_t)gy1 * nx + gx1;
        const size_t plane = (size_t)ny * nx;

        float R[T][3][4];
#pragma unroll
        for (int t = 0; t < T; t++)
#pragma unroll
            for (int q = 0; q < 3; q++)
#pragma unroll
                for (int c = 0; c < 4; c++) R[t][q][c] = 0.f;
        // level t+1's plane computed in iteration i is plane i - 2t - 1 of the
        // level-0 sequence, which starts at z0 - T: the output (level T) of
        // iteration i is plane z0 - 3T + 1 + i
        const int iters = (z1 - z0) + 3 * T - 1;
        int zload = wrapi(z0 - T, nz);
        {
            const size_t zo = (size_t)zload * plane;
            R[0][0][0] = __ldg(src + zo + o00);
            R[0][0][1] = __ldg(src + zo + o01);
            R[0][0][2] = __ldg(src + zo + o10);
            R[0][0][3] = __ldg(src + zo + o11);
            if (++zload == nz) zload = 0;
        }
        const int zout0 = z0 - 3 * T + 1;
        int i = 0;
        for (; i + 3 <= iters; i += 3) {
            heat3d_iter<T, 0>(R, S, src, dst, plane, o00, o01, o10, o11, i, iters, zload, nz, zout0,
                              z0, z1, ox0, ox1, oy0, oy1, r, rx, ry, ryu, ryd);
            heat3d_iter<T, 1>(R, S, src, dst, plane, o00, o01, o10, o11, i + 1, iters, zload, nz,
                              zout0, z0, z1, ox0, ox1, oy0, oy1, r, rx, ry, ryu, ryd);
            heat3d_iter<T, 2>(R, S, src, dst, plane, o00, o01, o10, o11, i + 2, iters, zload, nz,
                              zout0, z0, z1, ox0, ox1, oy0, oy1, r, rx, ry, ryu, ryd);
        }
        if (i < iters)
            heat3d_iter<T, 0>(R, S, src, dst, plane, o00, o01, o10, o11, i, iters, zload, nz, zout0,
                              z0, z1, ox0, ox1, oy0, oy1, r, rx, ry, ryu, ryd);
        if (i + 1 < iters)
            heat3d_iter<T, 1>(R, S, src, dst, plane, o00, o01, o10, o11, i + 1, iters, zload, nz,
                              zout0, z0, z1, ox0, ox1, oy0, oy1, r, rx, ry, ryu, ryd);
        __syncthreads();  // the shared planes are reused by the next block item
    }
}

int heat3d_blocks(int nz, int ny, int nx, int T, int zchunk) {
    const int BX = RX - 2 * T, BY = RY - 2 * T;
    return ((nx + BX - 1) / BX) * ((ny + BY - 1) / BY) * ((nz + zchunk - 1) / zchunk);
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

template <int T>
static cudaError_t launch3d(unsigned g, const float *src, float *dst, int nz, int ny, int nx,
                            float r, int zchunk, cudaStream_t s) {
    const size_t smem = 2 * (size_t)T * RY * RX * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_heat3d_tb<T>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_heat3d_tb<T><<<g, NT, smem, s>>>(src, dst, nz, ny, nx, r, zchunk);
    return cudaGetLastError();
}

cudaError_t heat3d(const float *src, float *dst, int nz, int ny, int nx, float r, int steps,
                   int zchunk, const hxc_launch_cfg *cfg, cudaStream_t s) {
    if (steps < 1 || steps > 4) return cudaErrorInvalidValue;
    if (zchunk <= 0) zchunk = heat3d_default_zchunk(nz, ny, nx, steps);
    const int blocks = heat3d_blocks(nz, ny, nx, steps, zchunk);
    unsigned g = cfg ? cfg->grid[0] * cfg->grid[1] * cfg->grid[2] : (unsigned)blocks;
    if (cfg && cfg->block[0] * cfg->block[1] * cfg->block[2] != NT) return cudaErrorInvalidValue;
    switch (steps) {
        case 1: return launch3d<1>(g, src, dst, nz, ny, nx, r, zchunk, s);
        case 2: return launch3d<2>(g, src, dst, nz, ny, nx, r, zchunk, s);
        case 3: return launch3d<3>(g, src, dst, nz, ny, nx, r, zchunk, s);
        case 4: return launch3d<4>(g, src, dst, nz, ny, nx, r, zchunk, s);
    }
    return cudaGetLastError();
}

}  // namespace k
}  // namespace hxc
