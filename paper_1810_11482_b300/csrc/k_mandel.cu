// Sec. 5.1.3 Mandelbrot kernel: escape-time iteration of z <- z^2 + c from
// z = 0, one pixel per thread, in binary32 with an explicit rounding
// sequence (round-to-nearest intrinsics, so the compiler fuses nothing
// else):  xx = x*x, yy = y*y, escape when xx + yy > 4,
// Im z' = fma(x + x, y, Im c), Re z' = (xx - yy) + Re c.
// Pixel (i, j) is c = (x0 + i*dx) + (y0 + j*dy) i, each step rounded.
//
// The work per pixel ranges from one iteration to max_iter, so a warp owns
// an 8 x 4 pixel tile (neighbouring pixels tend to escape together, which
// keeps the warp's lanes busy) and warps stride over the tiles of the image
// in an interleaved order, spreading the expensive interior over all SMs.
#include <algorithm>

#include "f32x2.cuh"
#include "kernels.cuh"
#include "tune.hpp"

namespace hxc {
namespace k {

namespace {

constexpr int kTileW = 8, kTileH = 4;

// One iteration from (x, y): the escape test of z_k and z_{k+1}.
struct Iter {
    float x, y;
    bool escaped;
};
__device__ __forceinline__ Iter step(float x, float y, float cr, float ci) {
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y);
    return {__fadd_rn(__fsub_rn(xx, yy), cr), __fmaf_rn(__fadd_rn(x, x), y, ci),
            __fadd_rn(xx, yy) > 4.0f};
}

// The escape count.  Iterations run in groups of four with the four escape
// tests joined into one branch; on an escape the first test that fired, in
// order, gives the count, so the result is that of testing after every
// iteration (values past the escape may overflow; they are never used).
//
// Where |c|^2 <= 3.99 an escape cannot undo itself: if |z_j| > 2 (to within
// rounding) then |z_{j+1}| >= |z_j|^2 - |c| > 2.002, far outside rounding, and
// the orbit keeps growing (three iterations past an escape stay below 1e5,
// so nothing overflows).  There only the last of every four iterates is
// tested; when it has escaped, the group is run again from its first
// iterate with a test after every iteration, which gives the exact count.
__device__ __forceinline__ bool fast_ok(float cr, float ci) {
    return __fmaf_rn(cr, cr, __fmul_rn(ci, ci)) <= 3.99f;
}

// The escape count from iterate k = (x, y), k a multiple of 4 or the start.
__device__ __forceinline__ int32_t escape_from(float x, float y, int32_t k, float cr, float ci,
                                               int32_t max_iter, bool fast) {
    if (fast) {
        for (; k + 4 <= max_iter; k += 4) {
            float px = x, py = y;
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const float xx = __fmul_rn(px, px), yy = __fmul_rn(py, py);
                const float nx = __fadd_rn(__fsub_rn(xx, yy), cr);
                py = __fmaf_rn(__fadd_rn(px, px), py, ci);
                px = nx;
            }
            const Iter d = step(px, py, cr, ci);  // tests z_{k+3}
            if (d.escaped) {
                for (;; k++) {  // the first escape in z_k .. z_{k+3}
                    const Iter a = step(x, y, cr, ci);
                    if (a.escaped) return k;
                    x = a.x;
                    y = a.y;
                }
            }
            x = d.x;
            y = d.y;
        }
    }
    for (; k + 4 <= max_iter; k += 4) {
        const Iter a = step(x, y, cr, ci);
        const Iter b = step(a.x, a.y, cr, ci);
        const Iter c = step(b.x, b.y, cr, ci);
        const Iter d = step(c.x, c.y, cr, ci);
        if (a.escaped | b.escaped | c.escaped | d.escaped)
            return k + (a.escaped ? 0 : b.escaped ? 1 : c.escaped ? 2 : 3);
        x = d.x;
        y = d.y;
    }
    for (; k < max_iter; k++) {
        const Iter a = step(x, y, cr, ci);
        if (a.escaped) return k;
        x = a.x;
        y = a.y;
    }
    return max_iter;
}

__device__ __forceinline__ int32_t escape_count(float cr, float ci, int32_t max_iter) {
    return escape_from(0.0f, 0.0f, 0, cr, ci, max_iter, fast_ok(cr, ci));
}

// Two horizontally adjacent pixels (the same ci) on paired FP32
// instructions, each half rounding exactly as the scalar step: products as
// fma(a, b, -0) and the difference as fma(yy, -1, xx), with -0 and -1 taken
// from kernel arguments so that the code generator cannot turn them into a
// paired multiplication and fuse it with a neighbour.  Used where both pixels
// take the grouped test; at the first group in which either escapes, both
// continue on the scalar path from their exact state.
__device__ __forceinline__ void escape_pair(float cra, float crb, float ci, int32_t max_iter,
                                            f2 nz, f2 m1, int32_t &ka, int32_t &kb) {
    const f2 CR = pk(cra, crb), CI = pk(ci, ci);
    f2 X = 0ull, Y = 0ull;
    int32_t k = 0;
    for (; k + 4 <= max_iter; k += 4) {
        const f2 sx = X, sy = Y;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const f2 xx = fma2(X, X, nz), yy = fma2(Y, Y, nz);
            const f2 nx = add2(fma2(yy, m1, xx), CR);
            Y = fma2(add2(X, X), Y, CI);
            X = nx;
        }
        const f2 xx = fma2(X, X, nz), yy = fma2(Y, Y, nz);
        const f2 s = add2(xx, yy);  // |z_{k+3}|^2 of both pixels
        const f2 nx = add2(fma2(yy, m1, xx), CR);
        const f2 ny = fma2(add2(X, X), Y, CI);
        const bool ea = lo_of(s) > 4.0f, eb = hi_of(s) > 4.0f;
        if (ea | eb) {
            ka = ea ? escape_from(lo_of(sx), lo_of(sy), k, cra, ci, k + 4, false)
                    : escape_from(lo_of(nx), lo_of(ny), k + 4, cra, ci, max_iter, true);
            kb = eb ? escape_from(hi_of(sx), hi_of(sy), k, crb, ci, k + 4, false)
                    : escape_from(hi_of(nx), hi_of(ny), k + 4, crb, ci, max_iter, true);
            return;
        }
        X = nx;
        Y = ny;
    }
    ka = escape_from(lo_of(X), lo_of(Y), k, cra, ci, max_iter, true);
    kb = escape_from(hi_of(X), hi_of(Y), k, crb, ci, max_iter, true);
}

__device__ __forceinline__ void put_pixel(uint8_t *__restrict__ rgb, int32_t *__restrict__ counts,
                                          int64_t p, int32_t k, int32_t max_iter) {
    if (counts) counts[p] = k;
    const uint32_t u = (uint32_t)k;
    const bool member = k == max_iter;
    rgb[3 * p + 0] = member ? 0 : (uint8_t)(u * 9u);
    rgb[3 * p + 1] = member ? 0 : (uint8_t)(u * 5u);
    rgb[3 * p + 2] = member ? 0 : (uint8_t)(u * 13u);
}

__global__ void __launch_bounds__(256) k_mandelbrot(uint8_t *__restrict__ rgb,
                                                     int32_t *__restrict__ counts, int64_t width,
                                                     int64_t height, float x0, float y0, float dx,
                                                     float dy, int32_t max_iter) {
    const int lane = threadIdx.x & 31;
    const int64_t tiles_x = (width + kTileW - 1) / kTileW;
    const int64_t tiles = tiles_x * ((height + kTileH - 1) / kTileH);
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < tiles;
         t += warps) {
        const int64_t i = (t % tiles_x) * kTileW + (lane % kTileW);
        const int64_t j = (t / tiles_x) * kTileH + (lane / kTileW);
        if (i >= width || j >= height) continue;
        const float cr = __fadd_rn(x0, __fmul_rn((float)(int)i, dx));
        const float ci = __fadd_rn(y0, __fmul_rn((float)(int)j, dy));
        put_pixel(rgb, counts, j * width + i, escape_count(cr, ci, max_iter), max_iter);
    }
}

// Two pixels per thread: a warp owns a 16 x 4 pixel tile.
__global__ void __launch_bounds__(256) k_mandelbrot2(uint8_t *__restrict__ rgb,
                                                      int32_t *__restrict__ counts, int64_t width,
                                                      int64_t height, float x0, float y0, float dx,
                                                      float dy, int32_t max_iter, float nzf,
                                                      float m1f) {
    const int lane = threadIdx.x & 31;
    const int64_t tiles_x = (width + 15) / 16;
    const int64_t tiles = tiles_x * ((height + kTileH - 1) / kTileH);
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const f2 nz = pk(nzf, nzf), m1 = pk(m1f, m1f);
    for (int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < tiles;
         t += warps) {
        const int64_t i = (t % tiles_x) * 16 + (lane % 8) * 2;
        const int64_t j = (t / tiles_x) * kTileH + (lane / 8);
        if (i >= width || j >= height) continue;
        const float ci = __fadd_rn(y0, __fmul_rn((float)(int)j, dy));
        const float cra = __fadd_rn(x0, __fmul_rn((float)(int)i, dx));
        const int64_t p = j * width + i;
        if (i + 1 >= width) {
            put_pixel(rgb, counts, p, escape_count(cra, ci, max_iter), max_iter);
            continue;
        }
        const float crb = __fadd_rn(x0, __fmul_rn((float)(int)(i + 1), dx));
        int32_t ka, kb;
        if (fast_ok(cra, ci) && fast_ok(crb, ci)) {
            escape_pair(cra, crb, ci, max_iter, nz, m1, ka, kb);
        } else {
            ka = escape_count(cra, ci, max_iter);
            kb = escape_count(crb, ci, max_iter);
        }
        put_pixel(rgb, counts, p, ka, max_iter);
        put_pixel(rgb, counts, p + 1, kb, max_iter);
    }
}

}  // namespace

cudaError_t mandelbrot(uint8_t *rgb, int32_t *counts, int64_t width, int64_t height, float x0,
                       float y0, float dx, float dy, int32_t max_iter, const hxc_launch_cfg *cfg,
                       cudaStream_t s) {
    if (width == 0 || height == 0) return cudaSuccess;
    const int64_t tiles = ((width + kTileW - 1) / kTileW) * ((height + kTileH - 1) / kTileH);
    unsigned b = 256, g;
    if (cfg) {
        b = cfg->block[0] * cfg->block[1] * cfg->block[2];
        g = cfg->grid[0] * cfg->grid[1] * cfg->grid[2];
    } else {
        g = (unsigned)std::min<int64_t>((tiles + 7) / 8, (int64_t)sm_count() * 8);
    }
    if (tune::get("mandel.pair") == 1) {
        if (!cfg) {
            const int64_t t2 = ((width + 15) / 16) * ((height + kTileH - 1) / kTileH);
            g = (unsigned)std::min<int64_t>((t2 + 7) / 8, (int64_t)sm_count() * 8);
        }
        k_mandelbrot2<<<g, b, 0, s>>>(rgb, counts, width, height, x0, y0, dx, dy, max_iter, -0.0f,
                                      -1.0f);
        return cudaGetLastError();
    }
    k_mandelbrot<<<g, b, 0, s>>>(rgb, counts, width, height, x0, y0, dx, dy, max_iter);
    return cudaGetLastError();
}

}  // namespace k
}  // namespace hxc
