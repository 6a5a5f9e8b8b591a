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

#include "kernels.cuh"

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
__device__ __forceinline__ int32_t escape_count(float cr, float ci, int32_t max_iter) {
    float x = 0.0f, y = 0.0f;
    int32_t k = 0;
    if (__fmaf_rn(cr, cr, __fmul_rn(ci, ci)) <= 3.99f) {
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
        const int32_t k = escape_count(cr, ci, max_iter);
        const int64_t p = j * width + i;
        if (counts) counts[p] = k;
        const uint32_t u = (uint32_t)k;
        const bool member = k == max_iter;
        rgb[3 * p + 0] = member ? 0 : (uint8_t)(u * 9u);
        rgb[3 * p + 1] = member ? 0 : (uint8_t)(u * 5u);
        rgb[3 * p + 2] = member ? 0 : (uint8_t)(u * 13u);
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
    k_mandelbrot<<<g, b, 0, s>>>(rgb, counts, width, height, x0, y0, dx, dy, max_iter);
    return cudaGetLastError();
}

}  // namespace k
}  // namespace hxc
