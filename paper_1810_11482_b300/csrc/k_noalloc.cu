// Tile L2 norms without any device allocation (hxc_tile_norms_noalloc).
//
// Why it exists: the regular tile-norm launch (HXC_K_TILE_NORM2 through
// hxc_launch) takes its reduction scratch from a per-device cache that is
// filled by cudaMalloc on first use.  Some callers cannot let the library
// allocate: a real-time loop in which cudaMalloc would synchronise the whole
// device, a process whose device memory is owned by another allocator, or a
// deployment that forbids allocation after start-up.  This entry point
// computes the same per-tile norms with its scratch in a fixed-size array
// that is part of the library image on every GPU that loads it.
#include <mutex>

#include "hxc.h"
#include "kernels.cuh"
#include "runtime.hpp"

namespace hxc {
namespace k {
namespace {

// Scratch: per tile kNormBands partial sums, then one counter per tile.
constexpr int kMaxTiles = HXC_NOALLOC_MAX_TILES;
constexpr size_t kPartialBytes = (size_t)kMaxTiles * kNormBands * sizeof(double);
constexpr size_t kScratchBytes = kPartialBytes + (size_t)kMaxTiles * sizeof(unsigned);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Same reduction order as the tile-norm kernel: band g of a tile covers rows
// [g*ty/B, (g+1)*ty/B); thread t of a band accumulates the squares of the
// band's elements whose row-major index within the band is t mod 256, in
// increasing order; lanes combine by a butterfly, warps by a fixed tree;
// the last band of a tile adds the band sums in order and stores the root.
__global__ void __launch_bounds__(256) k_tile_norms_noalloc(const double *__restrict__ src,
                                                            int64_t ny, int64_t nx,
                                                            int64_t tiles_y, int64_t tiles_x,
                                                            double *norms,
                                                            unsigned char *scratch) {
    const int g = blockIdx.x;
    const int64_t tile = blockIdx.y;
    const int64_t p = tile / tiles_x, q = tile % tiles_x;
    // tile bounds: rows split evenly, columns split on even indices when nx
    // is even (the partition used by the whole-run entry points)
    const int64_t y0 = p * ny / tiles_y, y1 = (p + 1) * ny / tiles_y;
    int64_t x0, x1;
    if (nx % 2 == 0) {
        x0 = (q * (nx / 2) / tiles_x) * 2;
        x1 = q + 1 == tiles_x ? nx : ((q + 1) * (nx / 2) / tiles_x) * 2;
    } else {
        x0 = q * nx / tiles_x;
        x1 = (q + 1) * nx / tiles_x;
    }
    const int64_t ty = y1 - y0, tx = x1 - x0;
    double *partials = reinterpret_cast<double *>(scratch) + tile * kNormBands;
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + kPartialBytes) + tile;

    const int64_t r0 = (int64_t)g * ty / kNormBands, r1 = (int64_t)(g + 1) * ty / kNormBands;
    const int64_t m = (r1 - r0) * tx;
    double acc = 0.0;
    if (tx > 0) {
        int64_t i = r0 + threadIdx.x / tx, j = threadIdx.x % tx;
        for (int64_t k = threadIdx.x; k < m; k += 256) {
            const double v = __ldg(src + (y0 + i) * nx + x0 + j);
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
        const double s = __dadd_rn(__dadd_rn(__dadd_rn(ws[0], ws[1]), __dadd_rn(ws[2], ws[3])),
                                   __dadd_rn(__dadd_rn(ws[4], ws[5]), __dadd_rn(ws[6], ws[7])));
        partials[g] = s;
        __threadfence();
        is_last = atomicAdd(counter, 1u) == kNormBands - 1;
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (int b = 0; b < kNormBands; b++) s = __dadd_rn(s, __ldcg(partials + b));
        norms[tile] = __dsqrt_rn(s);
    }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_m;
unsigned char *g_addr[64] = {};

cudaError_t scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_m);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace k
}  // namespace hxc

extern "C" hxc_status hxc_tile_norms_noalloc(const double *src, int64_t ny, int64_t nx,
                                             int64_t tiles_y, int64_t tiles_x, double *norms,
                                             void *stream) {
    using namespace hxc::k;
    if (!src || !norms || ny <= 0 || nx <= 0 || tiles_y < 1 || tiles_x < 1 || tiles_y > ny ||
        tiles_x > nx) {
        hxc::set_error("hxc_tile_norms_noalloc: invalid field or tile grid");
        return HXC_E_INVALID;
    }
    if (tiles_y * tiles_x > kMaxTiles) {
        hxc::set_error("hxc_tile_norms_noalloc: %lld tiles exceed the fixed scratch of %d tiles",
                       (long long)(tiles_y * tiles_x), kMaxTiles);
        return HXC_E_INVALID;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    unsigned char *scratch = nullptr;
    if (e == cudaSuccess) e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) return hxc::cuda_status(e, "hxc_tile_norms_noalloc: scratch address");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t T = tiles_y * tiles_x;
    // the per-tile counters must start at zero
    e = cudaMemsetAsync(scratch + kPartialBytes, 0, (size_t)T * sizeof(unsigned), s);
    if (e != cudaSuccess) return hxc::cuda_status(e, "hxc_tile_norms_noalloc: clear counters");
    dim3 grid(kNormBands, (unsigned)T);
    k_tile_norms_noalloc<<<grid, 256, 0, s>>>(src, ny, nx, tiles_y, tiles_x, norms, scratch);
    return hxc::cuda_status(cudaGetLastError(), "hxc_tile_norms_noalloc: launch");
}
