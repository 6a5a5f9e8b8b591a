// Tile L2 norms without any device allocation (hxc_tile_norms_noalloc).
//
// Why it exists: the regular tile-norm launch (HXC_K_TILE_NORM2 through
// hxc_launch) takes its reduction scratch from a per-device cache that is
// filled by cudaMalloc on first use.  Some callers cannot let the library
// allocate: a real-time loop in which cudaMalloc would synchronise the whole
// device, a process whose device memory is owned by another allocator, or a
// deployment that forbids allocation after start-up.  This entry point runs
// the library's one-launch tile-norm grid kernel (the one the 2D runs use for
// their device norms, so the same reduction order and the same bits) with
// its scratch in a fixed-size array that is part of the library image on
// every GPU that loads it.
#include "hxc.h"
#include "kernels.cuh"
#include "runtime.hpp"

namespace hxc {
namespace k {
namespace {

// Scratch of tile_norm_grid for the largest accepted grid: per tile
// kNormBands partial sums, then one counter per tile.
constexpr int kMaxTiles = HXC_NOALLOC_MAX_TILES;
constexpr size_t kScratchBytes =
    (size_t)kMaxTiles * (kNormBands * sizeof(double) + sizeof(unsigned)) + 16;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

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
    // The array's name is only a host-side stand-in: its device address is
    // looked up on every call, with the caller's device current, so the
    // address always belongs to the context that runs the kernel (also
    // after a device reset or with several devices).
    void *scratch = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
    if (e != cudaSuccess) return hxc::cuda_status(e, "hxc_tile_norms_noalloc: scratch address");
    if (hxc::k::tile_norm_grid_scratch_bytes(tiles_y * tiles_x) > kScratchBytes) {
        hxc::set_error("hxc_tile_norms_noalloc: scratch layout exceeds the fixed array");
        return HXC_E_INVALID;
    }
    // tile_norm_grid clears the per-tile counters on the stream, then
    // launches the grid kernel (no snapshot)
    e = tile_norm_grid(src, nullptr, 0, norms, scratch, ny, nx, tiles_y, tiles_x,
                       static_cast<cudaStream_t>(stream));
    return hxc::cuda_status(e, "hxc_tile_norms_noalloc: launch");
}
