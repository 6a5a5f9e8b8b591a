// The 2D FTCS run with the field in host memory and every step streamed
// through the device tile by tile: Algorithm 1's copy in / kernel / copy out
// per partition, applied to each step of the stencil (Sec. 5.1.1 measures
// exactly this contrast: a sequential native loop against the same work
// issued asynchronously, where copies of one tile overlap the kernels and
// copies of others).
//
// Tile p with rows [y0, y1) and columns [x0, x1) is copied with its one-cell
// halo (clipped to the field) into a device buffer of (ty + 2) rows of pitch
// W, the interior starting at row 1, column 2 (so that the interior starts
// on a 16-byte boundary and the vectorised kernel applies); halo cells
// outside the field stay zero (the Dirichlet ghosts).  The step kernel
// writes a second buffer of the same shape, whose interior is copied back.
// Host arrays alternate between steps.  Step s of tile p waits for step
// s - 1 of the tiles whose interiors its halo rectangle touches (itself and
// its up to eight neighbours); its copy in, kernel and copy out run on the
// tile's stream slot as one operation.
#include <algorithm>
#include <cstring>
#include <vector>

#include "drivers_util.hpp"
#include "ftcs_plan.hpp"
#include "kernels.cuh"
#include "runtime.hpp"

using namespace hxc;
using namespace hxc::drv;

namespace {

struct StreamPlan {
    int64_t ny, nx, TY, TX, H, W;
    std::vector<int64_t> by, bx;
    double *base;  // 2 * T buffers of H * W doubles
    int64_t count() const { return TY * TX; }
    double *in(int64_t t) const { return base + (size_t)t * H * W; }
    double *out(int64_t t) const { return base + (size_t)(count() + t) * H * W; }
};

// Copy in, step, copy out of tile t from src to dst (host arrays).
cudaError_t tile_step(const StreamPlan &pl, int64_t t, const double *src, double *dst,
                      const k::FtcsStep &kind, cudaStream_t s) {
    const int64_t p = t / pl.TX, q = t % pl.TX;
    const int64_t y0 = pl.by[p], y1 = pl.by[p + 1], x0 = pl.bx[q], x1 = pl.bx[q + 1];
    const int64_t r0 = std::max<int64_t>(y0 - 1, 0), r1 = std::min<int64_t>(y1 + 1, pl.ny);
    const int64_t c0 = std::max<int64_t>(x0 - 1, 0), c1 = std::min<int64_t>(x1 + 1, pl.nx);
    double *in = pl.in(t), *out = pl.out(t);
    cudaError_t e = cudaMemcpy2DAsync(in + (r0 - (y0 - 1)) * pl.W + (c0 - (x0 - 2)), pl.W * 8,
                                      src + r0 * pl.nx + c0, pl.nx * 8, (c1 - c0) * 8, r1 - r0,
                                      cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = k::heat2d_step(in, out, (y1 - y0) + 2, pl.W, 1, 2, y1 - y0, x1 - x0, kind, 0, s);
    if (e != cudaSuccess) return e;
    return cudaMemcpy2DAsync(dst + y0 * pl.nx + x0, pl.nx * 8, out + pl.W + 2, pl.W * 8,
                             (x1 - x0) * 8, y1 - y0, cudaMemcpyDeviceToHost, s);
}

}  // namespace

extern "C" hxc_status hxc_heat2d_stream_run(hxc_device dh, double *host_a, double *host_b,
                                            int64_t ny, int64_t nx, int64_t tiles_y,
                                            int64_t tiles_x, double r, int steps, int sequential,
                                            const hxc_future *deps, int ndeps, hxc_future *out,
                                            hxc_run_stats *stats) {
    hxc::drv::NvtxRange nvtx_range("hxc_heat2d_stream_run");
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    if (!out || !host_a || !host_b || host_a == host_b || ny < 1 || nx < 1 || tiles_y < 1 ||
        tiles_x < 1 || tiles_y > ny || tiles_x > nx || tiles_y * tiles_x > kCopySlot0 ||
        steps < 0) {
        set_error("hxc_heat2d_stream_run: invalid arguments");
        return HXC_E_INVALID;
    }
    std::vector<FutRef> dv;
    hxc_status st = deps_from_handles(deps, ndeps, &dv);
    if (st) return st;
    if (stats) memset(stats, 0, sizeof *stats);
    if ((st = d->make_current())) return st;
    StreamPlan pl;
    pl.ny = ny;
    pl.nx = nx;
    pl.TY = tiles_y;
    pl.TX = tiles_x;
    pl.by = split(ny, tiles_y, false);
    pl.bx = split(nx, tiles_x, true);
    int64_t mty = 0, mtx = 0;
    for (int64_t p = 0; p < tiles_y; p++) mty = std::max(mty, pl.by[p + 1] - pl.by[p]);
    for (int64_t q = 0; q < tiles_x; q++) mtx = std::max(mtx, pl.bx[q + 1] - pl.bx[q]);
    pl.H = mty + 2;
    pl.W = (mtx + 4 + 1) / 2 * 2;  // even pitch keeps every row 16-byte aligned
    const int64_t T = pl.count();
    const size_t bytes = (size_t)2 * T * pl.H * pl.W * 8;
    void *base = nullptr;
    if ((st = d->scratch_get("heat2d_stream", bytes, &base))) return st;
    pl.base = static_cast<double *>(base);
    Stats sc{stats};
    // the step kinds of the device-resident run without snapshots
    // (intervals of at most 100 steps), so that both give the same bits
    const int64_t every = std::min<int64_t>(steps, 100);
    auto step_kind = [every, steps, r](int64_t step) {
        const int64_t s0 = step / every * every;
        return ftcs2_step(r, step - s0, std::min<int64_t>(every, steps - s0));
    };
    auto count_step = [&]() {
        for (int64_t t = 0; t < T; t++) {
            const int64_t p = t / pl.TX, q = t % pl.TX;
            const int64_t hy = std::min<int64_t>(pl.by[p + 1] + 1, ny) - std::max<int64_t>(pl.by[p] - 1, 0);
            const int64_t hx = std::min<int64_t>(pl.bx[q + 1] + 1, nx) - std::max<int64_t>(pl.bx[q] - 1, 0);
            sc.copy(hy * hx * 8, 0);
            sc.copy(0, (pl.by[p + 1] - pl.by[p]) * (pl.bx[q + 1] - pl.bx[q]) * 8);
            sc.launch();
        }
    };

    if (sequential) {
        // the native sequential loop: every tile's three calls, then a wait
        for (auto &f : dv)
            if ((st = fut_wait(f, -1))) return st;
        cudaStream_t s;
        if ((st = d->stream(0, &s))) return st;
        cudaError_t e = cudaMemsetAsync(base, 0, bytes, s);
        for (int step = 0; step < steps && e == cudaSuccess; step++) {
            const double *src = step % 2 ? host_b : host_a;
            double *dst = step % 2 ? host_a : host_b;
            const k::FtcsStep kind = step_kind(step);
            for (int64_t t = 0; t < T && e == cudaSuccess; t++) {
                e = tile_step(pl, t, src, dst, kind, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            }
            count_step();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        st = e == cudaSuccess ? HXC_OK : cuda_status(e, "hxc_heat2d_stream_run");
        *out = to_handle(make_done(st));
        return st;
    }

    // asynchronous: one future per tile and step
    FutRef zero;
    if ((st = issue_device_op(d.get(), 0, dv,
                              [base, bytes](cudaStream_t s) { return cudaMemsetAsync(base, 0, bytes, s); },
                              {}, &zero)))
        return st;
    std::vector<FutRef> prev(T), cur(T);
    auto pp = std::make_shared<StreamPlan>(pl);
    for (int step = 0; step < steps; step++) {
        const double *src = step % 2 ? host_b : host_a;
        double *dst = step % 2 ? host_a : host_b;
        const k::FtcsStep kind = step_kind(step);
        for (int64_t t = 0; t < T; t++) {
            std::vector<FutRef> deps_t;
            if (step == 0) {
                deps_t.push_back(zero);
            } else {
                const int64_t p = t / pl.TX, q = t % pl.TX;
                for (int64_t a = std::max<int64_t>(p - 1, 0); a <= std::min(p + 1, pl.TY - 1); a++)
                    for (int64_t b = std::max<int64_t>(q - 1, 0); b <= std::min(q + 1, pl.TX - 1); b++)
                        deps_t.push_back(prev[a * pl.TX + b]);
            }
            if ((st = issue_device_op(d.get(), (int)t, deps_t,
                                      [pp, t, src, dst, kind](cudaStream_t s) {
                                          return tile_step(*pp, t, src, dst, kind, s);
                                      },
                                      {}, &cur[t])))
                return st;
        }
        count_step();
        prev.swap(cur);
    }
    std::vector<FutRef> finals = steps ? prev : std::vector<FutRef>{zero};
    return finish(d.get(), finals, out);
}
