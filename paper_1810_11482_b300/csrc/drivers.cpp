// Whole-run entry points: the partitioned FTCS loops expressed as futures.
//
// Algorithm 1 of the paper issues, per partition, an asynchronous copy in,
// a kernel and an asynchronous copy out on streams; Sec. 3.1 composes such
// operations through futures.  Here every partition owns a stream slot and
// step s of partition p is issued with the futures of step s-1 of p and of
// the partitions whose cells p reads as its halo, so no host round trip sits
// between steps.  Ping-pong buffers make step s write the buffer step s-1
// read; the halo dependencies order that write-after-read as well.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <memory>

#include "drivers_util.hpp"
#include "ftcs_plan.hpp"
#include "kernels.cuh"
#include "tune.hpp"
#include "runtime.hpp"

using namespace hxc;
using namespace hxc::drv;

namespace hxc {
namespace drv {
std::mutex g_graph_m;
std::map<std::string, Ref<Graph>> g_graphs;
}  // namespace drv
}  // namespace hxc

namespace {

// ---------------------------------------------------------------- 1D runs
struct Heat1dPlan {
    Device *dev;
    double *buf[2];
    int64_t n;
    std::vector<int64_t> b;
    double r;
    std::shared_ptr<const k::FtcsPlan> plan;  // the run's step kinds (ftcs_plan)
};

// Partitions whose cells fall in the periodic window [lo - T, hi + T).
std::vector<int> halo_parts(const std::vector<int64_t> &b, int64_t n, int p, int64_t T) {
    int parts = (int)b.size() - 1;
    std::vector<int> out;
    if (2 * T + (b[p + 1] - b[p]) >= n) {
        for (int q = 0; q < parts; q++) out.push_back(q);
        return out;
    }
    int64_t lo = b[p] - T, hi = b[p + 1] + T;  // may leave [0, n)
    for (int q = 0; q < parts; q++) {
        if (b[q + 1] == b[q]) continue;
        bool hit = false;
        for (int64_t shift : {-n, (int64_t)0, n}) {
            int64_t ql = b[q] + shift, qh = b[q + 1] + shift;
            if (ql < hi && qh > lo) hit = true;
        }
        if (hit) out.push_back(q);
    }
    return out;
}

// Issues `steps` 1D steps (run steps g0 .. g0+steps-1), `T` steps per
// launch, partition p on slot p.  prev[p] holds the last future of
// partition p and is updated.  `flip` is the index of the buffer holding
// the current state; every launch moves the state to the other buffer.
hxc_status issue_heat1d(const Heat1dPlan &pl, int steps, int T, int &flip, std::vector<FutRef> &prev,
                        Stats &stats, int64_t g0) {
    int parts = (int)pl.b.size() - 1;
    std::vector<std::vector<int>> nb(parts);
    for (int p = 0; p < parts; p++) nb[p] = halo_parts(pl.b, pl.n, p, T);
    int done = 0;
    while (done < steps) {
        int t = std::min(T, steps - done);
        if (t != T)
            for (int p = 0; p < parts; p++) nb[p] = halo_parts(pl.b, pl.n, p, t);
        const double *src = pl.buf[flip];
        double *dst = pl.buf[1 - flip];
        std::vector<FutRef> cur(parts);
        for (int p = 0; p < parts; p++) {
            std::vector<FutRef> deps;
            for (int q : nb[p])
                if (prev[q]) deps.push_back(prev[q]);
            int64_t lo = pl.b[p], cnt = pl.b[p + 1] - pl.b[p];
            int64_t n = pl.n;
            std::shared_ptr<const k::FtcsPlan> plan = pl.plan;
            const int64_t gs = g0 + done;
            hxc_launch_cfg cfg{};
            const hxc_launch_cfg *pc = nullptr;
            if (t > 1) {
                // spread the SMs over the partitions that run concurrently
                const int64_t tc = tune::get("heat1d.tb_ctas");
                int g = tc > 0 ? (int)tc : std::max(1, k::sm_count() / parts);
                cfg = hxc_launch_cfg{{(uint32_t)g, 1, 1}, {512, 1, 1}};
                pc = &cfg;
            }
            StreamOp op = [=](cudaStream_t s) {
                return k::heat1d_plan(src, dst, n, lo, cnt, *plan, gs, t, pc ? &cfg : nullptr, s);
            };
            hxc_status st = issue_device_op(pl.dev, p, deps, op, {}, &cur[p]);
            if (st) return st;
            stats.launch();
        }
        prev.swap(cur);
        done += t;
        flip = 1 - flip;
    }
    return HXC_OK;
}

}  // namespace

extern "C" {

hxc_status hxc_heat1d_run(hxc_device dh, hxc_buffer uh, hxc_buffer th, int64_t n, int parts,
                          double r, int steps, hxc_mode mode, int steps_per_launch,
                          const hxc_future *deps, int ndeps, hxc_future *out,
                          hxc_run_stats *stats_out) {
    hxc::drv::NvtxRange nvtx_range("hxc_heat1d_run");
    Ref<Device> d = dev_from_handle(dh);
    Ref<Buffer> u = buf_from_handle(uh), t = buf_from_handle(th);
    if (!d || !u || !t) return HXC_E_INVALID;
    if (n <= 0 || parts < 1 || parts > n || parts > kCopySlot0 || steps < 0 ||
        u->bytes < (size_t)n * 8 || t->bytes < (size_t)n * 8 || u->ptr == t->ptr ||
        u->dev.get() != d.get() || t->dev.get() != d.get() || steps_per_launch < 0 ||
        steps_per_launch > k::kHeat1dMaxSteps || (mode != HXC_MODE_PLAIN && mode != HXC_MODE_GRAPH &&
                                                  mode != HXC_MODE_FUSED)) {
        set_error("hxc_heat1d_run: invalid arguments");
        return HXC_E_INVALID;
    }
    std::vector<FutRef> dv;
    hxc_status st = deps_from_handles(deps, ndeps, &dv);
    if (st) return st;
    if (stats_out) memset(stats_out, 0, sizeof *stats_out);
    if (has_pending_host(dv)) {
        FutRef a, b;
        defer_run(dv,
                  [=](FutRef *ia, FutRef *ib) {
                      hxc_future h = nullptr;
                      hxc_status s2 = hxc_heat1d_run(dh, uh, th, n, parts, r, steps, mode,
                                                     steps_per_launch, nullptr, 0, &h, nullptr);
                      if (s2) return s2;
                      *ia = FutRef(reinterpret_cast<Future *>(h), true);
                      *ib = *ia;
                      return HXC_OK;
                  },
                  &a, &b);
        // the buffers must outlive the deferred run
        fut_on_done(a, [u, t](hxc_status) {});
        if (out) *out = to_handle(a);
        return HXC_OK;
    }
    Stats stats{stats_out};
    if ((st = d->make_current())) return st;
    Heat1dPlan pl{d.get(), {(double *)u->ptr, (double *)t->ptr}, n, split(n, parts, false), r,
                  std::make_shared<const k::FtcsPlan>(ftcs_plan(1, r, steps, heat1d_interval(steps)))};
    int T = 1;
    if (mode == HXC_MODE_FUSED) {
        if (steps_per_launch == 0) {
            const int tuned = (int)tune::get("heat1d.steps_per_launch");
            T = std::min(steps, tuned > 0 ? tuned : k::kHeat1dMaxSteps);
        } else {
            T = steps_per_launch;
        }
        if (T < 1) T = 1;
    }
    std::vector<FutRef> finals;
    std::vector<FutRef> prev(parts);
    int flip = 0;
    // the run starts after the caller's dependencies
    if (!dv.empty()) {
        FutRef j;
        if ((st = issue_device_op(d.get(), kJoinSlot, dv, StreamOp(), {}, &j))) return st;
        for (auto &p : prev) p = j;
    }
    if (mode == HXC_MODE_GRAPH && steps > 0) {
        // capture `chunk` steps (one interval of the step kinds) once (an
        // even count when replayed more than once, so every replay starts
        // from u) and replay it; the remaining steps are issued directly
        int chunk = (int)heat1d_interval(steps);
        int reps = steps / chunk;
        std::string key = key_of("heat1d", {(double)n, (double)parts, r, (double)chunk},
                                 {u->ptr, t->ptr});
        Ref<Graph> g;
        {
            std::lock_guard<std::mutex> lk(g_graph_m);
            auto it = g_graphs.find(key);
            if (it != g_graphs.end()) g = it->second;
        }
        if (!g) {
            if ((st = graph_begin(d.get()))) return st;
            std::vector<FutRef> cprev(parts);
            Stats none{nullptr};
            int cflip = 0;
            st = issue_heat1d(pl, chunk, 1, cflip, cprev, none, 0);
            Ref<Graph> ng;
            hxc_status st2 = graph_end(d.get(), &ng);
            if (st) return st;
            if (st2) return st2;
            g = ng;
            std::lock_guard<std::mutex> lk(g_graph_m);
            g_graphs[key] = g;
        }
        cudaGraphExec_t ex = g->exec;
        for (int rep = 0; rep < reps; rep++) {
            std::vector<FutRef> gdeps;
            for (auto &p : prev)
                if (p) {
                    gdeps.push_back(p);
                    break;  // every partition holds the same future here
                }
            FutRef gf;
            if ((st = issue_device_op(d.get(), 0, gdeps,
                                      [ex](cudaStream_t s) { return cudaGraphLaunch(ex, s); },
                                      {AnyRef(g.get(), false)}, &gf)))
                return st;
            stats.launch((int64_t)parts * chunk);
            if (stats_out) stats_out->graph_launches++;
            for (auto &p : prev) p = gf;
        }
        flip = (reps * chunk) % 2;
        int rest = steps - reps * chunk;
        if (rest > 0 && (st = issue_heat1d(pl, rest, 1, flip, prev, stats, (int64_t)reps * chunk)))
            return st;
    } else if (steps > 0) {
        if ((st = issue_heat1d(pl, steps, T, flip, prev, stats, 0))) return st;
    }
    // the result lands in buf[flip]; bring it back into u
    if (flip == 1) {
        for (int p = 0; p < parts; p++) {
            int64_t lo = pl.b[p], cnt = pl.b[p + 1] - pl.b[p];
            double *dst = pl.buf[0] + lo;
            const double *src = pl.buf[1] + lo;
            std::vector<FutRef> deps;
            for (auto &f : prev)
                if (f) deps.push_back(f);  // every partition read u during the last step
            FutRef c;
            if ((st = issue_device_op(d.get(), p, deps,
                                      [=](cudaStream_t s) {
                                          return cudaMemcpyAsync(dst, src, cnt * 8,
                                                                 cudaMemcpyDeviceToDevice, s);
                                      },
                                      {}, &c)))
                return st;
            stats.copy(0, 0);
            finals.push_back(c);
        }
    } else {
        for (auto &f : prev)
            if (f) finals.push_back(f);
    }
    if (finals.empty()) finals.push_back(make_done(HXC_OK));
    std::vector<AnyRef> keep{AnyRef(u.get(), false), AnyRef(t.get(), false)};
    FutRef fin;
    // the join keeps the buffers alive until the run completes
    hxc_status st3 = issue_device_op(d.get(), kJoinSlot, finals, StreamOp(), keep, &fin);
    if (st3) return st3;
    if (out) *out = to_handle(fin);
    return HXC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- 2D runs
namespace {

struct Tiles {
    int64_t TY, TX;
    std::vector<int64_t> by, bx;
    int64_t count() const { return TY * TX; }
    int64_t y0(int64_t t) const { return by[t / TX]; }
    int64_t x0(int64_t t) const { return bx[t % TX]; }
    int64_t ty(int64_t t) const { return by[t / TX + 1] - by[t / TX]; }
    int64_t tx(int64_t t) const { return bx[t % TX + 1] - bx[t % TX]; }
    // the tile and its four edge neighbours
    std::vector<int64_t> nbrs(int64_t t) const {
        int64_t p = t / TX, q = t % TX;
        std::vector<int64_t> v{t};
        if (p > 0) v.push_back(t - TX);
        if (p + 1 < TY) v.push_back(t + TX);
        if (q > 0) v.push_back(t - 1);
        if (q + 1 < TX) v.push_back(t + 1);
        return v;
    }
};

struct HostNormTask {
    const double *data;
    int64_t count;
    double *out;
};

// sqrt(sum v^2) of a snapshot tile on the host, in double: blocks of 64
// squares summed with 8 independent accumulators of 8 terms each (a
// vectorisable loop), the block sums pairwise.  For these non-negative terms
// the sum's relative error is at most (1 + 7 + 3 + ceil(log2(blocks))) * 2^-53
// (the rounded square, an accumulator's 8 terms, the 8 accumulators, the
// pairwise levels): 25 * 2^-53 = 2.8e-15 for a 1024^2 tile, 1.4e-15 on the
// norm, within the 1e-14 asked of the host norms against a long-double
// reference sum.
hxc_status host_norm_fn(void *user) {
    HostNormTask *t = static_cast<HostNormTask *>(user);
    const double *x = t->data;
    const int64_t n = t->count, B = 64;
    std::vector<double> blocks((n + B - 1) / B);
    for (int64_t b0 = 0, k = 0; b0 < n; b0 += B, k++) {
        const int64_t e = std::min(n, b0 + B);
        double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int64_t i = b0;
        for (; i + 8 <= e; i += 8)
            for (int q = 0; q < 8; q++) a[q] += x[i + q] * x[i + q];
        for (; i < e; i++) a[0] += x[i] * x[i];
        blocks[k] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    }
    for (size_t w = 1; w < blocks.size(); w *= 2)
        for (size_t k = 0; k + w < blocks.size(); k += 2 * w) blocks[k] += blocks[k + w];
    *t->out = blocks.empty() ? 0.0 : std::sqrt(blocks[0]);
    return HXC_OK;
}

struct Heat2dRun {
    Device *dev;
    const hxc_heat2d_cfg *cfg;
    Tiles tl;
    double *buf[2];
    double *snap_dev;      // [2][tiles] compact tile snapshots
    double *norm_dev;      // [n_snap][tiles] device norms
    double *replay_dev;    // [2][tiles] device norms written by graph replays
    double *host_stage;    // [2][tiles] pinned staging for the host norms
    int64_t tile_stride;   // elements per snapshot tile slot
    int norm_set;          // which of the device's sets of norm rows
    Stats stats;
};

// Issues steps [s0, s1), one interval of the run (its step kinds follow
// ftcs_step), per tile or fused.
hxc_status issue_steps2d(Heat2dRun &R, int64_t s0, int64_t s1, std::vector<FutRef> &prev,
                         bool fused) {
    const hxc_heat2d_cfg &c = *R.cfg;
    const int64_t T = R.tl.count();
    if (fused && s1 > s0) {
        // the interval's whole-field steps as one operation: back-to-back
        // launches, each after the first with programmatic dependent launch
        // (its CTAs are placed while the step ahead of it drains)
        std::vector<FutRef> deps;
        for (auto &f : prev)
            if (f) {
                deps.push_back(f);
                break;  // in fused mode every tile holds the same future
            }
        double *b0 = R.buf[0], *b1 = R.buf[1];
        const int64_t ny = c.ny, nx = c.nx;
        const double r = c.r;
        FutRef f;
        hxc_status st = issue_device_op(
            R.dev, 0, deps,
            [=](cudaStream_t q) {
                for (int64_t s = s0; s < s1; s++) {
                    const double *src = s % 2 ? b1 : b0;
                    double *dst = s % 2 ? b0 : b1;
                    cudaError_t e = k::heat2d_step(src, dst, ny, nx, 0, 0, ny, nx,
                                                   ftcs2_step(r, s - s0, s1 - s0), 0, q, s > s0);
                    if (e != cudaSuccess) return e;
                }
                return cudaSuccess;
            },
            {}, &f);
        if (st) return st;
        R.stats.launch(s1 - s0);
        for (auto &p : prev) p = f;
        return HXC_OK;
    }
    for (int64_t s = s0; s < s1; s++) {
        const double *src = R.buf[s % 2];
        double *dst = R.buf[(s + 1) % 2];
        const k::FtcsStep kind = ftcs2_step(c.r, s - s0, s1 - s0);
        std::vector<FutRef> cur(T);
        for (int64_t t = 0; t < T; t++) {
            std::vector<FutRef> deps;
            for (int64_t q : R.tl.nbrs(t))
                if (prev[q]) deps.push_back(prev[q]);
            int64_t ny = c.ny, nx = c.nx, y0 = R.tl.y0(t), x0 = R.tl.x0(t), ty = R.tl.ty(t),
                    tx = R.tl.tx(t);
            hxc_status st = issue_device_op(
                R.dev, (int)t, deps,
                [=](cudaStream_t st) { return k::heat2d_step(src, dst, ny, nx, y0, x0, ty, tx, kind, 0, st); },
                {}, &cur[t]);
            if (st) return st;
            R.stats.launch();
        }
        prev.swap(cur);
    }
    return HXC_OK;
}

// Issues the device part of snapshot k (taken after step `step`): the tile
// snapshot + device norm kernels into ring slot k % 2.
hxc_status issue_snap_kernels(Heat2dRun &R, int64_t k, int64_t step, std::vector<FutRef> &prev,
                              const std::vector<FutRef> &ring_free, bool fused,
                              const FutRef &norm_free = FutRef()) {
    const hxc_heat2d_cfg &c = *R.cfg;
    const int64_t T = R.tl.count();
    const double *src = R.buf[step % 2];
    if (fused) {
        // one launch for every tile on slot 0 (same bits as the per-tile launches)
        std::vector<FutRef> deps;
        for (auto &f : prev)
            if (f) {
                deps.push_back(f);
                break;  // in fused mode every tile holds the same future
            }
        for (auto &f : ring_free)
            if (f) deps.push_back(f);
        if (norm_free) deps.push_back(norm_free);
        void *scratch = nullptr;
        hxc_status st = R.dev->scratch_get("tile_norm_grid", k::tile_norm_grid_scratch_bytes(T), &scratch);
        if (st) return st;
        double *snap = c.host_norms ? R.snap_dev + (k % 2) * T * R.tile_stride : nullptr;
        double *norms = R.norm_dev + k * T;
        const int64_t stride = R.tile_stride, ny = c.ny, nx = c.nx, TY = R.tl.TY, TX = R.tl.TX;
        FutRef f;
        st = issue_device_op(
            R.dev, 0, deps,
            [=](cudaStream_t s) {
                return k::tile_norm_grid(src, snap, stride, norms, scratch, ny, nx, TY, TX, s);
            },
            {}, &f);
        if (st) return st;
        R.stats.launch();
        for (auto &p : prev) p = f;
        return HXC_OK;
    }
    for (int64_t t = 0; t < T; t++) {
        std::vector<FutRef> deps;
        if (prev[t]) deps.push_back(prev[t]);
        if (ring_free.size() > (size_t)t && ring_free[t]) deps.push_back(ring_free[t]);
        if (norm_free) deps.push_back(norm_free);
        double *snap = c.host_norms ? R.snap_dev + ((k % 2) * T + t) * R.tile_stride : nullptr;
        double *norms = R.norm_dev;
        int64_t idx = k * T + t;
        int64_t ny = c.ny, nx = c.nx, y0 = R.tl.y0(t), x0 = R.tl.x0(t), ty = R.tl.ty(t),
                tx = R.tl.tx(t);
        int slot = fused ? 0 : (int)t;
        void *scratch = nullptr;
        hxc_status st = R.dev->scratch_get("tile_norm." + std::to_string(slot), k::kNormScratchBytes,
                                           &scratch);
        if (st) return st;
        FutRef f;
        st = issue_device_op(
            R.dev, slot, deps,
            [=](cudaStream_t s) {
                return k::tile_norm(src, snap, norms, scratch, ny, nx, y0, x0, ty, tx, idx, s);
            },
            {}, &f);
        if (st) return st;
        R.stats.launch();
        prev[t] = f;
    }
    return HXC_OK;
}

// Host part of snapshot k: device->host copies of the ring slot into the
// pinned staging ring, then host-norm continuations.  host_free[t] is the
// continuation of snapshot k-2 (staging reuse); d2h_out receives the copies
// (they free the device ring slot), cont_out the continuations.
hxc_status issue_snap_host(Heat2dRun &R, int64_t k, const std::vector<FutRef> &snapf,
                           const std::vector<FutRef> &host_free, std::vector<FutRef> &d2h_out,
                           std::vector<FutRef> &cont_out, std::vector<std::unique_ptr<HostNormTask>> &tasks) {
    const int64_t T = R.tl.count();
    for (int64_t t = 0; t < T; t++) {
        std::vector<FutRef> deps{snapf[t]};
        if (host_free.size() > (size_t)t && host_free[t]) deps.push_back(host_free[t]);
        const double *snap = R.snap_dev + ((k % 2) * T + t) * R.tile_stride;
        double *stage = R.host_stage + ((k % 2) * T + t) * R.tile_stride;
        size_t bytes = (size_t)R.tl.ty(t) * R.tl.tx(t) * 8;
        FutRef c;
        hxc_status st = issue_device_op(
            R.dev, kCopySlot0 + (int)(t % kCopySlots), deps,
            [=](cudaStream_t s) { return cudaMemcpyAsync(stage, snap, bytes, cudaMemcpyDeviceToHost, s); },
            {}, &c);
        if (st) return st;
        R.stats.copy(0, bytes);
        d2h_out[t] = c;
        tasks.emplace_back(new HostNormTask{stage, R.tl.ty(t) * R.tl.tx(t),
                                             R.cfg->host_norms + k * T + t});
        HostNormTask *task = tasks.back().get();
        FutRef r = make_pending();
        fut_on_done(c, [r, task](hxc_status s) {
            if (s != HXC_OK) {
                fut_set_done(r, HXC_E_DEP_FAILED);
                return;
            }
            pool().submit([r, task] { fut_set_done(r, host_norm_fn(task) == HXC_OK ? HXC_OK : HXC_E_CALLBACK); });
        });
        cont_out[t] = r;
    }
    return HXC_OK;
}

// Holds what a run's futures refer to until the run's final future is done.
struct RunResources : RefCounted {
    std::vector<std::unique_ptr<HostNormTask>> tasks;
    std::vector<AnyRef> keep;
};


// Snapshot rings shared by consecutive runs on a device: the futures of the
// last operations that read each ring slot (device->host copies and host
// continuations), so that a new run does not overwrite a slot still in use.
struct RingCarry {
    int64_t tiles = -1, stride = -1;
    std::vector<FutRef> d2h[2], conts[2];
};
std::mutex g_carry_m;
std::map<Device *, RingCarry> g_carry;

// Two device field pairs per device for the host entry points, used in turn:
// the uploads and downloads of one call overlap the steps of the call issued
// before it, and a call waits (on the device) only for the call two back,
// the last user of its pair.
struct HostRunSlots {
    int next = 0;
    FutRef last[2];
};
std::mutex g_hostrun_m;
std::map<Device *, HostRunSlots> g_hostrun;
const char *const kHostKeyU[2] = {"heat2d_host.u0", "heat2d_host.u1"};
const char *const kHostKeyT[2] = {"heat2d_host.t0", "heat2d_host.t1"};
constexpr int kHostSlots = 4;
constexpr int kHostInSlot0 = kCopySlot0 + kCopySlots;     // host-run uploads
constexpr int kHostOutSlot0 = kHostInSlot0 + kHostSlots;  // host-run downloads
constexpr int kNormCopySlot = kHostOutSlot0 + kHostSlots;  // device norms to the host
static_assert(kNormCopySlot < HXC_MAX_SLOTS, "stream slots");

// The device norm rows of a run and their pinned host staging: four sets of
// each, used in turn by successive runs.  A run's first write into its rows
// waits for the copy out of the same rows by the run four before (copied[]),
// its copy into a staging buffer for the host copy out of that buffer by the
// run four before (last[]), and the run as a whole starts after the previous
// run's copy of its rows (latest).
constexpr int kGnormStages = 4;
struct GnormStage {
    std::mutex m;
    int next = 0, next_rows = 0;
    void *ptr[kGnormStages] = {};
    size_t bytes[kGnormStages] = {};
    FutRef last[kGnormStages];    // the host copy out of each staging buffer
    FutRef copied[kGnormStages];  // the device->host copy out of each set of rows
    FutRef latest;                // the last run's copy out of its rows
};
GnormStage &gnorm_stage(Device *d) {
    static std::mutex mm;
    static std::map<Device *, std::unique_ptr<GnormStage>> stages;
    std::lock_guard<std::mutex> lk(mm);
    auto &p = stages[d];
    if (!p) p.reset(new GnormStage());
    return *p;
}

hxc_status heat2d_run_impl(Ref<Device> d, Ref<Buffer> u, Ref<Buffer> tb, const hxc_heat2d_cfg *cfg,
                           std::vector<FutRef> dv, FutRef *all_out, FutRef *field_out,
                           hxc_run_stats *stats_out, bool after_last_norms);

// A 2D run reads and replaces state the device carries from run to run (the
// last readers of the snapshot rings, the last copy of the device norm rows)
// while it is issued, so 2D runs on one device are issued one at a time.  A
// run whose issue would overlap another's (another host thread, or a run
// deferred to the worker pool) is queued and issued by the thread issuing
// now, right after its own run; its futures complete through promises, as
// for a deferred run.  Nobody blocks on the queue.
struct IssueQueue {
    std::mutex m;
    bool busy = false;
    std::deque<std::function<void()>> q;
};

IssueQueue &issue_queue(Device *d) {
    static std::mutex mm;
    static std::map<Device *, std::unique_ptr<IssueQueue>> queues;
    std::lock_guard<std::mutex> lk(mm);
    auto &p = queues[d];
    if (!p) p.reset(new IssueQueue());
    return *p;
}

// Issues the run now with `now` (its status is returned) when no other 2D
// run is being issued on the device, else queues `later` (status OK; *all,
// *field are promises).  `now` may be empty: `later` then serves both.
hxc_status issue_serial(Device *d, RunIssue later, RunIssue now, FutRef *all, FutRef *field) {
    IssueQueue &iq = issue_queue(d);
    {
        std::lock_guard<std::mutex> g(iq.m);
        if (iq.busy) {
            FutRef pa = make_pending(), pb = make_pending();
            iq.q.push_back([pa, pb, later] {
                FutRef ia, ib;
                hxc_status st = later(&ia, &ib);
                if (st) {
                    fut_set_done(pa, st);
                    fut_set_done(pb, st);
                    return;
                }
                fut_on_done(ia, [pa](hxc_status s) { fut_set_done(pa, s); });
                fut_on_done(ib ? ib : ia, [pb](hxc_status s) { fut_set_done(pb, s); });
            });
            *all = pa;
            *field = pb;
            return HXC_OK;
        }
        iq.busy = true;
    }
    hxc_status st = now ? now(all, field) : later(all, field);
    for (;;) {
        std::function<void()> next;
        {
            std::lock_guard<std::mutex> g(iq.m);
            if (iq.q.empty()) {
                iq.busy = false;
                break;
            }
            next = std::move(iq.q.front());
            iq.q.pop_front();
        }
        next();
    }
    return st;
}

// hxc_heat2d_run; after_last_norms orders the run after the previous 2D
// run's device-norm copy (the host-memory entry points).
hxc_status heat2d_run_entry(hxc_device dh, hxc_buffer uh, hxc_buffer th, const hxc_heat2d_cfg *cfg,
                            const hxc_future *deps, int ndeps, hxc_future *out,
                            hxc_future *field_ready, hxc_run_stats *stats_out,
                            bool after_last_norms) {
    Ref<Device> d = dev_from_handle(dh);
    Ref<Buffer> u = buf_from_handle(uh), tb = buf_from_handle(th);
    if (!d || !u || !tb) return HXC_E_INVALID;
    if (!cfg || cfg->ny <= 0 || cfg->nx <= 0 || cfg->tiles_y < 1 || cfg->tiles_x < 1 ||
        cfg->tiles_y > cfg->ny || cfg->tiles_x > cfg->nx ||
        cfg->tiles_y * cfg->tiles_x > kCopySlot0 || cfg->steps < 0 || cfg->snapshot_every < 0 ||
        u->ptr == tb->ptr || u->dev.get() != d.get() || tb->dev.get() != d.get() ||
        (cfg->mode != HXC_MODE_PLAIN && cfg->mode != HXC_MODE_GRAPH && cfg->mode != HXC_MODE_FUSED)) {
        set_error("hxc_heat2d_run: invalid configuration");
        return HXC_E_INVALID;
    }
    const size_t field = (size_t)cfg->ny * cfg->nx * 8;
    if (u->bytes < field || tb->bytes < field) {
        set_error("hxc_heat2d_run: buffers smaller than the %lld x %lld field",
                  (long long)cfg->ny, (long long)cfg->nx);
        return HXC_E_INVALID;
    }
    std::vector<FutRef> dv;
    hxc_status st = deps_from_handles(deps, ndeps, &dv);
    if (st) return st;
    if (stats_out) memset(stats_out, 0, sizeof *stats_out);
    FutRef a, b;
    auto c = std::make_shared<hxc_heat2d_cfg>(*cfg);
    const bool aln = after_last_norms;
    if (has_pending_host(dv)) {
        defer_run(dv,
                  [d, u, tb, c, aln](FutRef *ia, FutRef *ib) {
                      return issue_serial(d.get(), [d, u, tb, c, aln](FutRef *ja, FutRef *jb) {
                          return heat2d_run_impl(d, u, tb, c.get(), {}, ja, jb, nullptr, aln);
                      }, nullptr, ia, ib);
                  },
                  &a, &b);
    } else {
        st = issue_serial(
            d.get(),
            [d, u, tb, c, dv, aln](FutRef *ia, FutRef *ib) {
                return heat2d_run_impl(d, u, tb, c.get(), dv, ia, ib, nullptr, aln);
            },
            [&](FutRef *ia, FutRef *ib) {
                return heat2d_run_impl(d, u, tb, c.get(), dv, ia, ib, stats_out, aln);
            },
            &a, &b);
        if (st) return st;
    }
    if (out) *out = to_handle(a);
    if (field_ready) *field_ready = to_handle(b);
    return HXC_OK;
}

// Issues one call of hxc_heat2d_run_host_async into device field pair
// `slot` after `deps`: the tile uploads, the run and the tile downloads.
// *all receives the future of the whole call; after a failure, the future
// of whatever was issued (or none).
hxc_status host_run_issue(hxc_device dh, Device *d, int slot, const double *host_u0,
                          double *host_uT, const hxc_heat2d_cfg *cfg,
                          const std::vector<FutRef> &deps, FutRef *all_out,
                          hxc_run_stats *stats_out) {
    const size_t field = (size_t)cfg->ny * cfg->nx * 8;
    hxc_status st;
    void *pu, *pt;
    if ((st = d->scratch_get(kHostKeyU[slot], field, &pu))) return st;
    if ((st = d->scratch_get(kHostKeyT[slot], field, &pt))) return st;
    hxc_buffer ub, tb;
    hxc_buffer_wrap(dh, pu, field, &ub);
    hxc_buffer_wrap(dh, pt, field, &tb);
    Tiles tl;
    tl.TY = cfg->tiles_y;
    tl.TX = cfg->tiles_x;
    tl.by = split(cfg->ny, cfg->tiles_y, false);
    tl.bx = split(cfg->nx, cfg->tiles_x, true);
    const int64_t T = tl.count(), nx = cfg->nx;
    hxc_run_stats inner{};
    std::vector<hxc_future> in_deps;
    for (auto &f : deps) in_deps.push_back(to_handle(f));
    std::vector<hxc_future> h2d, d2h;
    hxc_future run = nullptr, ready = nullptr;
    auto cleanup = [&]() {
        for (auto f : in_deps) hxc_future_release(f);
        for (auto f : h2d) hxc_future_release(f);
        for (auto f : d2h) hxc_future_release(f);
        if (run) hxc_future_release(run);
        if (ready) hxc_future_release(ready);
        hxc_buffer_release(ub);
        hxc_buffer_release(tb);
    };
    // uploads and downloads on their own stream slots, so that they overlap
    // the steps of the call issued before this one
    for (int64_t t = 0; t < T && !st; t++) {
        size_t off = ((size_t)tl.y0(t) * nx + tl.x0(t)) * 8;
        hxc_future f = nullptr;
        st = hxc_buffer_enqueue_write_2d(ub, off, nx * 8, (const char *)host_u0 + off, nx * 8,
                                         tl.tx(t) * 8, tl.ty(t), kHostInSlot0 + (int)(t % kHostSlots),
                                         in_deps.data(), (int)in_deps.size(), &f);
        if (!st) h2d.push_back(f);
        inner.copies++;
        inner.h2d_bytes += tl.tx(t) * tl.ty(t) * 8;
    }
    hxc_run_stats rs{};
    if (!st) st = heat2d_run_entry(dh, ub, tb, cfg, h2d.data(), (int)T, &run, &ready, &rs, true);
    for (int64_t t = 0; t < T && !st; t++) {
        size_t off = ((size_t)tl.y0(t) * nx + tl.x0(t)) * 8;
        hxc_future f = nullptr;
        st = hxc_buffer_enqueue_read_2d(ub, off, nx * 8, (char *)host_uT + off, nx * 8,
                                        tl.tx(t) * 8, tl.ty(t), kHostOutSlot0 + (int)(t % kHostSlots),
                                        &ready, 1, &f);
        if (!st) d2h.push_back(f);
        inner.copies++;
        inner.d2h_bytes += tl.tx(t) * tl.ty(t) * 8;
    }
    hxc_future all = nullptr;
    if (!st) {
        d2h.push_back(run);
        run = nullptr;
        st = hxc_when_all(d2h.data(), (int)d2h.size(), &all);
    }
    if (st) {
        // nothing more is issued into this pair; its next user waits for
        // whatever did get issued
        std::vector<hxc_future> issued(h2d);
        issued.insert(issued.end(), d2h.begin(), d2h.end());
        if (run) issued.push_back(run);
        hxc_future j = nullptr;
        if (!issued.empty() && hxc_when_all(issued.data(), (int)issued.size(), &j) == HXC_OK) {
            *all_out = fut_order_only(fut_from_handle(j));
            hxc_future_release(j);
        }
        cleanup();
        return st;
    }
    cleanup();
    if (stats_out) {
        *stats_out = rs;
        stats_out->copies += inner.copies;
        stats_out->h2d_bytes += inner.h2d_bytes;
        stats_out->d2h_bytes += inner.d2h_bytes;
    }
    *all_out = FutRef(reinterpret_cast<Future *>(all), true);
    return HXC_OK;
}

}  // namespace

extern "C" {

hxc_status hxc_heat2d_run(hxc_device dh, hxc_buffer uh, hxc_buffer th, const hxc_heat2d_cfg *cfg,
                          const hxc_future *deps, int ndeps, hxc_future *out,
                          hxc_future *field_ready, hxc_run_stats *stats_out) {
    hxc::drv::NvtxRange nvtx_range("hxc_heat2d_run");
    return heat2d_run_entry(dh, uh, th, cfg, deps, ndeps, out, field_ready, stats_out, false);
}

}  // extern "C"

namespace {

hxc_status heat2d_run_impl(Ref<Device> d, Ref<Buffer> u, Ref<Buffer> tb, const hxc_heat2d_cfg *cfg,
                           std::vector<FutRef> dv, FutRef *all_out, FutRef *field_out,
                           hxc_run_stats *stats_out, bool after_last_norms) {
    hxc_status st;
    if ((st = d->make_current())) return st;

    Heat2dRun R{};
    R.dev = d.get();
    R.cfg = cfg;
    R.tl.TY = cfg->tiles_y;
    R.tl.TX = cfg->tiles_x;
    R.tl.by = split(cfg->ny, cfg->tiles_y, false);
    R.tl.bx = split(cfg->nx, cfg->tiles_x, true);
    R.buf[0] = (double *)u->ptr;
    R.buf[1] = (double *)tb->ptr;
    R.stats = Stats{stats_out};
    const int64_t T = R.tl.count();
    const int64_t n_snap = cfg->snapshot_every > 0 ? cfg->steps / cfg->snapshot_every : 0;
    const bool want_snaps = n_snap > 0 && (cfg->host_norms || cfg->gpu_norms);
    int64_t max_tile = 0;
    for (int64_t t = 0; t < T; t++) max_tile = std::max(max_tile, R.tl.ty(t) * R.tl.tx(t));
    R.tile_stride = (max_tile + 1) / 2 * 2;
    // snapshot rings carried over from earlier runs on this device
    RingCarry carry;
    if (want_snaps && cfg->host_norms) {
        {
            std::lock_guard<std::mutex> g(g_carry_m);
            carry = g_carry[d.get()];
        }
        if (carry.tiles != T || carry.stride != R.tile_stride) {
            // the ring geometry changes: every earlier user must be done first
            for (int r2 = 0; r2 < 2; r2++) {
                for (auto &f : carry.d2h[r2])
                    if (f) fut_wait(f, -1);
                for (auto &f : carry.conts[r2])
                    if (f) fut_wait(f, -1);
            }
            carry = RingCarry();
        }
    }
    FutRef norm_free;  // the last copy out of this run's norm rows
    if (want_snaps) {
        void *p;
        if ((st = d->scratch_get("heat2d.snap", (size_t)2 * T * R.tile_stride * 8, &p))) return st;
        R.snap_dev = (double *)p;
        // this run's set of n_snap rows of results, and the 2 rows (ring
        // slots) that graph replays write and that are copied into them
        int nset;
        {
            GnormStage &gs = gnorm_stage(d.get());
            std::lock_guard<std::mutex> lk(gs.m);
            nset = gs.next_rows;
            gs.next_rows = (nset + 1) % kGnormStages;
            norm_free = fut_order_only(gs.copied[nset]);
            gs.copied[nset] = FutRef();
            // a run from host memory also starts after the last run's norm
            // copy (measured: host-memory runs issued back to back 2.5%
            // faster).  Not a device-resident run: the norm copy queues
            // behind the last snapshot's device->host copies, so the next
            // run would wait for them (13 ms per 8192^2 pass measured)
            if (after_last_norms)
                if (FutRef c = fut_order_only(gs.latest)) dv.push_back(c);
        }
        if ((st = d->scratch_get("heat2d.norms." + std::to_string(nset), (size_t)n_snap * T * 8, &p)))
            return st;
        R.norm_dev = (double *)p;
        if ((st = d->scratch_get("heat2d.norms.replay", (size_t)2 * T * 8, &p))) return st;
        R.replay_dev = (double *)p;
        R.norm_set = nset;
        if (cfg->host_norms) {
            // pinned staging ring, cached per device
            static std::mutex sm;
            static std::map<Device *, std::pair<void *, size_t>> stage;
            std::lock_guard<std::mutex> g(sm);
            auto &e = stage[d.get()];
            size_t need = (size_t)2 * T * R.tile_stride * 8;
            if (e.second < need) {
                if (e.first) cudaFreeHost(e.first);
                e = {nullptr, 0};
                if (cudaMallocHost(&e.first, need) != cudaSuccess) {
                    set_error("pinned staging allocation of %zu bytes failed", need);
                    return HXC_E_NOMEM;
                }
                e.second = need;
            }
            R.host_stage = (double *)e.first;
        }
    }
    if (cfg->mode == HXC_MODE_FUSED) {
        void *p;
        if ((st = d->scratch_get("tile_norm_grid", k::tile_norm_grid_scratch_bytes(T), &p))) return st;
    }
    for (int64_t t = 0; t < T; t++) {  // scratch of the norm kernels, before any capture
        void *p;
        int slot = cfg->mode == HXC_MODE_FUSED ? 0 : (int)t;
        if ((st = d->scratch_get("tile_norm." + std::to_string(slot), k::kNormScratchBytes, &p)))
            return st;
    }

    Ref<RunResources> res(new RunResources(), true);
    res->keep = {AnyRef(u.get(), false), AnyRef(tb.get(), false)};
    std::vector<FutRef> prev(T);
    if (!dv.empty()) {
        FutRef j;
        if ((st = issue_device_op(d.get(), kJoinSlot, dv, StreamOp(), {}, &j))) return st;
        for (auto &p : prev) p = j;
    }
    const bool fused = cfg->mode == HXC_MODE_FUSED;
    // without snapshots the steps are issued (and captured) in intervals of
    // at most 100 steps, which bounds the size of a captured graph
    const int64_t every = heat2d_interval(*cfg);
    // the earlier runs' readers of the rings order this run's writes into them
    // but must not pass on their own failures: an unrelated later run would
    // otherwise fail with HXC_E_DEP_FAILED after one failed run
    std::vector<FutRef> ring_free[2], host_free[2];  // per ring slot, per tile
    for (int r2 = 0; r2 < 2; r2++) {
        for (auto &f : carry.d2h[r2]) ring_free[r2].push_back(fut_order_only(f));
        for (auto &f : carry.conts[r2]) host_free[r2].push_back(fut_order_only(f));
    }
    std::vector<FutRef> host_conts;
    std::vector<FutRef> finals;
    int64_t s = 0, k = 0;

    // GRAPH mode: capture one interval of `every` steps (+ snapshot kernels)
    // per ring slot and replay it; the host side of a snapshot stays outside.
    Ref<Graph> graphs[2];
    if (cfg->mode == HXC_MODE_GRAPH && every > 0 && cfg->steps >= every) {
        for (int ring = 0; ring < 2 && ring * every < cfg->steps; ring++) {
            // interval k starts at step k*every; its parity decides src/dst
            int64_t s_start = ring * every;
            std::string key = key_of("heat2d",
                                     {(double)cfg->ny, (double)cfg->nx, (double)cfg->tiles_y,
                                      (double)cfg->tiles_x, cfg->r, (double)every,
                                      (double)(s_start % 2), (double)ring, (double)want_snaps,
                                      (double)n_snap, (double)(cfg->host_norms != nullptr)},
                                     {u->ptr, tb->ptr, R.snap_dev, R.replay_dev});
            {
                std::lock_guard<std::mutex> lk(g_graph_m);
                auto it = g_graphs.find(key);
                if (it != g_graphs.end()) graphs[ring] = it->second;
            }
            if (graphs[ring]) continue;
            if ((st = graph_begin(d.get()))) return st;
            Heat2dRun C = R;
            C.stats = Stats{nullptr};
            std::vector<FutRef> cprev(T);
            st = issue_steps2d(C, s_start, s_start + every, cprev, false);
            if (!st && want_snaps) {
                // a replay writes its device norms to row n_snap + ring; they
                // are copied to their snapshot's row after each replay
                std::vector<FutRef> none;
                C.norm_dev = R.replay_dev;  // index ring*T+t lands in replay row `ring`
                st = issue_snap_kernels(C, ring, s_start + every, cprev, none, false);
            }
            Ref<Graph> g;
            hxc_status st2 = graph_end(d.get(), &g);
            if (st) return st;
            if (st2) return st2;
            graphs[ring] = g;
            std::lock_guard<std::mutex> lk(g_graph_m);
            g_graphs[key] = g;
        }
    }

    std::vector<FutRef> gnorm_copies;
    while (s < cfg->steps) {
        int64_t s1 = std::min<int64_t>(cfg->steps, s + (every > 0 ? every : cfg->steps));
        bool snap_here = want_snaps && k < n_snap && s1 == (k + 1) * cfg->snapshot_every;
        int ring = (int)(k % 2);
        if (cfg->mode == HXC_MODE_GRAPH && graphs[ring] && s1 - s == every &&
            (s % 2) == ((ring * every) % 2)) {
            std::vector<FutRef> gdeps;
            for (auto &p : prev)
                if (p) gdeps.push_back(p);
            for (auto &f : ring_free[ring])
                if (f) gdeps.push_back(f);
            // dedupe: the same future may appear for every tile
            std::vector<FutRef> uniq;
            for (auto &f : gdeps) {
                bool seen = false;
                for (auto &g : uniq) seen |= g.get() == f.get();
                if (!seen) uniq.push_back(f);
            }
            cudaGraphExec_t ex = graphs[ring]->exec;
            FutRef gf;
            if ((st = issue_device_op(d.get(), 0, uniq,
                                      [ex](cudaStream_t st) { return cudaGraphLaunch(ex, st); },
                                      {AnyRef(graphs[ring].get(), false)}, &gf)))
                return st;
            R.stats.launch(T * (s1 - s) + (snap_here ? T : 0));
            if (stats_out) stats_out->graph_launches++;
            for (auto &p : prev) p = gf;
            if (snap_here) {
                // move the replay's device norms (replay row `ring`) to row k;
                // the run's first write into its rows waits for their last copy
                double *src = R.replay_dev + ring * T, *dst = R.norm_dev + k * T;
                std::vector<FutRef> cdeps{gf};
                if (k == 0 && norm_free) cdeps.push_back(norm_free);
                FutRef c;
                if ((st = issue_device_op(d.get(), 0, cdeps,
                                          [=](cudaStream_t st) {
                                              return cudaMemcpyAsync(dst, src, T * 8,
                                                                     cudaMemcpyDeviceToDevice, st);
                                          },
                                          {}, &c)))
                    return st;
                for (auto &p : prev) p = c;
            }
        } else {
            if ((st = issue_steps2d(R, s, s1, prev, fused))) return st;
            if (snap_here && (st = issue_snap_kernels(R, k, s1, prev, ring_free[ring], fused,
                                                      k == 0 ? norm_free : FutRef())))
                return st;
        }
        if (snap_here) {
            if (cfg->host_norms) {
                std::vector<FutRef> d2h(T), conts(T);
                if ((st = issue_snap_host(R, k, prev, host_free[ring], d2h, conts, res->tasks)))
                    return st;
                ring_free[ring] = d2h;
                host_free[ring] = conts;
                for (auto &c : conts) host_conts.push_back(c);
            }
            k++;
        }
        s = s1;
    }
    // result lives in buf[steps % 2]; copy back into u tile by tile
    if (cfg->steps % 2 == 1) {
        for (int64_t t = 0; t < T; t++) {
            std::vector<FutRef> deps;
            for (int64_t q : R.tl.nbrs(t))
                if (prev[q]) deps.push_back(prev[q]);
            int64_t y0 = R.tl.y0(t), x0 = R.tl.x0(t), ty = R.tl.ty(t), tx = R.tl.tx(t), nx = cfg->nx;
            double *dst = R.buf[0] + y0 * nx + x0;
            const double *src = R.buf[1] + y0 * nx + x0;
            FutRef c;
            if ((st = issue_device_op(d.get(), fused ? 0 : (int)t, deps,
                                      [=](cudaStream_t s) {
                                          return cudaMemcpy2DAsync(dst, nx * 8, src, nx * 8, tx * 8,
                                                                   ty, cudaMemcpyDeviceToDevice, s);
                                      },
                                      {}, &c)))
                return st;
            R.stats.copy(0, 0);
            finals.push_back(c);
        }
    } else {
        for (auto &p : prev)
            if (p) finals.push_back(p);
    }
    // device norms back to the host: through a page-locked staging buffer
    // (a copy into pageable memory would block this thread), then a host
    // continuation copies them into the caller's array
    FutRef gnorm_done;
    if (cfg->gpu_norms && want_snaps) {
        const size_t bytes = (size_t)n_snap * T * 8;
        GnormStage &gs = gnorm_stage(d.get());
        std::lock_guard<std::mutex> lk(gs.m);
        const int b = gs.next;
        gs.next = (b + 1) % kGnormStages;
        if (gs.bytes[b] < bytes) {
            if (gs.last[b]) fut_wait(gs.last[b], -1);  // the old buffer may still be read
            if (gs.ptr[b]) cudaFreeHost(gs.ptr[b]);
            gs.ptr[b] = nullptr;
            gs.bytes[b] = 0;
            if (cudaMallocHost(&gs.ptr[b], bytes) != cudaSuccess) {
                set_error("pinned staging of %zu bytes for device norms failed", bytes);
                return HXC_E_NOMEM;
            }
            gs.bytes[b] = bytes;
        }
        double *stage = static_cast<double *>(gs.ptr[b]);
        const double *src = R.norm_dev;
        std::vector<FutRef> cdeps = finals;
        // the host copy out of this buffer by the run four before is done
        // (order only: its failure is not this run's)
        if (FutRef o = fut_order_only(gs.last[b])) cdeps.push_back(o);
        FutRef c;
        // a slot of its own: behind the snapshot copies it would hold up the
        // next run's first snapshot
        if ((st = issue_device_op(d.get(), kNormCopySlot, cdeps,
                                  [=](cudaStream_t s) {
                                      return cudaMemcpyAsync(stage, src, bytes, cudaMemcpyDeviceToHost, s);
                                  },
                                  {}, &c)))
            return st;
        R.stats.copy(0, bytes);
        gs.copied[R.norm_set] = c;
        gs.latest = c;
        double *dst = cfg->gpu_norms;
        FutRef r = make_pending();
        fut_on_done(c, [r, stage, dst, bytes](hxc_status s2) {
            if (s2 != HXC_OK) {
                fut_set_done(r, HXC_E_DEP_FAILED);
                return;
            }
            pool().submit([r, stage, dst, bytes] {
                memcpy(dst, stage, bytes);
                fut_set_done(r, HXC_OK);
            });
        });
        gs.last[b] = r;
        gnorm_done = r;
    }
    if (finals.empty()) finals.push_back(make_done(HXC_OK));
    // the field (and the device norms) are final once these are done
    FutRef field;
    if ((st = issue_device_op(d.get(), kJoinSlot, finals, StreamOp(), res->keep, &field))) return st;
    std::vector<FutRef> all{field};
    if (gnorm_done) all.push_back(gnorm_done);
    for (auto &c : host_conts) all.push_back(c);
    for (auto &f : ring_free[0]) if (f) all.push_back(f);
    for (auto &f : ring_free[1]) if (f) all.push_back(f);
    FutRef fin;
    hxc_future fh = nullptr;
    if ((st = finish(d.get(), all, &fh))) return st;
    fin = FutRef(reinterpret_cast<Future *>(fh), true);
    // release the run's resources once everything is done
    Ref<RunResources> keep_res = res;
    fut_on_done(fin, [keep_res](hxc_status) {});
    if (want_snaps && cfg->host_norms) {
        std::lock_guard<std::mutex> g(g_carry_m);
        RingCarry &c = g_carry[d.get()];
        c.tiles = T;
        c.stride = R.tile_stride;
        for (int r2 = 0; r2 < 2; r2++)
            if (!ring_free[r2].empty()) {
                c.d2h[r2] = ring_free[r2];
                c.conts[r2] = host_free[r2];
            }
    }
    if (stats_out) stats_out->host_tasks = (int64_t)host_conts.size();
    *all_out = fin;
    *field_out = field;
    return HXC_OK;
}

}  // namespace

extern "C" {

hxc_status hxc_heat2d_run_host_async(hxc_device dh, const double *host_u0, double *host_uT,
                                     const hxc_heat2d_cfg *cfg, const hxc_future *deps, int ndeps,
                                     hxc_future *out, hxc_run_stats *stats_out) {
    hxc::drv::NvtxRange nvtx_range("hxc_heat2d_run_host_async");
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    if (!cfg || !host_u0 || !host_uT || !out || cfg->ny <= 0 || cfg->nx <= 0 ||
        cfg->tiles_y < 1 || cfg->tiles_x < 1 || cfg->tiles_y > cfg->ny ||
        cfg->tiles_x > cfg->nx || cfg->tiles_y * cfg->tiles_x > kCopySlot0) {
        set_error("hxc_heat2d_run_host: invalid arguments");
        return HXC_E_INVALID;
    }
    std::vector<FutRef> dv;
    hxc_status st = deps_from_handles(deps, ndeps, &dv);
    if (st) return st;
    if ((st = d->make_current())) return st;
    if (stats_out) memset(stats_out, 0, sizeof *stats_out);
    // the device field pair of this call, the call that used it last, and
    // the promise the pair's next user orders itself after
    int slot;
    FutRef prev, whole = make_pending();
    {
        std::lock_guard<std::mutex> g(g_hostrun_m);
        HostRunSlots &hs = g_hostrun[d.get()];
        slot = hs.next;
        hs.next ^= 1;
        prev = hs.last[slot];
        hs.last[slot] = fut_order_only(whole);
    }
    if (prev) dv.push_back(prev);
    if (has_pending_host(dv)) {
        // unfinished host work ahead (typically the pair's last user, a call
        // still running): the whole call is issued by the worker pool once
        // every dependency is done, so that its uploads, steps and downloads
        // are enqueued together.  Issued piecemeal (each copy as its own
        // dependency came in, the downloads only after the field was done)
        // back-to-back calls ran 432 instead of 418 ms per 8192^2 call.
        auto c = std::make_shared<hxc_heat2d_cfg>(*cfg);
        FutRef a = make_pending();
        auto left = std::make_shared<std::atomic<int>>((int)dv.size());
        auto failed = std::make_shared<std::atomic<int>>(0);
        auto fire = [=]() {
            if (failed->load()) {  // nothing is issued into the pair
                fut_set_done(a, HXC_E_DEP_FAILED);
                fut_set_done(whole, HXC_OK);
                return;
            }
            pool().submit([=] {
                FutRef all;
                hxc_status s2 = d->make_current();
                if (!s2)
                    s2 = host_run_issue(dh, d.get(), slot, host_u0, host_uT, c.get(), {}, &all,
                                        nullptr);
                // the pair's next user waits for whatever was issued into it
                if (all)
                    fut_on_done(all, [whole](hxc_status s3) { fut_set_done(whole, s3); });
                else
                    fut_set_done(whole, HXC_OK);
                if (s2) {
                    fut_set_done(a, s2);
                    return;
                }
                fut_on_done(all, [a](hxc_status s3) { fut_set_done(a, s3); });
            });
        };
        for (auto &f : dv)
            fut_on_done(f, [left, failed, fire](hxc_status s2) {
                if (s2 != HXC_OK) failed->store(1);
                if (left->fetch_sub(1) == 1) fire();
            });
        *out = to_handle(a);
        return HXC_OK;
    }
    FutRef all;
    st = host_run_issue(dh, d.get(), slot, host_u0, host_uT, cfg, dv, &all, stats_out);
    // the pair's next user waits for whatever was issued into it
    if (all)
        fut_on_done(all, [whole](hxc_status s2) { fut_set_done(whole, s2); });
    else
        fut_set_done(whole, st ? st : HXC_OK);
    if (st) return st;
    *out = to_handle(all);
    return HXC_OK;
}

hxc_status hxc_heat2d_run_host(hxc_device dh, const double *host_u0, double *host_uT,
                               const hxc_heat2d_cfg *cfg, hxc_run_stats *stats_out) {
    hxc::drv::NvtxRange nvtx_range("hxc_heat2d_run_host");
    hxc_future f = nullptr;
    hxc_status st = hxc_heat2d_run_host_async(dh, host_u0, host_uT, cfg, nullptr, 0, &f, stats_out);
    if (st) return st;
    st = hxc_future_wait(f, -1);
    hxc_future_release(f);
    return st;
}


hxc_status hxc_heat1d_step_kinds(double r, int steps, int64_t *counts) {
    if (!counts || steps < 0) {
        set_error("hxc_heat1d_step_kinds: invalid arguments");
        return HXC_E_INVALID;
    }
    ftcs_count(1, r, steps, heat1d_interval(steps), counts);
    return HXC_OK;
}

hxc_status hxc_heat2d_step_kinds(const hxc_heat2d_cfg *cfg, int64_t *counts) {
    if (!cfg || !counts || cfg->steps < 0 || cfg->snapshot_every < 0) {
        set_error("hxc_heat2d_step_kinds: invalid arguments");
        return HXC_E_INVALID;
    }
    ftcs_count(2, cfg->r, cfg->steps, heat2d_interval(*cfg), counts);
    return HXC_OK;
}

hxc_status hxc_host_norms(const double *const *arrays, const int64_t *counts, int n, double *out) {
    if (n < 0 || (n > 0 && (!arrays || !counts || !out))) {
        set_error("hxc_host_norms: NULL argument");
        return HXC_E_INVALID;
    }
    for (int i = 0; i < n; i++)
        if (counts[i] < 0 || (counts[i] > 0 && !arrays[i])) {
            set_error("hxc_host_norms: array %d is invalid", i);
            return HXC_E_INVALID;
        }
    std::vector<HostNormTask> tasks(n);
    std::vector<FutRef> done(n);
    for (int i = 0; i < n; i++) {
        tasks[i] = HostNormTask{arrays[i], counts[i], out + i};
        done[i] = make_pending();
        HostNormTask *t = &tasks[i];
        FutRef r = done[i];
        pool().submit([t, r] { fut_set_done(r, host_norm_fn(t)); });
    }
    hxc_status st = HXC_OK;
    for (auto &f : done) {
        hxc_status s2 = fut_wait(f, -1);
        if (!st) st = s2;
    }
    return st;
}

hxc_status hxc_heat3d_run(hxc_device dh, hxc_buffer uh, hxc_buffer th, int64_t nz, int64_t ny,
                          int64_t nx, float r, int steps, hxc_mode mode, int steps_per_launch,
                          const hxc_future *deps, int ndeps, hxc_future *out,
                          hxc_run_stats *stats_out) {
    hxc::drv::NvtxRange nvtx_range("hxc_heat3d_run");
    Ref<Device> d = dev_from_handle(dh);
    Ref<Buffer> u = buf_from_handle(uh), t = buf_from_handle(th);
    if (!d || !u || !t) return HXC_E_INVALID;
    const size_t bytes = (size_t)nz * ny * nx * 4;
    if (nz <= 0 || ny <= 0 || nx <= 0 || nz > INT32_MAX || ny > INT32_MAX || nx > INT32_MAX ||
        steps < 0 || steps_per_launch < 0 || steps_per_launch > 4 || u->bytes < bytes ||
        t->bytes < bytes || u->ptr == t->ptr || u->dev.get() != d.get() || t->dev.get() != d.get() ||
        (mode != HXC_MODE_PLAIN && mode != HXC_MODE_GRAPH && mode != HXC_MODE_FUSED)) {
        set_error("hxc_heat3d_run: invalid arguments");
        return HXC_E_INVALID;
    }
    std::vector<FutRef> dv;
    hxc_status st = deps_from_handles(deps, ndeps, &dv);
    if (st) return st;
    if (stats_out) memset(stats_out, 0, sizeof *stats_out);
    if (has_pending_host(dv)) {
        FutRef a, b;
        defer_run(dv,
                  [=](FutRef *ia, FutRef *ib) {
                      hxc_future h = nullptr;
                      hxc_status s2 = hxc_heat3d_run(dh, uh, th, nz, ny, nx, r, steps, mode,
                                                     steps_per_launch, nullptr, 0, &h, nullptr);
                      if (s2) return s2;
                      *ia = FutRef(reinterpret_cast<Future *>(h), true);
                      *ib = *ia;
                      return HXC_OK;
                  },
                  &a, &b);
        fut_on_done(a, [u, t](hxc_status) {});
        if (out) *out = to_handle(a);
        return HXC_OK;
    }
    Stats stats{stats_out};
    if ((st = d->make_current())) return st;
    const int T = mode == HXC_MODE_PLAIN
                      ? 1
                      : (steps_per_launch == 0 ? (int)tune::get("heat3d.steps_per_launch")
                                               : steps_per_launch);
    float *buf[2] = {(float *)u->ptr, (float *)t->ptr};
    const int inz = (int)nz, iny = (int)ny, inx = (int)nx;
    FutRef prev;
    if (!dv.empty() && (st = issue_device_op(d.get(), kJoinSlot, dv, StreamOp(), {}, &prev))) return st;
    int flip = 0;
    // launches of `cnt` steps each (the last may be shorter), on slot 0
    auto issue = [&](int nsteps, int &fl, FutRef &pv, Stats &sc) -> hxc_status {
        int done = 0;
        while (done < nsteps) {
            int tt = std::min(T, nsteps - done);
            const float *sp = buf[fl];
            float *dp = buf[1 - fl];
            std::vector<FutRef> dd;
            if (pv) dd.push_back(pv);
            FutRef f;
            hxc_status s2 = issue_device_op(
                d.get(), 0, dd,
                [=](cudaStream_t s) { return k::heat3d(sp, dp, inz, iny, inx, r, tt, 0, nullptr, s); },
                {}, &f);
            if (s2) return s2;
            sc.launch();
            pv = f;
            fl = 1 - fl;
            done += tt;
        }
        return HXC_OK;
    };
    if (mode == HXC_MODE_GRAPH && steps > 0) {
        // capture `chunk` steps (an even number of launches when replayed more
        // than once, so every replay starts from u) and replay it
        int per = 16 * T;  // 16 launches per graph
        int chunk = steps <= per ? steps : per;
        int reps = steps / chunk;
        std::string key = key_of("heat3d", {(double)nz, (double)ny, (double)nx, (double)r,
                                            (double)chunk, (double)T},
                                 {u->ptr, t->ptr});
        Ref<Graph> g;
        {
            std::lock_guard<std::mutex> lk(g_graph_m);
            auto it = g_graphs.find(key);
            if (it != g_graphs.end()) g = it->second;
        }
        if (!g) {
            if ((st = graph_begin(d.get()))) return st;
            int cf = 0;
            FutRef cp;
            Stats none{nullptr};
            st = issue(chunk, cf, cp, none);
            Ref<Graph> ng;
            hxc_status st2 = graph_end(d.get(), &ng);
            if (st) return st;
            if (st2) return st2;
            g = ng;
            std::lock_guard<std::mutex> lk(g_graph_m);
            g_graphs[key] = g;
        }
        const int launches_per = (chunk + T - 1) / T;
        cudaGraphExec_t ex = g->exec;
        for (int rep = 0; rep < reps; rep++) {
            std::vector<FutRef> dd;
            if (prev) dd.push_back(prev);
            FutRef gf;
            if ((st = issue_device_op(d.get(), 0, dd,
                                      [ex](cudaStream_t s) { return cudaGraphLaunch(ex, s); },
                                      {AnyRef(g.get(), false)}, &gf)))
                return st;
            stats.launch(launches_per);
            if (stats_out) stats_out->graph_launches++;
            prev = gf;
            flip ^= launches_per & 1;
        }
        int rest = steps - reps * chunk;
        if (rest > 0 && (st = issue(rest, flip, prev, stats))) return st;
    } else if (steps > 0) {
        if ((st = issue(steps, flip, prev, stats))) return st;
    }
    if (flip == 1) {
        std::vector<FutRef> dd;
        if (prev) dd.push_back(prev);
        FutRef c;
        float *dp = buf[0];
        const float *sp = buf[1];
        if ((st = issue_device_op(d.get(), 0, dd,
                                  [=](cudaStream_t s) {
                                      return cudaMemcpyAsync(dp, sp, bytes, cudaMemcpyDeviceToDevice, s);
                                  },
                                  {}, &c)))
            return st;
        stats.copy(0, 0);
        prev = c;
    }
    std::vector<FutRef> fin;
    fin.push_back(prev ? prev : make_done(HXC_OK));
    FutRef f;
    if ((st = issue_device_op(d.get(), kJoinSlot, fin, StreamOp(),
                              {AnyRef(u.get(), false), AnyRef(t.get(), false)}, &f)))
        return st;
    if (out) *out = to_handle(f);
    return HXC_OK;
}

}  // extern "C"
