// Helpers shared by the whole-run entry points (drivers*.cpp).
#pragma once

#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "runtime.hpp"
#include "tune.hpp"

namespace hxc {
namespace drv {

// An NVTX range around the host-side issue of a run entry point (a no-op
// unless a profiler is attached): `ncu --nvtx --nvtx-include "<name>/"`
// then captures only the kernels that entry point launches.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kCopySlot0 = 224;  // slots used for snapshot device->host copies
constexpr int kCopySlots = 16;

// Partition bounds: [bounds[p], bounds[p+1]).  With `even` the interior
// bounds are even (keeps 16-byte alignment of rows of doubles).
inline std::vector<int64_t> split(int64_t n, int64_t parts, bool even) {
    std::vector<int64_t> b(parts + 1);
    for (int64_t p = 0; p <= parts; p++) {
        if (p == parts)
            b[p] = n;
        else if (even && n % 2 == 0)
            b[p] = (p * (n / 2) / parts) * 2;
        else
            b[p] = p * n / parts;
    }
    return b;
}

struct Stats {
    hxc_run_stats *s;
    void launch(int64_t k = 1) {
        if (s) s->kernel_launches += k;
    }
    void copy(int64_t h2d, int64_t d2h) {
        if (!s) return;
        s->copies++;
        s->h2d_bytes += h2d;
        s->d2h_bytes += d2h;
    }
};

// Cache of captured graphs, keyed by the full description of the captured
// work (buffers, shapes, parameters), shared by all drivers.
extern std::mutex g_graph_m;
extern std::map<std::string, Ref<Graph>> g_graphs;

inline std::string key_of(const char *what, std::initializer_list<double> vals,
                   std::initializer_list<const void *> ptrs) {
    std::string k = what;
    char buf[64];
    snprintf(buf, sizeof buf, "|tune%llu", (unsigned long long)tune::generation());
    k += buf;
    for (double v : vals) {
        snprintf(buf, sizeof buf, "|%.17g", v);
        k += buf;
    }
    for (const void *p : ptrs) {
        snprintf(buf, sizeof buf, "|%p", p);
        k += buf;
    }
    return k;
}

inline hxc_status finish(Device *dev, std::vector<FutRef> &finals, hxc_future *out) {
    FutRef r;
    // join on the host only if some final future is host work
    bool host = false;
    for (auto &f : finals) {
        std::lock_guard<std::mutex> g(f->m);
        host |= f->state == Future::PENDING || (f->state == Future::DONE && !f->dev);
    }
    if (!host) {
        hxc_status st = issue_device_op(dev, kJoinSlot, finals, StreamOp(), {}, &r);
        if (st) return st;
    } else {
        r = make_pending();
        struct J {
            std::atomic<int> left{0};
            std::atomic<int> failed{0};
        };
        auto j = std::make_shared<J>();
        j->left = (int)finals.size();
        if (finals.empty()) fut_set_done(r, HXC_OK);
        for (auto &f : finals)
            fut_on_done(f, [r, j](hxc_status s) {
                if (s != HXC_OK) j->failed = 1;
                if (j->left.fetch_sub(1) == 1) fut_set_done(r, j->failed ? HXC_E_DEP_FAILED : HXC_OK);
            });
    }
    if (out) *out = to_handle(r);
    return HXC_OK;
}

// True if some dependency is host work that has not finished.
inline bool has_pending_host(const std::vector<FutRef> &dv) {
    for (auto &f : dv) {
        std::lock_guard<std::mutex> g(f->m);
        if (f->state == Future::PENDING) return true;
    }
    return false;
}

// Issues a whole run later: once every dependency is done, `issue` runs on
// the worker pool; the returned futures follow the ones it produces.
using RunIssue = std::function<hxc_status(FutRef *all, FutRef *field)>;

inline void defer_run(const std::vector<FutRef> &dv, RunIssue issue, FutRef *all_out, FutRef *field_out) {
    FutRef a = make_pending(), b = make_pending();
    struct J {
        std::atomic<int> left{0};
        std::atomic<int> failed{0};
    };
    auto js = std::make_shared<J>();
    js->left = (int)dv.size();
    auto fire = [a, b, js, issue]() {
        if (js->failed) {
            fut_set_done(a, HXC_E_DEP_FAILED);
            fut_set_done(b, HXC_E_DEP_FAILED);
            return;
        }
        pool().submit([a, b, issue] {
            FutRef ia, ib;
            hxc_status st = issue(&ia, &ib);
            if (st) {
                fut_set_done(a, st);
                fut_set_done(b, st);
                return;
            }
            fut_on_done(ia, [a](hxc_status s) { fut_set_done(a, s); });
            fut_on_done(ib ? ib : ia, [b](hxc_status s) { fut_set_done(b, s); });
        });
    };
    for (auto &f : dv)
        fut_on_done(f, [js, fire](hxc_status s) {
            if (s != HXC_OK) js->failed = 1;
            if (js->left.fetch_sub(1) == 1) fire();
        });
    *all_out = a;
    *field_out = b;
}


// Looks up a captured graph under `key`, capturing it with `body` (which
// issues the operations on `dev` and reports how many kernels they launch)
// on a miss.
inline hxc_status cached_graph(Device *dev, const std::string &key,
                               const std::function<hxc_status(int64_t *kernels)> &body,
                               Ref<Graph> *out) {
    {
        std::lock_guard<std::mutex> lk(g_graph_m);
        auto it = g_graphs.find(key);
        if (it != g_graphs.end()) {
            *out = it->second;
            return HXC_OK;
        }
    }
    hxc_status st = graph_begin(dev);
    if (st) return st;
    int64_t kernels = 0;
    st = body(&kernels);
    Ref<Graph> g;
    hxc_status st2 = graph_end(dev, &g);
    if (st) return st;
    if (st2) return st2;
    g->kernels = kernels;
    std::lock_guard<std::mutex> lk(g_graph_m);
    g_graphs[key] = g;
    *out = g;
    return HXC_OK;
}

// Issues a replay of `g` on `slot` after `deps`.
inline hxc_status launch_graph(Device *dev, const Ref<Graph> &g, int slot,
                               const std::vector<FutRef> &deps, FutRef *out) {
    cudaGraphExec_t ex = g->exec;
    return issue_device_op(dev, slot, deps, [ex](cudaStream_t s) { return cudaGraphLaunch(ex, s); },
                           {AnyRef(g.get(), false)}, out);
}

}  // namespace drv
}  // namespace hxc
