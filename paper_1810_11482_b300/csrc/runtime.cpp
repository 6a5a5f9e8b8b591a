// Future layer, devices, buffers and graphs (see runtime.hpp).
#include "runtime.hpp"

#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>

namespace hxc {

// ------------------------------------------------------------------ errors
static thread_local std::string tl_error = "";

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    tl_error = buf;
}

const char *last_error() { return tl_error.c_str(); }

hxc_status cuda_status(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return HXC_OK;
    if (e == cudaErrorMemoryAllocation) {
        set_error("%s: out of device memory", what);
        return HXC_E_NOMEM;
    }
    set_error("%s: %s", what, cudaGetErrorString(e));
    return HXC_E_CUDA;
}

// ------------------------------------------------------------- worker pool
WorkerPool::WorkerPool(int n) {
    for (int i = 0; i < n; i++) threads_.emplace_back([this] { loop(); });
}
WorkerPool::~WorkerPool() { shutdown(); }

void WorkerPool::submit(std::function<void()> fn) {
    {
        std::lock_guard<std::mutex> g(m_);
        if (!stop_) {
            q_.push_back(std::move(fn));
            cv_.notify_one();
            return;
        }
    }
    fn();  // after shutdown: run inline so that no continuation is lost
}

void WorkerPool::loop() {
    for (;;) {
        std::function<void()> fn;
        {
            std::unique_lock<std::mutex> lk(m_);
            cv_.wait(lk, [&] { return stop_ || !q_.empty(); });
            if (q_.empty()) return;  // stop_ and drained
            fn = std::move(q_.front());
            q_.pop_front();
            busy_++;
        }
        fn();
        tasks_run_.fetch_add(1);
        {
            std::lock_guard<std::mutex> g(m_);
            busy_--;
        }
        idle_cv_.notify_all();
    }
}

void WorkerPool::shutdown() {
    {
        std::unique_lock<std::mutex> lk(m_);
        if (stop_ && threads_.empty()) return;
        stop_ = true;
    }
    cv_.notify_all();
    for (auto &t : threads_)
        if (t.joinable()) t.join();
    threads_.clear();
}

static WorkerPool *g_pool = nullptr;
static std::once_flag g_pool_once;

WorkerPool &pool() {
    std::call_once(g_pool_once, [] {
        int n = (int)std::thread::hardware_concurrency();
        const char *env = getenv("HXC_WORKERS");
        if (env && atoi(env) > 0) n = atoi(env);
        if (n < 2) n = 2;
        if (n > 32) n = 32;
        g_pool = new WorkerPool(n);  // intentionally never deleted
    });
    return *g_pool;
}

// ------------------------------------------------------------------ device
static thread_local int tl_current_dev = -1;

hxc_status Device::make_current() {
    if (tl_current_dev == ordinal) return HXC_OK;
    cudaError_t e = cudaSetDevice(ordinal);
    if (e != cudaSuccess) return cuda_status(e, "cudaSetDevice");
    tl_current_dev = ordinal;
    return HXC_OK;
}

Device::~Device() {
    cudaSetDevice(ordinal);
    tl_current_dev = ordinal;
    for (auto s : slots)
        if (s) cudaStreamDestroy(s);
    if (notify) cudaStreamDestroy(notify);
    if (join) cudaStreamDestroy(join);
    if (cap_origin) cudaStreamDestroy(cap_origin);
    if (cap_fork) cudaEventDestroy(cap_fork);
    for (auto e : free_events) cudaEventDestroy(e);
    for (auto &kv : scratch) cudaFree(kv.second.first);
    for (auto p : retired) cudaFree(p);
}

hxc_status Device::stream(int slot, cudaStream_t *s) {
    if (slot < kJoinSlot || slot >= HXC_MAX_SLOTS) {
        set_error("stream slot %d out of range [0, %d)", slot, HXC_MAX_SLOTS);
        return HXC_E_INVALID;
    }
    std::lock_guard<std::mutex> g(m);
    if (capturing && slot == kJoinSlot) {
        *s = cap_origin;
        return HXC_OK;
    }
    cudaStream_t *ps = slot == kJoinSlot ? &join : &slots[slot];
    if (!*ps) {
        hxc_status st = make_current();
        if (st) return st;
        cudaError_t e = cudaStreamCreateWithFlags(ps, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_status(e, "cudaStreamCreate");
    }
    if (capturing && slot >= 0) {
        bool joined = false;
        for (int j : cap_joined) joined |= (j == slot);
        if (!joined) {
            cudaError_t e = cudaStreamWaitEvent(*ps, cap_fork, 0);
            if (e != cudaSuccess) return cuda_status(e, "join capture");
            cap_joined.push_back(slot);
        }
    }
    *s = *ps;
    return HXC_OK;
}

cudaEvent_t Device::get_event() {
    {
        std::lock_guard<std::mutex> g(m);
        if (!free_events.empty()) {
            cudaEvent_t e = free_events.back();
            free_events.pop_back();
            return e;
        }
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

void Device::put_event(cudaEvent_t e) {
    std::lock_guard<std::mutex> g(m);
    free_events.push_back(e);
}

hxc_status Device::scratch_get(const std::string &key, size_t bytes, void **p) {
    std::lock_guard<std::mutex> g(m);
    auto it = scratch.find(key);
    if (it != scratch.end() && it->second.second >= bytes) {
        *p = it->second.first;
        return HXC_OK;
    }
    hxc_status st = make_current();
    if (st) return st;
    if (it != scratch.end()) {
        // operations already issued, or still to be issued from the worker
        // pool, may hold the old pointer: it is kept until the device goes
        retired.push_back(it->second.first);
        scratch.erase(it);
    }
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return cuda_status(e, "scratch cudaMalloc");
    // the library's streams do not synchronize with the legacy stream, so
    // the zero fill is waited for here: work issued after this call must
    // not overtake it
    e = cudaMemsetAsync(q, 0, bytes, cudaStreamLegacy);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
    if (e != cudaSuccess) {
        cudaFree(q);
        return cuda_status(e, "scratch cudaMemset");
    }
    scratch[key] = {q, bytes};
    *p = q;
    return HXC_OK;
}

Buffer::~Buffer() {
    if (owned && ptr) {
        cudaSetDevice(dev->ordinal);
        tl_current_dev = dev->ordinal;
        cudaFree(ptr);
    }
}

// ------------------------------------------------------------------ future
Future::~Future() {
    if (ev) {
        if (captured)
            cudaEventDestroy(ev);
        else
            dev->put_event(ev);
    }
}

FutRef make_pending() { return FutRef(new Future(), true); }

FutRef make_done(hxc_status st) {
    FutRef f(new Future(), true);
    f->state = Future::DONE;
    f->status = st;
    return f;
}

static void CUDART_CB notify_cb(void *p);

// Arms a host notification for an issued device future (caller holds f->m).
static void arm_notify_locked(Future *f) {
    if (f->notify_armed || f->captured) return;
    f->notify_armed = true;
    Device *d = f->dev.get();
    f->retain();  // released by the worker task behind notify_cb
    cudaStream_t ns = nullptr;
    {
        std::lock_guard<std::mutex> g(d->m);
        if (!d->notify) {
            d->make_current();
            cudaStreamCreateWithFlags(&d->notify, cudaStreamNonBlocking);
        }
        ns = d->notify;
    }
    d->make_current();
    cudaError_t e = cudaStreamWaitEvent(ns, f->ev, 0);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(ns, notify_cb, f);
    if (e != cudaSuccess) {
        // could not arm: resolve on the pool by polling instead
        Future *ff = f;
        pool().submit([ff] {
            FutRef r(ff, true);
            fut_wait(r, -1);
        });
    }
}

static void CUDART_CB notify_cb(void *p) {
    // CUDA's callback thread: no CUDA calls here, hand over to the pool.
    Future *f = static_cast<Future *>(p);
    pool().submit([f] {
        FutRef r(f, true);
        int ready = 0;
        fut_poll(r, &ready);
        if (!ready) fut_wait(r, -1);
    });
}

void fut_set_issued(const FutRef &f, Device *dev, cudaEvent_t ev, int slot, bool captured) {
    std::vector<std::function<void()>> leave;
    {
        std::lock_guard<std::mutex> g(f->m);
        f->dev = Ref<Device>(dev, false);
        f->ev = ev;
        f->slot = slot;
        f->captured = captured;
        f->state = Future::ISSUED;
        leave.swap(f->on_leave_pending);
        if (!f->on_done.empty()) arm_notify_locked(f.get());
    }
    f->cv.notify_all();
    for (auto &fn : leave) fn();
}

void fut_set_done(const FutRef &f, hxc_status st) {
    std::vector<std::function<void()>> leave;
    std::vector<std::function<void(hxc_status)>> done;
    {
        std::lock_guard<std::mutex> g(f->m);
        if (f->state == Future::DONE) return;
        f->state = Future::DONE;
        f->status = st;
        leave.swap(f->on_leave_pending);
        done.swap(f->on_done);
    }
    f->cv.notify_all();
    for (auto &fn : leave) fn();
    for (auto &fn : done) fn(st);
}

hxc_status fut_poll(const FutRef &f, int *ready) {
    cudaEvent_t ev;
    Device *d;
    {
        std::lock_guard<std::mutex> g(f->m);
        if (f->state == Future::DONE) {
            *ready = 1;
            return f->status;
        }
        if (f->state == Future::PENDING || f->captured) {
            *ready = 0;
            return HXC_OK;
        }
        ev = f->ev;
        d = f->dev.get();
    }
    d->make_current();
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaErrorNotReady) {
        *ready = 0;
        return HXC_OK;
    }
    hxc_status st = HXC_OK;
    if (e != cudaSuccess) st = cuda_status(e, "device operation");
    fut_set_done(f, st);
    *ready = 1;
    std::lock_guard<std::mutex> g(f->m);
    return f->status;
}

hxc_status fut_wait(const FutRef &f, int64_t timeout_ns) {
    using clk = std::chrono::steady_clock;
    auto t0 = clk::now();
    auto deadline = timeout_ns < 0 ? clk::time_point::max() : t0 + std::chrono::nanoseconds(timeout_ns);
    {
        std::unique_lock<std::mutex> lk(f->m);
        while (f->state == Future::PENDING) {
            if (timeout_ns < 0)
                f->cv.wait(lk);
            else if (f->cv.wait_until(lk, deadline) == std::cv_status::timeout &&
                     f->state == Future::PENDING) {
                set_error("future not ready within the timeout");
                return HXC_E_TIMEOUT;
            }
        }
        if (f->state == Future::DONE) return f->status;
        if (f->captured) {
            set_error("a future recorded during graph capture cannot be waited on");
            return HXC_E_INVALID;
        }
    }
    int spins = 0;
    for (;;) {
        int ready = 0;
        hxc_status st = fut_poll(f, &ready);
        if (ready) return st;
        if (clk::now() >= deadline) {
            set_error("future not ready within the timeout");
            return HXC_E_TIMEOUT;
        }
        if (++spins < 64)
            std::this_thread::yield();
        else
            std::this_thread::sleep_for(std::chrono::microseconds(spins < 1024 ? 5 : 50));
    }
}

void fut_on_done(const FutRef &f, std::function<void(hxc_status)> cb) {
    hxc_status st;
    {
        std::lock_guard<std::mutex> g(f->m);
        if (f->state != Future::DONE) {
            f->on_done.push_back(std::move(cb));
            if (f->state == Future::ISSUED) arm_notify_locked(f.get());
            return;
        }
        st = f->status;
    }
    cb(st);
}

// Calls fn once f is issued or done (inline if it already is).
static void fut_on_leave_pending(const FutRef &f, std::function<void()> fn) {
    {
        std::lock_guard<std::mutex> g(f->m);
        if (f->state == Future::PENDING) {
            f->on_leave_pending.push_back(std::move(fn));
            return;
        }
    }
    fn();
}

FutRef fut_from_handle(hxc_future h) {
    Future *f = reinterpret_cast<Future *>(h);
    if (!f || f->magic != kFutMagic) {
        set_error("invalid future handle");
        return FutRef();
    }
    return FutRef(f, false);
}

Ref<Device> dev_from_handle(hxc_device h) {
    Device *d = reinterpret_cast<Device *>(h);
    if (!d || d->magic != kDevMagic) {
        set_error("invalid device handle");
        return Ref<Device>();
    }
    return Ref<Device>(d, false);
}

Ref<Buffer> buf_from_handle(hxc_buffer h) {
    Buffer *b = reinterpret_cast<Buffer *>(h);
    if (!b || b->magic != kBufMagic) {
        set_error("invalid buffer handle");
        return Ref<Buffer>();
    }
    return Ref<Buffer>(b, false);
}

hxc_status deps_from_handles(const hxc_future *deps, int ndeps, std::vector<FutRef> *v) {
    if (ndeps < 0 || (ndeps > 0 && !deps)) {
        set_error("invalid dependency list");
        return HXC_E_INVALID;
    }
    v->reserve(ndeps);
    for (int i = 0; i < ndeps; i++) {
        FutRef f = fut_from_handle(deps[i]);
        if (!f) return HXC_E_INVALID;
        v->push_back(std::move(f));
    }
    return HXC_OK;
}

// ---------------------------------------------------------- device issue
namespace {
enum DepCheck { DEPS_READY, DEPS_PENDING, DEPS_FAILED, DEPS_INVALID };

// Classifies the dependencies of an operation on `dev`.  Device futures that
// must be waited on are returned in *waits.
DepCheck check_deps(Device *dev, const std::vector<FutRef> &deps, bool capturing,
                    std::vector<std::pair<cudaEvent_t, int>> *waits) {
    for (const auto &f : deps) {
        std::unique_lock<std::mutex> lk(f->m);
        if (f->state == Future::DONE) {
            if (f->status != HXC_OK) return DEPS_FAILED;
            continue;
        }
        if (f->state == Future::PENDING) return DEPS_PENDING;
        // ISSUED
        if (f->captured && !capturing) {
            set_error("a future recorded during graph capture used outside the capture");
            return DEPS_INVALID;
        }
        if (capturing && !f->captured) {
            lk.unlock();
            int ready = 0;
            hxc_status st = fut_poll(f, &ready);
            if (!ready) {
                set_error("dependencies from before a graph capture must be ready");
                return DEPS_INVALID;
            }
            if (st != HXC_OK) return DEPS_FAILED;
            continue;
        }
        (void)dev;
        waits->push_back({f->ev, f->dev.get() == dev ? f->slot : -2});
    }
    return DEPS_READY;
}

struct PendingOp {
    Ref<Device> dev;
    int slot;
    std::vector<FutRef> deps;
    StreamOp op;
    std::vector<AnyRef> keep;
    FutRef out;
};

void issue_now(PendingOp &p);

std::atomic<int64_t> g_inject_left{-1};
std::atomic<int> g_inject_status{HXC_E_CUDA};

// True for exactly one operation: the one the armed countdown reaches.
bool inject_fires() {
    int64_t v = g_inject_left.load(std::memory_order_relaxed);
    while (v >= 0)
        if (g_inject_left.compare_exchange_weak(v, v - 1)) return v == 0;
    return false;
}

void issue_deferred(std::shared_ptr<PendingOp> p) {
    std::vector<std::pair<cudaEvent_t, int>> waits;
    DepCheck c = check_deps(p->dev.get(), p->deps, false, &waits);
    if (c == DEPS_FAILED || c == DEPS_INVALID) {
        fut_set_done(p->out, HXC_E_DEP_FAILED);
        return;
    }
    if (c == DEPS_PENDING) {
        // still waiting on some host future: re-arm on the first pending one
        for (auto &d : p->deps) {
            bool pend;
            {
                std::lock_guard<std::mutex> g(d->m);
                pend = d->state == Future::PENDING;
            }
            if (pend) {
                fut_on_leave_pending(d, [p] { pool().submit([p] { issue_deferred(p); }); });
                return;
            }
        }
    }
    issue_now(*p);
}

// Operations from other threads wait while a thread captures a graph on the
// device (they would otherwise land in its graph); captures are host-side
// recordings, so the wait is short.  Called with dev->m held; false if the
// capture did not end within the bound.
constexpr auto kCaptureWaitBound = std::chrono::seconds(60);

bool wait_foreign_capture(Device *dev, std::unique_lock<std::mutex> &lk) {
    const auto me = std::this_thread::get_id();
    return dev->cap_cv.wait_for(lk, kCaptureWaitBound,
                                [dev, me] { return !dev->capturing || dev->cap_thread == me; });
}

void issue_now(PendingOp &p) {
    Device *dev = p.dev.get();
    bool capturing;
    {
        std::unique_lock<std::mutex> lk(dev->m);
        if (!wait_foreign_capture(dev, lk)) {
            set_error("deferred operation: another thread's graph capture did not end within 60 s");
            lk.unlock();
            fut_set_done(p.out, HXC_E_TIMEOUT);
            return;
        }
        capturing = dev->capturing;
    }
    std::vector<std::pair<cudaEvent_t, int>> waits;
    DepCheck c = check_deps(dev, p.deps, capturing, &waits);
    if (c != DEPS_READY) {
        fut_set_done(p.out, HXC_E_DEP_FAILED);
        return;
    }
    hxc_status st = dev->make_current();
    cudaStream_t s = nullptr;
    if (!st) st = dev->stream(p.slot, &s);
    if (st) {
        fut_set_done(p.out, st);
        return;
    }
    cudaError_t e = cudaSuccess;
    for (auto &w : waits) {
        if (w.second == p.slot && p.slot >= 0) continue;  // same stream: already ordered
        e = cudaStreamWaitEvent(s, w.first, 0);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess && inject_fires()) {
        set_error("injected failure of a device operation");
        if (capturing) {
            std::lock_guard<std::mutex> g(dev->m);
            dev->cap_failed = true;
        }
        fut_set_done(p.out, (hxc_status)g_inject_status.load());
        return;
    }
    if (e == cudaSuccess && p.op) e = p.op(s);
    if (e != cudaSuccess) {
        hxc_status es = cuda_status(e, "enqueue");
        if (capturing) {
            std::lock_guard<std::mutex> g(dev->m);
            dev->cap_failed = true;
        }
        fut_set_done(p.out, es);
        return;
    }
    cudaEvent_t ev = nullptr;
    if (capturing) {
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    } else {
        ev = dev->get_event();
        if (!ev) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev, s);
    if (e != cudaSuccess) {
        fut_set_done(p.out, cuda_status(e, "cudaEventRecord"));
        return;
    }
    {
        std::lock_guard<std::mutex> g(p.out->m);
        for (auto &k : p.keep) p.out->keep.push_back(k);
    }
    if (capturing) {
        std::lock_guard<std::mutex> g(dev->m);
        for (auto &k : p.keep) dev->cap_keep.push_back(k);
    }
    fut_set_issued(p.out, dev, ev, p.slot, capturing);
}
}  // namespace

FutRef fut_order_only(const FutRef &f) {
    if (!f) return f;
    {
        std::lock_guard<std::mutex> g(f->m);
        if (f->state == Future::DONE) return FutRef();
        if (f->state == Future::ISSUED) return f;
    }
    FutRef p = make_pending();
    fut_on_done(f, [p](hxc_status) { fut_set_done(p, HXC_OK); });
    return p;
}

void inject_arm(int64_t after, hxc_status status) {
    g_inject_status.store((int)status);
    g_inject_left.store(after < 0 ? -1 : after);
}

hxc_status issue_device_op(Device *dev, int slot, const std::vector<FutRef> &deps, StreamOp op,
                           std::vector<AnyRef> keep, FutRef *out) {
    if (slot < kJoinSlot || slot >= HXC_MAX_SLOTS) {
        set_error("stream slot %d out of range [0, %d)", slot, HXC_MAX_SLOTS);
        return HXC_E_INVALID;
    }
    bool capturing;
    {
        std::unique_lock<std::mutex> lk(dev->m);
        if (!wait_foreign_capture(dev, lk)) {
            set_error("another thread's graph capture did not end within 60 s");
            return HXC_E_TIMEOUT;
        }
        capturing = dev->capturing;
    }
    std::vector<std::pair<cudaEvent_t, int>> waits;
    DepCheck c = check_deps(dev, deps, capturing, &waits);
    if (c == DEPS_INVALID) return HXC_E_INVALID;
    FutRef f = make_pending();
    if (c == DEPS_FAILED) {
        fut_set_done(f, HXC_E_DEP_FAILED);
        *out = f;
        return HXC_OK;
    }
    auto p = std::make_shared<PendingOp>();
    p->dev = Ref<Device>(dev, false);
    p->slot = slot;
    p->deps = deps;
    p->op = std::move(op);
    p->keep = std::move(keep);
    p->out = f;
    if (c == DEPS_PENDING) {
        if (capturing) {
            set_error("host-side dependencies cannot be captured into a graph");
            return HXC_E_UNSUPPORTED;
        }
        issue_deferred(p);
    } else {
        issue_now(*p);
    }
    *out = f;
    return HXC_OK;
}

// ------------------------------------------------------------------- graph
Graph::~Graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
}

hxc_status graph_begin(Device *dev) {
    hxc_status st = dev->make_current();
    if (st) return st;
    // operations deferred on host futures that become ready during the
    // capture are issued by the worker pool after it (wait_foreign_capture)
    std::unique_lock<std::mutex> g(dev->m);
    if (dev->capturing && dev->cap_thread == std::this_thread::get_id()) {
        set_error("this thread is already capturing a graph on the device");
        return HXC_E_INVALID;
    }
    if (!wait_foreign_capture(dev, g)) {
        set_error("graph_begin: another thread's graph capture did not end within 60 s");
        return HXC_E_TIMEOUT;
    }
    cudaError_t e = cudaSuccess;
    if (!dev->cap_origin) e = cudaStreamCreateWithFlags(&dev->cap_origin, cudaStreamNonBlocking);
    if (e == cudaSuccess && !dev->cap_fork)
        e = cudaEventCreateWithFlags(&dev->cap_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(dev->cap_origin, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) e = cudaEventRecord(dev->cap_fork, dev->cap_origin);
    if (e != cudaSuccess) return cuda_status(e, "graph begin");
    dev->capturing = true;
    dev->cap_thread = std::this_thread::get_id();
    dev->cap_joined.clear();
    dev->cap_keep.clear();
    dev->cap_failed = false;
    return HXC_OK;
}

hxc_status graph_end(Device *dev, Ref<Graph> *out) {
    hxc_status st = dev->make_current();
    if (st) return st;
    std::vector<int> joined;
    std::vector<AnyRef> keep;
    bool failed;
    {
        std::lock_guard<std::mutex> g(dev->m);
        if (!dev->capturing || dev->cap_thread != std::this_thread::get_id()) {
            set_error("no graph capture in progress on this thread");
            return HXC_E_INVALID;
        }
        joined = dev->cap_joined;
        keep.swap(dev->cap_keep);
        failed = dev->cap_failed;
    }
    cudaError_t e = cudaSuccess;
    std::vector<cudaEvent_t> evs;
    for (int slot : joined) {
        cudaEvent_t ev;
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        evs.push_back(ev);
        cudaError_t e1 = cudaEventRecord(ev, dev->slots[slot]);
        if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(dev->cap_origin, ev, 0);
        if (e == cudaSuccess) e = e1;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(dev->cap_origin, &graph);
    for (auto ev : evs) cudaEventDestroy(ev);
    {
        std::lock_guard<std::mutex> g(dev->m);
        dev->capturing = false;
        dev->cap_joined.clear();
    }
    dev->cap_cv.notify_all();
    if (e == cudaSuccess) e = e2;
    if (failed && e == cudaSuccess) {
        set_error("an operation failed during graph capture");
        if (graph) cudaGraphDestroy(graph);
        return HXC_E_CUDA;
    }
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_status(e, "graph end");
    }
    Ref<Graph> gr(new Graph(), true);
    gr->dev = Ref<Device>(dev, false);
    gr->graph = graph;
    gr->keep = std::move(keep);
    e = cudaGraphGetNodes(graph, nullptr, &gr->nodes);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gr->exec, graph, 0);
    if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate");
    *out = gr;
    return HXC_OK;
}

}  // namespace hxc
