// Future layer, devices, buffers and graphs behind the C ABI (hxc.h).
//
// Sec. 3.1 of the paper: every asynchronous operation returns a future and
// futures compose with then / when_all.  Sec. 4: a device owns asynchronous
// work queues, a buffer is device memory with asynchronous copies, a program
// launch takes buffers as arguments.  Here a device is one CUDA GPU with a
// set of stream slots, a device future is a CUDA event recorded after its
// operation, and a host future is completed by host code (a continuation, a
// promise, or a join of host futures).
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <functional>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "hxc.h"

namespace hxc {

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
hxc_status cuda_status(cudaError_t e, const char *what);

// -------------------------------------------------------- reference counts
struct RefCounted {
    std::atomic<int> refs{1};
    virtual ~RefCounted() {}
    void retain() { refs.fetch_add(1, std::memory_order_relaxed); }
    void release() {
        if (refs.fetch_sub(1, std::memory_order_acq_rel) == 1) delete this;
    }
};

template <class T>
struct Ref {
    T *p = nullptr;
    Ref() {}
    Ref(T *q, bool adopt) : p(q) {
        if (p && !adopt) p->retain();
    }
    Ref(const Ref &o) : p(o.p) {
        if (p) p->retain();
    }
    Ref(Ref &&o) noexcept : p(o.p) { o.p = nullptr; }
    Ref &operator=(Ref o) {
        std::swap(p, o.p);
        return *this;
    }
    ~Ref() {
        if (p) p->release();
    }
    T *operator->() const { return p; }
    T *get() const { return p; }
    explicit operator bool() const { return p != nullptr; }
    T *detach() {
        T *q = p;
        p = nullptr;
        return q;
    }
};
using AnyRef = Ref<RefCounted>;

// ------------------------------------------------------------- worker pool
class WorkerPool {
  public:
    explicit WorkerPool(int n);
    ~WorkerPool();
    void submit(std::function<void()> fn);
    void shutdown();
    int size() const { return (int)threads_.size(); }
    int64_t tasks_run() const { return tasks_run_.load(); }

  private:
    void loop();
    std::mutex m_;
    std::condition_variable cv_, idle_cv_;
    std::deque<std::function<void()>> q_;
    std::vector<std::thread> threads_;
    bool stop_ = false;
    int busy_ = 0;
    std::atomic<int64_t> tasks_run_{0};
};
WorkerPool &pool();

// ------------------------------------------------------------------ device
constexpr uint32_t kDevMagic = 0xD0E1CE01u, kBufMagic = 0xB0FFE901u, kFutMagic = 0xF07E0001u,
                   kGraphMagic = 0x96A9F001u;
constexpr int kJoinSlot = -1;  // internal stream used for device-side joins

struct Device : RefCounted {
    uint32_t magic = kDevMagic;
    int ordinal = 0;
    cudaDeviceProp prop{};
    std::mutex m;
    std::vector<cudaStream_t> slots;  // HXC_MAX_SLOTS entries, created on first use
    cudaStream_t notify = nullptr;    // host notifications (cudaLaunchHostFunc)
    cudaStream_t join = nullptr;      // device-side when_all joins
    std::vector<cudaEvent_t> free_events;
    // graph capture state
    bool capturing = false;
    std::thread::id cap_thread;
    std::condition_variable cap_cv;  // signalled when a capture ends
    cudaStream_t cap_origin = nullptr;
    cudaEvent_t cap_fork = nullptr;
    std::vector<int> cap_joined;
    std::vector<AnyRef> cap_keep;
    bool cap_failed = false;
    // scratch allocations cached by key (released with the device)
    std::unordered_map<std::string, std::pair<void *, size_t>> scratch;
    std::vector<void *> retired;  // outgrown scratch, freed with the device

    ~Device() override;
    hxc_status make_current();
    // Stream of a slot (kJoinSlot: the join stream); joins an ongoing capture.
    hxc_status stream(int slot, cudaStream_t *s);
    cudaEvent_t get_event();
    void put_event(cudaEvent_t e);
    // Device memory cached under `key`, at least `bytes` large, zero-filled
    // when first allocated.  Valid until the device is destroyed, also after
    // a larger request for the same key has replaced it (devices live until
    // the process ends).
    hxc_status scratch_get(const std::string &key, size_t bytes, void **p);
};

struct Buffer : RefCounted {
    uint32_t magic = kBufMagic;
    Ref<Device> dev;
    void *ptr = nullptr;
    size_t bytes = 0;
    bool owned = false;
    ~Buffer() override;
};

// ------------------------------------------------------------------ future
struct Future : RefCounted {
    enum State { PENDING, ISSUED, DONE };
    uint32_t magic = kFutMagic;
    std::mutex m;
    std::condition_variable cv;
    State state = PENDING;
    hxc_status status = HXC_OK;
    Ref<Device> dev;          // device futures
    cudaEvent_t ev = nullptr;  // device futures: recorded after the operation
    int slot = 0;
    bool captured = false;     // recorded inside a graph capture
    bool notify_armed = false;
    std::vector<std::function<void()>> on_leave_pending;   // issued or done
    std::vector<std::function<void(hxc_status)>> on_done;  // done
    std::vector<AnyRef> keep;
    ~Future() override;
};
using FutRef = Ref<Future>;

FutRef make_pending();
FutRef make_done(hxc_status st);
void fut_set_issued(const FutRef &f, Device *dev, cudaEvent_t ev, int slot, bool captured);
void fut_set_done(const FutRef &f, hxc_status st);
// Non-blocking readiness probe; *ready = 1 when final.  Returns the status if
// ready (HXC_OK otherwise).
hxc_status fut_poll(const FutRef &f, int *ready);
hxc_status fut_wait(const FutRef &f, int64_t timeout_ns);
// Calls cb(status) once f is done (inline if it already is).
void fut_on_done(const FutRef &f, std::function<void(hxc_status)> cb);
// A dependency on f that orders without passing on f's failure: null when
// f is final (nothing left to wait for), f itself when it is an issued
// device operation (its event orders; an issued operation does not fail
// afterwards short of a lost context), else a host future that completes
// with HXC_OK once f is final.
FutRef fut_order_only(const FutRef &f);

// Checks a C handle and returns a new reference (null on error, with the
// thread-local error set).
FutRef fut_from_handle(hxc_future h);
Ref<Device> dev_from_handle(hxc_device h);
Ref<Buffer> buf_from_handle(hxc_buffer h);
inline hxc_future to_handle(FutRef f) { return reinterpret_cast<hxc_future>(f.detach()); }

// The operation issued by issue_device_op: enqueues work on `s`.
using StreamOp = std::function<cudaError_t(cudaStream_t s)>;

// Issues `op` on `slot` of `dev` after `deps`.  If a dependency is a host
// future that is not complete yet, the issue is deferred to the worker pool
// and runs when it completes.  A failed dependency makes the result
// HXC_E_DEP_FAILED without running op.  Returns a synchronous status; the
// asynchronous result is in *out.
hxc_status issue_device_op(Device *dev, int slot, const std::vector<FutRef> &deps, StreamOp op,
                           std::vector<AnyRef> keep, FutRef *out);
hxc_status deps_from_handles(const hxc_future *deps, int ndeps, std::vector<FutRef> *v);

// Host-side fault injection: the device operation that reaches issue after
// `after` further ones (0: the next) is not enqueued and completes with
// `status`, as if its CUDA call had failed.  after < 0 disarms.
void inject_arm(int64_t after, hxc_status status);

// ------------------------------------------------------------------- graph
struct Graph : RefCounted {
    uint32_t magic = kGraphMagic;
    Ref<Device> dev;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t nodes = 0;
    int64_t kernels = 0;  // kernels one replay launches (set by the capturer)
    std::vector<AnyRef> keep;
    ~Graph() override;
};

hxc_status graph_begin(Device *dev);
hxc_status graph_end(Device *dev, Ref<Graph> *out);

}  // namespace hxc
