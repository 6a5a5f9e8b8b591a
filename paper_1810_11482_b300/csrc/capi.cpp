// extern "C" entry points of hxc.h: argument validation and marshalling onto
// the future layer (runtime.hpp) and the kernel launchers (kernels.cuh).
#include <cstdlib>
#include <cstring>

#include "kernels.cuh"
#include "runtime.hpp"
#include "tune.hpp"

using namespace hxc;

namespace hxc {
const char *last_error();
}

#define CHECK_OUT(p)                                   \
    do {                                               \
        if (!(p)) {                                    \
            set_error("%s: output pointer is NULL", __func__); \
            return HXC_E_INVALID;                      \
        }                                              \
    } while (0)

extern "C" {

const char *hxc_status_string(hxc_status s) {
    switch (s) {
        case HXC_OK: return "ok";
        case HXC_E_INVALID: return "invalid argument";
        case HXC_E_NOMEM: return "out of memory";
        case HXC_E_CUDA: return "CUDA error";
        case HXC_E_TIMEOUT: return "timeout";
        case HXC_E_DEP_FAILED: return "dependency failed";
        case HXC_E_CALLBACK: return "host continuation failed";
        case HXC_E_UNSUPPORTED: return "unsupported";
        case HXC_E_NODEV: return "no matching device";
    }
    return "unknown status";
}

const char *hxc_last_error(void) { return hxc::last_error(); }
int hxc_abi_version(void) { return HXC_ABI_VERSION; }

hxc_status hxc_shutdown(void) {
    pool().shutdown();
    return HXC_OK;
}

// ----------------------------------------------------------------- devices
static std::mutex g_dev_m;
static std::vector<Device *> g_devs;  // one Device per ordinal, kept for the process

hxc_status hxc_get_all_devices(int min_major, int min_minor, hxc_device *out, int cap,
                               int *n_out) {
    CHECK_OUT(n_out);
    if (cap < 0 || (cap > 0 && !out)) {
        set_error("hxc_get_all_devices: bad output array");
        return HXC_E_INVALID;
    }
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        *n_out = 0;
        set_error("no CUDA device: %s", cudaGetErrorString(e));
        return HXC_E_NODEV;
    }
    std::lock_guard<std::mutex> g(g_dev_m);
    if (g_devs.empty()) {
        g_devs.assign(count, nullptr);
        cudaDeviceProp p0;
        if (cudaGetDeviceProperties(&p0, 0) == cudaSuccess) tune::load_default(p0.major, p0.minor);
    }
    int found = 0;
    for (int i = 0; i < count; i++) {
        if (!g_devs[i]) {
            Device *d = new Device();
            d->ordinal = i;
            if (cudaGetDeviceProperties(&d->prop, i) != cudaSuccess) {
                delete d;
                continue;
            }
            d->slots.assign(HXC_MAX_SLOTS, nullptr);
            g_devs[i] = d;  // the table's own reference
        }
        Device *d = g_devs[i];
        if (d->prop.major < min_major || (d->prop.major == min_major && d->prop.minor < min_minor))
            continue;
        if (found < cap) {
            d->retain();
            out[found] = reinterpret_cast<hxc_device>(d);
        }
        found++;
    }
    *n_out = found;
    if (!found) {
        set_error("no device with compute capability >= %d.%d", min_major, min_minor);
        return HXC_E_NODEV;
    }
    return HXC_OK;
}

hxc_status hxc_device_info(hxc_device dh, int *major, int *minor, int *sm_count,
                           size_t *global_mem) {
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    if (major) *major = d->prop.major;
    if (minor) *minor = d->prop.minor;
    if (sm_count) *sm_count = d->prop.multiProcessorCount;
    if (global_mem) *global_mem = d->prop.totalGlobalMem;
    return HXC_OK;
}

hxc_status hxc_device_synchronize(hxc_device dh) {
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    hxc_status st = d->make_current();
    if (st) return st;
    std::vector<cudaStream_t> ss;
    {
        std::lock_guard<std::mutex> g(d->m);
        for (auto s : d->slots)
            if (s) ss.push_back(s);
        if (d->join) ss.push_back(d->join);
    }
    for (auto s : ss) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e, "cudaStreamSynchronize");
    }
    return HXC_OK;
}

hxc_status hxc_device_stream(hxc_device dh, int slot, void **stream) {
    CHECK_OUT(stream);
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    if (slot < 0) {
        set_error("slot must be >= 0");
        return HXC_E_INVALID;
    }
    cudaStream_t s;
    hxc_status st = d->stream(slot, &s);
    if (!st) *stream = s;
    return st;
}

hxc_status hxc_device_retain(hxc_device dh) {
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    d->retain();
    return HXC_OK;
}

hxc_status hxc_device_release(hxc_device dh) {
    Device *d = reinterpret_cast<Device *>(dh);
    if (!d || d->magic != kDevMagic) {
        set_error("invalid device handle");
        return HXC_E_INVALID;
    }
    d->release();  // the device table keeps its own reference
    return HXC_OK;
}

// ------------------------------------------------------------ host memory
hxc_status hxc_host_alloc(size_t bytes, void **p) {
    CHECK_OUT(p);
    cudaError_t e = cudaMallocHost(p, bytes ? bytes : 1);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("cudaMallocHost(%zu): %s", bytes, cudaGetErrorString(e));
        return HXC_E_NOMEM;
    }
    return HXC_OK;
}

hxc_status hxc_host_free(void *p) {
    if (!p) return HXC_OK;
    return cuda_status(cudaFreeHost(p), "cudaFreeHost");
}

// ----------------------------------------------------------------- buffers
hxc_status hxc_device_create_buffer(hxc_device dh, size_t bytes, hxc_buffer *out) {
    CHECK_OUT(out);
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    hxc_status st = d->make_current();
    if (st) return st;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        return HXC_E_NOMEM;
    }
    Buffer *b = new Buffer();
    b->dev = d;
    b->ptr = p;
    b->bytes = bytes;
    b->owned = true;
    *out = reinterpret_cast<hxc_buffer>(b);
    return HXC_OK;
}

hxc_status hxc_buffer_wrap(hxc_device dh, void *device_ptr, size_t bytes, hxc_buffer *out) {
    CHECK_OUT(out);
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    if (!device_ptr && bytes) {
        set_error("hxc_buffer_wrap: NULL pointer");
        return HXC_E_INVALID;
    }
    Buffer *b = new Buffer();
    b->dev = d;
    b->ptr = device_ptr;
    b->bytes = bytes;
    b->owned = false;
    *out = reinterpret_cast<hxc_buffer>(b);
    return HXC_OK;
}

hxc_status hxc_buffer_device_ptr(hxc_buffer bh, void **device_ptr, size_t *bytes) {
    Ref<Buffer> b = buf_from_handle(bh);
    if (!b) return HXC_E_INVALID;
    if (device_ptr) *device_ptr = b->ptr;
    if (bytes) *bytes = b->bytes;
    return HXC_OK;
}

hxc_status hxc_buffer_retain(hxc_buffer bh) {
    Ref<Buffer> b = buf_from_handle(bh);
    if (!b) return HXC_E_INVALID;
    b->retain();
    return HXC_OK;
}

hxc_status hxc_buffer_release(hxc_buffer bh) {
    Buffer *b = reinterpret_cast<Buffer *>(bh);
    if (!b || b->magic != kBufMagic) {
        set_error("invalid buffer handle");
        return HXC_E_INVALID;
    }
    b->release();
    return HXC_OK;
}

static bool range_ok(const Buffer *b, size_t off, size_t bytes) {
    return off <= b->bytes && bytes <= b->bytes - off;
}

static hxc_status copy_common(Ref<Buffer> b, int slot, const hxc_future *deps, int ndeps,
                              StreamOp op, std::vector<AnyRef> keep, hxc_future *out) {
    std::vector<FutRef> dv;
    hxc_status st = deps_from_handles(deps, ndeps, &dv);
    if (st) return st;
    FutRef f;
    st = issue_device_op(b->dev.get(), slot, dv, std::move(op), std::move(keep), &f);
    if (st) return st;
    *out = to_handle(f);
    return HXC_OK;
}

hxc_status hxc_buffer_enqueue_write(hxc_buffer bh, size_t off, size_t bytes, const void *host,
                                    int slot, const hxc_future *deps, int ndeps,
                                    hxc_future *out) {
    CHECK_OUT(out);
    Ref<Buffer> b = buf_from_handle(bh);
    if (!b) return HXC_E_INVALID;
    if (!range_ok(b.get(), off, bytes) || (!host && bytes)) {
        set_error("enqueue_write: range [%zu, +%zu) outside buffer of %zu bytes or NULL host",
                  off, bytes, b->bytes);
        return HXC_E_INVALID;
    }
    char *dst = static_cast<char *>(b->ptr) + off;
    StreamOp op = [=](cudaStream_t s) {
        return bytes ? cudaMemcpyAsync(dst, host, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    return copy_common(b, slot, deps, ndeps, op, {AnyRef(b.get(), false)}, out);
}

hxc_status hxc_buffer_enqueue_read(hxc_buffer bh, size_t off, size_t bytes, void *host, int slot,
                                   const hxc_future *deps, int ndeps, hxc_future *out) {
    CHECK_OUT(out);
    Ref<Buffer> b = buf_from_handle(bh);
    if (!b) return HXC_E_INVALID;
    if (!range_ok(b.get(), off, bytes) || (!host && bytes)) {
        set_error("enqueue_read: range [%zu, +%zu) outside buffer of %zu bytes or NULL host",
                  off, bytes, b->bytes);
        return HXC_E_INVALID;
    }
    const char *src = static_cast<const char *>(b->ptr) + off;
    StreamOp op = [=](cudaStream_t s) {
        return bytes ? cudaMemcpyAsync(host, src, bytes, cudaMemcpyDeviceToHost, s) : cudaSuccess;
    };
    return copy_common(b, slot, deps, ndeps, op, {AnyRef(b.get(), false)}, out);
}

hxc_status hxc_buffer_enqueue_read_sync(hxc_buffer bh, size_t off, size_t bytes, void *host,
                                        int slot, const hxc_future *deps, int ndeps) {
    hxc_future f = nullptr;
    hxc_status st = hxc_buffer_enqueue_read(bh, off, bytes, host, slot, deps, ndeps, &f);
    if (st) return st;
    st = fut_wait(FutRef(reinterpret_cast<Future *>(f), false), -1);
    hxc_future_release(f);
    return st;
}

hxc_status hxc_buffer_enqueue_copy(hxc_buffer dh, size_t dst_off, hxc_buffer sh, size_t src_off,
                                   size_t bytes, int slot, const hxc_future *deps, int ndeps,
                                   hxc_future *out) {
    CHECK_OUT(out);
    Ref<Buffer> d = buf_from_handle(dh), s = buf_from_handle(sh);
    if (!d || !s) return HXC_E_INVALID;
    if (d->dev.get() != s->dev.get()) {
        set_error("enqueue_copy: buffers live on different devices");
        return HXC_E_UNSUPPORTED;
    }
    if (!range_ok(d.get(), dst_off, bytes) || !range_ok(s.get(), src_off, bytes)) {
        set_error("enqueue_copy: range outside a buffer");
        return HXC_E_INVALID;
    }
    char *dp = static_cast<char *>(d->ptr) + dst_off;
    const char *sp = static_cast<const char *>(s->ptr) + src_off;
    StreamOp op = [=](cudaStream_t st) {
        return bytes ? cudaMemcpyAsync(dp, sp, bytes, cudaMemcpyDeviceToDevice, st) : cudaSuccess;
    };
    return copy_common(d, slot, deps, ndeps, op, {AnyRef(d.get(), false), AnyRef(s.get(), false)},
                       out);
}

static bool range2d_ok(const Buffer *b, size_t off, size_t pitch, size_t row_bytes, size_t rows) {
    if (rows == 0 || row_bytes == 0) return true;
    if (row_bytes > pitch) return false;
    size_t last = off + (rows - 1) * pitch + row_bytes;
    return last <= b->bytes && last >= off;
}

hxc_status hxc_buffer_enqueue_write_2d(hxc_buffer bh, size_t off, size_t buf_pitch,
                                       const void *host, size_t host_pitch, size_t row_bytes,
                                       size_t rows, int slot, const hxc_future *deps, int ndeps,
                                       hxc_future *out) {
    CHECK_OUT(out);
    Ref<Buffer> b = buf_from_handle(bh);
    if (!b) return HXC_E_INVALID;
    if (!range2d_ok(b.get(), off, buf_pitch, row_bytes, rows) || row_bytes > host_pitch ||
        (!host && rows)) {
        set_error("enqueue_write_2d: bad range or pitch");
        return HXC_E_INVALID;
    }
    char *dst = static_cast<char *>(b->ptr) + off;
    StreamOp op = [=](cudaStream_t s) {
        return rows ? cudaMemcpy2DAsync(dst, buf_pitch, host, host_pitch, row_bytes, rows,
                                        cudaMemcpyHostToDevice, s)
                    : cudaSuccess;
    };
    return copy_common(b, slot, deps, ndeps, op, {AnyRef(b.get(), false)}, out);
}

hxc_status hxc_buffer_enqueue_read_2d(hxc_buffer bh, size_t off, size_t buf_pitch, void *host,
                                      size_t host_pitch, size_t row_bytes, size_t rows, int slot,
                                      const hxc_future *deps, int ndeps, hxc_future *out) {
    CHECK_OUT(out);
    Ref<Buffer> b = buf_from_handle(bh);
    if (!b) return HXC_E_INVALID;
    if (!range2d_ok(b.get(), off, buf_pitch, row_bytes, rows) || row_bytes > host_pitch ||
        (!host && rows)) {
        set_error("enqueue_read_2d: bad range or pitch");
        return HXC_E_INVALID;
    }
    const char *src = static_cast<const char *>(b->ptr) + off;
    StreamOp op = [=](cudaStream_t s) {
        return rows ? cudaMemcpy2DAsync(host, host_pitch, src, buf_pitch, row_bytes, rows,
                                        cudaMemcpyDeviceToHost, s)
                    : cudaSuccess;
    };
    return copy_common(b, slot, deps, ndeps, op, {AnyRef(b.get(), false)}, out);
}

// ----------------------------------------------------------------- futures
hxc_status hxc_future_is_ready(hxc_future fh, int *ready) {
    CHECK_OUT(ready);
    FutRef f = fut_from_handle(fh);
    if (!f) return HXC_E_INVALID;
    fut_poll(f, ready);
    return HXC_OK;
}

hxc_status hxc_future_wait(hxc_future fh, int64_t timeout_ns) {
    FutRef f = fut_from_handle(fh);
    if (!f) return HXC_E_INVALID;
    return fut_wait(f, timeout_ns);
}

hxc_status hxc_wait_all(const hxc_future *fs, int n, int64_t timeout_ns) {
    std::vector<FutRef> v;
    hxc_status st = deps_from_handles(fs, n, &v);
    if (st) return st;
    auto t0 = std::chrono::steady_clock::now();
    hxc_status first = HXC_OK;
    for (auto &f : v) {
        int64_t left = -1;
        if (timeout_ns >= 0) {
            int64_t used = std::chrono::duration_cast<std::chrono::nanoseconds>(
                               std::chrono::steady_clock::now() - t0)
                               .count();
            left = timeout_ns > used ? timeout_ns - used : 0;
        }
        hxc_status s = fut_wait(f, left);
        if (s == HXC_E_TIMEOUT) return s;
        if (s && !first) first = s;
    }
    return first;
}

hxc_status hxc_future_then(hxc_future fh, hxc_host_fn fn, void *user, hxc_future *out) {
    CHECK_OUT(out);
    FutRef f = fut_from_handle(fh);
    if (!f) return HXC_E_INVALID;
    if (!fn) {
        set_error("hxc_future_then: NULL function");
        return HXC_E_INVALID;
    }
    {
        std::lock_guard<std::mutex> g(f->m);
        if (f->captured) {
            set_error("host continuations cannot be attached inside a graph capture");
            return HXC_E_UNSUPPORTED;
        }
    }
    FutRef r = make_pending();
    fut_on_done(f, [r, fn, user](hxc_status st) {
        if (st != HXC_OK) {
            fut_set_done(r, HXC_E_DEP_FAILED);
            return;
        }
        pool().submit([r, fn, user] {
            hxc_status s = fn(user);
            fut_set_done(r, s == HXC_OK ? HXC_OK : HXC_E_CALLBACK);
        });
    });
    *out = to_handle(r);
    return HXC_OK;
}

hxc_status hxc_when_all(const hxc_future *fs, int n, hxc_future *out) {
    CHECK_OUT(out);
    std::vector<FutRef> v;
    hxc_status st = deps_from_handles(fs, n, &v);
    if (st) return st;
    // Device-side join when every input is issued device work on one device.
    Device *dev = nullptr;
    bool device_join = true;
    for (auto &f : v) {
        std::lock_guard<std::mutex> g(f->m);
        if (f->state == Future::PENDING) {
            device_join = false;
            break;
        }
        if (f->state == Future::ISSUED) {
            if (dev && dev != f->dev.get()) device_join = false;
            dev = f->dev.get();
        }
    }
    if (device_join && dev) {
        FutRef r;
        st = issue_device_op(dev, kJoinSlot, v, StreamOp(), {}, &r);
        if (st) return st;
        *out = to_handle(r);
        return HXC_OK;
    }
    FutRef r = make_pending();
    if (v.empty()) {
        fut_set_done(r, HXC_OK);
        *out = to_handle(r);
        return HXC_OK;
    }
    struct JoinState {
        std::atomic<int> left;
        std::atomic<int> failed{0};
    };
    auto js = std::make_shared<JoinState>();
    js->left = (int)v.size();
    for (auto &f : v) {
        fut_on_done(f, [r, js](hxc_status s) {
            if (s != HXC_OK) js->failed = 1;
            if (js->left.fetch_sub(1) == 1) fut_set_done(r, js->failed ? HXC_E_DEP_FAILED : HXC_OK);
        });
    }
    *out = to_handle(r);
    return HXC_OK;
}

hxc_status hxc_make_ready_future(hxc_status status, hxc_future *out) {
    CHECK_OUT(out);
    *out = to_handle(make_done(status));
    return HXC_OK;
}

hxc_status hxc_promise_create(hxc_future *out) {
    CHECK_OUT(out);
    *out = to_handle(make_pending());
    return HXC_OK;
}

hxc_status hxc_promise_set(hxc_future ph, hxc_status status) {
    FutRef f = fut_from_handle(ph);
    if (!f) return HXC_E_INVALID;
    {
        std::lock_guard<std::mutex> g(f->m);
        if (f->state != Future::PENDING || f->dev) {
            set_error("hxc_promise_set: not an unset promise");
            return HXC_E_INVALID;
        }
    }
    fut_set_done(f, status);
    return HXC_OK;
}

hxc_status hxc_debug_inject(int64_t after_ops, hxc_status status) {
    if (after_ops >= 0 && status == HXC_OK) {
        set_error("hxc_debug_inject: an injected failure needs a non-OK status");
        return HXC_E_INVALID;
    }
    inject_arm(after_ops, status);
    return HXC_OK;
}

hxc_status hxc_debug_wait_errors(hxc_device dh, uint32_t *flags) {
    CHECK_OUT(flags);
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    hxc_status st = d->make_current();
    if (st) return st;
    if ((st = hxc_device_synchronize(dh))) return st;
    unsigned v = 0;
    cudaError_t e = k::heat3d_wait_errors(&v);
    if (e != cudaSuccess) return cuda_status(e, "hxc_debug_wait_errors");
    *flags = v;
    return HXC_OK;
}

hxc_status hxc_future_from_stream(hxc_device dh, void *stream, hxc_future *out) {
    CHECK_OUT(out);
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    hxc_status st = d->make_current();
    if (st) return st;
    cudaEvent_t ev = d->get_event();
    if (!ev) return cuda_status(cudaErrorMemoryAllocation, "event");
    cudaError_t e = cudaEventRecord(ev, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        d->put_event(ev);
        return cuda_status(e, "cudaEventRecord on foreign stream");
    }
    FutRef f = make_pending();
    fut_set_issued(f, d.get(), ev, -3, false);
    *out = to_handle(f);
    return HXC_OK;
}

hxc_status hxc_future_stream_wait(hxc_future fh, void *stream) {
    FutRef f = fut_from_handle(fh);
    if (!f) return HXC_E_INVALID;
    hxc_status st = fut_wait(f, 0);
    if (st == HXC_OK) return HXC_OK;  // already complete
    std::unique_lock<std::mutex> lk(f->m);
    if (f->state == Future::DONE) return f->status == HXC_OK ? HXC_OK : HXC_E_DEP_FAILED;
    if (f->state == Future::PENDING) {
        lk.unlock();
        st = fut_wait(f, -1);  // host work: wait on the host
        return st == HXC_OK ? HXC_OK : HXC_E_DEP_FAILED;
    }
    cudaEvent_t ev = f->ev;
    Device *d = f->dev.get();
    lk.unlock();
    d->make_current();
    return cuda_status(cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), ev, 0),
                       "cudaStreamWaitEvent");
}

hxc_status hxc_future_retain(hxc_future fh) {
    FutRef f = fut_from_handle(fh);
    if (!f) return HXC_E_INVALID;
    f->retain();
    return HXC_OK;
}

hxc_status hxc_future_release(hxc_future fh) {
    Future *f = reinterpret_cast<Future *>(fh);
    if (!f || f->magic != kFutMagic) {
        set_error("invalid future handle");
        return HXC_E_INVALID;
    }
    f->release();
    return HXC_OK;
}

// --------------------------------------------------------- kernel launches
static hxc_status need_buf(hxc_buffer h, Device *dev, size_t bytes, const char *what,
                           Ref<Buffer> *out) {
    Ref<Buffer> b = buf_from_handle(h);
    if (!b) {
        set_error("%s: invalid buffer", what);
        return HXC_E_INVALID;
    }
    if (b->dev.get() != dev) {
        set_error("%s: buffer belongs to another device", what);
        return HXC_E_INVALID;
    }
    if (b->bytes < bytes) {
        set_error("%s: buffer holds %zu bytes, %zu needed", what, b->bytes, bytes);
        return HXC_E_INVALID;
    }
    *out = b;
    return HXC_OK;
}

static bool cfg_ok(const hxc_launch_cfg *cfg, unsigned min_block, unsigned max_block) {
    if (!cfg) return true;
    uint64_t g = (uint64_t)cfg->grid[0] * cfg->grid[1] * cfg->grid[2];
    uint64_t b = (uint64_t)cfg->block[0] * cfg->block[1] * cfg->block[2];
    if (g == 0 || g > 0x7fffffffu) return false;
    return b >= min_block && b <= max_block && b % 32 == 0;
}

hxc_status hxc_launch(hxc_device dh, hxc_kernel_id id, const void *args, size_t args_size,
                      const hxc_launch_cfg *cfg_in, int slot, const hxc_future *deps, int ndeps,
                      hxc_future *out) {
    CHECK_OUT(out);
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    if (!args) {
        set_error("hxc_launch: NULL args");
        return HXC_E_INVALID;
    }
    std::vector<FutRef> dv;
    hxc_status st = deps_from_handles(deps, ndeps, &dv);
    if (st) return st;
    bool has_cfg = cfg_in != nullptr;
    hxc_launch_cfg cfg{};
    if (has_cfg) cfg = *cfg_in;
    const hxc_launch_cfg *pc = has_cfg ? &cfg : nullptr;
    StreamOp op;
    std::vector<AnyRef> keep;
#define ARGS(T)                                                                   \
    if (args_size != sizeof(T)) {                                                 \
        set_error("hxc_launch: args_size %zu != sizeof(" #T ") %zu", args_size, sizeof(T)); \
        return HXC_E_INVALID;                                                     \
    }                                                                             \
    T a;                                                                          \
    memcpy(&a, args, sizeof(T));
#define BUF(var, h, bytes, what)                                   \
    Ref<Buffer> var;                                               \
    if ((st = need_buf(h, d.get(), bytes, what, &var))) return st; \
    keep.push_back(AnyRef(var.get(), false));
    switch (id) {
        case HXC_K_SUM_U32: {
            ARGS(hxc_sum_args);
            if (a.n < 0 || !cfg_ok(pc, 32, 1024)) goto bad;
            BUF(in, a.input, (size_t)a.n * 4, "sum.input");
            BUF(res, a.result, 8, "sum.result");
            const uint32_t *ip = (const uint32_t *)in->ptr;
            unsigned long long *rp = (unsigned long long *)res->ptr;
            int64_t n = a.n;
            op = [=](cudaStream_t s) { return k::sum_u32(ip, rp, n, pc ? &cfg : nullptr, s); };
            break;
        }
        case HXC_K_PRK_STENCIL: {
            ARGS(hxc_prk_args);
            if (a.n <= 0 || !cfg_ok(pc, 32, 1024)) goto bad;
            BUF(in, a.in, (size_t)a.n * 8, "prk.in");
            BUF(o, a.out, (size_t)a.n * 8, "prk.out");
            if (in->ptr == o->ptr) goto bad;
            const double *ip = (const double *)in->ptr;
            double *optr = (double *)o->ptr;
            int64_t n = a.n;
            op = [=](cudaStream_t s) { return k::prk(ip, optr, n, pc ? &cfg : nullptr, s); };
            break;
        }
        case HXC_K_MANDELBROT: {
            ARGS(hxc_mandelbrot_args);
            if (a.width < 0 || a.height < 0 || a.max_iter < 1 || !cfg_ok(pc, 32, 256)) goto bad;
            if (a.width > ((int64_t)1 << 24) || a.height > ((int64_t)1 << 24)) goto bad;
            const size_t npx = (size_t)a.width * (size_t)a.height;
            BUF(img, a.rgb, npx * 3, "mandelbrot.rgb");
            uint8_t *rp = (uint8_t *)img->ptr;
            int32_t *cp = nullptr;
            if (a.counts) {
                BUF(cb, a.counts, npx * 4, "mandelbrot.counts");
                cp = (int32_t *)cb->ptr;
            }
            const hxc_mandelbrot_args m = a;
            op = [=](cudaStream_t s) {
                return k::mandelbrot(rp, cp, m.width, m.height, m.x0, m.y0, m.dx, m.dy, m.max_iter,
                                     pc ? &cfg : nullptr, s);
            };
            break;
        }
        case HXC_K_PARTITION: {
            ARGS(hxc_partition_args);
            if (a.n < 0 || a.offset < 0 || !cfg_ok(pc, 32, 1024)) goto bad;
            BUF(o, a.x, (size_t)(a.offset + a.n) * 8, "partition.x");
            double *xptr = (double *)o->ptr + a.offset;
            int64_t n = a.n;
            op = [=](cudaStream_t s) { return k::partition(xptr, n, pc ? &cfg : nullptr, s); };
            break;
        }
        case HXC_K_HEAT1D: {
            ARGS(hxc_heat1d_args);
            if (a.n <= 0 || a.lo < 0 || a.count < 0 || a.lo > a.n || a.count > a.n - a.lo ||
                a.steps < 1 || a.steps > k::kHeat1dMaxSteps || !cfg_ok(pc, 32, 1024))
                goto bad;
            BUF(src, a.src, (size_t)a.n * 8, "heat1d.src");
            BUF(dst, a.dst, (size_t)a.n * 8, "heat1d.dst");
            if (src->ptr == dst->ptr) goto bad;
            const double *sp = (const double *)src->ptr;
            double *dp = (double *)dst->ptr;
            hxc_heat1d_args v = a;
            op = [=](cudaStream_t s) {
                return k::heat1d(sp, dp, v.n, v.lo, v.count, v.r, v.steps, pc ? &cfg : nullptr, s);
            };
            break;
        }
        case HXC_K_HEAT2D: {
            ARGS(hxc_heat2d_args);
            if (a.ny <= 0 || a.nx <= 0 || a.y0 < 0 || a.x0 < 0 || a.ty < 0 || a.tx < 0 ||
                a.y0 + a.ty > a.ny || a.x0 + a.tx > a.nx || !cfg_ok(pc, 32, 256))
                goto bad;
            size_t bytes = (size_t)a.ny * a.nx * 8;
            BUF(src, a.src, bytes, "heat2d.src");
            BUF(dst, a.dst, bytes, "heat2d.dst");
            if (src->ptr == dst->ptr) goto bad;
            const double *sp = (const double *)src->ptr;
            double *dp = (double *)dst->ptr;
            hxc_heat2d_args v = a;
            op = [=](cudaStream_t s) {
                return k::heat2d(sp, dp, v.ny, v.nx, v.y0, v.x0, v.ty, v.tx, v.r, 0,
                                 pc ? &cfg : nullptr, s);
            };
            break;
        }
        case HXC_K_TILE_NORM2: {
            ARGS(hxc_tile_norm2_args);
            if (a.ny <= 0 || a.nx <= 0 || a.y0 < 0 || a.x0 < 0 || a.ty < 0 || a.tx < 0 ||
                a.y0 + a.ty > a.ny || a.x0 + a.tx > a.nx || a.sum_index < 0 || pc)
                goto bad;
            BUF(src, a.src, (size_t)a.ny * a.nx * 8, "tile_norm.src");
            BUF(sums, a.sums, (size_t)(a.sum_index + 1) * 8, "tile_norm.sums");
            double *snap = nullptr;
            if (a.snap) {
                BUF(sn, a.snap, (size_t)a.ty * a.tx * 8, "tile_norm.snap");
                snap = (double *)sn->ptr;
            }
            // scratch per stream slot: launches on one slot never overlap
            void *scratch = nullptr;
            if ((st = d->scratch_get("tile_norm." + std::to_string(slot),
                                     k::kNormScratchBytes, &scratch)))
                return st;
            const double *sp = (const double *)src->ptr;
            double *np = (double *)sums->ptr;
            hxc_tile_norm2_args v = a;
            op = [=](cudaStream_t s) {
                return k::tile_norm(sp, snap, np, scratch, v.ny, v.nx, v.y0, v.x0, v.ty, v.tx,
                                    v.sum_index, s);
            };
            break;
        }
        case HXC_K_HEAT3D: {
            ARGS(hxc_heat3d_args);
            if (a.nz <= 0 || a.ny <= 0 || a.nx <= 0 || a.nz > INT32_MAX || a.ny > INT32_MAX ||
                a.nx > INT32_MAX || a.steps < 1 || a.steps > 4 || (pc && !cfg_ok(pc, 512, 512)))
                goto bad;
            size_t bytes = (size_t)a.nz * a.ny * a.nx * 4;
            BUF(src, a.src, bytes, "heat3d.src");
            BUF(dst, a.dst, bytes, "heat3d.dst");
            if (src->ptr == dst->ptr) goto bad;
            const float *sp = (const float *)src->ptr;
            float *dp = (float *)dst->ptr;
            hxc_heat3d_args v = a;
            op = [=](cudaStream_t s) {
                return k::heat3d(sp, dp, (int)v.nz, (int)v.ny, (int)v.nx, v.r, v.steps, 0,
                                 pc ? &cfg : nullptr, s);
            };
            break;
        }
        case HXC_K_VARCOEF2D: {
            ARGS(hxc_varcoef2d_args);
            if (a.ny <= 0 || a.nx <= 0 || !cfg_ok(pc, 32, 1024)) goto bad;
            size_t bytes = (size_t)a.ny * a.nx * 8;
            BUF(src, a.src, bytes, "varcoef2d.src");
            BUF(dst, a.dst, bytes, "varcoef2d.dst");
            BUF(kap, a.kappa, bytes, "varcoef2d.kappa");
            if (src->ptr == dst->ptr || kap->ptr == dst->ptr) goto bad;
            const double *sp = (const double *)src->ptr, *kp = (const double *)kap->ptr;
            double *dp = (double *)dst->ptr;
            hxc_varcoef2d_args v = a;
            op = [=](cudaStream_t s) {
                return k::vc_step_otf(sp, dp, kp, v.c, v.ny, v.nx, pc ? &cfg : nullptr, s);
            };
            break;
        }
        case HXC_K_ADJOINT2D: {
            ARGS(hxc_adjoint2d_args);
            if (a.ny <= 0 || a.nx <= 0 || !cfg_ok(pc, 32, 1024)) goto bad;
            size_t bytes = (size_t)a.ny * a.nx * 8;
            BUF(li, a.lam_in, bytes, "adjoint2d.lam_in");
            BUF(lo, a.lam_out, bytes, "adjoint2d.lam_out");
            BUF(ub, a.u, bytes, "adjoint2d.u");
            BUF(kap, a.kappa, bytes, "adjoint2d.kappa");
            BUF(gk, a.grad_kappa, bytes, "adjoint2d.grad_kappa");
            if (li->ptr == lo->ptr || lo->ptr == ub->ptr || lo->ptr == gk->ptr ||
                li->ptr == gk->ptr || ub->ptr == gk->ptr || kap->ptr == gk->ptr ||
                kap->ptr == lo->ptr)
                goto bad;
            const double *lip = (const double *)li->ptr, *up = (const double *)ub->ptr,
                         *kp = (const double *)kap->ptr;
            double *lop = (double *)lo->ptr, *gp = (double *)gk->ptr;
            hxc_adjoint2d_args v = a;
            op = [=](cudaStream_t s) {
                return k::vc_adjoint_otf(lip, lop, up, kp, gp, v.c, v.ny, v.nx, pc ? &cfg : nullptr,
                                         s);
            };
            break;
        }
        default:
            set_error("hxc_launch: unknown or unavailable kernel id %d", (int)id);
            return HXC_E_UNSUPPORTED;
    }
#undef ARGS
#undef BUF
    {
        FutRef f;
        st = issue_device_op(d.get(), slot, dv, std::move(op), std::move(keep), &f);
        if (st) return st;
        *out = to_handle(f);
        return HXC_OK;
    }
bad:
    set_error("hxc_launch: kernel %d: arguments out of range or launch shape unsupported", (int)id);
    return HXC_E_INVALID;
}

// ------------------------------------------------------------------ tuning
hxc_status hxc_tune_set(const char *key, int64_t value) {
    if (!tune::set(key, value)) {
        set_error("hxc_tune_set: unknown key '%s'", key ? key : "(null)");
        return HXC_E_INVALID;
    }
    return HXC_OK;
}

hxc_status hxc_tune_get(const char *key, int64_t *value) {
    CHECK_OUT(value);
    if (!tune::known(key)) {
        set_error("hxc_tune_get: unknown key '%s'", key ? key : "(null)");
        return HXC_E_INVALID;
    }
    *value = tune::get(key);
    return HXC_OK;
}

hxc_status hxc_tune_load(const char *path, int major, int minor) {
    if (!path) {
        set_error("hxc_tune_load: NULL path");
        return HXC_E_INVALID;
    }
    return tune::load_file(path, major, minor);
}

// ------------------------------------------------------------------ graphs
hxc_status hxc_graph_begin(hxc_device dh) {
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    return graph_begin(d.get());
}

hxc_status hxc_graph_end(hxc_device dh, hxc_graph *out) {
    CHECK_OUT(out);
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    Ref<Graph> g;
    hxc_status st = graph_end(d.get(), &g);
    if (st) return st;
    *out = reinterpret_cast<hxc_graph>(g.detach());
    return HXC_OK;
}

static Ref<Graph> graph_from_handle(hxc_graph h) {
    Graph *g = reinterpret_cast<Graph *>(h);
    if (!g || g->magic != kGraphMagic) {
        set_error("invalid graph handle");
        return Ref<Graph>();
    }
    return Ref<Graph>(g, false);
}

hxc_status hxc_graph_launch(hxc_graph gh, int slot, const hxc_future *deps, int ndeps,
                            hxc_future *out) {
    CHECK_OUT(out);
    Ref<Graph> g = graph_from_handle(gh);
    if (!g) return HXC_E_INVALID;
    std::vector<FutRef> dv;
    hxc_status st = deps_from_handles(deps, ndeps, &dv);
    if (st) return st;
    cudaGraphExec_t ex = g->exec;
    FutRef f;
    st = issue_device_op(
        g->dev.get(), slot, dv, [ex](cudaStream_t s) { return cudaGraphLaunch(ex, s); },
        {AnyRef(g.get(), false)}, &f);
    if (st) return st;
    *out = to_handle(f);
    return HXC_OK;
}

hxc_status hxc_graph_node_count(hxc_graph gh, size_t *nodes) {
    CHECK_OUT(nodes);
    Ref<Graph> g = graph_from_handle(gh);
    if (!g) return HXC_E_INVALID;
    *nodes = g->nodes;
    return HXC_OK;
}

hxc_status hxc_graph_release(hxc_graph gh) {
    Graph *g = reinterpret_cast<Graph *>(gh);
    if (!g || g->magic != kGraphMagic) {
        set_error("invalid graph handle");
        return HXC_E_INVALID;
    }
    g->release();
    return HXC_OK;
}

}  // extern "C"
