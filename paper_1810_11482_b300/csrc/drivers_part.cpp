// The partition benchmark of Sec. 5.1.2 (Algorithm 1): a vector split into
// partitions, each copied to the device, transformed by the partition kernel
// and copied back, with the three loops over the partitions issued
// asynchronously so that the copies of one partition overlap the kernel of
// another.  Two forms: composed from the public futures calls (write,
// launch, read, when_all), and the same sequence as plain CUDA runtime calls
// on the same streams (the native comparison of Sec. 5.1.2).
#include <vector>

#include "drivers_util.hpp"
#include "kernels.cuh"
#include "runtime.hpp"

using namespace hxc;
using namespace hxc::drv;

namespace {

hxc_status check_args(const double *hx, const double *hr, int64_t n, int parts, hxc_buffer work,
                      const char *who) {
    if (n < 0 || parts < 1 || parts > 64 || (n > 0 && (!hx || !hr))) {
        set_error("%s: need n >= 0, 1 <= parts <= 64 and host arrays", who);
        return HXC_E_INVALID;
    }
    Ref<Buffer> b = buf_from_handle(work);
    if (!b) return HXC_E_INVALID;
    if (b->bytes < (size_t)n * 8) {
        set_error("%s: work buffer holds %zu bytes, %lld needed", who, b->bytes, (long long)n * 8);
        return HXC_E_INVALID;
    }
    return HXC_OK;
}

}  // namespace

extern "C" {

hxc_status hxc_partition_run(hxc_device dh, const double *host_x, double *host_r, int64_t n,
                             int parts, hxc_buffer work, const hxc_future *deps, int ndeps,
                             hxc_future *out) {
    hxc::drv::NvtxRange nvtx_range("hxc_partition_run");
    if (!out) {
        set_error("hxc_partition_run: NULL output");
        return HXC_E_INVALID;
    }
    hxc_status st = check_args(host_x, host_r, n, parts, work, "hxc_partition_run");
    if (st) return st;
    if (!dev_from_handle(dh)) return HXC_E_INVALID;
    const std::vector<int64_t> b = split(n, parts, false);
    std::vector<hxc_future> w(parts, nullptr), k(parts, nullptr), r;
    auto release = [](std::vector<hxc_future> &v) {
        for (hxc_future f : v)
            if (f) hxc_future_release(f);
    };
    // loop 1: every partition's copy to the device
    for (int i = 0; i < parts && !st; i++) {
        const int64_t m = b[i + 1] - b[i];
        if (m == 0) continue;
        st = hxc_buffer_enqueue_write(work, (size_t)b[i] * 8, (size_t)m * 8, host_x + b[i], i, deps,
                                      ndeps, &w[i]);
    }
    // loop 2: the kernel on every partition, after its copy
    for (int i = 0; i < parts && !st; i++) {
        if (!w[i]) continue;
        hxc_partition_args a{work, b[i + 1] - b[i], b[i]};
        st = hxc_launch(dh, HXC_K_PARTITION, &a, sizeof a, nullptr, i, &w[i], 1, &k[i]);
    }
    // loop 3: every partition's result back to the host, after its kernel
    for (int i = 0; i < parts && !st; i++) {
        if (!k[i]) continue;
        hxc_future f = nullptr;
        st = hxc_buffer_enqueue_read(work, (size_t)b[i] * 8, (size_t)(b[i + 1] - b[i]) * 8,
                                     host_r + b[i], i, &k[i], 1, &f);
        if (!st) r.push_back(f);
    }
    if (!st) {
        if (r.empty())
            st = hxc_when_all(deps, ndeps, out);  // nothing to move: ready with the deps
        else
            st = hxc_when_all(r.data(), (int)r.size(), out);
    }
    release(w);
    release(k);
    release(r);
    return st;
}

hxc_status hxc_partition_run_native(hxc_device dh, const double *host_x, double *host_r, int64_t n,
                                    int parts, hxc_buffer work) {
    hxc::drv::NvtxRange nvtx_range("hxc_partition_run_native");
    hxc_status st = check_args(host_x, host_r, n, parts, work, "hxc_partition_run_native");
    if (st) return st;
    Ref<Device> d = dev_from_handle(dh);
    Ref<Buffer> buf = buf_from_handle(work);
    if (!d || !buf) return HXC_E_INVALID;
    if (buf->dev.get() != d.get()) {
        set_error("hxc_partition_run_native: work buffer lives on another device");
        return HXC_E_INVALID;
    }
    if ((st = d->make_current())) return st;
    const std::vector<int64_t> b = split(n, parts, false);
    std::vector<cudaStream_t> s(parts);
    for (int i = 0; i < parts; i++)
        if ((st = d->stream(i, &s[i]))) return st;
    double *x = static_cast<double *>(buf->ptr);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < parts && e == cudaSuccess; i++)
        if (b[i + 1] > b[i])
            e = cudaMemcpyAsync(x + b[i], host_x + b[i], (size_t)(b[i + 1] - b[i]) * 8,
                                cudaMemcpyHostToDevice, s[i]);
    for (int i = 0; i < parts && e == cudaSuccess; i++)
        if (b[i + 1] > b[i]) e = k::partition(x + b[i], b[i + 1] - b[i], nullptr, s[i]);
    for (int i = 0; i < parts && e == cudaSuccess; i++)
        if (b[i + 1] > b[i])
            e = cudaMemcpyAsync(host_r + b[i], x + b[i], (size_t)(b[i + 1] - b[i]) * 8,
                                cudaMemcpyDeviceToHost, s[i]);
    for (int i = 0; i < parts; i++) {
        cudaError_t e2 = cudaStreamSynchronize(s[i]);
        if (e == cudaSuccess) e = e2;
    }
    return e == cudaSuccess ? HXC_OK : cuda_status(e, "hxc_partition_run_native");
}

}  // extern "C"
