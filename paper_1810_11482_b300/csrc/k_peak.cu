// Arithmetic-pipe throughput of the device (hxc_pipe_rate).
//
// The FP64 stencils of this library are bound by the FP64 pipe, not by HBM,
// so their rooflines need the rate that pipe actually sustains.  This file
// measures it: a kernel of independent dependency chains (eight per thread,
// eight 256-thread CTAs per SM) that issues nothing but the measured
// instruction, timed with CUDA events, and the SM clock seen by the first
// CTA during the run (clock64 ticks over globaltimer nanoseconds).
#include "hxc.h"
#include "runtime.hpp"

namespace hxc {
namespace k {
namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;
constexpr int kCtasPerSm = 8;

template <int KIND>
struct PipeT {
    using T = double;
};
template <>
struct PipeT<HXC_PIPE_F32_FMA> {
    using T = float;
};

template <int KIND>
__device__ __forceinline__ typename PipeT<KIND>::T pipe_op(typename PipeT<KIND>::T x,
                                                           typename PipeT<KIND>::T a,
                                                           typename PipeT<KIND>::T b) {
    if constexpr (KIND == HXC_PIPE_F64_FMA) return __fma_rn(x, a, b);
    else if constexpr (KIND == HXC_PIPE_F64_ADD) return __dadd_rn(x, a);
    else return __fmaf_rn(x, a, b);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// x <- fma(x, a, b) (or x + a) on kChains independent chains per thread,
// `iters` times.  With a = 1 - 2^-10, b = 2^-10 the FMA chains converge to 1
// and the add chains grow slowly, so every value stays normal.  The results
// are stored only when `store` is set (never, in practice), which the
// compiler cannot know, so no operation is removed.
template <int KIND>
__global__ void __launch_bounds__(kBlock) k_pipe(typename PipeT<KIND>::T a,
                                                 typename PipeT<KIND>::T b, int iters, int store,
                                                 typename PipeT<KIND>::T *sink,
                                                 unsigned long long *clk) {
    using T = typename PipeT<KIND>::T;
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = (T)(threadIdx.x + 1) * (T)0.001 + (T)c;
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long c0 = 0, t0 = 0;
    if (timer) {
        t0 = global_ns();
        c0 = clock64();
    }
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) x[c] = pipe_op<KIND>(x[c], a, b);
    }
    if (timer) {
        const unsigned long long c1 = clock64();
        const unsigned long long t1 = global_ns();
        clk[0] = c1 - c0;
        clk[1] = t1 - t0;
    }
    if (store) {
        T s = x[0];
#pragma unroll
        for (int c = 1; c < kChains; c++) s += x[c];
        sink[blockIdx.x * kBlock + threadIdx.x] = s;
    }
}

template <int KIND>
cudaError_t launch_pipe(int ctas, int iters, cudaStream_t s, void *sink,
                        unsigned long long *clk) {
    using T = typename PipeT<KIND>::T;
    const T a = (T)1 - (T)1 / (T)1024, b = (T)1 / (T)1024;
    const T aa = KIND == HXC_PIPE_F64_ADD ? (T)1e-9 : a;
    k_pipe<KIND><<<ctas, kBlock, 0, s>>>(aa, b, iters, 0, static_cast<T *>(sink), clk);
    return cudaGetLastError();
}

cudaError_t launch_kind(int kind, int ctas, int iters, cudaStream_t s, void *sink,
                        unsigned long long *clk) {
    switch (kind) {
        case HXC_PIPE_F64_FMA: return launch_pipe<HXC_PIPE_F64_FMA>(ctas, iters, s, sink, clk);
        case HXC_PIPE_F64_ADD: return launch_pipe<HXC_PIPE_F64_ADD>(ctas, iters, s, sink, clk);
        default: return launch_pipe<HXC_PIPE_F32_FMA>(ctas, iters, s, sink, clk);
    }
}

}  // namespace
}  // namespace k
}  // namespace hxc

extern "C" hxc_status hxc_pipe_rate(hxc_device dev, int kind, double *ops_per_s,
                                    double *sm_mhz) {
    using namespace hxc;
    Ref<Device> d = dev_from_handle(dev);
    if (!d) return HXC_E_INVALID;
    if (!ops_per_s || (kind != HXC_PIPE_F64_FMA && kind != HXC_PIPE_F64_ADD &&
                       kind != HXC_PIPE_F32_FMA)) {
        set_error("hxc_pipe_rate: invalid kind or output pointer");
        return HXC_E_INVALID;
    }
    hxc_status st = d->make_current();
    if (st) return st;
    const int ctas = d->prop.multiProcessorCount * k::kCtasPerSm;
    // about 0.1 s per timed launch on B300 (FP64 ~0.5 Top/s, FP32 ~38 Top/s)
    const int iters = kind == HXC_PIPE_F32_FMA ? 1000000 : 20000;
    void *sink = nullptr;
    unsigned long long *clk = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    unsigned long long hclk[2] = {0, 0};
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&sink, (size_t)ctas * k::kBlock * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&clk, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // warm-up (clocks up, code loaded), then the timed launch
    if (e == cudaSuccess) e = k::launch_kind(kind, ctas, iters / 10, s, sink, clk);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = k::launch_kind(kind, ctas, iters, s, sink, clk);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess)
        e = cudaMemcpy(hclk, clk, sizeof(hclk), cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (clk) cudaFree(clk);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) return cuda_status(e, "hxc_pipe_rate");
    const double ops = (double)ctas * k::kBlock * (double)iters * k::kChains;
    *ops_per_s = ops / (ms * 1e-3);
    if (sm_mhz) *sm_mhz = hclk[1] ? (double)hclk[0] / (double)hclk[1] * 1e3 : 0.0;
    return HXC_OK;
}
