// sop_peak.cu -- FMA throughput of the GPU the library runs on (the
// denominator of the arithmetic roofline of the FP64 split step).
//
// Every thread runs 8 independent FMA chains a = a * b + c for kIters
// iterations, on a grid of 8 CTAs of 256 threads per SM; the flop count is
// 2 per FMA.  The chains' results feed one conditional store, so the
// arithmetic cannot be dropped, and the store never happens for these inputs.
#include <cuda_runtime.h>

#include <string>

#include "sop.h"
#include "sop_internal.h"

namespace sop {
void set_last_error(const std::string &msg);   // defined in sop_api.cu
namespace {

constexpr int kChains = 8;
constexpr int kIters = 1 << 14;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;

template <typename R> __global__ void __launch_bounds__(kThreads) fma_chains(R b, R c, R *sink) {
    R a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = R(threadIdx.x + k);
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    R s = R(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == R(-12345.678)) sink[0] = s;   // never true for b = 1 - 2^-20, c = 2^-30
}

template <typename R> int measure(double *flops_per_s, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    R *sink = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(R));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    const dim3 grid((unsigned)(sms * kCtasPerSm));
    const R b = R(1) - R(1.0 / (1 << 20)), c = R(1.0 / (1 << 30));
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch is a warm-up
        cudaEventRecord(e0, s);
        fma_chains<R><<<grid, kThreads, 0, s>>>(b, c, sink);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) {
        set_last_error(std::string("sop_fma_peak: ") + cudaGetErrorString(e));
        return SOP_ECUDA;
    }
    const double fmas = (double)grid.x * kThreads * kChains * (double)kIters;
    *flops_per_s = 2.0 * fmas / (best * 1e-3);
    return SOP_OK;
}

}  // namespace
}  // namespace sop

extern "C" int sop_fma_peak(int f64, double *flops_per_s, void *cuda_stream) {
    if (!flops_per_s) {
        sop::set_last_error("sop_fma_peak: null output");
        return SOP_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    return f64 ? sop::measure<double>(flops_per_s, s) : sop::measure<float>(flops_per_s, s);
}
