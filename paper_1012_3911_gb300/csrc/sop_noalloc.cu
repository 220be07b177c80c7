// sop_noalloc.cu -- sop_norm_noalloc: the norm reduction for callers that
// may not allocate device memory.
//
// Who needs it: sop_norm works on a plan, and a plan takes device memory
// from cudaMalloc (its tables and the reduction partials).  Some host
// programs cannot allow that: frameworks that hand all of HBM to their own
// pool allocator and forbid any other device allocation, and latency-bound
// loops where cudaMalloc/cudaFree, which can synchronise the whole device,
// would stall work on other streams.  This entry point takes the state and
// the output from the caller and keeps its only scratch -- one FP64 partial
// sum per block -- in the file-scope array below, so it never allocates.
//
// The array is part of the library image: every GPU that loads libsop.so
// holds it (256 KB) until the process exits.  All calls share it and each
// call leaves its partial sums there; calls that may run at the same time on
// the GPU (unordered streams, or several host threads) race on it and must be
// serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "sop.h"

namespace sop {
void set_last_error(const std::string &msg);   // defined in sop_api.cu
}

namespace {
constexpr int kThreads = 256;
constexpr int64_t kValuesPerBlock = 16384;            // complex values per partial sum
constexpr int kMaxPartials = 32768;                   // slots in the scratch array
constexpr int64_t kMaxValues = kValuesPerBlock * kMaxPartials;   // 2^29 complex values
constexpr int kMaxDevices = 64;
}  // namespace

// One FP64 partial sum per block of the last call.
static __device__ __align__(256) double sop_noalloc_scratch[kMaxPartials];

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[kThreads / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < kThreads / 32 ? ws[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;   // valid in thread 0
}

// Block b sums |psi|^2 over values [b * kValuesPerBlock, (b + 1) * kValuesPerBlock) in FP64.
template <typename C>
__global__ void __launch_bounds__(kThreads) k_partials(const C *psi, int64_t n, double *partials) {
    const int64_t begin = (int64_t)blockIdx.x * kValuesPerBlock;
    const int64_t end = begin + kValuesPerBlock < n ? begin + kValuesPerBlock : n;
    double acc = 0.0;
    for (int64_t i = begin + threadIdx.x; i < end; i += kThreads) {
        const C z = psi[i];
        const double x = (double)z.x, y = (double)z.y;
        acc = fma(x, x, fma(y, y, acc));
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Fixed-order sum of the nb partials written by the same call, times scale.
__global__ void __launch_bounds__(kThreads) k_final(const double *partials, int nb, double scale, double *out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) acc += partials[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) out[0] = scale * acc;
}

// Device address of the scratch array on the current device.  Host code must
// not pass the symbol itself to a kernel (on the host it names a host-side
// stand-in); the address is looked up once per device with that device
// current and cached for the life of the process (a cudaDeviceReset after
// the first call would leave it stale; the header says so).
int scratch_address(double **out) {
    static std::mutex mu;
    static double *addr[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        sop::set_last_error(std::string("sop_norm_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return SOP_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        sop::set_last_error("sop_norm_noalloc: device index beyond 63");
        return SOP_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (addr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, sop_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            sop::set_last_error(std::string("sop_norm_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return SOP_ECUDA;
        }
        addr[dev] = static_cast<double *>(p);
    }
    *out = addr[dev];
    return SOP_OK;
}

}  // namespace

extern "C" int sop_norm_noalloc(const void *psi_dev, int64_t n_values, int dtype, double scale, double *out_dev,
                                void *cuda_stream) {
    if (!psi_dev || !out_dev) {
        sop::set_last_error("sop_norm_noalloc: psi_dev and out_dev must be device pointers");
        return SOP_EINVAL;
    }
    if (dtype != SOP_C64 && dtype != SOP_C128) {
        sop::set_last_error("sop_norm_noalloc: dtype must be SOP_C64 or SOP_C128");
        return SOP_EINVAL;
    }
    const size_t csz = dtype == SOP_C128 ? 16 : 8;
    if (reinterpret_cast<uintptr_t>(psi_dev) % csz != 0 || reinterpret_cast<uintptr_t>(out_dev) % 8 != 0) {
        sop::set_last_error("sop_norm_noalloc: misaligned psi_dev or out_dev");
        return SOP_EINVAL;
    }
    if (n_values < 0) {
        sop::set_last_error("sop_norm_noalloc: n_values < 0");
        return SOP_EINVAL;
    }
    if (n_values > kMaxValues) {
        sop::set_last_error("sop_norm_noalloc: n_values = " + std::to_string(n_values) +
                            " exceeds the limit of 536870912 (2^29) complex values per call set by the "
                            "fixed scratch array; use sop_norm on a plan");
        return SOP_EUNSUPPORTED;
    }
    double *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != SOP_OK) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    const int nb = (int)((n_values + kValuesPerBlock - 1) / kValuesPerBlock);
    if (nb > 0) {
        if (dtype == SOP_C128)
            k_partials<double2><<<nb, kThreads, 0, s>>>(static_cast<const double2 *>(psi_dev), n_values, scratch);
        else
            k_partials<float2><<<nb, kThreads, 0, s>>>(static_cast<const float2 *>(psi_dev), n_values, scratch);
    }
    k_final<<<1, kThreads, 0, s>>>(scratch, nb, scale, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        sop::set_last_error(std::string("sop_norm_noalloc: kernel launch: ") + cudaGetErrorString(e));
        return SOP_ECUDA;
    }
    return SOP_OK;
}
