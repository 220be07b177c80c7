// sop_adjoint.cu -- reductions of the adjoint gradient (a follow-on of the
// split-operator method of Bauke & Keitel, Eqs. 6-8 / 10a-b; the paper has no
// adjoint).
//
// For J = |<phi|psi_N>|^2 with costates lambda_m (lambda_N = phi,
// lambda_m = U_m^dagger lambda_{m+1}) the gradient needs, for every m,
//   <lambda_m|psi_m>, <lambda_m|X_a|psi_m>   (inner products, k_inner)
//   acc_j += w_m conj(lambda_{m,j}) psi_{m,j}  (per point, k_accum)
// and finally dJ/dV_j = 2 Re(conj(c) k_V dV acc_j) (k_grad_v).
//
// Reductions use a fixed grid and a fixed-order final sum in FP64, like
// sop_reduce.cu, so results are deterministic run to run.
#include "sop_fft.cuh"
#include "sop_internal.h"

namespace sop {

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 152 * 2;
constexpr int kVals = 8;   // re/im of <a|b> and of <a|X_a|b>, a < 3

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct InnerGeom {
    int ndim;
    int64_t dims[3];
    double x0[3], h[3];   // x_{a,i} = x0[a] + i h[a]
};

// Products and coordinates are formed in the precision of the state (FP32
// for complex64); each thread sums kChunk points in that precision and adds
// the chunk sums in FP64 (FP64 arithmetic is a small fraction of the FP32
// rate on GB300, and a 16-term FP32 sum errs by ~1e-6 relative).
constexpr int kChunk = 16;

template <typename C>
__global__ void __launch_bounds__(kThreads) k_inner(const C *a, const C *b, int64_t npts, InnerGeom g, double *partial) {
    using R = decltype(C{}.x);
    double acc[kVals];
#pragma unroll
    for (int k = 0; k < kVals; ++k) acc[k] = 0.0;
    R x0[3], hh[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        x0[ax] = (R)g.x0[ax];
        hh[ax] = (R)g.h[ax];
    }
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    while (j < npts) {
        R loc[kVals];
#pragma unroll
        for (int k = 0; k < kVals; ++k) loc[k] = R(0);
        for (int q = 0; q < kChunk && j < npts; ++q, j += stride) {
            const C u = a[j], v = b[j];
            const R re = u.x * v.x + u.y * v.y;   // conj(u) v
            const R im = u.x * v.y - u.y * v.x;
            loc[0] += re;
            loc[1] += im;
            // lattice index per axis, in 32 bits (sop_adjoint_gradient accepts
            // lattices of fewer than 2^31 points)
            uint32_t r = (uint32_t)j;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                if (ax < g.ndim) {
                    const uint32_t n = (uint32_t)g.dims[ax];
                    const uint32_t i = r % n;
                    r /= n;
                    const R x = x0[ax] + (R)i * hh[ax];
                    loc[2 + 2 * ax] += x * re;
                    loc[3 + 2 * ax] += x * im;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kVals; ++k) acc[k] += (double)loc[k];
    }
    __shared__ double ws[kVals][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kVals; ++k) {
        const double sum = warp_sum(acc[k]);
        if (lane == 0) ws[k][wid] = sum;
    }
    __syncthreads();
    if (threadIdx.x < kVals) {
        double sum = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) sum += ws[threadIdx.x][w];
        partial[(int64_t)blockIdx.x * kVals + threadIdx.x] = sum;
    }
}

// out[k] = scale * sum over blocks: warp k sums value k (fixed order).
__global__ void k_inner_final(const double *partial, int nb, double scale, double *out) {
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k < kVals) {
        double sum = 0.0;
        for (int i = lane; i < nb; i += 32) sum += partial[(int64_t)i * kVals + k];
        sum = warp_sum(sum);
        if (lane == 0) out[k] = scale * sum;
    }
}

// acc_j += w conj(a_j) b_j: the product in the state's precision, the sum in FP64.
template <typename C>
__global__ void __launch_bounds__(kThreads) k_accum(const C *a, const C *b, int64_t npts, double w, double2 *acc) {
    using R = decltype(C{}.x);
    const R wr = (R)w;
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < npts; j += (int64_t)gridDim.x * kThreads) {
        const C u = a[j], v = b[j];
        double2 s = acc[j];
        s.x += (double)(wr * (u.x * v.x + u.y * v.y));
        s.y += (double)(wr * (u.x * v.y - u.y * v.x));
        acc[j] = s;
    }
}

// g_j = 2 Re(z acc_j) with z = conj(c) k_V dV given as (zr, zi).
__global__ void __launch_bounds__(kThreads) k_grad_v(const double2 *acc, int64_t npts, double zr, double zi, double *g) {
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < npts; j += (int64_t)gridDim.x * kThreads) {
        const double2 s = acc[j];
        g[j] = 2.0 * (zr * s.x - zi * s.y);
    }
}

}  // namespace

int inner_partials() { return kBlocks * kVals; }

cudaError_t launch_inner(const void *a, const void *b, bool f64, int ndim, const int64_t *dims, const double *h,
                         double dV, double *partial, double *out, cudaStream_t s) {
    InnerGeom g{};
    g.ndim = ndim;
    int64_t npts = 1;
    for (int ax = 0; ax < 3; ++ax) {
        g.dims[ax] = ax < ndim ? dims[ax] : 1;
        g.h[ax] = ax < ndim ? h[ax] : 0.0;
        g.x0[ax] = ax < ndim ? -0.5 * (double)dims[ax] * h[ax] : 0.0;
        npts *= g.dims[ax];
    }
    if (f64)
        k_inner<double2><<<kBlocks, kThreads, 0, s>>>(static_cast<const double2 *>(a), static_cast<const double2 *>(b),
                                                         npts, g, partial);
    else
        k_inner<float2><<<kBlocks, kThreads, 0, s>>>(static_cast<const float2 *>(a), static_cast<const float2 *>(b),
                                                       npts, g, partial);
    k_inner_final<<<1, 32 * kVals, 0, s>>>(partial, kBlocks, dV, out);
    return cudaGetLastError();
}

cudaError_t launch_accum(const void *a, const void *b, bool f64, int64_t npts, double w, double *acc,
                         cudaStream_t s) {
    double2 *ac = reinterpret_cast<double2 *>(acc);
    if (f64)
        k_accum<double2><<<kBlocks * 4, kThreads, 0, s>>>(static_cast<const double2 *>(a),
                                                            static_cast<const double2 *>(b), npts, w, ac);
    else
        k_accum<float2><<<kBlocks * 4, kThreads, 0, s>>>(static_cast<const float2 *>(a),
                                                           static_cast<const float2 *>(b), npts, w, ac);
    return cudaGetLastError();
}

cudaError_t launch_grad_v(const double *acc, int64_t npts, double zr, double zi, double *g, cudaStream_t s) {
    k_grad_v<<<kBlocks * 4, kThreads, 0, s>>>(reinterpret_cast<const double2 *>(acc), npts, zr, zi, g);
    return cudaGetLastError();
}

}  // namespace sop
