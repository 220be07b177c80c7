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

template <typename C>
__global__ void __launch_bounds__(kThreads) k_inner(const C *a, const C *b, int64_t npts, InnerGeom g, double *partial) {
    double acc[kVals];
#pragma unroll
    for (int k = 0; k < kVals; ++k) acc[k] = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < npts; j += (int64_t)gridDim.x * kThreads) {
        const C u = a[j], v = b[j];
        // conj(u) v
        const double re = (double)u.x * (double)v.x + (double)u.y * (double)v.y;
        const double im = (double)u.x * (double)v.y - (double)u.y * (double)v.x;
        acc[0] += re;
        acc[1] += im;
        // lattice index per axis, in 32 bits (sop_adjoint_gradient accepts
        // lattices of fewer than 2^31 points)
        uint32_t r = (uint32_t)j;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            if (ax < g.ndim) {
                const uint32_t n = (uint32_t)g.dims[ax];
                const uint32_t i = r % n;
                r /= n;
                const double x = g.x0[ax] + (double)i * g.h[ax];
                acc[2 + 2 * ax] = fma(x, re, acc[2 + 2 * ax]);
                acc[3 + 2 * ax] = fma(x, im, acc[3 + 2 * ax]);
            }
        }
    }
    __shared__ double ws[kVals][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kVals; ++k) {
        const double s = warp_sum(acc[k]);
        if (lane == 0) ws[k][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < kVals) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += ws[threadIdx.x][w];
        partial[(int64_t)blockIdx.x * kVals + threadIdx.x] = s;
    }
}

// out[k] = scale * sum over blocks, fixed order.
__global__ void k_inner_final(const double *partial, int nb, double scale, double *out) {
    const int k = threadIdx.x;
    if (k < kVals) {
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += partial[(int64_t)i * kVals + k];
        out[k] = scale * s;
    }
}

template <typename C>
__global__ void __launch_bounds__(kThreads) k_accum(const C *a, const C *b, int64_t npts, double w, double2 *acc) {
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < npts; j += (int64_t)gridDim.x * kThreads) {
        const C u = a[j], v = b[j];
        double2 s = acc[j];
        s.x = fma(w, (double)u.x * (double)v.x + (double)u.y * (double)v.y, s.x);
        s.y = fma(w, (double)u.x * (double)v.y - (double)u.y * (double)v.x, s.y);
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
    k_inner_final<<<1, 32, 0, s>>>(partial, kBlocks, dV, out);
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
