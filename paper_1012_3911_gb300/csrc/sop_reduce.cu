// sop_reduce.cu -- FP64 reductions for sop_norm and sop_energy.
//
// Each reduction runs a fixed grid (the block count never depends on the
// data), every thread accumulates its grid-stride subset in FP64, blocks
// reduce by warp shuffles, and one final single-block kernel adds the block
// partials in a fixed order.  The result is deterministic run to run.
#include "sop_fft.cuh"
#include "sop_internal.h"

namespace sop {

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 152 * 4;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void block_store(double acc, double *partial) {
    __shared__ double ws[kThreads / 32];
    acc = warp_sum(acc);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        double v = lane < kThreads / 32 ? ws[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) partial[blockIdx.x] = v;
    }
}

template <typename C> __global__ void __launch_bounds__(kThreads) k_norm(const C *psi, int64_t n, double *partial) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const C z = psi[i];
        const double x = (double)z.x, y = (double)z.y;
        acc = fma(x, x, fma(y, y, acc));
    }
    block_store(acc, partial);
}

template <typename C>
__global__ void __launch_bounds__(kThreads) k_energy_v(const C *psi, const double *V, int64_t npts, int comps,
                                                        double *partial) {
    double acc = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < npts; j += (int64_t)gridDim.x * kThreads) {
        double r = 0.0;
        for (int c = 0; c < comps; ++c) {
            const C z = psi[c * npts + j];
            const double x = (double)z.x, y = (double)z.y;
            r = fma(x, x, fma(y, y, r));
        }
        acc = fma(V[j], r, acc);
    }
    block_store(acc, partial);
}

struct KGeom {
    int ndim;
    int64_t dims[3];
    int64_t off[3];   // offsets of each axis' momenta in pgrid
};

// Schroedinger: sum_k |p_k|^2/(2m) |psi~_k|^2.
// Dirac (2D, four components): sum_k psi~^dag (c alpha.p + m c^2 beta) psi~,
// written out on the coupled pairs (1,4) and (2,3); 1D, two components:
// alpha_1 = sigma_x, beta = sigma_z.
template <typename C>
__global__ void __launch_bounds__(kThreads) k_energy_t(const C *pt, KGeom g, const double *pgrid, int comps,
                                                        double mass, double c, double *partial) {
    int64_t npts = 1;
    for (int a = 0; a < g.ndim; ++a) npts *= g.dims[a];
    double acc = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x; k < npts; k += (int64_t)gridDim.x * kThreads) {
        double p[3] = {0.0, 0.0, 0.0};
        int64_t r = k;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a < g.ndim) {
                const int64_t ka = r % g.dims[a];
                r /= g.dims[a];
                p[a] = pgrid[g.off[a] + ka];
            }
        }
        if (comps == 1) {
            const C z = pt[k];
            const double x = (double)z.x, y = (double)z.y;
            const double p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
            acc = fma(p2 / (2.0 * mass), fma(x, x, y * y), acc);
        } else if (comps == 2) {
            // 1D: H = c p sigma_x + m c^2 sigma_z
            const C z0 = pt[k], z1 = pt[npts + k];
            const double n0 = (double)z0.x * z0.x + (double)z0.y * z0.y;
            const double n1 = (double)z1.x * z1.x + (double)z1.y * z1.y;
            const double sr = (double)z0.x * z1.x + (double)z0.y * z1.y;   // Re conj(z0) z1
            acc += mass * c * c * (n0 - n1) + 2.0 * c * p[0] * sr;
        } else {
            const C z0 = pt[k], z1 = pt[npts + k], z2 = pt[2 * npts + k], z3 = pt[3 * npts + k];
            const double mc2 = mass * c * c;
            const double n0 = (double)z0.x * z0.x + (double)z0.y * z0.y;
            const double n1 = (double)z1.x * z1.x + (double)z1.y * z1.y;
            const double n2 = (double)z2.x * z2.x + (double)z2.y * z2.y;
            const double n3 = (double)z3.x * z3.x + (double)z3.y * z3.y;
            // s = conj(z0) z3 ; u = conj(z1) z2
            const double sr = (double)z0.x * z3.x + (double)z0.y * z3.y;
            const double si = (double)z0.x * z3.y - (double)z0.y * z3.x;
            const double ur = (double)z1.x * z2.x + (double)z1.y * z2.y;
            const double ui = (double)z1.x * z2.y - (double)z1.y * z2.x;
            // Re[(p_x - i p_y) s] = p_x sr + p_y si ; Re[(p_x + i p_y) u] = p_x ur - p_y ui;
            // alpha_3 (3D): p_z Re[conj(z0) z2 - conj(z1) z3]
            const double zr = (double)z0.x * z2.x + (double)z0.y * z2.y - (double)z1.x * z3.x - (double)z1.y * z3.y;
            const double off = 2.0 * c * (p[0] * sr + p[1] * si + p[0] * ur - p[1] * ui + p[2] * zr);
            acc += mc2 * (n0 + n1 - n2 - n3) + off;
        }
    }
    block_store(acc, partial);
}

__global__ void __launch_bounds__(kThreads) k_final(const double *partial, int nb, double scale, double *out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) acc += partial[i];
    __shared__ double ws[kThreads / 32];
    acc = warp_sum(acc);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        double v = lane < kThreads / 32 ? ws[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) out[0] = scale * v;
    }
}

}  // namespace

int reduce_blocks() { return kBlocks; }

cudaError_t reduce_norm(const void *psi, int64_t n, bool f64, double *partial, double *out, double scale,
                        cudaStream_t s) {
    if (f64) k_norm<double2><<<kBlocks, kThreads, 0, s>>>(reinterpret_cast<const double2 *>(psi), n, partial);
    else k_norm<float2><<<kBlocks, kThreads, 0, s>>>(reinterpret_cast<const float2 *>(psi), n, partial);
    k_final<<<1, kThreads, 0, s>>>(partial, kBlocks, scale, out);
    return cudaGetLastError();
}

cudaError_t reduce_energy_v(const void *psi, const double *V, int64_t npts, int comps, bool f64, double *partial,
                            double *out, double scale, cudaStream_t s) {
    if (f64)
        k_energy_v<double2><<<kBlocks, kThreads, 0, s>>>(reinterpret_cast<const double2 *>(psi), V, npts, comps, partial);
    else
        k_energy_v<float2><<<kBlocks, kThreads, 0, s>>>(reinterpret_cast<const float2 *>(psi), V, npts, comps, partial);
    k_final<<<1, kThreads, 0, s>>>(partial, kBlocks, scale, out);
    return cudaGetLastError();
}

cudaError_t reduce_energy_t(const void *psit, int ndim, const int64_t *dims, const double *pgrid, int comps,
                            double mass, double c, bool f64, double *partial, double *out, double scale,
                            cudaStream_t s) {
    KGeom g{};
    g.ndim = ndim;
    int64_t off = 0;
    for (int a = 0; a < 3; ++a) {
        g.dims[a] = a < ndim ? dims[a] : 1;
        g.off[a] = off;
        if (a < ndim) off += dims[a];
    }
    if (f64)
        k_energy_t<double2><<<kBlocks, kThreads, 0, s>>>(reinterpret_cast<const double2 *>(psit), g, pgrid, comps,
                                                         mass, c, partial);
    else
        k_energy_t<float2><<<kBlocks, kThreads, 0, s>>>(reinterpret_cast<const float2 *>(psit), g, pgrid, comps,
                                                        mass, c, partial);
    k_final<<<1, kThreads, 0, s>>>(partial, kBlocks, scale, out);
    return cudaGetLastError();
}

}  // namespace sop
