// sop_adjoint.cu -- reductions of the adjoint gradient (a follow-on of the
// split-operator method of Bauke & Keitel, Eqs. 6-8 / 10a-b; the paper has no
// adjoint).
//
// For J = |<phi|psi_N>|^2 with costates lambda_m (lambda_N = phi,
// lambda_m = U_m^dagger lambda_{m+1}) the gradient needs, for every m,
//   <lambda_m|psi_m>, <lambda_m|X_a|psi_m>   (inner products, k_inner)
//   acc_j += w_m conj(lambda_{m,j}) psi_{m,j}  (per point, k_accum)
// and finally dJ/dV_j = 2 Re(conj(c) k_V dV acc_j) (k_grad_v).  The same
// file holds the reductions of the spectral method (k_spectral_*).
//
// Reductions use a fixed grid and a fixed-order final sum, so results are
// deterministic run to run.  Per-point work avoids FP64 instructions (GB300
// runs about one FP64 operation per SM per clock): sums stay in the state's
// precision, as float pairs (two-sum) for complex64, and reach FP64 per warp.
#include <type_traits>

#include "sop_fft.cuh"
#include "sop_internal.h"

namespace sop {

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 152 * 2;
constexpr int kVals = 8;   // re/im of <a|b> and of <a|X_a|b>, a < 3
constexpr int kMaxEnergies = SOP_SPECTRAL_MAX_ENERGIES;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// s + e = a + b exactly (Knuth's two-sum; explicit round-to-nearest adds so
// that nothing is contracted or reassociated).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// A running sum kept as an unevaluated pair hi + lo of the state's real
// type: for float, two-sum keeps about 48 significant bits without any FP64
// instruction (FP64 throughput on this part is a small fraction of FP32);
// for double, lo stays zero.
template <typename R> struct PairSum {
    R hi = R(0), lo = R(0);
    __device__ __forceinline__ void add(R v) {
        if constexpr (sizeof(R) == 4) {
            float s, e;
            two_sum(hi, v, s, e);
            hi = s;
            lo += e;
        } else {
            hi += v;
        }
    }
    __device__ __forceinline__ void add(const PairSum &o) {
        add(o.hi);
        lo += o.lo;
    }
    __device__ __forceinline__ PairSum shfl_xor(int o) const {
        PairSum r;
        r.hi = __shfl_xor_sync(0xffffffffu, hi, o);
        r.lo = __shfl_xor_sync(0xffffffffu, lo, o);
        return r;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

struct InnerGeom {
    int ndim;
    int64_t dims[3];
    double x0[3], h[3];   // x_{a,i} = x0[a] + i h[a]
};

// Products and coordinates are formed in the precision of the state (FP32
// for complex64); each thread sums kChunk points in that precision, keeps
// the chunk sums as float pairs (PairSum: no FP64 instruction per point, the
// FP64 pipe being a small fraction of FP32 on this part), reduces them over
// the warp as pairs and only then adds in FP64 (per warp and block).
constexpr int kChunk = 16;

template <typename C>
__global__ void __launch_bounds__(kThreads) k_inner(const C *a, const C *b, int64_t npts, InnerGeom g, double *partial) {
    using R = decltype(C{}.x);
    PairSum<R> acc[kVals];
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
        for (int k = 0; k < kVals; ++k) acc[k].add(loc[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < kVals; ++k) acc[k].add(acc[k].shfl_xor(o));
    __shared__ double ws[kVals][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < kVals; ++k) ws[k][wid] = acc[k].value();
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

// acc_j += w conj(a_j) b_j, the product in the state's precision.  Complex128:
// FP64 accumulators; complex64: float pairs (hi.re, hi.im, lo.re, lo.im) in
// the same 16 bytes, updated by two-sum (read back by k_grad_v).
template <typename C>
__global__ void __launch_bounds__(kThreads) k_accum(const C *a, const C *b, int64_t npts, double w, double2 *acc) {
    using R = decltype(C{}.x);
    constexpr bool kPair = sizeof(R) == 4;
    using A = typename std::conditional<kPair, float4, double2>::type;
    A *ac = reinterpret_cast<A *>(acc);
    const R wr = (R)w;
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < npts; j += (int64_t)gridDim.x * kThreads) {
        const C u = a[j], v = b[j];
        A s = ac[j];
        const R px = wr * (u.x * v.x + u.y * v.y), py = wr * (u.x * v.y - u.y * v.x);
        if constexpr (kPair) {
            float hx, ex, hy, ey;
            two_sum(s.x, px, hx, ex);
            two_sum(s.y, py, hy, ey);
            s = make_float4(hx, hy, s.z + ex, s.w + ey);
        } else {
            s.x += px;
            s.y += py;
        }
        ac[j] = s;
    }
}

// One checkpoint segment at once: slots k < count of lam and psi hold the
// costate and the state at step m0 + k.  For every k the block sums
// <lam_k|psi_k> and <lam_k|X_a|psi_k> (products in the state's precision,
// float pairs over the warp, FP64 per warp slot and block, fixed order) into
// partial[(k gridDim.x + block) 8 + v]; every point adds
// sum_k w_k conj(lam_k) psi_k to its accumulator once (w = 1 for step 0,
// else 2), instead of once per step.
constexpr int kSegPts = 2;          // points per thread and chunk
constexpr int kSegGrid = 152 * 8;   // blocks at most (one chunk each where the lattice allows)

template <typename C>
__global__ void __launch_bounds__(kThreads) k_seg_reduce(const C *__restrict__ lam, const C *__restrict__ psi,
                                                         int64_t npts, int count, int64_t m0, InnerGeom g,
                                                         double2 *acc, double *partial) {
    using R = decltype(C{}.x);
    constexpr bool kPair = sizeof(R) == 4;
    using A = typename std::conditional<kPair, float4, double2>::type;
    extern __shared__ double wsum[];   // [warp][count][kVals]
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (kThreads / 32) * count * kVals; i += kThreads) wsum[i] = 0.0;
    __syncthreads();
    R x0[3], hh[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        x0[ax] = (R)g.x0[ax];
        hh[ax] = (R)g.h[ax];
    }
    const int64_t span = (int64_t)kThreads * kSegPts;
    for (int64_t base = (int64_t)blockIdx.x * span; base < npts; base += (int64_t)gridDim.x * span) {
        R xs[kSegPts][3];
        PairSum<R> ax_[kSegPts], ay_[kSegPts];   // sum_k w_k conj(lam) psi per point
#pragma unroll
        for (int q = 0; q < kSegPts; ++q) {
            uint32_t r = (uint32_t)(base + threadIdx.x + (int64_t)q * kThreads);
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                xs[q][ax] = R(0);
                if (ax < g.ndim) {
                    const uint32_t n = (uint32_t)g.dims[ax];
                    const uint32_t i = r % n;
                    r /= n;
                    xs[q][ax] = x0[ax] + (R)i * hh[ax];
                }
            }
        }
        // slot k + 1 is fetched before slot k's block sums, so its load
        // latency overlaps the shuffles
        C un[kSegPts], vn[kSegPts];
        auto fetch = [&](int k) {
#pragma unroll
            for (int q = 0; q < kSegPts; ++q) {
                const int64_t j = base + threadIdx.x + (int64_t)q * kThreads;
                if (j < npts) {
                    un[q] = lam[(int64_t)k * npts + j];
                    vn[q] = psi[(int64_t)k * npts + j];
                }
            }
        };
        fetch(0);
        for (int k = 0; k < count; ++k) {
            const R w = (m0 + k == 0) ? R(1) : R(2);
            C uc[kSegPts], vc[kSegPts];
#pragma unroll
            for (int q = 0; q < kSegPts; ++q) {
                uc[q] = un[q];
                vc[q] = vn[q];
            }
            if (k + 1 < count) fetch(k + 1);
            R loc[kVals];
#pragma unroll
            for (int v = 0; v < kVals; ++v) loc[v] = R(0);
#pragma unroll
            for (int q = 0; q < kSegPts; ++q) {
                const int64_t j = base + threadIdx.x + (int64_t)q * kThreads;
                if (j < npts) {
                    const C u = uc[q], vv = vc[q];
                    const R re = u.x * vv.x + u.y * vv.y;   // conj(u) v
                    const R im = u.x * vv.y - u.y * vv.x;
                    ax_[q].add(w * re);
                    ay_[q].add(w * im);
                    loc[0] += re;
                    loc[1] += im;
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        loc[2 + 2 * ax] += xs[q][ax] * re;
                        loc[3 + 2 * ax] += xs[q][ax] * im;
                    }
                }
            }
            PairSum<R> ps[kVals];
#pragma unroll
            for (int v = 0; v < kVals; ++v) ps[v].add(loc[v]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int v = 0; v < kVals; ++v) ps[v].add(ps[v].shfl_xor(o));
            if (lane == 0)
#pragma unroll
                for (int v = 0; v < kVals; ++v) wsum[(wid * count + k) * kVals + v] += ps[v].value();
        }
        A *ac = reinterpret_cast<A *>(acc);
#pragma unroll
        for (int q = 0; q < kSegPts; ++q) {
            const int64_t j = base + threadIdx.x + (int64_t)q * kThreads;
            if (j < npts) {
                A sacc = ac[j];
                if constexpr (kPair) {
                    float hx, ex, hy, ey;
                    two_sum(sacc.x, ax_[q].hi, hx, ex);
                    two_sum(sacc.y, ay_[q].hi, hy, ey);
                    sacc = make_float4(hx, hy, sacc.z + (ex + ax_[q].lo), sacc.w + (ey + ay_[q].lo));
                } else {
                    sacc.x += ax_[q].hi;
                    sacc.y += ay_[q].hi;
                }
                ac[j] = sacc;
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < count * kVals; i += kThreads) {
        double sum = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) sum += wsum[w * count * kVals + i];
        const int k = i / kVals, v = i % kVals;
        partial[((int64_t)k * gridDim.x + blockIdx.x) * kVals + v] = sum;
    }
}

// out[(m0 + k) 8 + v] = scale * sum over the nb blocks of slot k (block k,
// warp v, fixed order).
__global__ void k_seg_final(const double *partial, int nb, double scale, double *out, int64_t m0) {
    const int k = blockIdx.x, v = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (v < kVals) {
        double sum = 0.0;
        for (int i = lane; i < nb; i += 32) sum += partial[((int64_t)k * nb + i) * kVals + v];
        sum = warp_sum(sum);
        if (lane == 0) out[(m0 + k) * kVals + v] = scale * sum;
    }
}

// Spectral method.  Per time sample, k_spectral_sample forms the partial
// sums of conj(psi0_j) psi_j (products in the state's precision, summed over
// kUnroll points per thread in that precision, then as a float pair per
// thread and warp, then in FP64 per block) and, for the
// eigenfunctions, copies psi_n into one slot of a ring of up to kRing states;
// every kRing samples k_spectral_accum adds sum_b w_{b,k} psi_b,j into the
// FP64 accumulator of each energy k, so that the accumulators are read and
// written once per kRing steps instead of every step.  Loads of kUnroll
// points are issued before any is used (the memory-level parallelism a
// bandwidth-bound reduction needs with 16 warps per SM).
constexpr int kUnroll = 4;
constexpr int kSampleBlocks = kBlocks * 4;
static_assert(2 * kSampleBlocks <= kBlocks * kVals, "sample partials fit the inner-product partial buffer");
constexpr int kRing = SOP_SPECTRAL_RING;

template <typename C>
__global__ void __launch_bounds__(kThreads) k_spectral_sample(const C *__restrict__ psi0, const C *__restrict__ psi,
                                                              int64_t len, C *__restrict__ slot, double *partial,
                                                              unsigned *done, double scale, double *chi) {
    using R = decltype(C{}.x);
    PairSum<R> sr, si;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t base = (int64_t)blockIdx.x * kThreads + threadIdx.x; base < len; base += kUnroll * stride) {
        C u[kUnroll], v[kUnroll];
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) {
            const int64_t j = base + q * stride;
            if (j < len) {
                u[q] = psi0[j];
                v[q] = psi[j];
            } else {
                u[q] = C{R(0), R(0)};
                v[q] = C{R(0), R(0)};
            }
        }
        if (slot) {
#pragma unroll
            for (int q = 0; q < kUnroll; ++q)
                if (base + q * stride < len) slot[base + q * stride] = v[q];
        }
        R lr = R(0), li = R(0);
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) {
            lr += u[q].x * v[q].x + u[q].y * v[q].y;
            li += u[q].x * v[q].y - u[q].y * v[q].x;
        }
        sr.add(lr);
        si.add(li);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sr.add(sr.shfl_xor(o));
        si.add(si.shfl_xor(o));
    }
    __shared__ double ws[2][kThreads / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        ws[0][wid] = sr.value();
        ws[1][wid] = si.value();
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double sum = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) sum += ws[threadIdx.x][i];
        partial[2 * blockIdx.x + threadIdx.x] = sum;
        __threadfence();
    }
    __syncthreads();
    // the last block to finish adds the block sums (a fixed partition and
    // order, whichever block it is) and re-arms the counter
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double sum = 0.0;   // thread t meets values of parity t & 1 only (kThreads is even)
    for (int i = threadIdx.x; i < 2 * (int)gridDim.x; i += kThreads) sum += __ldcg(partial + i);
#pragma unroll
    for (int o = 16; o > 1; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    __syncthreads();
    if (lane < 2) ws[lane][wid] = sum;
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += ws[threadIdx.x][w];
        chi[threadIdx.x] = scale * t;
    }
    if (threadIdx.x == 0) *done = 0u;
}

// Weights w_{b,k} of the B <= kRing ring states for K <= kMaxEnergies
// energies, rounded to the state's real type on the host (a conversion per
// point would run on the FP64 pipe).
template <typename R> struct RingWeights {
    R re[kRing][kMaxEnergies], im[kRing][kMaxEnergies];
};

// acc_k[j] += sum_{b < B} w_{b,k} ring_b[j] (ring_b at ring + b * len): the B
// products summed in the state's precision.  Complex128 states add into FP64
// accumulators.  Complex64 states keep each accumulator as an unevaluated
// float sum (hi.re, hi.im, lo.re, lo.im) in the same 16 bytes, updated with
// two-sum, so that no FP64 instruction runs per point (FP64 throughput on
// this part is a small fraction of FP32); k_float_pair_to_double turns it
// into complex128 at the end.
template <typename C>
__global__ void __launch_bounds__(kThreads) k_spectral_accum(const C *__restrict__ ring, int B, int64_t len, int K,
                                                             RingWeights<decltype(C{}.x)> w,
                                                             double2 *__restrict__ acc) {
    using R = decltype(C{}.x);
    constexpr bool kPair = sizeof(R) == 4;
    using A = typename std::conditional<kPair, float4, double2>::type;
    A *ac = reinterpret_cast<A *>(acc);
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < len; j += (int64_t)gridDim.x * kThreads) {
        C v[kRing];
#pragma unroll
        for (int b = 0; b < kRing; ++b) v[b] = b < B ? ring[(int64_t)b * len + j] : C{R(0), R(0)};
        // energies four at a time: four accumulator loads in flight per thread
        for (int k0 = 0; k0 < K; k0 += 4) {
            A a[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (k0 + q < K) a[q] = ac[(int64_t)(k0 + q) * len + j];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (k0 + q >= K) continue;
                R sx = R(0), sy = R(0);
#pragma unroll
                for (int b = 0; b < kRing; ++b) {
                    if (b < B) {
                        const R wr = w.re[b][k0 + q], wi = w.im[b][k0 + q];
                        sx += wr * v[b].x - wi * v[b].y;
                        sy += wr * v[b].y + wi * v[b].x;
                    }
                }
                if constexpr (kPair) {
                    float hx, ex, hy, ey;
                    two_sum(a[q].x, sx, hx, ex);
                    two_sum(a[q].y, sy, hy, ey);
                    a[q] = make_float4(hx, hy, a[q].z + ex, a[q].w + ey);
                } else {
                    a[q].x += sx;
                    a[q].y += sy;
                }
                ac[(int64_t)(k0 + q) * len + j] = a[q];
            }
        }
    }
}

// In place: (hi.re, hi.im, lo.re, lo.im) floats -> complex128 (hi + lo).
__global__ void __launch_bounds__(kThreads) k_float_pair_to_double(double2 *acc, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < n; j += (int64_t)gridDim.x * kThreads) {
        const float4 f = reinterpret_cast<const float4 *>(acc)[j];
        acc[j] = make_double2((double)f.x + (double)f.z, (double)f.y + (double)f.w);
    }
}

// spec[k] = dt sum_n (1 - cos(2 pi n / N)) chi_n exp(i E_k n dt / hbar) with
// chi_n = chi[2 n] + i chi[2 n + 1], n = 0..N; one block per energy, fixed-order sums.
__global__ void __launch_bounds__(kThreads) k_spectrum(const double *chi, int64_t N, double dt, double hbar,
                                                       const double *E, double *spec) {
    const int k = blockIdx.x;
    const double e = E[k];
    double sr = 0.0, si = 0.0;
    for (int64_t n = threadIdx.x; n <= N; n += kThreads) {
        const double t = (double)n * dt;
        const double w = 1.0 - cospi(2.0 * (double)n / (double)N);
        double sn, cn;
        sincos(t * e / hbar, &sn, &cn);
        const double cr = chi[2 * n], ci = chi[2 * n + 1];
        sr += w * (cr * cn - ci * sn);
        si += w * (cr * sn + ci * cn);
    }
    __shared__ double ws[2][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    sr = warp_sum(sr);
    si = warp_sum(si);
    if (lane == 0) {
        ws[0][wid] = sr;
        ws[1][wid] = si;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) {
            a += ws[0][i];
            b += ws[1][i];
        }
        spec[2 * k] = dt * a;
        spec[2 * k + 1] = dt * b;
    }
}

// g_j = 2 Re(z acc_j) with z = conj(c) k_V dV given as (zr, zi); acc as
// k_accum left it (float pairs for complex64 states).
template <bool kPair>
__global__ void __launch_bounds__(kThreads) k_grad_v(const double2 *acc, int64_t npts, double zr, double zi, double *g) {
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < npts; j += (int64_t)gridDim.x * kThreads) {
        double sx, sy;
        if constexpr (kPair) {
            const float4 f = reinterpret_cast<const float4 *>(acc)[j];
            sx = (double)f.x + (double)f.z;
            sy = (double)f.y + (double)f.w;
        } else {
            sx = acc[j].x;
            sy = acc[j].y;
        }
        g[j] = 2.0 * (zr * sx - zi * sy);
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

constexpr int kSegMax = 64;   // slots per k_seg_reduce launch (shared memory: 512 B per slot)

int seg_partials(int count) { return (count < kSegMax ? count : kSegMax) * kSegGrid * kVals; }

cudaError_t launch_seg_reduce(const void *lam, const void *psi, bool f64, int count, int64_t m0, int ndim,
                              const int64_t *dims, const double *h, double dV, double *acc, double *partial,
                              double *out, cudaStream_t s) {
    InnerGeom g{};
    g.ndim = ndim;
    int64_t npts = 1;
    for (int ax = 0; ax < 3; ++ax) {
        g.dims[ax] = ax < ndim ? dims[ax] : 1;
        g.h[ax] = ax < ndim ? h[ax] : 0.0;
        g.x0[ax] = ax < ndim ? -0.5 * (double)dims[ax] * h[ax] : 0.0;
        npts *= g.dims[ax];
    }
    double2 *ac = reinterpret_cast<double2 *>(acc);
    const int64_t chunks = (npts + (int64_t)kThreads * kSegPts - 1) / ((int64_t)kThreads * kSegPts);
    const int nb = (int)(chunks < kSegGrid ? chunks : kSegGrid);
    for (int k0 = 0; k0 < count; k0 += kSegMax) {
        const int c = count - k0 < kSegMax ? count - k0 : kSegMax;
        const size_t smem = (size_t)(kThreads / 32) * c * kVals * sizeof(double);
        if (f64)
            k_seg_reduce<double2><<<nb, kThreads, smem, s>>>(static_cast<const double2 *>(lam) + k0 * npts,
                                                             static_cast<const double2 *>(psi) + k0 * npts, npts, c,
                                                             m0 + k0, g, ac, partial);
        else
            k_seg_reduce<float2><<<nb, kThreads, smem, s>>>(static_cast<const float2 *>(lam) + k0 * npts,
                                                            static_cast<const float2 *>(psi) + k0 * npts, npts, c,
                                                            m0 + k0, g, ac, partial);
        k_seg_final<<<c, 32 * kVals, 0, s>>>(partial, nb, dV, out, m0 + k0);
    }
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

cudaError_t launch_spectral_sample(const void *psi0, const void *psi, bool f64, int64_t len, void *slot, double dV,
                                   double *partial, unsigned *done, double *chi, cudaStream_t s) {
    if (f64)
        k_spectral_sample<double2><<<kSampleBlocks, kThreads, 0, s>>>(
            static_cast<const double2 *>(psi0), static_cast<const double2 *>(psi), len, static_cast<double2 *>(slot),
            partial, done, dV, chi);
    else
        k_spectral_sample<float2><<<kSampleBlocks, kThreads, 0, s>>>(
            static_cast<const float2 *>(psi0), static_cast<const float2 *>(psi), len, static_cast<float2 *>(slot),
            partial, done, dV, chi);
    return cudaGetLastError();
}

template <typename C>
static cudaError_t spectral_accum_t(const void *ring, int B, int64_t len, int K, const double *wre, const double *wim,
                                   double *acc, cudaStream_t s) {
    using R = decltype(C{}.x);
    RingWeights<R> w{};
    for (int b = 0; b < B; ++b)
        for (int k = 0; k < K; ++k) {
            w.re[b][k] = (R)wre[b * K + k];
            w.im[b][k] = (R)wim[b * K + k];
        }
    k_spectral_accum<C><<<kSampleBlocks, kThreads, 0, s>>>(static_cast<const C *>(ring), B, len, K, w,
                                                            reinterpret_cast<double2 *>(acc));
    return cudaGetLastError();
}

cudaError_t launch_spectral_accum(const void *ring, bool f64, int B, int64_t len, int K, const double *wre,
                                  const double *wim, double *acc, cudaStream_t s) {
    if (B < 1 || B > kRing || K < 1 || K > kMaxEnergies) return cudaErrorInvalidValue;
    return f64 ? spectral_accum_t<double2>(ring, B, len, K, wre, wim, acc, s)
               : spectral_accum_t<float2>(ring, B, len, K, wre, wim, acc, s);
}

cudaError_t launch_spectral_finish(double *acc, bool f64, int64_t n, cudaStream_t s) {
    if (f64) return cudaSuccess;
    k_float_pair_to_double<<<kSampleBlocks, kThreads, 0, s>>>(reinterpret_cast<double2 *>(acc), n);
    return cudaGetLastError();
}

cudaError_t launch_spectrum(const double *chi, int64_t N, double dt, double hbar, const double *E, int K,
                            double *spec, cudaStream_t s) {
    if (K <= 0) return cudaSuccess;
    k_spectrum<<<K, kThreads, 0, s>>>(chi, N, dt, hbar, E, spec);
    return cudaGetLastError();
}

cudaError_t launch_grad_v(const double *acc, bool f64, int64_t npts, double zr, double zi, double *g,
                          cudaStream_t s) {
    const double2 *ac = reinterpret_cast<const double2 *>(acc);
    if (f64)
        k_grad_v<false><<<kBlocks * 4, kThreads, 0, s>>>(ac, npts, zr, zi, g);
    else
        k_grad_v<true><<<kBlocks * 4, kThreads, 0, s>>>(ac, npts, zr, zi, g);
    return cudaGetLastError();
}

}  // namespace sop
