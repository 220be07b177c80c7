// sop_kernels.cuh -- fused split-operator pencil passes for sm_103a.
//
// Each pass streams psi through HBM once along one axis: it loads whole
// pencils (coalesced), optionally transforms them, applies a pointwise factor
// of the split step, optionally transforms again and stores in place:
//   real-space axis (x):  [inverse FFT_x] -> U_A1 -> [forward FFT_x]
//   last axis:            forward FFT -> U~_A2 and 1/N -> inverse FFT
//   middle axis (3D):     forward or inverse FFT only
// (Bauke & Keitel, arXiv:1012.3911, Eq. 8; the FFTs are separable per axis,
// Sec. 2.1).  A d-dimensional step therefore costs one HBM round trip per
// pass and adjacent real-space half factors are merged into one pass.
#pragma once

#include <type_traits>

#include "sop_dirac4.cuh"
#include "sop_fft.cuh"
#include "sop_internal.h"

namespace sop {

// Phase factors in the working precision.  FP32 stores z = w - 1 ("z-form")
// and applies psi + z psi, so a factor close to 1 keeps its full relative
// precision and its rounding error does not recur as a systematic modulus
// error every step; FP64 stores and multiplies w itself.
template <typename Real> struct Phase;
template <> struct Phase<float> {
    using C = float2;
    __device__ __forceinline__ static C one() { return mk<C>(0.f, 0.f); }
    __device__ __forceinline__ static C combine(C a, C b) {   // (1+a)(1+b) - 1 = a + b + ab
        return mk<C>(fmar(a.x, b.x, fmar(-a.y, b.y, a.x + b.x)), fmar(a.x, b.y, fmar(a.y, b.x, a.y + b.y)));
    }
    __device__ __forceinline__ static C apply(C psi, C z) {
        return mk<C>(fmar(z.x, psi.x, fmar(-z.y, psi.y, psi.x)), fmar(z.x, psi.y, fmar(z.y, psi.x, psi.y)));
    }
};
template <> struct Phase<double> {
    using C = double2;
    __device__ __forceinline__ static C one() { return mk<C>(1.0, 0.0); }
    __device__ __forceinline__ static C combine(C a, C b) { return cmul(a, b); }
    __device__ __forceinline__ static C apply(C psi, C w) { return cmul(psi, w); }
};

// psi * (hi + lo): 1/N with N = 2^a 3^b carried as an unevaluated sum so the
// factor has no systematic rounding bias in FP32.
template <typename C, typename R> __device__ __forceinline__ C scale2(C a, R hi, R lo) {
    return mk<C>(fmar(a.x, hi, a.x * lo), fmar(a.y, hi, a.y * lo));
}

// ---------------------------------------------------------------------------
// Launch geometry
// ---------------------------------------------------------------------------

template <typename Real, int N, int NC, bool CONTIG> struct PassCfg {
    using G = Geometry<N, NC>;
    static constexpr int E = G::E;
    static constexpr int T = G::T;
    static constexpr int CSZ = 2 * (int)sizeof(Real);
    static constexpr int wp_contig() {
        int w = 256 / T;
        return w < 1 ? 1 : w;
    }
    static constexpr int wp_strided() {
        int w = 128 / CSZ;                         // 128-byte row segments
        while (w > 1 && (long)w * T > 512) w /= 2; // at most 512 threads
        while (w > 1 && (long)w * NC * N * CSZ > 96 * 1024) w /= 2;
        return w;
    }
    static constexpr int WP = CONTIG ? wp_contig() : wp_strided();
    static constexpr int THREADS = T * WP;
    static constexpr int PITCH = N + (N >> G::LR);
    static constexpr int ROWLINES = (128 / (WP * CSZ)) < 1 ? 1 : 128 / (WP * CSZ);  // rows per bank line
    static constexpr int LM = ROWLINES - 1;
    static constexpr int SH = G::LR > ilog2c(ROWLINES) ? G::LR : ilog2c(ROWLINES);
    static constexpr bool NEEDS_SMEM = G::P.S > 1;
    static constexpr size_t SMEM = !NEEDS_SMEM ? 0
                                   : CONTIG ? (size_t)WP * NC * PITCH * CSZ
                                            : (size_t)NC * N * WP * CSZ;
    static_assert(THREADS <= 1024, "block too large");
};

// ---------------------------------------------------------------------------
// Pointwise factors
// ---------------------------------------------------------------------------

// Lattice coordinates (ix, iy, iz) of linear point index lin.
__device__ __forceinline__ void unravel3(int64_t lin, const int64_t *dims, int ndim, int *co) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        co[a] = 0;
        if (a < ndim) {
            co[a] = (int)(lin % dims[a]);
            lin /= dims[a];
        }
    }
}

// Pointwise factor of a pass on the E values per component a thread holds
// (axis index i = t + T m of the pencil starting at linear point index base).
// vrow/vstride: the per-point phase values of this pencil (global or shared
// memory), or null.  pz: component pair (nc == 2).
// Loads and stores that bypass L1 but keep the normal L2 policy: psi and the
// per-point tables stream through each pass once and must not push the
// twiddle and field tables out of L1, while psi should stay in L2 for the
// next pass.
// Check builds (-DSOP_CHECK=1): SOP_IN(flag, cond) is cond, and a false cond
// sets bit 2 of the error word at flag so the caller can skip the access; in
// normal builds it is the constant true and cond is not evaluated.
#ifndef SOP_CHECK
#define SOP_CHECK 0
#endif
__device__ __forceinline__ bool sop_in(int *flag, bool cond) {
    if (!cond && flag) atomicOr(flag, 4);
    return cond;
}
#if SOP_CHECK
#define SOP_IN(flag, cond) sop_in((flag), (cond))
#else
#define SOP_IN(flag, cond) true
#endif

template <typename C> __device__ __forceinline__ C ld_stream(const C *p) { return __ldcg(p); }
template <typename C> __device__ __forceinline__ void st_stream(C *p, C v) { __stcg(p, v); }

// VGLOBAL: vrow points to global memory (read with ld_stream); otherwise it
// points to shared memory.
template <typename Real, int E, int T, int NC, bool VGLOBAL = false>
__device__ __forceinline__ void apply_op(cplx_t<Real> (&v)[NC][E], const PassArgs &a, int64_t base, int64_t stride,
                                         int t, int pz, const cplx_t<Real> *vrow, int64_t vstride) {
    using C = cplx_t<Real>;
    using Ph = Phase<Real>;
    if constexpr (NC == 1) {
        if (a.op == OP_V || a.op == OP_T) {
            // Pencil-constant part: factors of the axes other than this one.
            const bool is_v = a.op == OP_V;
            const C *tab[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) tab[ax] = reinterpret_cast<const C *>(is_v ? a.ftab[ax] : a.ttab[ax]);
            int co[3];
            unravel3(base, a.dims, a.ndim, co);
            C g = Ph::one();
#pragma unroll
            for (int ax = 0; ax < 3; ++ax)
                if (ax < a.ndim && ax != a.axis && tab[ax] != nullptr) g = Ph::combine(g, ldg_c(tab[ax] + co[ax]));
            const C *ta = a.axis == 0 ? tab[0] : (a.axis == 1 ? tab[1] : tab[2]);
            const C *vt = vrow;
            const Real shi = Real(a.scale_hi), slo = Real(a.scale_lo);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int i = t + T * m;
                C f = g;
                if (ta != nullptr) f = Ph::combine(ldg_c(ta + i), f);
                if (is_v) {
                    if (vt != nullptr) {
                        const C vv = VGLOBAL ? ld_stream(vt + (int64_t)i * vstride) : vt[(int64_t)i * vstride];
                        f = Ph::combine(vv, f);
                    }
                    v[0][m] = Ph::apply(v[0][m], f);
                } else {
                    v[0][m] = scale2(Ph::apply(v[0][m], f), shi, slo);
                }
            }
        }
    } else {
        if (a.op == OP_DV) {
            // (psi_a, psi_b) <- exp(-i V tau') M (psi_a, psi_b), M the 2x2 block of
            // the spinor-mixing factor on this component pair.
            const double *mx = a.mix[pz];
            const C m00 = mk<C>(Real(mx[0]), Real(mx[1])), m01 = mk<C>(Real(mx[2]), Real(mx[3]));
            const C m10 = mk<C>(Real(mx[4]), Real(mx[5])), m11 = mk<C>(Real(mx[6]), Real(mx[7]));
            const C *vt = vrow;
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int i = t + T * m;
                C u0 = cadd(cmul(m00, v[0][m]), cmul(m01, v[1][m]));
                C u1 = cadd(cmul(m10, v[0][m]), cmul(m11, v[1][m]));
                if (vt != nullptr) {
                    const C f = VGLOBAL ? ld_stream(vt + (int64_t)i * vstride) : vt[(int64_t)i * vstride];
                    u0 = Ph::apply(u0, f);
                    u1 = Ph::apply(u1, f);
                }
                v[0][m] = u0;
                v[1][m] = u1;
            }
        } else if (a.op == OP_DT) {
            // U = cos(th) - i sin(th) H/E on the pair, H/E = [[mu, k],[k*, -mu]] with
            // k = kappa* on pair (1,4) and k = kappa on pair (2,3), kappa = c(p_x + i p_y)/E;
            // table entry q = (cos th, sin th mu, sin th c p_x/E, sin th c p_y/E).
            const C *dt2 = reinterpret_cast<const C *>(a.dtab);
            const Real sgn = pz == 0 ? Real(1) : Real(-1);
            const Real shi = Real(a.scale_hi), slo = Real(a.scale_lo);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int i = t + T * m;
                const int64_t k = base + (int64_t)i * stride;
                C q0, q1;
                if (!SOP_IN(a.errflag, k >= 0 && k < a.comp_stride)) continue;
                if constexpr (sizeof(Real) == 4) {
                    const float4 q = __ldcg(reinterpret_cast<const float4 *>(dt2) + k);
                    q0 = mk<C>(q.x, q.y);
                    q1 = mk<C>(q.z, q.w);
                } else {
                    q0 = ld_stream(dt2 + 2 * k);
                    q1 = ld_stream(dt2 + 2 * k + 1);
                }
                const C u00 = mk<C>(q0.x, -q0.y), u11 = mk<C>(q0.x, q0.y);
                const C u01 = mk<C>(-sgn * q1.y, -q1.x), u10 = mk<C>(sgn * q1.y, -q1.x);
                const C r0 = cadd(cmul(u00, v[0][m]), cmul(u01, v[1][m]));
                const C r1 = cadd(cmul(u10, v[0][m]), cmul(u11, v[1][m]));
                v[0][m] = scale2(r0, shi, slo);
                v[1][m] = scale2(r1, shi, slo);
            }
        }
    }
}

// The four-component factors of the 3D Dirac step on the E values per
// component a thread holds (axis index i = t + T m of the pencil at linear
// point index base; stride along the axis).  OP_D3V runs on the contiguous
// x pass: vrow are the pencil's phase values (global, or null) and a.rows4
// the per-column mixing rows indexed by x = i.  OP_D3T reads the
// per-momentum table a.dtab at base + i stride.
template <typename Real, int E, int T>
__device__ __forceinline__ void apply_op4(cplx_t<Real> (&v)[4][E], const PassArgs &a, int64_t base, int64_t stride,
                                          int t, const cplx_t<Real> *vrow) {
    using C = cplx_t<Real>;
    using Ph = Phase<Real>;
    if (a.op == OP_D3V) {
        const Real *rows = reinterpret_cast<const Real *>(a.rows4);
        C M[16];
        if (!rows) {
#pragma unroll
            for (int q = 0; q < 16; ++q) M[q] = mk<C>(Real(a.mix4[2 * q]), Real(a.mix4[2 * q + 1]));
        }
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int i = t + T * m;
            const C x[4] = {v[0][m], v[1][m], v[2][m], v[3][m]};
            C w[4];
            if (rows) {
                Real q[8];
                dirac4_load_row(rows + (int64_t)i * 8, q);
                dirac4_mix_compact(q, x, w);
            } else {
                dirac4_mix(M, x, w);
            }
            if (vrow) {
                const C f = ld_stream(vrow + i);
#pragma unroll
                for (int c = 0; c < 4; ++c) w[c] = Ph::apply(w[c], f);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c][m] = w[c];
        }
    } else if (a.op == OP_D3T) {
        const Real *tab = reinterpret_cast<const Real *>(a.dtab);
        const Real shi = Real(a.scale_hi), slo = Real(a.scale_lo);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int64_t k = base + (int64_t)(t + T * m) * stride;
            if (!SOP_IN(a.errflag, k >= 0 && k < a.comp_stride)) continue;
            Real co, sm, sx, sy, sz;
            dirac4_load_kin(tab, k, co, sm, sx, sy, sz);
            const C x[4] = {v[0][m], v[1][m], v[2][m], v[3][m]};
            C r[4];
            dirac4_kinetic(co, sm, sx, sy, sz, x, r);
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c][m] = scale2(r[c], shi, slo);
        }
    }
}

// ---------------------------------------------------------------------------
// The pass kernel
// ---------------------------------------------------------------------------

template <typename Real, int N, int NC, bool CONTIG>
__global__ void __launch_bounds__(PassCfg<Real, N, NC, CONTIG>::THREADS)
    pass_kernel(const __grid_constant__ PassArgs a) {
    using C = cplx_t<Real>;
    using Cfg = PassCfg<Real, N, NC, CONTIG>;
    using Ph = Phase<Real>;
    constexpr int E = Cfg::E, T = Cfg::T, WP = Cfg::WP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);

    const int t = CONTIG ? threadIdx.x : threadIdx.y;   // thread within the pencil
    const int w = CONTIG ? threadIdx.y : threadIdx.x;   // pencil within the CTA
    const int64_t stride = CONTIG ? 1 : a.stride;

    // Pencil and component offsets.  NC == 1: the batch index (e.g. the
    // component of a spinor transformed as independent fields) is folded into
    // the pencil index.  NC == 2: blockIdx.z selects a coupled component pair.
    const int64_t per_batch = a.n_pencils;
    const int64_t total = (NC == 1) ? per_batch * a.n_batch : per_batch;
    const int64_t pg = (int64_t)blockIdx.x * WP + w;
    const bool active = pg < total;
    const int64_t pc = active ? pg : 0;
    int64_t bidx = 0, p = pc;
    if (NC == 1) {
        bidx = pc / per_batch;
        p = pc - bidx * per_batch;
    }
    const int64_t base = CONTIG ? p * N : (p / stride) * stride * N + (p % stride);
    int64_t coff[NC];
    if constexpr (NC == 1) {
        coff[0] = bidx * a.comp_stride;
    } else {
        coff[0] = (int64_t)a.pair_comp[blockIdx.z][0] * a.comp_stride;
        coff[1] = (int64_t)a.pair_comp[blockIdx.z][1] * a.comp_stride;
    }
    C *psi = reinterpret_cast<C *>(a.psi);
    const C *tw = reinterpret_cast<const C *>(a.tw);

    C v[NC][E];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int m = 0; m < E; ++m)
            v[c][m] = active ? ld_stream(psi + coff[c] + base + (int64_t)(t + T * m) * stride) : mk<C>(Real(0), Real(0));

    // Exchange layouts, one per component.
    using LayC = LayContig<C, Cfg::G::LR>;
    using LayS = LayStrided<C, WP, Cfg::SH, Cfg::LM>;
    using Lay = typename std::conditional<CONTIG, LayC, LayS>::type;
    Lay lay[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        if constexpr (CONTIG) lay[c].p = sm + (w * NC + c) * Cfg::PITCH;
        else lay[c].p = sm + c * N * WP + w;
    }

    if (a.pre != 0) fft_dir<C, N, E, NC>(v, lay, t, tw, a.pre);

    apply_op<Real, E, T, NC, true>(v, a, base, stride, t, blockIdx.z, reinterpret_cast<const cplx_t<Real> *>(a.vtab) + (a.vtab ? base : 0), stride);

    if (a.post != 0) {
        if (a.pre != 0) __syncthreads();   // the exchange buffer is reused
        fft_dir<C, N, E, NC>(v, lay, t, tw, a.post);
    }

    if (active) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int m = 0; m < E; ++m) st_stream(psi + coff[c] + base + (int64_t)(t + T * m) * stride, v[c][m]);
    }
}

// ---------------------------------------------------------------------------
// One-dimensional whole-step kernel: a CTA keeps one lattice line on chip for
// a run of steps, so in 1D a step costs no HBM traffic at all.
//   for each real-space index P in [p_begin, p_end):
//     psi <- U_A1 psi  (half factor for P = 0 and P = n_steps, merged otherwise)
//     if P < n_steps:  psi <- F^-1 (U~_A2 / N) F psi
// ---------------------------------------------------------------------------

template <typename Real, int N>
__global__ void __launch_bounds__(Geometry<N, 1>::T) fso1d_kernel(const __grid_constant__ Args1D a) {
    using C = cplx_t<Real>;
    using G = Geometry<N, 1>;
    using Ph = Phase<Real>;
    constexpr int E = G::E, T = G::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    const int t = threadIdx.x;
    const int64_t row = blockIdx.x;
    C *psi = reinterpret_cast<C *>(a.psi) + row * N;
    const C *tw = reinterpret_cast<const C *>(a.tw);
    const C *vh = reinterpret_cast<const C *>(a.vhalf);
    const C *vf = reinterpret_cast<const C *>(a.vfull);
    const C *ft = reinterpret_cast<const C *>(a.ftab);
    const C *tt = reinterpret_cast<const C *>(a.ttab);
    const Real shi = Real(a.scale_hi), slo = Real(a.scale_lo);

    C v[1][E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[0][m] = psi[t + T * m];
    LayContig<C, G::LR> lay[1];
    lay[0].p = sm;

    for (int64_t P = a.p_begin; P < a.p_end; ++P) {
        const C *vt = (P == 0 || P == a.n_steps) ? vh : vf;
        const C *fr = ft ? ft + (P - a.p_table0) * N : nullptr;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int i = t + T * m;
            C f = Ph::one();
            if (fr != nullptr) f = ldg_c(fr + i);
            if (vt != nullptr) f = Ph::combine(ldg_c(vt + i), f);
            v[0][m] = Ph::apply(v[0][m], f);
        }
        if (P < a.n_steps) {
            fft_forward<C, N, E, 1>(v, lay, t, tw);
            const C *tr = tt + (P - a.p_table0) * a.ttab_stride;
#pragma unroll
            for (int m = 0; m < E; ++m) v[0][m] = scale2(Ph::apply(v[0][m], ldg_c(tr + t + T * m)), shi, slo);
            __syncthreads();
            fft_dir<C, N, E, 1>(v, lay, t, tw, +1);
            __syncthreads();
        }
    }
#pragma unroll
    for (int m = 0; m < E; ++m) psi[t + T * m] = v[0][m];
}

// One-dimensional two-component Dirac equation (end of Sec. 2.3), whole
// steps on chip: one CTA holds both components of a line in registers.  Per
// real-space index P: psi <- exp(-i V tau') M_P psi (M_P the merged 2x2
// mixing of the two adjacent half steps, uniform along the line), then, for
// P < n_steps, FFT, the per-momentum factor
//   U = cos(E tau) - i sin(E tau) (c p sigma_x + m c^2 sigma_z) / E
// (equal to u^dagger diag(e^{-iE tau}, e^{iE tau}) u) with 1/N, inverse FFT.
template <typename Real, int N>
__global__ void __launch_bounds__(Geometry<N, 2>::T) fso1d_dirac_kernel(const __grid_constant__ Args1D a) {
    using C = cplx_t<Real>;
    using G = Geometry<N, 2>;
    using Ph = Phase<Real>;
    constexpr int E = G::E, T = G::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    const int t = threadIdx.x;
    C *psi = reinterpret_cast<C *>(a.psi) + blockIdx.x * (int64_t)(2 * N);
    const C *tw = reinterpret_cast<const C *>(a.tw);
    const C *vh = reinterpret_cast<const C *>(a.vhalf);
    const C *vf = reinterpret_cast<const C *>(a.vfull);
    const C *mt = reinterpret_cast<const C *>(a.mtab);
    const C *dt2 = reinterpret_cast<const C *>(a.dtab);
    const Real shi = Real(a.scale_hi), slo = Real(a.scale_lo);

    C v[2][E];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int m = 0; m < E; ++m) v[c][m] = psi[c * N + t + T * m];
    LayContig<C, G::LR> lay[2];
    lay[0].p = sm;
    lay[1].p = sm + (N + (N >> G::LR));

    for (int64_t P = a.p_begin; P < a.p_end; ++P) {
        const C *vt = (P == 0 || P == a.n_steps) ? vh : vf;
        const C *mr = mt + (P - a.p_table0) * 4;
        const C m00 = ldg_c(mr), m01 = ldg_c(mr + 1), m10 = ldg_c(mr + 2), m11 = ldg_c(mr + 3);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            C u0 = cadd(cmul(m00, v[0][m]), cmul(m01, v[1][m]));
            C u1 = cadd(cmul(m10, v[0][m]), cmul(m11, v[1][m]));
            if (vt != nullptr) {
                const C f = ldg_c(vt + t + T * m);
                u0 = Ph::apply(u0, f);
                u1 = Ph::apply(u1, f);
            }
            v[0][m] = u0;
            v[1][m] = u1;
        }
        if (P < a.n_steps) {
            fft_forward<C, N, E, 2>(v, lay, t, tw);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int k = t + T * m;
                C q0, q1;
                if constexpr (sizeof(Real) == 4) {
                    const float4 q = __ldg(reinterpret_cast<const float4 *>(dt2) + k);
                    q0 = mk<C>(q.x, q.y);
                    q1 = mk<C>(q.z, q.w);
                } else {
                    q0 = ldg_c(dt2 + 2 * k);
                    q1 = ldg_c(dt2 + 2 * k + 1);
                }
                // q0 = (cos, sin mc^2/E), q1.x = sin c p / E
                const C u00 = mk<C>(q0.x, -q0.y), u11 = mk<C>(q0.x, q0.y), u01 = mk<C>(Real(0), -q1.x);
                const C r0 = cadd(cmul(u00, v[0][m]), cmul(u01, v[1][m]));
                const C r1 = cadd(cmul(u01, v[0][m]), cmul(u11, v[1][m]));
                v[0][m] = scale2(r0, shi, slo);
                v[1][m] = scale2(r1, shi, slo);
            }
            __syncthreads();
            fft_dir<C, N, E, 2>(v, lay, t, tw, +1);
            __syncthreads();
        }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int m = 0; m < E; ++m) psi[c * N + t + T * m] = v[c][m];
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------

// Opt a kernel into more than 48 KB of dynamic shared memory once per device.
cudaError_t ensure_smem_attr(const void *kern, int bytes);

template <typename Real, int N, int NC, bool CONTIG>
cudaError_t launch_pass_t(const PassArgs &a, cudaStream_t s) {
    using Cfg = PassCfg<Real, N, NC, CONTIG>;
    auto kern = pass_kernel<Real, N, NC, CONTIG>;
    if (Cfg::SMEM > 48 * 1024) {
        cudaError_t e = ensure_smem_attr(reinterpret_cast<const void *>(kern), (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
    }
    const int64_t total = (NC == 1) ? a.n_pencils * a.n_batch : a.n_pencils;
    const int64_t blocks = (total + Cfg::WP - 1) / Cfg::WP;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 grid((unsigned)blocks, 1, NC == 2 ? 2 : 1);
    dim3 block = CONTIG ? dim3(Cfg::T, Cfg::WP, 1) : dim3(Cfg::WP, Cfg::T, 1);
    kern<<<grid, block, Cfg::SMEM, s>>>(a);
    return cudaGetLastError();
}

template <typename Real, int N> cudaError_t launch_1d_dirac_t(const Args1D &a, cudaStream_t s) {
    using G = Geometry<N, 2>;
    constexpr size_t SMEM = G::P.S > 1 ? (size_t)(N + (N >> G::LR)) * 2 * 2 * sizeof(Real) : 0;
    auto kern = fso1d_dirac_kernel<Real, N>;
    if (SMEM > 48 * 1024) {
        cudaError_t e = ensure_smem_attr(reinterpret_cast<const void *>(kern), (int)SMEM);
        if (e != cudaSuccess) return e;
    }
    if (a.n_rows <= 0) return cudaSuccess;
    kern<<<(unsigned)a.n_rows, G::T, SMEM, s>>>(a);
    return cudaGetLastError();
}

template <typename Real, int N> cudaError_t launch_1d_t(const Args1D &a, cudaStream_t s) {
    using G = Geometry<N, 1>;
    constexpr size_t SMEM = G::P.S > 1 ? (size_t)(N + (N >> G::LR)) * 2 * sizeof(Real) : 0;
    auto kern = fso1d_kernel<Real, N>;
    if (SMEM > 48 * 1024) {
        cudaError_t e = ensure_smem_attr(reinterpret_cast<const void *>(kern), (int)SMEM);
        if (e != cudaSuccess) return e;
    }
    if (a.n_rows <= 0) return cudaSuccess;
    kern<<<(unsigned)a.n_rows, G::T, SMEM, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sop
