// sop_fft.cuh -- in-register / shared-memory Stockham FFT engine for sm_103a.
//
// Sec. 2.1 of Bauke & Keitel (arXiv:1012.3911): on a lattice of N points the
// Fourier transforms of the split step become DFTs, X_k = sum_j x_j
// exp(-2 pi i jk/n) per axis, computed here by mixed-radix FFTs.
//
// Design (one pencil of n points, one CTA-resident exchange buffer):
//  * T = n/E threads per pencil, each holding E complex values in registers.
//    Thread t always holds the elements t + T*m, m = 0..E-1, of the current
//    stage's input ("natural mapping"); global loads/stores in this mapping
//    are coalesced along t.
//  * Stage s (radix R, Ns = product of the earlier radices) is the Stockham
//    autosort step: butterfly j (j < n/R) reads x[j + r n/R], multiplies
//    input r by W_{Ns R}^{(j mod Ns) r}, does an R-point DFT in registers and
//    writes output r to y[(j div Ns) Ns R + (j mod Ns) + r Ns].  With
//    j = t + T q the inputs of thread t are exactly its registers
//    q + r (E/R), so only the outputs go through shared memory; the last
//    stage's outputs land back in the natural mapping without an exchange.
//  * The inverse transform is conj(F(conj(x))): only the forward code is
//    compiled.
//  * Stage twiddles come from a per-size table W_n^e, e < n, formed in FP64
//    on the device (FP32 keeps z = w - 1, see tw_apply); each thread loads only
//    its R-1 distinct twiddles per stage (StageTw).  Constants inside the
//    radix-3/4/8/16 butterflies and the compile-time roots that complete the
//    stage twiddles are applied as hi + lo in FP32 (kmul, rot48), so no
//    rounded constant biases the modulus of a transform.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace sop {

template <typename R> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename R> using cplx_t = typename CplxOf<R>::type;

__device__ __forceinline__ float fmar(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename C> __device__ __forceinline__ C mk(decltype(C::x) re, decltype(C::x) im) {
    C r;
    r.x = re;
    r.y = im;
    return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
// Complex64 sums and differences as one paired FP32 instruction (the
// .f32x2 forms of sm_100 and later): both lanes round to nearest like two
// scalar adds, so results are bit-identical, at half the issue slots of the
// butterflies' additions.
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "add.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return mk<C>(fmar(a.x, b.x, -(a.y * b.y)), fmar(a.x, b.y, a.y * b.x));
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C mul_mi(C a) { return mk<C>(a.y, -a.x); }  // a * (-i)
template <typename C> __device__ __forceinline__ C mul_pi(C a) { return mk<C>(-a.y, a.x); }  // a * (+i)
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }

// Butterfly constants.  In FP32 every non-trivial constant is applied as an
// unevaluated sum hi + lo (x*c = fma(x, hi, x*lo)): a rounded constant alone
// would give each twiddle a modulus |w| != 1 with a fixed sign, and a
// decimation-in-time combine e +- w o changes the norm by 2(|w|^2 - 1)|o|^2,
// which then recurs identically in every transform of every step.  With the
// pair the constant is exact to ~2^-48 and only the unbiased rounding of the
// data remains.  FP64 uses the constants directly.
enum KId { K_C1 = 0, K_S1 = 1, K_R2 = 2, K_R3 = 3 };
template <int ID> struct KVal;
template <> struct KVal<K_C1> { static constexpr double v = 0.92387953251128675612818318939678828682; };  // cos(pi/8)
template <> struct KVal<K_S1> { static constexpr double v = 0.38268343236508977172845998403039886676; };  // sin(pi/8)
template <> struct KVal<K_R2> { static constexpr double v = 0.70710678118654752440084436210484903928; };  // cos(pi/4)
template <> struct KVal<K_R3> { static constexpr double v = 0.86602540378443864676372317075293618347; };  // sin(pi/3)

template <int ID> __device__ __forceinline__ float kmul(float x) {
    constexpr float hi = (float)KVal<ID>::v;
    constexpr float lo = (float)(KVal<ID>::v - (double)hi);
    return fmar(x, hi, x * lo);
}
template <int ID> __device__ __forceinline__ double kmul(double x) { return x * KVal<ID>::v; }

// a*c_A + b*c_B
template <int A, int B> __device__ __forceinline__ float kdot(float a, float b) {
    constexpr float ah = (float)KVal<A>::v, al = (float)(KVal<A>::v - (double)ah);
    constexpr float bh = (float)KVal<B>::v, bl = (float)(KVal<B>::v - (double)bh);
    return fmar(a, ah, fmar(b, bh, fmar(a, al, b * bl)));
}
template <int A, int B> __device__ __forceinline__ double kdot(double a, double b) {
    return fmar(a, KVal<A>::v, b * KVal<B>::v);
}

// Stage twiddles.  FP32 stores z = w - 1 of w = exp(-2 pi i e/n) (formed in
// FP64, rounded once) and applies x + z x: the same four FMAs as a complex
// product, but twiddles near 1 -- the ones a smooth field's energy flows
// through -- keep their full relative precision, so their rounding does not
// bias the norm.  FP64 stores and multiplies w.
__device__ __forceinline__ float2 tw_apply(float2 x, float2 z) {
    return mk<float2>(fmar(z.x, x.x, fmar(-z.y, x.y, x.x)), fmar(z.x, x.y, fmar(z.y, x.x, x.y)));
}
__device__ __forceinline__ double2 tw_apply(double2 x, double2 w) { return cmul(x, w); }

// cos(2 pi j / 48) for any integer j (first-quadrant decimal expansions and
// symmetry); used only in constant expressions.
__host__ __device__ constexpr double cos48(int j) {
    const double q[13] = {1.0,
                          0.99144486137381041114455752692856287128,
                          0.96592582628906828674974319972889736763,
                          0.92387953251128675612818318939678828682,
                          0.86602540378443864676372317075293618347,
                          0.79335334029123516457977696150129927663,
                          0.70710678118654752440084436210484903928,
                          0.60876142900872063941609754289816400452,
                          0.5,
                          0.38268343236508977172845998403039886676,
                          0.25881904510252076234889883762404832835,
                          0.13052619222005159154840622789548901019,
                          0.0};
    j %= 48;
    if (j < 0) j += 48;
    if (j <= 12) return q[j];
    if (j <= 24) return -q[24 - j];
    if (j <= 36) return -q[j - 24];
    return q[48 - j];
}
__host__ __device__ constexpr double sin48(int j) { return cos48(j - 12); }

// Shear coefficients tan(pi j/48) and sin(2 pi j/48), j = 1..11.
__host__ __device__ constexpr double shear_t48(int j) {
    const double t[12] = {0.0,
                          0.065543462815238228564543724879942794922,
                          0.13165249758739585347152645740971710359,
                          0.1989123673796580069115976226446762286,
                          0.26794919243112270647255365849412763306,
                          0.33945425886337581553711890089328069302,
                          0.41421356237309504880168872420969807857,
                          0.49314542603130412392530089399243144889,
                          0.57735026918962576450914878050195745565,
                          0.66817863791929891999775768652308076155,
                          0.76732698797896034292304169200206568034,
                          0.87697646299275686724868856712992232268};
    return t[j];
}

// x * exp(-2 pi i J / 48).  The quarter turns (-i)^q are exact swaps and
// negations; the remaining angle phi = 2 pi j/48 < pi/2 is applied as three
// shears, x += t y; y -= s x; x += t y with t = tan(phi/2), s = sin(phi)
// (3 FMAs).  A shear has determinant 1 whatever its rounded coefficient, so
// the product is area-preserving exactly: a rounded constant cannot bias the
// norm to first order (a rounded cos/sin pair would, with a fixed sign, in
// every transform).
template <int J, typename C> __device__ __forceinline__ C rot48(C x) {
    using R = decltype(x.x);
    constexpr int jj = ((J % 48) + 48) % 48;
    constexpr int q = jj / 12, j = jj % 12;
    C y = x;
    if constexpr (q == 1) y = mul_mi(x);
    else if constexpr (q == 2) y = mk<C>(-x.x, -x.y);
    else if constexpr (q == 3) y = mul_pi(x);
    if constexpr (j == 0) {
        return y;
    } else {
        constexpr R t = R(shear_t48(j));
        constexpr R sn = R(sin48(j));
        R a = fmar(t, y.y, y.x);
        const R b = fmar(-sn, a, y.y);
        a = fmar(t, b, a);
        return mk<C>(a, b);
    }
}

// a * exp(-2 pi i J / 16) for the radix-2^k butterflies.
template <int J, typename C> __device__ __forceinline__ C w16(C a) { return rot48<3 * J>(a); }

// sin x and cos x for |x| <= pi/2 in constant expressions (Taylor series
// summed to 16 terms; the next term is below 1e-25 there).
__host__ __device__ constexpr double ct_sin(double x) {
    double term = x, sum = x;
    for (int k = 1; k < 16; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double ct_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 16; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
constexpr double kPiD = 3.14159265358979323846264338327950288;

// x * exp(-2 pi i J / O) for any order O that is a multiple of 4: quarter
// turns, then the remaining angle phi = 2 pi j / O < pi/2 as the three
// shears of rot48 (determinant 1 whatever the rounding of tan(phi/2) and
// sin(phi)).  Orders dividing 48 use rot48's constants.
template <int J, int O, typename C> __device__ __forceinline__ C rotq(C x) {
    if constexpr (48 % O == 0) {
        return rot48<(((J % O) + O) % O) * (48 / O)>(x);
    } else {
        static_assert(O % 4 == 0, "root order");
        using R = decltype(x.x);
        constexpr int jj = ((J % O) + O) % O;
        constexpr int q = (4 * jj) / O, j = jj - q * (O / 4);
        C y = x;
        if constexpr (q == 1) y = mul_mi(x);
        else if constexpr (q == 2) y = mk<C>(-x.x, -x.y);
        else if constexpr (q == 3) y = mul_pi(x);
        if constexpr (j == 0) {
            return y;
        } else {
            constexpr double half = kPiD * j / O;
            constexpr R t = R(ct_sin(half) / ct_cos(half));
            constexpr R sn = R(ct_sin(2.0 * half));
            R a = fmar(t, y.y, y.x);
            const R b = fmar(-sn, a, y.y);
            a = fmar(t, b, a);
            return mk<C>(a, b);
        }
    }
}

// Compile-time loop: f(std::integral_constant<int, I>) for I in [B, E).
template <int B, int E, typename F> __device__ __forceinline__ void sfor(F &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        sfor<B + 1, E>(f);
    }
}

template <int R> struct Dft;

template <int R, int K, typename C> __device__ __forceinline__ void dit_combine(C *x, const C *e, const C *o) {
    if constexpr (K < R / 2) {
        const C t = rotq<K, R>(o[K]);
        x[K] = cadd(e[K], t);
        x[K + R / 2] = csub(e[K], t);
        dit_combine<R, K + 1>(x, e, o);
    }
}

// Forward R-point DFT in registers, natural order in and out.
template <int R> struct Dft {
    template <typename C> __device__ __forceinline__ static void run(C *x) {
        if constexpr (R == 1) {
        } else if constexpr (R == 2) {
            const C a = x[0], b = x[1];
            x[0] = cadd(a, b);
            x[1] = csub(a, b);
        } else if constexpr (R == 3) {
            using T = decltype(x[0].x);
            constexpr T h = T(0.5);
            const C a = x[0];
            const C s = cadd(x[1], x[2]);
            const C d = csub(x[1], x[2]);
            x[0] = cadd(a, s);
            const C m = mk<C>(fmar(-h, s.x, a.x), fmar(-h, s.y, a.y));
            const C u = mk<C>(kmul<K_R3>(d.x), kmul<K_R3>(d.y));   // d sin(pi/3)
            x[1] = mk<C>(m.x + u.y, m.y - u.x);  // m - i u
            x[2] = mk<C>(m.x - u.y, m.y + u.x);  // m + i u
        } else {
            static_assert(R == 4 || R == 8 || R == 16 || R == 32 || R == 64, "radix");
            constexpr int H = R / 2;
            C e[H], o[H];
#pragma unroll
            for (int k = 0; k < H; ++k) {
                e[k] = x[2 * k];
                o[k] = x[2 * k + 1];
            }
            Dft<H>::run(e);
            Dft<H>::run(o);
            dit_combine<R, 0>(x, e, o);
        }
    }
};

// ---------------------------------------------------------------------------
// Compile-time stage plan
// ---------------------------------------------------------------------------

struct StagePlan {
    int S;       // number of stages
    int R[8];    // radix of each stage
    int NS[8];   // product of the radices before each stage
};

__host__ __device__ constexpr int pow2_part(int x) {
    int p = 1;
    while (x % 2 == 0) {
        x /= 2;
        p *= 2;
    }
    return p;
}

// Radices: the largest power of two dividing E while it fits, then the
// power-of-two remainder, then one radix-3 stage if 3 | n.
__host__ __device__ constexpr StagePlan make_plan(int n, int E) {
    StagePlan p{0, {0, 0, 0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0, 0, 0}};
    const bool has3 = (n % 3) == 0;
    int rem = has3 ? n / 3 : n;
    const int rmax = pow2_part(E);
    while (rem >= rmax && rem > 1) {
        p.R[p.S++] = rmax;
        rem /= rmax;
    }
    if (rem > 1) p.R[p.S++] = rem;
    if (has3) p.R[p.S++] = 3;
    int ns = 1;
    for (int s = 0; s < p.S; ++s) {
        p.NS[s] = ns;
        ns *= p.R[s];
    }
    return p;
}

__host__ __device__ constexpr int ilog2c(int x) {
    int r = 0;
    while ((1 << r) < x) ++r;
    return r;
}

// Elements per thread: 16 (scalar) or 8 (two coupled components) for powers
// of two; for n = 3*2^k, 8*3 or 4*3.  Small sizes use one thread per pencil.
template <int N, int NC, int EOV = 0> struct Geometry {
    static constexpr int E_calc() {
        if (EOV > 0) return EOV;   // an explicit choice (launch-shape variants)
        if (N % 3 == 0) {
            int base = (NC == 1) ? 8 : 4;
            const int p2 = N / 3;
            if (p2 < base) base = p2;
            return base * 3;
        }
        const int e = (NC == 1) ? 16 : 8;
        return N < e ? N : e;
    }
    static constexpr int E = E_calc();
    static constexpr int T = N / E;
    static constexpr StagePlan P = make_plan(N, E);
    static constexpr int LR = ilog2c(P.R[0] == 3 ? 2 : P.R[0]);   // log2 of the first radix
    static_assert(N % E == 0, "E must divide N");
};

// ---------------------------------------------------------------------------
// Shared-memory exchange layouts
// ---------------------------------------------------------------------------

// One pencil stored contiguously with one pad element per 2^LR elements, so
// the stride-R writes of the first stage and the unit-stride reads both map
// consecutive threads to distinct banks.
template <typename C, int LR> struct LayContig {
    C *p;
    __device__ __forceinline__ static int off(int i) { return i + (i >> LR); }
    __device__ __forceinline__ void st(int i, C v) const { p[off(i)] = v; }
    __device__ __forceinline__ C ld(int i) const { return p[off(i)]; }
};

__host__ __device__ constexpr int pad_off(int i, int lr) { return i + (i >> lr); }

// Padded rows admit immediate addressing: when every exchange index of a
// stage is one per-thread base b(t) plus a compile-time term X, and the pad
// of the sum splits as pad_off(b + X) = pad_off(b) + pad_off(X) for every
// thread t, a thread computes one base address per stage and each access
// is that base plus a constant.  The two checks below prove the split by
// enumerating all threads at compile time; where they fail the generic
// per-element address is used.
template <typename Lay> struct LayFast {
    static constexpr bool value = false;
    static constexpr int LR = 0;
};
template <typename C, int LR_> struct LayFast<LayContig<C, LR_>> {
    static constexpr bool value = true;
    static constexpr int LR = LR_;
};

// Stage S writes output r of butterfly j = t + T q to ob(j) + r NS; base
// b(t) = ob(t) when NS <= T, else t.
template <int N, int E, int S, int LR> constexpr bool write_split_ok() {
    constexpr StagePlan P = make_plan(N, E);
    const int R = P.R[S], NS = P.NS[S], T = N / E, Q = E / R;
    if (!(NS % T == 0 || T % NS == 0)) return false;
    for (int t = 0; t < T; ++t) {
        const int b = NS <= T ? (t / NS) * NS * R + t % NS : t;
        for (int q = 0; q < Q; ++q) {
            const int j = t + T * q, j0 = T * q;
            const int ob = (j / NS) * NS * R + j % NS, ob0 = (j0 / NS) * NS * R + j0 % NS;
            for (int r = 0; r < R; ++r) {
                const int i = ob + r * NS, X = ob0 + r * NS;
                if (i - b != X) return false;
                if (pad_off(i, LR) != pad_off(b, LR) + pad_off(X, LR)) return false;
            }
        }
    }
    return true;
}
// Exchange reads take element t + T m; base t.
template <int N, int E, int LR> constexpr bool read_split_ok() {
    const int T = N / E;
    for (int t = 0; t < T; ++t)
        for (int m = 0; m < E; ++m)
            if (pad_off(t + T * m, LR) != pad_off(t, LR) + pad_off(T * m, LR)) return false;
    return true;
}

// WP pencils interleaved as rows [i][w] (w fastest, matching the coalesced
// global layout of a strided axis).  When a row is shorter than 128 bytes,
// LM+1 rows share a bank line; the row index is XOR-swizzled so the
// stride-R first-stage writes of the warp spread over the line.
template <typename C, int WP, int SH, int LM> struct LayStrided {
    C *p;  // tile base + pencil column
    __device__ __forceinline__ static int off(int i) { return (i ^ ((i >> SH) & LM)) * WP; }
    __device__ __forceinline__ void st(int i, C v) const { p[off(i)] = v; }
    __device__ __forceinline__ C ld(int i) const { return p[off(i)]; }
};

template <typename C> __device__ __forceinline__ C ldg_c(const C *p) { return __ldg(p); }

// Barrier of the threads that share an exchange buffer: the whole CTA, or
// (BarGroup) the warps of one pencil, a named barrier of n threads.
struct BarCTA {
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct BarGroup {
    int id, n;   // barrier 1..15 (0 is __syncthreads), thread count (a multiple of 32)
    __device__ __forceinline__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
};

// Stage twiddles of one thread.  In stage s (radix R, Ns = product of the
// earlier radices) butterfly j = t + T q multiplies input r by
// W_{Ns R}^{(j mod Ns) r}.  Either Ns divides T, and j mod Ns = t mod Ns for
// every q, or T divides Ns, and W_{Ns R}^{(j mod Ns) r} =
// W_{Ns R}^{t r} W_{Ns R / T}^{(q mod Ns/T) r}, the second factor a root of
// unity of an order dividing E, known at compile time.  So a thread loads only
// W_{Ns R}^{(t mod Ns) r}, r = 1..R-1, per stage (fetched one stage ahead,
// before the exchange barrier, so the load latency overlaps the barrier).
template <typename C, int N, int E, int S> struct StageTw {
    static constexpr StagePlan P = make_plan(N, E);
    static constexpr int R = (S < P.S) ? P.R[S] : 2;
    static constexpr int NS = (S < P.S) ? P.NS[S] : 1;
    static constexpr int T = N / E;
    C z[R > 1 ? R - 1 : 1];
    // Twiddle source TWM & 3: 0 = the full W_n table in global memory; 1 =
    // this size's per-stage table (see StageTable) in shared memory; 2 = the
    // same per-stage table in global memory, read through L1.  TWM & 4: the
    // next stage's twiddles are fetched after the exchange instead of before
    // it (fewer registers live across the exchange).
    template <int TWM>
    __device__ __forceinline__ void load(const C *__restrict__ tab, int t);
};

// Per-stage twiddle table laid out for conflict-free shared-memory reads:
// stage s (s >= 1) holds W_{Ns R}^{k r} at off(s) + (r - 1) KS + k for
// k < KS = min(Ns, T), r = 1..R-1; thread t reads k = t mod KS.
template <typename C, int N, int E> struct StageTable {
    static constexpr StagePlan P = make_plan(N, E);
    static constexpr int T = N / E;
    static constexpr int ks(int s) { return P.NS[s] < T ? P.NS[s] : T; }
    static constexpr int off(int s) {
        int o = 0;
        for (int i = 1; i < s; ++i) o += (P.R[i] - 1) * ks(i);
        return o;
    }
    static constexpr int ENTRIES = off(P.S);
    // Fill from the global W_n table; all nthreads threads of the CTA call it.
    __device__ __forceinline__ static void fill(C *dst, const C *__restrict__ tab, int tid, int nthreads) {
        sfor<1, P.S>([&](auto sc) {
            constexpr int S = decltype(sc)::value;
            constexpr int KS = ks(S), OFF = off(S), R = P.R[S], STEP = N / (P.NS[S] * P.R[S]);
            for (int loc = tid; loc < (R - 1) * KS; loc += nthreads) {
                const int k = loc % KS, r = loc / KS + 1;
                dst[OFF + loc] = ldg_c(tab + k * r * STEP);
            }
        });
    }
};

template <typename C, int N, int E, int S>
template <int TWM>
__device__ __forceinline__ void StageTw<C, N, E, S>::load(const C *__restrict__ tab, int t) {
    if constexpr (S > 0 && S < P.S) {
        static_assert(NS % T == 0 || T % NS == 0, "stage twiddles must split");
        if constexpr ((TWM & 3) != 0) {
            constexpr int KS = StageTable<C, N, E>::ks(S), OFF = StageTable<C, N, E>::off(S);
            const int k = t % KS;
#pragma unroll
            for (int r = 1; r < R; ++r)
                z[r - 1] = (TWM & 3) == 1 ? tab[OFF + (r - 1) * KS + k] : ldg_c(tab + OFF + (r - 1) * KS + k);
        } else {
            const int k = t % NS;
#pragma unroll
            for (int r = 1; r < R; ++r) z[r - 1] = ldg_c(tab + k * r * (N / (NS * R)));
        }
    }
}

// One Stockham stage (see the header comment).
template <typename C, int N, int E, int S, typename Lay>
__device__ __forceinline__ void fft_stage(C (&v)[E], const Lay &lay, int t, const StageTw<C, N, E, S> &tw) {
    constexpr StagePlan P = make_plan(N, E);
    constexpr int R = P.R[S];
    constexpr int NS = P.NS[S];
    constexpr int T = N / E;
    constexpr int Q = E / R;
    constexpr bool LAST = (S == P.S - 1);
    static_assert(E % R == 0, "radix must divide E");
    constexpr bool FASTW = !LAST && LayFast<Lay>::value && write_split_ok<N, E, S, LayFast<Lay>::LR>();
    C *pw = nullptr;
    if constexpr (FASTW) {
        const unsigned ut = (unsigned)t;
        const int b = NS <= T ? (int)((ut / NS) * NS * R + ut % NS) : t;
        pw = lay.p + Lay::off(b);
    }
    sfor<0, Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const int j = t + T * q;
        C x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = v[q + r * Q];
        if constexpr (NS > 1) {
            sfor<1, R>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                x[r] = tw_apply(x[r], tw.z[r - 1]);
                if constexpr (NS > T) {
                    constexpr int M = NS / T;           // distinct j mod Ns per thread
                    constexpr int O = NS * R / T;       // order of the extra root
                    x[r] = rotq<((q % M) * r) % O, O>(x[r]);
                }
            });
        }
        Dft<R>::run(x);
        if constexpr (LAST) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[q + r * Q] = x[r];
        } else if constexpr (FASTW) {
            constexpr int j0 = T * q;
            constexpr int ob0 = (j0 / NS) * NS * R + j0 % NS;
            sfor<0, R>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                pw[pad_off(ob0 + r * NS, LayFast<Lay>::LR)] = x[r];
            });
        } else {
            const int k = j % NS;
            const int ob = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) lay.st(ob + r * NS, x[r]);
        }
    });
}

// The same stage split in two halves, for callers that synchronise between
// them: the butterflies of every butterfly group of the thread (results back
// into v in the natural order of the stage's outputs), then the writes of v
// to the exchange row.
template <typename C, int N, int E, int S>
__device__ __forceinline__ void fft_stage_compute(C (&v)[E], int t, const StageTw<C, N, E, S> &tw) {
    constexpr StagePlan P = make_plan(N, E);
    constexpr int R = P.R[S];
    constexpr int NS = P.NS[S];
    constexpr int T = N / E;
    constexpr int Q = E / R;
    static_assert(E % R == 0, "radix must divide E");
    sfor<0, Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        C x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = v[q + r * Q];
        if constexpr (NS > 1) {
            sfor<1, R>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                x[r] = tw_apply(x[r], tw.z[r - 1]);
                if constexpr (NS > T) {
                    constexpr int M = NS / T;
                    constexpr int O = NS * R / T;
                    x[r] = rotq<((q % M) * r) % O, O>(x[r]);
                }
            });
        }
        Dft<R>::run(x);
#pragma unroll
        for (int r = 0; r < R; ++r) v[q + r * Q] = x[r];
    });
}
template <typename C, int N, int E, int S, typename Lay>
__device__ __forceinline__ void fft_stage_write(const C (&v)[E], const Lay &lay, int t) {
    constexpr StagePlan P = make_plan(N, E);
    constexpr int R = P.R[S];
    constexpr int NS = P.NS[S];
    constexpr int T = N / E;
    constexpr int Q = E / R;
    constexpr bool FASTW = LayFast<Lay>::value && write_split_ok<N, E, S, LayFast<Lay>::LR>();
    if constexpr (FASTW) {
        const unsigned ut = (unsigned)t;
        const int b = NS <= T ? (int)((ut / NS) * NS * R + ut % NS) : t;
        C *pw = lay.p + Lay::off(b);
        sfor<0, Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            constexpr int j0 = T * q;
            constexpr int ob0 = (j0 / NS) * NS * R + j0 % NS;
            sfor<0, R>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                pw[pad_off(ob0 + r * NS, LayFast<Lay>::LR)] = v[q + r * Q];
            });
        });
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int j = t + T * q;
            const int ob = (j / NS) * NS * R + j % NS;
#pragma unroll
            for (int r = 0; r < R; ++r) lay.st(ob + r * NS, v[q + r * Q]);
        }
    }
}

// Forward FFT of NC pencils held by this thread group, natural mapping in
// and out.  Every thread of the CTA must call it (it contains barriers).
//
// SMEM & 8 ("late barrier"): the barrier that keeps a stage's writes from
// overtaking other threads' reads of the previous exchange is taken after the
// stage's butterflies, just before the writes, instead of right after the
// reads, so a thread's arithmetic overlaps the other threads' reads.  Then
// every stage's writes, including the first stage's, wait at that barrier,
// and no barrier follows the last exchange: the caller must synchronise
// before it overwrites the exchange rows by other means.
// tw holds the twiddles of stage S; those of stage S+1 are fetched before the
// exchange barrier.
template <typename C, int N, int E, int NC, int S, int SMEM, typename Lay, typename Bar>
__device__ __forceinline__ void fft_forward_from(C (&v)[NC][E], const Lay (&lay)[NC], int t, const C *__restrict__ tab,
                                                 const StageTw<C, N, E, S> &tw, const Bar &bar) {
    constexpr StagePlan P = make_plan(N, E);
    constexpr bool LATEBAR = (SMEM & 8) != 0;
    if constexpr (S < P.S) {
        if constexpr (LATEBAR) {
#pragma unroll
            for (int c = 0; c < NC; ++c) fft_stage_compute<C, N, E, S>(v[c], t, tw);
            if constexpr (S + 1 < P.S) {
                bar.sync();   // every read of the previous exchange (or landing) is done
#pragma unroll
                for (int c = 0; c < NC; ++c) fft_stage_write<C, N, E, S>(v[c], lay[c], t);
            }
        } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) fft_stage<C, N, E, S>(v[c], lay[c], t, tw);
        }
        if constexpr (S + 1 < P.S) {
            constexpr int T = N / E;
            StageTw<C, N, E, S + 1> nxt;
            if constexpr ((SMEM & 4) == 0) nxt.template load<SMEM>(tab, t);
            bar.sync();
            if constexpr (LayFast<Lay>::value && read_split_ok<N, E, LayFast<Lay>::LR>()) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const C *pr = lay[c].p + Lay::off(t);
                    sfor<0, E>([&](auto mc) {
                        constexpr int m = decltype(mc)::value;
                        v[c][m] = pr[pad_off(T * m, LayFast<Lay>::LR)];
                    });
                }
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int m = 0; m < E; ++m) v[c][m] = lay[c].ld(t + T * m);
            }
            if constexpr (!LATEBAR) bar.sync();
            if constexpr ((SMEM & 4) != 0) nxt.template load<SMEM>(tab, t);
            fft_forward_from<C, N, E, NC, S + 1, SMEM>(v, lay, t, tab, nxt, bar);
        }
    }
}

template <typename C, int N, int E, int NC, int SMEM = 0, typename Lay, typename Bar = BarCTA>
__device__ __forceinline__ void fft_forward(C (&v)[NC][E], const Lay (&lay)[NC], int t, const C *__restrict__ tab,
                                            const Bar &bar = Bar()) {
    StageTw<C, N, E, 0> none;
    fft_forward_from<C, N, E, NC, 0, SMEM>(v, lay, t, tab, none, bar);
}

template <typename C, int E, int NC> __device__ __forceinline__ void conj_all(C (&v)[NC][E]) {
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int m = 0; m < E; ++m) v[c][m].y = -v[c][m].y;
}

// dir < 0: forward DFT; dir > 0: inverse DFT without the 1/n factor.
template <typename C, int N, int E, int NC, int SMEM = 0, typename Lay, typename Bar = BarCTA>
__device__ __forceinline__ void fft_dir(C (&v)[NC][E], const Lay (&lay)[NC], int t, const C *__restrict__ tw,
                                        int dir, const Bar &bar = Bar()) {
    if (dir > 0) conj_all<C, E, NC>(v);
    fft_forward<C, N, E, NC, SMEM>(v, lay, t, tw, bar);
    if (dir > 0) conj_all<C, E, NC>(v);
}

}  // namespace sop
