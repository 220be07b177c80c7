// sop_async.cuh -- persistent pencil passes with asynchronous tile prefetch.
//
// Same arithmetic as pass_kernel (sop_kernels.cuh): load a group of pencils,
// [transform] -> pointwise factor -> [transform], store in place.  The
// difference is how data reaches shared memory.  Each CTA loops over tiles
// (persistent grid sized to the GPU) and keeps two tile buffers: while it
// transforms tile k in one buffer, the copy engine fills the other with tile
// k+1:
//   axis 0 (rows contiguous):  cp.async.bulk of each row
//   strided axes:              cp.async.bulk.tensor (TMA) 3D/4D boxes of
//                              W adjacent pencils x <=256 points
// Completion is tracked with mbarrier transaction counts.  The tile buffer is
// also the Stockham exchange buffer, so a pencil is read from HBM once and
// never staged through registers before its first stage.  The stage
// twiddles (a per-stage table, built once per CTA) and the factor table of
// the pass axis (the laser-phase row of the real-space pass or the kinetic
// row of the momentum pass, copied once per launch) live in shared memory;
// the per-point phase values of the real-space pass are fetched into
// registers at the start of each tile, bypassing L1.
//
// Every wait on an mbarrier is bounded in wall time (globaltimer).  If a wait
// gives up, the CTA agrees on it with a block vote, sets bit 0 of *errflag,
// waits (again bounded) for copies it still has in flight, and returns; the
// host reports SOP_ETIMEOUT at its next synchronising call.
#pragma once

#include <cuda.h>

#include "sop_kernels.cuh"

#ifndef SOP_SINGLE_BUFFER
#define SOP_SINGLE_BUFFER 1
#endif
#ifndef SOP_LEAN_TABLES
#define SOP_LEAN_TABLES 1
#endif

namespace sop {

// ---------------------------------------------------------------------------
// PTX wrappers (sm_90 and later)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Non-blocking probe of the phase (no suspend hint): used when a short wait
// limit must be honoured to the timer's resolution.
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity to complete, at most limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
// The same with a caller-set limit (sop_set_wait_limit): polled with the
// non-blocking probe and timed on the SM's cycle counter (two cycles per ns,
// the clock rounded down), so even a limit of a few ns gives up on a copy
// still in flight; try_wait may suspend, and the global timer may advance in
// steps, for longer than such a limit.
__device__ __forceinline__ bool mbar_wait_limit(uint32_t bar, uint32_t parity, uint64_t limit_ns, bool custom) {
    if (!custom) return mbar_wait_bounded(bar, parity, limit_ns);
    const long long c0 = clock64();
    const long long lim = (long long)(limit_ns > (1ull << 40) ? (1ull << 41) : 2 * limit_ns);
    while (!mbar_test_wait(bar, parity))
        if (clock64() - c0 > lim) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, int c0, int c1, int c2, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map),
                 "r"(c0), "r"(c1), "r"(c2), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, int c0, int c1, int c2, int c3, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(map),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(src)
                 : "memory");
}
// Programmatic dependent launch: the next kernel of the stream may be
// scheduled once every CTA of this one has signalled (or exited), and
// griddep_wait() blocks until the preceding kernel has completed and its
// writes are visible.
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// The shared-memory sources of this thread's committed bulk stores have been read.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// This thread's committed bulk stores are complete (globally visible).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s: far beyond any tile copy

__host__ __device__ constexpr int largest_divisor_le(int n, int cap) {
    int d = n < cap ? n : cap;
    while (n % d != 0) --d;
    return d;
}

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------

// Launch-shape variants of the persistent pass (the autotuner picks one per
// pass-axis size, component count and axis kind; 0 is the default shape):
//   WP1   : contiguous axis, one pencil group of ~128 threads per CTA instead of ~256
//   NBUF  : 1 = one tile buffer (the next tile is fetched once the current one
//           no longer needs it; other CTAs on the SM cover the wait), 2 = two
//           (prefetch of the next tile while this one is transformed), 0 = the
//           default rule
//   VPRE  : the per-point phase values of the real-space factor are fetched
//           into registers before the tile is waited for (else just before use)
//   L1TAB : stage twiddles and the pass-axis factor row are read through L1
//           instead of being copied into shared memory
//   REGS  : register budget per thread that sets the resident CTAs per SM
//   E     : values per thread (0: the size's default, 16 for a power of two)
//   LATE  : stage twiddles fetched after each exchange instead of before it
//   AXL1  : only the pass-axis factor row is read through L1
//   CT    : threads per CTA on the contiguous axis (0: 128 with WP1, else 256)
template <int VAR> struct PassPolicy;
//   PMAJOR: strided axes with pencil-major threads (each pencil's threads are
//           whole warps, so its exchanges synchronise only its own warps;
//           the lane-interleaved landing reads then touch two bank lines)
struct PolBase {
    static constexpr bool LATE = false, AXL1 = false, PMAJOR = false;
    static constexpr int E = 0, CT = 0;
};
template <> struct PassPolicy<0> : PolBase {
    static constexpr bool WP1 = false, VPRE = true, L1TAB = false;
    static constexpr int NBUF = 0, REGS = 104;
};
template <> struct PassPolicy<1> : PolBase {
    static constexpr bool WP1 = true, VPRE = false, L1TAB = false;
    static constexpr int NBUF = 1, REGS = 80;
};
template <> struct PassPolicy<2> : PolBase {
    static constexpr bool WP1 = true, VPRE = false, L1TAB = true, PMAJOR = true;
    static constexpr int NBUF = 2, REGS = 80;
};
template <> struct PassPolicy<3> : PolBase {
    static constexpr bool WP1 = true, VPRE = false, L1TAB = true;
    static constexpr int NBUF = 2, REGS = 64;
};
template <> struct PassPolicy<4> : PolBase {
    static constexpr bool WP1 = true, VPRE = false, L1TAB = true;
    static constexpr int NBUF = 1, REGS = 72;
};
// one pencil group per CTA with the phase values prefetched (as variant 0)
template <> struct PassPolicy<5> : PolBase {
    static constexpr bool WP1 = true, VPRE = true, L1TAB = false;
    static constexpr int NBUF = 1, REGS = 112;
};
// stage twiddles in shared memory, the pass-axis row through L1
template <> struct PassPolicy<6> : PolBase {
    static constexpr bool WP1 = true, VPRE = false, L1TAB = false, AXL1 = true;
    static constexpr int NBUF = 2, REGS = 80;
};
template <> struct PassPolicy<7> : PolBase {
    static constexpr bool WP1 = true, VPRE = false, L1TAB = false, AXL1 = true;
    static constexpr int NBUF = 1, REGS = 80;
};
static_assert(kPassVariants == 8, "one PassPolicy per variant");

// Values per thread of the persistent passes where they differ from the
// Geometry default (0: the default).  Complex64 component pairs on power-of-
// two sides >= 512 hold 16 values per component instead of 8: 1024 points
// then take 16·16·4 (two exchanges per transform) instead of 8·8·8·2 (three),
// and the two-exchange transform wins despite the doubled register set
// (measured on GB300, 1024^2 Dirac pairs: 62.5 -> 56.2 us per split step
// with the default shapes).  Complex128 pairs would spill and keep 8.
template <typename Real, int N, int NC> constexpr int pass_ev() {
    return (sizeof(Real) == 4 && NC == 2 && N >= 512 && (N & (N - 1)) == 0) ? 16 : 0;
}

template <typename Real, int N, int NC, bool CONTIG, int VAR = 0> struct AsyncCfg {
    using Pol = PassPolicy<VAR>;
    static constexpr int EV0 = pass_ev<Real, N, NC>();
    // 32 values per thread only where the size's default is 16
    static constexpr int EV = (Pol::E > 0 && Geometry<N, NC, EV0>::E == 16 && N >= 512) ? Pol::E : EV0;
    using G = Geometry<N, NC, EV>;
    using C = cplx_t<Real>;
    static constexpr int E = G::E;
    static constexpr int T = G::T;
    static constexpr int CSZ = 2 * (int)sizeof(Real);
    static constexpr int PITCH = ((N + (N >> G::LR)) + 1) & ~1;   // even: rows stay 16-byte aligned
    static constexpr int wp_contig() {
        int w = (Pol::CT > 0 ? Pol::CT : (Pol::WP1 || NC == 4 ? 128 : 256)) / T;
        return w < 1 ? 1 : w;
    }
    static constexpr int wp_strided() {
        const int wmin = CSZ == 8 ? 2 : 1;                 // a TMA box row is at least 16 bytes
        int w = (32 * 1024) / (NC * N * CSZ);              // ~32 KB per tile buffer
        const int wmax = CSZ == 8 ? 128 : 64;              // box row <= 256 8-byte elements
        if (w > wmax) w = wmax;
        int p = 1;
        while (p * 2 <= w) p *= 2;
        w = p;
        while (w > wmin && w * T > 512) w /= 2;
        return w < wmin ? wmin : w;
    }
    static constexpr int WP = CONTIG ? wp_contig() : wp_strided();
    static constexpr int THREADS = T * WP;
    static constexpr int BR = largest_divisor_le(N, 256);   // box extent along the axis
    // Strided axes interleave the WP pencils of a tile over the lanes of a
    // warp (pencil w = tid mod WP), so a warp reads whole landing rows of
    // 16 bytes or more.  Shared-memory accesses of 8-byte (16-byte) elements
    // are served per half (quarter) warp, PER lanes per 128-byte wavefront,
    // which then cover PER / WP threads of each pencil; the exchange rows get
    // a pitch RPITCH >= USED with RPITCH = SKEW_B = PER / (WP NC) (mod PER), so
    // that the pencil rows of one wavefront fall on different banks.  The rule
    // was checked against a bank model of every access of the pass (landing
    // read, exchanges, write-back) for all sizes.
    static constexpr int LANES = CONTIG ? 32 : (WP >= 32 ? 1 : 32 / WP);
    static constexpr int PER = 128 / CSZ;   // elements per 128-byte bank line
    static constexpr int SKEW_H = PER / (WP * NC) > 1 ? PER / (WP * NC) : 1;
    static constexpr int SKEW_B = SKEW_H % PER;
    static constexpr int USED = (N - 1) + ((N - 1) >> G::LR) + 1;   // exchange row length in use
    static constexpr int RPITCH = CONTIG ? PITCH : USED + ((SKEW_B - USED % PER) % PER + PER) % PER;
    static constexpr size_t al128(size_t x) { return (x + 127) & ~size_t(127); }
    static constexpr size_t LAND = (size_t)NC * N * WP * CSZ;        // strided: TMA landing layout [c][i][w]
    static constexpr size_t XCHG = (size_t)WP * NC * RPITCH * CSZ;   // padded per-pencil exchange rows
    static constexpr size_t BUF = al128(CONTIG ? XCHG : (LAND > XCHG ? LAND : XCHG));
    static constexpr size_t TWZ = al128((size_t)StageTable<C, N, E>::ENTRIES * CSZ + 16);
    static constexpr size_t AXT = al128((size_t)N * CSZ);   // pass-axis table (field row / kinetic row)
    // Strided complex128 passes keep one tile buffer instead of two when that
    // lets one more CTA share the SM: the next tile is then fetched after the
    // tile store has read the buffer, and the other CTAs cover the wait.
    // (Measured on GB300: 2048^2 c128 split steps 1394 -> 1354 us; for
    // complex64 the second buffer is worth more than the extra CTA.)
    static constexpr int ctas_smem(size_t bytes) { return (int)((228 * 1024) / (bytes + 1024)); }
    // Four-component passes also keep one buffer: their tiles are four times
    // larger, and more CTAs per SM pay more than the prefetch.
    static constexpr bool SINGLE = Pol::NBUF == 1 || (Pol::NBUF == 0 && NC == 4) ||
                                   (Pol::NBUF == 0 && SOP_SINGLE_BUFFER != 0 && !CONTIG && CSZ == 16 && NC == 1 &&
                                    ctas_smem(128 + BUF + TWZ + AXT) > ctas_smem(128 + 2 * BUF + TWZ + AXT));
    static constexpr int NBUF = SINGLE ? 1 : 2;
    static constexpr size_t OFF_BUF = 128, OFF_TWZ = OFF_BUF + NBUF * BUF, OFF_AXT = OFF_TWZ + TWZ;
    // Lean layout: the stage twiddles are read from global memory through L1
    // instead of shared memory, when that lets one more CTA share the SM.
    // Used for the complex64 Dirac pair passes on strided axes, which read
    // no axis table.  (Measured on GB300: for the single-component passes
    // the extra CTA does not pay for the L1 reads of the axis row and the
    // twiddles; 2048^2 complex64 split steps took 61.0 instead of 56.2 us.)
    static constexpr int ctas_for(size_t bytes) { return (int)((228 * 1024) / (bytes + 1024)); }
    static constexpr bool LEAN = Pol::L1TAB || (SOP_LEAN_TABLES != 0 && CSZ == 8 && NC == 2 && !CONTIG &&
                                                ctas_for(OFF_BUF + NBUF * BUF) > ctas_for(OFF_AXT + AXT));
    static_assert(!LEAN || EV == EV0, "the global stage table is laid out for the default values per thread");
    static constexpr bool AXL1 = LEAN || Pol::AXL1;   // pass-axis row through L1
    static constexpr size_t SMEM = LEAN ? OFF_BUF + NBUF * BUF : (AXL1 ? OFF_AXT : OFF_AXT + AXT);
    // buffer and mbarrier phase parity of iteration it
    __device__ __forceinline__ static int buf_of(int it) { return SINGLE ? 0 : (it & 1); }
    __device__ __forceinline__ static uint32_t par_of(int it) { return SINGLE ? (it & 1) : ((it >> 1) & 1); }
    static constexpr bool FITS = SMEM <= 227 * 1024 && THREADS <= 1024;
    // twiddle source of the FFT (see StageTw) and the late write barrier (see fft_forward_from)
    static constexpr int TWM = (LEAN ? 2 : 1) | (Pol::LATE ? 4 : 0) | 8;
    // On the contiguous axis a pencil is whole warps (threadIdx.y = pencil), so
    // its exchanges synchronise only its own warps (named barrier 1 + pencil).
    static constexpr bool PMAJOR = !CONTIG && Pol::PMAJOR && T % 32 == 0 && WP > 1 && WP <= 15;
    static constexpr bool PENCIL_BAR = (CONTIG || PMAJOR) && T % 32 == 0 && WP > 1 && WP <= 15;
    static_assert(USED <= PITCH && USED <= RPITCH, "exchange rows must not overlap");
    // CTAs per SM that shared memory allows; the register budget follows.
    static constexpr int minb() {
        int b = (int)((227 * 1024) / (SMEM > 0 ? SMEM : 1));
        const int bt = 2048 / THREADS;
        int regs = VAR == 0 ? (NC == 4 ? 128 : (LEAN ? 64 : 104)) : Pol::REGS;
        if (EV0 == 16 && NC == 2 && regs < 128) regs = 128;   // 32 values per thread: budgets below spill
        const int br = 65536 / (THREADS * regs);   // registers per thread to leave
        if (bt < b) b = bt;
        if (br < b) b = br;
        if (b > 8) b = 8;
        return b < 1 ? 1 : b;
    }
    static constexpr int MINB = minb();
};

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------

// MULTI: the tiles belong to several lattices (a.inst, one component each)
// that share the pass-axis size N; each tile takes its lattice's state,
// tables, geometry and tensor map from the instance descriptor.
template <typename Real, int N, int NC, bool CONTIG, bool MULTI, int VAR = 0>
__global__ void __launch_bounds__(AsyncCfg<Real, N, NC, CONTIG, VAR>::THREADS, AsyncCfg<Real, N, NC, CONTIG, VAR>::MINB)
    pass_kernel_async(const __grid_constant__ PassArgs a, const __grid_constant__ CUtensorMap tmap) {
    static_assert(!MULTI || NC == 1, "multi-instance passes have one component");
    using Cfg = AsyncCfg<Real, N, NC, CONTIG, VAR>;
    constexpr bool VPRE = Cfg::Pol::VPRE && NC != 4;   // the 4x4 factor reads its phase values itself
    using C = cplx_t<Real>;
    using Ph = Phase<Real>;
    constexpr int E = Cfg::E, T = Cfg::T, WP = Cfg::WP, CSZ = Cfg::CSZ;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);   // 0, 1: tile buffers; 2: axis table
    int64_t *s_tile = reinterpret_cast<int64_t *>(smem + 32);   // claimed tiles, by iteration parity
    unsigned char *const buf0 = smem + Cfg::OFF_BUF;       // tile buffer b starts at buf0 + b * BUF
    C *twz = reinterpret_cast<C *>(smem + Cfg::OFF_TWZ);   // per-stage twiddles
    C *axt = reinterpret_cast<C *>(smem + Cfg::OFF_AXT);   // pass-axis factor table

    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int t = (CONTIG || Cfg::PMAJOR) ? (int)threadIdx.x : tid / WP;   // thread within the pencil
    const int w = (CONTIG || Cfg::PMAJOR) ? (int)threadIdx.y : tid % WP;   // pencil within the tile
    const int pz = NC == 2 ? (int)blockIdx.z : 0;
    const int64_t stride = CONTIG ? 1 : a.stride;
    const bool op_v = a.op == OP_V, op_t = a.op == OP_T;
    // the factor table of this pass's axis (field row for OP_V, kinetic row for OP_T)
    const C *axsrc = nullptr;
    if (NC == 1 && (op_v || op_t)) {
        const void *p = op_v ? (a.axis == 0 ? a.ftab[0] : (a.axis == 1 ? a.ftab[1] : a.ftab[2]))
                             : (a.axis == 0 ? a.ttab[0] : (a.axis == 1 ? a.ttab[1] : a.ttab[2]));
        axsrc = reinterpret_cast<const C *>(p);
    }
    const uint32_t bar0 = smem_addr(&bars[0]), bar1 = smem_addr(&bars[1]), barx = smem_addr(&bars[2]);

    const int64_t ntiles = a.n_tiles;
    // The next pass may start its prologue (barriers, twiddle table) on SMs
    // this grid leaves; it reads psi and its tables only after griddep_wait.
    griddep_launch_dependents();
    // Tiles are claimed one at a time (thread 0), so SMs that run ahead take
    // more of them whatever the placement of the CTAs.
    // A claim below the launch's base can only follow a launch whose CTAs
    // gave up (their claims fell short); it counts as past the last tile.
    auto claim = [&]() -> int64_t {
        const int64_t c = (int64_t)(atomicAdd(a.tile_ctr + pz, 1ull) - a.tile_base[pz]);
        return c < 0 ? ntiles : c;
    };
    // tile copies wait at most this long (a.wait_ns > 0 shortens it to test
    // the error path); drains after giving up always use the full limit
    const uint64_t wait_ns = a.wait_ns > 0 ? a.wait_ns : kWaitLimitNs;

    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        mbar_init(barx, 1);
        fence_mbar_init();
    }
    if constexpr (!Cfg::LEAN) StageTable<C, N, E>::fill(twz, reinterpret_cast<const C *>(a.tw), tid, Cfg::THREADS);
    __syncthreads();

    // Multi-instance: the lattice of global tile g (the last instance whose
    // first tile is <= g).
    auto find_inst = [&](int64_t g) -> const InstDesc * {
        int lo = 0, hi = a.n_inst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.inst[mid].tile_begin <= g) lo = mid;
            else hi = mid - 1;
        }
        return a.inst + lo;
    };
    // Per-tile values, read where they are used (launch arguments of a
    // single lattice, or the instance descriptor through L1), so that they
    // hold no registers across the tile.
    auto pv_psi = [&](const InstDesc *d) -> C * {
        if constexpr (MULTI) return reinterpret_cast<C *>(d->psi);
        else return reinterpret_cast<C *>(a.psi);
    };
    // Field row of this launch's real-space index and whether it takes the
    // half factor (first and last index of a call); a graph-replayed middle
    // step reads its row from a device word (set after griddep_wait).
    int64_t frow = a.P - a.p_table0;
    const bool half_v = a.row_dev == nullptr && (a.P == 0 || a.P == a.n_total);
    auto pv_vtab = [&](const InstDesc *d) -> const C * {
        if constexpr (MULTI) return reinterpret_cast<const C *>(half_v ? d->vhalf : d->vfull);
        else return reinterpret_cast<const C *>(a.vtab);
    };
    auto pv_row = [&](const InstDesc *d, int ax) -> const C * {   // factor row of axis ax (field or kinetic)
        if constexpr (MULTI) {
            if (!op_v) return reinterpret_cast<const C *>(d->ttab[ax]);
            if (!d->ftab || d->foff[ax] < 0) return nullptr;
            return reinterpret_cast<const C *>(d->ftab) + frow * d->frow_len + d->foff[ax];
        } else {
            return reinterpret_cast<const C *>(op_v ? a.ftab[ax] : a.ttab[ax]);
        }
    };
    const int64_t tpb_single = CONTIG ? 0 : a.n_xgroups * (a.n_pencils / a.dims[0]);
    auto pv_i64 = [&](const InstDesc *d, int which) -> int64_t {
        // 0 pencils per batch, 1 pencils, 2 n0, 3 n1, 4 x groups, 5 o stride,
        // 6 component stride, 7 strided tiles per batch entry
        if constexpr (MULTI) {
            switch (which) {
                case 0: case 1: return d->n_pencils;
                case 2: return d->dims[0];
                case 3: return d->dims[1];
                case 4: return d->n_xgroups;
                case 5: return d->o_stride;
                case 7: return d->tiles_per_batch;
                default: return 0;
            }
        } else {
            switch (which) {
                case 0: return a.n_pencils;
                case 1: return (NC == 1) ? a.n_pencils * a.n_batch : a.n_pencils;
                case 2: return a.dims[0];
                case 3: return a.dims[1];
                case 4: return a.n_xgroups;
                case 5: return a.o_stride;
                case 7: return tpb_single;
                default: return a.comp_stride;
            }
        }
    };
    auto pv_map = [&](const InstDesc *d) -> const CUtensorMap * {
        if constexpr (MULTI) return reinterpret_cast<const CUtensorMap *>(d->tmap);
        else return &tmap;
    };
    // Check builds: elements of the state array (all components) and points
    // of one component that a tile of this launch may touch.
    auto lat_elems = [&](const InstDesc *d) -> int64_t {
        if constexpr (MULTI) return d->n_pencils * (int64_t)N;
        else return (int64_t)a.n_comp_total * a.comp_stride;
    };
    auto lat_pts = [&](const InstDesc *d) -> int64_t {
        if constexpr (MULTI) return d->n_pencils * (int64_t)N;
        else return a.comp_stride;
    };
    (void)lat_elems;
    (void)lat_pts;
    // Global tile g -> its lattice (null for a single lattice) and local index.
    auto locate = [&](int64_t g, int64_t &local) -> const InstDesc * {
        if constexpr (MULTI) {
            const InstDesc *d = find_inst(g);
            local = g - d->tile_begin;
            return d;
        } else {
            local = g;
            return nullptr;
        }
    };

    auto comp_index = [&](int c, int64_t b) -> int64_t {
        return NC == 1 ? b : (NC == 2 ? (int64_t)a.pair_comp[pz][c] : (int64_t)c);
    };

    // Strided axes: the TMA boxes of tile tl of lattice q, f(component slot,
    // box, coords...) with coordinates (x [in 8-byte units], axis 1, axis 2,
    // component).
    auto tile_boxes = [&](const InstDesc *d, int64_t tl, auto &&f) {
        const int64_t tiles_per_batch = pv_i64(d, 7);
        const uint32_t ut = (uint32_t)tl, ng = (uint32_t)pv_i64(d, 4);
        const uint32_t bidx = NC == 1 ? ut / (uint32_t)tiles_per_batch : 0u;
        const uint32_t rem = NC == 1 ? ut - bidx * (uint32_t)tiles_per_batch : ut;
        const uint32_t o = rem / ng;
        const uint32_t xg = rem - o * ng;
        const int x0 = (int)(xg * WP) * (CSZ / 8);
        for (int c = 0; c < NC; ++c) {
            const int cc = (int)comp_index(c, bidx);
            for (int r = 0; r < N / Cfg::BR; ++r) {
                if (a.ndim == 2) f(c, r, x0, r * Cfg::BR, 0, cc);
                else if (a.axis == 1) f(c, r, x0, r * Cfg::BR, (int)o, cc);
                else f(c, r, x0, (int)o, r * Cfg::BR, cc);
            }
        }
    };

    // Thread 0: start the copies of (global) tile g into buffer slot b.
    auto issue = [&](int64_t g, int b) {
        int64_t tl;
        const InstDesc *d = locate(g, tl);
        const int64_t per_batch = pv_i64(d, 0), total = pv_i64(d, 1);
        const uint32_t bar = b ? bar1 : bar0;
        const uint32_t dst0 = smem_addr(buf0 + b * Cfg::BUF);
        if constexpr (CONTIG) {
            const int64_t p0 = tl * WP;
            const int rows = (int)((total - p0) < WP ? (total - p0) : WP);
            mbar_expect_tx(bar, (uint32_t)(rows * NC * N * CSZ));
            for (int r = 0; r < rows; ++r) {
                const int64_t p = p0 + r;
                int64_t bidx = 0, pp = p;
                if (NC == 1) {
                    bidx = p / per_batch;
                    pp = p - bidx * per_batch;
                }
                for (int c = 0; c < NC; ++c) {
                    const int64_t off = comp_index(c, bidx) * pv_i64(d, 6) + pp * N;
                    if (SOP_IN(a.errflag, off >= 0 && off + N <= lat_elems(d)))
                        bulk_g2s(dst0 + (uint32_t)((r * NC + c) * Cfg::PITCH * CSZ), pv_psi(d) + off,
                                 (uint32_t)(N * CSZ), bar);
                }
            }
        } else {
            mbar_expect_tx(bar, (uint32_t)(NC * N * WP * CSZ));
            const CUtensorMap *map = pv_map(d);
            tile_boxes(d, tl, [&](int c, int r, int c0, int c1, int c2, int c3) {
                const uint32_t dst = dst0 + (uint32_t)((c * N + r * Cfg::BR) * WP * CSZ);
                if (!SOP_IN(a.errflag, ((c0 * 8) & 15) == 0)) return;   // a TMA x must be 16-byte aligned
                if (a.ndim == 2) tma_load_3d(dst, map, c0, c1, c3, bar);
                else tma_load_4d(dst, map, c0, c1, c2, c3, bar);
            });
        }
    };
    // Thread 0: write (global) tile g back from buffer slot b (strided axes).
    auto store_tile = [&](int64_t g, int b) {
        int64_t tl;
        const InstDesc *d = locate(g, tl);
        const CUtensorMap *map = pv_map(d);
        const uint32_t src0 = smem_addr(buf0 + b * Cfg::BUF);
        tile_boxes(d, tl, [&](int c, int r, int c0, int c1, int c2, int c3) {
            const uint32_t src = src0 + (uint32_t)((c * N + r * Cfg::BR) * WP * CSZ);
            if (!SOP_IN(a.errflag, ((c0 * 8) & 15) == 0 && c1 >= 0 && c2 >= 0)) return;
            if (a.ndim == 2) tma_store_3d(map, c0, c1, c3, src);
            else tma_store_4d(map, c0, c1, c2, c3, src);
        });
        bulk_commit();
    };
    // A wait gave up: record it, drain what this CTA still has in flight, leave.
    auto give_up = [&](int it, bool cur_pending, bool next_issued, bool ax_pending) {
        if (tid == 0) {
            atomicOr(a.errflag, 1);
            if (!CONTIG) bulk_wait_all();
            const int b = Cfg::buf_of(it);
            if (cur_pending) mbar_wait_bounded(b ? bar1 : bar0, Cfg::par_of(it), kWaitLimitNs);
            if (next_issued) mbar_wait_bounded(b ? bar0 : bar1, Cfg::par_of(it + 1), kWaitLimitNs);
            if (ax_pending) mbar_wait_bounded(barx, 0, kWaitLimitNs);
        }
    };

    // axis table copied into shared memory (single lattice; multi-instance
    // passes read each lattice's row through L1)
    const bool axt_smem = !Cfg::AXL1 && !MULTI && axsrc != nullptr;
    // Before this point only the stage twiddles (written when the plan was
    // made) are read.  psi and the phase tables may come from the kernel
    // just before this one in the stream.
    griddep_wait();
    // An earlier pass of this stream gave up waiting (its tiles are
    // unfinished and the tile counters are behind): do nothing until the
    // host, which reports SOP_ETIMEOUT, has reset them.
    if (*reinterpret_cast<volatile int *>(a.errflag) != 0) return;
    if constexpr (MULTI)
        if (a.row_dev) frow = *reinterpret_cast<const volatile int64_t *>(a.row_dev);
    // Thread 0 claims one tile ahead: the claim for the tile after the
    // current one is made when the current one is issued, so the latency of
    // the atomic is hidden behind a whole tile.  Claims stop after the first
    // one past the last tile.
    int64_t ahead = ntiles;
    if (tid == 0) {
        const int64_t first = claim();
        s_tile[0] = first;
        if (first < ntiles) {
            if (axt_smem) {
                mbar_expect_tx(barx, (uint32_t)(N * CSZ));
                bulk_g2s(smem_addr(axt), axsrc, (uint32_t)(N * CSZ), barx);
            }
            issue(first, 0);
            ahead = claim();
        }
    }
    __syncthreads();
    int64_t tile = s_tile[0];
    if (tile >= ntiles) return;   // nothing claimed, nothing in flight
    if (axt_smem) {
        const bool okx = mbar_wait_limit(barx, 0, wait_ns, a.wait_ns > 0);
        if (!__syncthreads_and(okx)) {
            give_up(0, true, false, true);
            return;
        }
    }
    const C *tw = Cfg::LEAN ? reinterpret_cast<const C *>(a.stw) : twz;

    for (int it = 0; tile < ntiles; ++it) {
        const int b = Cfg::buf_of(it);
        // Claim and prefetch of the next tile into buffer b ^ 1: at once on the
        // contiguous axis; on strided axes after the first transform, by which
        // time the tile store out of that buffer (issued at the end of the
        // previous iteration) has long been read, so no thread waits for it.
        // The claim reaches the other threads through s_tile[(it + 1) & 1].
        bool has_next = false;   // meaningful in thread 0
        int64_t next = ntiles;
        auto publish_next = [&]() {
            next = ahead;
            s_tile[(it + 1) & 1] = next;
            has_next = next < ntiles;
        };
        auto issue_next = [&]() {
            fence_proxy_async_smem();   // earlier generic accesses to the buffers precede the copies
            if (has_next) {
                issue(next, Cfg::buf_of(it + 1));
                ahead = claim();
            }
        };
        auto claim_next = [&]() {
            publish_next();
            issue_next();
        };
        if (CONTIG && tid == 0) {
            if constexpr (Cfg::SINGLE) publish_next();   // issued once the buffer is free
            else claim_next();
        }

        int64_t ltile = tile;
        const InstDesc *dp = nullptr;
        if constexpr (MULTI) {
            dp = find_inst(tile);
            ltile = tile - dp->tile_begin;
        }
        const int64_t per_batch = pv_i64(dp, 0), total = pv_i64(dp, 1), n0 = pv_i64(dp, 2);
        const int64_t tiles_per_batch = pv_i64(dp, 7);
        const bool want_v = CONTIG && pv_vtab(dp) != nullptr && (op_v || a.op == OP_DV || a.op == OP_D3V);
        // Pencil of this thread: first point (linear index base) and lattice
        // coordinates co (0 along the pass axis).  Pencil and tile counts are
        // below 2^31, so the index arithmetic runs in 32 bits.
        int64_t base, coff[NC];
        int co[3] = {0, 0, 0};
        bool active;
        if constexpr (CONTIG) {
            const uint32_t p = (uint32_t)ltile * WP + w;
            active = p < (uint32_t)total;
            const uint32_t pc = active ? p : 0u;
            uint32_t bidx = 0, pp = pc;
            if (NC == 1) {
                bidx = pc / (uint32_t)per_batch;
                pp = pc - bidx * (uint32_t)per_batch;
            }
            base = (int64_t)pp * N;
            const uint32_t n1 = (uint32_t)pv_i64(dp, 3);
            if (a.ndim >= 2) co[1] = (int)(pp % n1);
            if (a.ndim == 3) co[2] = (int)(pp / n1);
#pragma unroll
            for (int c = 0; c < NC; ++c) coff[c] = comp_index(c, bidx) * pv_i64(dp, 6);
        } else {
            const uint32_t ut = (uint32_t)ltile, ng = (uint32_t)pv_i64(dp, 4);
            const uint32_t bidx = NC == 1 ? ut / (uint32_t)tiles_per_batch : 0u;
            const uint32_t rem = NC == 1 ? ut - bidx * (uint32_t)tiles_per_batch : ut;
            const uint32_t o = rem / ng;   // the remaining coordinate (z for axis 1, y for axis 2)
            const uint32_t x = (rem - o * ng) * WP + w;
            active = x < (uint32_t)n0;
            const uint32_t xc = active ? x : 0u;
            base = (int64_t)xc + (int64_t)o * pv_i64(dp, 5);
            co[0] = (int)xc;
            if (a.ndim == 3) co[a.axis == 1 ? 2 : 1] = (int)o;
#pragma unroll
            for (int c = 0; c < NC; ++c) coff[c] = comp_index(c, bidx) * pv_i64(dp, 6);
        }

        // Per-point phase values of this pencil (bypassing L1): fetched now
        // and used after the first transform (VPRE), or loaded where used.
        const C *const vt = want_v ? pv_vtab(dp) + base : nullptr;
        C vpre[VPRE ? E : 1];
        if constexpr (VPRE) {
            if (want_v) {
#pragma unroll
                for (int m = 0; m < E; ++m)
                    vpre[m] = SOP_IN(a.errflag, base + t + T * m < lat_pts(dp)) ? ld_stream(vt + (t + T * m)) : Ph::one();
            } else {
#pragma unroll
                for (int m = 0; m < E; ++m) vpre[m] = Ph::one();
            }
        }
        auto vph = [&](int m) -> C {
            if constexpr (VPRE) return vpre[m];
            else return (want_v && SOP_IN(a.errflag, base + t + T * m < lat_pts(dp))) ? ld_stream(vt + (t + T * m))
                                                                                    : Ph::one();
        };

        bool ok = mbar_wait_limit(b ? bar1 : bar0, Cfg::par_of(it), wait_ns, a.wait_ns > 0);
        if (!__syncthreads_and(ok)) {
            give_up(it, true, CONTIG && !Cfg::SINGLE && has_next, false);
            return;
        }

        // Registers <- tile buffer (landing layout), then the buffer becomes
        // the exchange buffer.
        C *bufc = reinterpret_cast<C *>(buf0 + b * Cfg::BUF);
        using Bar = std::conditional_t<Cfg::PENCIL_BAR, BarGroup, BarCTA>;
        Bar pbar;
        if constexpr (Cfg::PENCIL_BAR) pbar = BarGroup{1 + w, T};
        C v[NC][E];
        using Lay = LayContig<C, Cfg::G::LR>;   // exchange rows, one per pencil and component
        Lay lay[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            C *row = bufc + (w * NC + c) * Cfg::RPITCH;
            lay[c].p = row;
            if constexpr (CONTIG) {
#pragma unroll
                for (int m = 0; m < E; ++m)
                    v[c][m] = SOP_IN(a.errflag, ((w * NC + c) * Cfg::RPITCH + t + T * m + 1) * CSZ <= (int)Cfg::BUF)
                                  ? row[t + T * m]
                                  : C{};
            } else {
                const C *col = bufc + c * N * WP + w;   // TMA landing layout [c][i][w]
#pragma unroll
                for (int m = 0; m < E; ++m)
                    v[c][m] = SOP_IN(a.errflag, (c * N * WP + w + (t + T * m) * WP + 1) * CSZ <= (int)Cfg::BUF)
                                  ? col[(t + T * m) * WP]
                                  : C{};
            }
        }
        // the landing rows become exchange rows: a transform's first writes
        // wait at its late barrier until every landing read is done (with
        // pencil-major threads the landing rows hold every pencil's values,
        // so all of the CTA's reads must be done first)
        if constexpr (Cfg::PMAJOR) __syncthreads();

        if (a.pre != 0) fft_dir<C, N, E, NC, Cfg::TWM>(v, lay, t, tw, a.pre, pbar);
        if (!CONTIG && !Cfg::SINGLE && tid == 0) {
            bulk_wait_read();   // the tile store out of buffer b ^ 1 has read it
            claim_next();
        }

        if constexpr (NC == 1 && CONTIG && !MULTI) {
            if (op_v && a.mat_out) {
                // psi_P = A_{P-1} u, stored; then A_P psi_P (A = half factor,
                // phase values and field rows of each half)
                const C *h1[3], *h2[3];
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    h1[ax] = ax < a.ndim ? reinterpret_cast<const C *>(a.ftab[ax]) : nullptr;
                    h2[ax] = ax < a.ndim ? reinterpret_cast<const C *>(a.fh2[ax]) : nullptr;
                }
                C g1 = Ph::one(), g2 = Ph::one();
#pragma unroll
                for (int ax = 1; ax < 3; ++ax) {
                    if (h1[ax]) g1 = Ph::combine(g1, ldg_c(h1[ax] + co[ax]));
                    if (h2[ax]) g2 = Ph::combine(g2, ldg_c(h2[ax] + co[ax]));
                }
                C *const mo = reinterpret_cast<C *>(a.mat_out) + coff[0] + base + t;
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const C vh = vph(m);
                    C f1 = Ph::combine(vh, g1), f2 = Ph::combine(vh, g2);
                    if (h1[0]) f1 = Ph::combine(ldg_c(h1[0] + t + T * m), f1);
                    if (h2[0]) f2 = Ph::combine(ldg_c(h2[0] + t + T * m), f2);
                    const C ps = Ph::apply(v[0][m], f1);
                    if (active && SOP_IN(a.errflag, coff[0] + base + t + T * m < lat_elems(dp))) st_stream(mo + T * m, ps);
                    v[0][m] = Ph::apply(ps, f2);
                }
            }
        }
        if constexpr (NC == 1) {
            if ((op_v || op_t) && !(CONTIG && !MULTI && op_v && a.mat_out)) {
                // Pencil-constant part g from the other axes' tables (absent when
                // none is set), per-point part from the axis table and, for the
                // real-space factor, the phase values.  The flags are uniform, so
                // the loop is specialised on them rather than branching per point.
                const C *tab[3];
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) tab[ax] = pv_row(dp, ax);
                const C *const axsrc_t = (MULTI || Cfg::AXL1) ? pv_row(dp, a.axis) : axsrc;
                const bool has_axt = axsrc_t != nullptr;
                C g = Ph::one();
                bool g_set = false;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax)
                    if (ax < a.ndim && ax != a.axis && tab[ax] != nullptr) {
                        const C x = ldg_c(tab[ax] + co[ax]);
                        g = g_set ? Ph::combine(g, x) : x;
                        g_set = true;
                    }
                Real shi, slo;
                if constexpr (MULTI) {
                    shi = Real(dp->scale_hi);
                    slo = Real(dp->scale_lo);
                } else {
                    shi = Real(a.scale_hi);
                    slo = Real(a.scale_lo);
                }
                auto axis_at = [&](int i) -> C { return (Cfg::AXL1 || MULTI) ? ldg_c(axsrc_t + i) : axt[i]; };
                // f = [V phase] [axis factor] [g], then psi <- psi (1 + f) [* 1/N].
                auto loop = [&](auto hv_c, auto axt_c, auto g_c, auto scale_c) {
                    constexpr bool HV = decltype(hv_c)::value, AX = decltype(axt_c)::value;
                    constexpr bool GG = decltype(g_c)::value;
                    constexpr int SC = decltype(scale_c)::value;   // 0: none, 1: hi only, 2: hi + lo
#pragma unroll
                    for (int m = 0; m < E; ++m) {
                        C f = HV ? vph(m) : (AX ? axis_at(t + T * m) : (GG ? g : Ph::one()));
                        if constexpr (HV && AX) f = Ph::combine(axis_at(t + T * m), f);
                        if constexpr (GG && (HV || AX)) f = Ph::combine(f, g);
                        C r = Ph::apply(v[0][m], f);
                        if constexpr (SC == 1) r = mk<C>(r.x * shi, r.y * shi);
                        if constexpr (SC == 2) r = scale2(r, shi, slo);
                        v[0][m] = r;
                    }
                };
                using F_ = std::false_type;
                using T_ = std::true_type;
                using S0 = std::integral_constant<int, 0>;
                using S1 = std::integral_constant<int, 1>;
                using S2 = std::integral_constant<int, 2>;
                // Specialised: the real-space factor on the contiguous axis and the
                // kinetic factor (axis row and g) on strided axes, the passes of a
                // step; any other combination takes the per-point flags.
                if (CONTIG && op_v && !g_set) {
                    if (has_axt) loop(T_{}, T_{}, F_{}, S0{});
                    else loop(T_{}, F_{}, F_{}, S0{});
                } else if (!CONTIG && op_t && has_axt && g_set) {
                    if (slo == Real(0)) loop(F_{}, T_{}, T_{}, S1{});
                    else loop(F_{}, T_{}, T_{}, S2{});
                } else {
#pragma unroll
                    for (int m = 0; m < E; ++m) {
                        C f = g;
                        if (has_axt) f = Ph::combine(axis_at(t + T * m), f);
                        if (op_v) {
                            f = Ph::combine(vph(m), f);
                            v[0][m] = Ph::apply(v[0][m], f);
                        } else {
                            v[0][m] = scale2(Ph::apply(v[0][m], f), shi, slo);
                        }
                    }
                }
            }
        } else if constexpr (NC == 4) {
            apply_op4<Real, E, T>(v, a, base, stride, t, want_v ? vt : nullptr);
        } else {
            if (a.op == OP_DV && a.rows4 != nullptr && CONTIG) {
                // A varying along x_1 (in the lattice plane): per-column merged
                // mixing a + i b.alpha + i d.Sigma with b_3 = d_1 = d_2 = 0, which
                // keeps the pairs (1,4) and (2,3); its 2x2 block on this pair is
                // [[a + i s d3, i b~], [i b~*, a - i s d3]] with s = +1, b~ = b1 - i b2
                // for (1,4) and s = -1, b~ = b1 + i b2 for (2,3).
                const Real *rows = reinterpret_cast<const Real *>(a.rows4);
                const Real sg = pz == 0 ? Real(1) : Real(-1);
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int i = t + T * m;   // x_1 column of this value
                    Real q[8];
                    dirac4_load_row(rows + (int64_t)i * 8, q);
                    const Real ar = q[0], b1 = q[1], b2 = q[2], d3 = sg * q[6];
                    const C m00 = mk<C>(ar, d3), m11 = mk<C>(ar, -d3);
                    const C m01 = mk<C>(sg * b2, b1), m10 = mk<C>(-sg * b2, b1);   // i (b1 -+ i b2)
                    C u0 = cadd(cmul(m00, v[0][m]), cmul(m01, v[1][m]));
                    C u1 = cadd(cmul(m10, v[0][m]), cmul(m11, v[1][m]));
                    if (want_v) {
                        const C vm = vph(m);
                        u0 = Ph::apply(u0, vm);
                        u1 = Ph::apply(u1, vm);
                    }
                    v[0][m] = u0;
                    v[1][m] = u1;
                }
            } else if (a.op == OP_DV) {
                // (psi_a, psi_b) <- exp(-i V tau') M (psi_a, psi_b) on this component pair
                const double *mx = a.mix[pz];
                const C m00 = mk<C>(Real(mx[0]), Real(mx[1])), m01 = mk<C>(Real(mx[2]), Real(mx[3]));
                const C m10 = mk<C>(Real(mx[4]), Real(mx[5])), m11 = mk<C>(Real(mx[6]), Real(mx[7]));
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    C u0 = cadd(cmul(m00, v[0][m]), cmul(m01, v[1][m]));
                    C u1 = cadd(cmul(m10, v[0][m]), cmul(m11, v[1][m]));
                    if (want_v) {
                        const C vm = vph(m);
                        u0 = Ph::apply(u0, vm);
                        u1 = Ph::apply(u1, vm);
                    }
                    v[0][m] = u0;
                    v[1][m] = u1;
                }
            } else {
                apply_op<Real, E, T, NC>(v, a, base, stride, t, pz, nullptr, 1);
            }
        }

        if (a.post != 0) fft_dir<C, N, E, NC, Cfg::TWM>(v, lay, t, tw, a.post, pbar);   // first writes wait inside

        if constexpr (CONTIG) {
            if constexpr (Cfg::SINGLE) {
                // Every read of the only buffer is done: fetch the next tile
                // into it while this one is stored from registers.  s_tile of
                // the next iteration was published before this barrier.
                __syncthreads();
                if (tid == 0) issue_next();
            }
            if (active) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    C *dst = pv_psi(dp) + coff[c] + base + t;
#pragma unroll
                    for (int m = 0; m < E; ++m)
                        if (SOP_IN(a.errflag, coff[c] + base + t + T * m < lat_elems(dp))) st_stream(dst + T * m, v[c][m]);
                }
            }
            if constexpr (!Cfg::SINGLE) __syncthreads();   // the tile buffer is free again; s_tile is set
        } else {
            // Back into the landing layout, then one TMA store per box (clipped at
            // the lattice edge, so inactive pencils are never written).
            __syncthreads();   // landing and exchange reads are done
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                C *col = bufc + c * N * WP + w;
#pragma unroll
                for (int m = 0; m < E; ++m)
                    if (SOP_IN(a.errflag, (c * N * WP + w + (t + T * m) * WP + 1) * CSZ <= (int)Cfg::BUF))
                        col[(t + T * m) * WP] = v[c][m];
            }
            fence_proxy_async_smem();   // make these writes visible to the bulk copy engine
            if (Cfg::SINGLE && tid == 0) publish_next();
            __syncthreads();            // also: s_tile of the next iteration is set
            if (tid == 0) {
                store_tile(tile, b);
                if constexpr (Cfg::SINGLE) {
                    bulk_wait_read();   // the store has read the only buffer
                    issue_next();
                }
            }
        }
        tile = s_tile[(it + 1) & 1];
    }
    if (!CONTIG && tid == 0) bulk_wait_all();   // the last stores are complete before the kernel ends
}

// Per-stage twiddle table of size N in global memory (lean passes), the
// layout of StageTable; one CTA fills it from the W_n table.
template <typename Real, int N, int NC>
__global__ void stage_table_kernel(void *out, const void *tw) {
    using C = cplx_t<Real>;
    StageTable<C, N, Geometry<N, NC, pass_ev<Real, N, NC>()>::E>::fill(
        reinterpret_cast<C *>(out), reinterpret_cast<const C *>(tw), (int)threadIdx.x, (int)blockDim.x);
}

// out == nullptr: the number of entries; else fill out (async on s).
template <typename Real, int N, int NC>
int stage_table_t(void *out, const void *tw, cudaStream_t s) {
    constexpr int entries = StageTable<cplx_t<Real>, N, Geometry<N, NC, pass_ev<Real, N, NC>()>::E>::ENTRIES;
    if (out != nullptr && entries > 0) stage_table_kernel<Real, N, NC><<<1, 256, 0, s>>>(out, tw);
    return entries;
}

// ---------------------------------------------------------------------------
// Launcher
// ---------------------------------------------------------------------------

cudaError_t ensure_smem_attr(const void *kern, int bytes);
cudaError_t persistent_grid(const void *kern, int threads, size_t smem, int *blocks_per_sm, int *sms);

template <typename Real, int N, int NC, bool CONTIG, int VAR = 0>
cudaError_t launch_async_t(const PassArgs &a0, const TensorMapBytes &tm, cudaStream_t s, int64_t *ctr_advance) {
    using Cfg = AsyncCfg<Real, N, NC, CONTIG, VAR>;
    if constexpr (!Cfg::FITS) {
        return cudaErrorInvalidValue;
    } else {
        PassArgs a = a0;
        // multi-instance launches: the host set n_tiles and the instance descriptors
        const bool multi = NC == 1 && a.inst != nullptr;
        if (!multi) {
            const int64_t total = (NC == 1) ? a.n_pencils * a.n_batch : a.n_pencils;
            if (CONTIG) {
                a.n_xgroups = 0;
                a.n_tiles = (total + Cfg::WP - 1) / Cfg::WP;
            } else {
                const int64_t n0 = a.dims[0];
                a.n_xgroups = (n0 + Cfg::WP - 1) / Cfg::WP;
                const int64_t others = a.n_pencils / n0;
                a.n_tiles = a.n_xgroups * others * (NC == 1 ? a.n_batch : 1);
            }
        }
        *ctr_advance = 0;
        if (a.n_tiles <= 0) return cudaSuccess;
        auto kern = pass_kernel_async<Real, N, NC, CONTIG, false, VAR>;
        if constexpr (NC == 1)
            if (multi) kern = pass_kernel_async<Real, N, NC, CONTIG, true, VAR>;
        cudaError_t e = ensure_smem_attr(reinterpret_cast<const void *>(kern), (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = persistent_grid(reinterpret_cast<const void *>(kern), Cfg::THREADS, Cfg::SMEM, &per_sm, &sms);
        if (e != cudaSuccess) return e;
        int64_t blocks = (int64_t)per_sm * sms / (NC == 2 ? 2 : 1);   // both component pairs resident
        if (blocks > a.n_tiles) blocks = a.n_tiles;
        if (blocks < 1) blocks = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)blocks, 1, NC == 2 ? 2 : 1);
        cfg.blockDim = dim3(Cfg::T, Cfg::WP, 1);
        cfg.dynamicSmemBytes = Cfg::SMEM;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, kern, a, *reinterpret_cast<const CUtensorMap *>(tm.b));
        if (e == cudaSuccess) *ctr_advance = a.n_tiles + blocks;
        return e;
    }
}

}  // namespace sop
