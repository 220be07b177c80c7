// sop_api.cu -- the sop_* C ABI: plans, table management and the split-step
// time loop of Bauke & Keitel (arXiv:1012.3911), Eq. 8.
//
// Time loop of one sop_step call with n steps (d >= 2, x = axis 0):
//   real-space index P = 0..n: pass over x with
//       [inverse FFT_x if P > 0] -> U_A1 -> [forward FFT_x if P < n]
//     where U_A1 is the half factor for P = 0 and P = n and the product of
//     the trailing half of step P-1 and the leading half of step P otherwise;
//   after every P < n, the momentum-space side of step P:
//       2D: pass over y: forward FFT_y -> U~_A2 / N -> inverse FFT_y
//       3D: forward FFT_y; pass over z: forward FFT_z -> U~_A2 / N -> inverse FFT_z;
//           inverse FFT_y
// so a 2D step costs two passes over psi and a 3D step four.  In 1D a single
// kernel keeps the line on chip for many steps.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <set>
#include <vector>

#include "sop.h"
#include "sop_internal.h"

namespace sop {

#define SOP_VAR_DECL(K)                                                                                          \
    cudaError_t launch_async_var_f32_contig_##K(const PassArgs &, int, const TensorMapBytes &, cudaStream_t,     \
                                                int64_t *);                                                      \
    cudaError_t launch_async_var_f32_strided_##K(const PassArgs &, int, const TensorMapBytes &, cudaStream_t,    \
                                                 int64_t *);
SOP_VAR_DECL(1)
SOP_VAR_DECL(2)
SOP_VAR_DECL(3)
SOP_VAR_DECL(4)
SOP_VAR_DECL(5)
SOP_VAR_DECL(6)
SOP_VAR_DECL(7)
#undef SOP_VAR_DECL

cudaError_t launch_async_variant(bool f64, bool contig, int var, const PassArgs &a, int nc, const TensorMapBytes &tmap,
                                 cudaStream_t s, int64_t *ctr_advance) {
    if (f64) return cudaErrorInvalidValue;
    switch (var) {
#define SOP_VAR_CASE(K)                                                                \
    case K:                                                                            \
        return contig ? launch_async_var_f32_contig_##K(a, nc, tmap, s, ctr_advance)   \
                      : launch_async_var_f32_strided_##K(a, nc, tmap, s, ctr_advance);
        SOP_VAR_CASE(1)
        SOP_VAR_CASE(2)
        SOP_VAR_CASE(3)
        SOP_VAR_CASE(4)
        SOP_VAR_CASE(5)
        SOP_VAR_CASE(6)
        SOP_VAR_CASE(7)
#undef SOP_VAR_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace sop

using namespace sop;
using cd = std::complex<double>;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(SOP_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int64_t kFieldChunk = 512;   // real-space indices per field-table chunk
constexpr int64_t kProfileChunk = 64;  // real-space indices per chunk of per-column mixing matrices
constexpr int kStageSlots = 8;         // pinned upload slots in flight

struct EventPair {
    cudaEvent_t a, b;
    int cls;
};

}  // namespace

struct sop_plan_s {
    int ndim = 0;
    int64_t dims[3] = {1, 1, 1};
    double h[3] = {1, 1, 1};
    int comps = 1;
    bool f64 = false;
    sop_params prm{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int64_t npts = 0;
    size_t csz = 0;

    void *psi = nullptr;
    double *V = nullptr;
    int *vbad = nullptr;            // set by the potential conversion for a non-finite value
    bool v_set = false;
    sop_plan rev = nullptr;         // same lattice, stepped with -dt (costates of sop_adjoint_gradient)
    uint64_t v_version = 0;         // count of successful sop_set_potential calls
    uint64_t rev_v_version = 0;     // the version rev's potential was copied from
    char *adj = nullptr;            // sop_adjoint_gradient buffers, kept across calls
    size_t adj_cap = 0;

    void *tw[3] = {nullptr, nullptr, nullptr};
    void *stw[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};   // per-stage tables, nc = 1, 2
    void *vhalf = nullptr, *vfull = nullptr;
    void *kin[3] = {nullptr, nullptr, nullptr};
    void *dtab = nullptr;
    void *mtab = nullptr;           // 1D Dirac: merged mixing rows of one call; Dirac with a
    size_t mtab_cap = 0;            // column-dependent A: kProfileChunk rows of per-column matrices
    bool profile = false;           // Dirac: field samples per lattice column of axis 0
    double *theta = nullptr;        // device scratch for per-axis angles
    double tables_dt = std::nan("");
    bool tables_valid = false;
    double scale_hi = 1.0, scale_lo = 0.0;

    int gauge = SOP_GAUGE_LENGTH;   // meaning of the Schroedinger field samples
    void *ftab = nullptr;           // kFieldChunk rows x row_len
    void *ftab_h = nullptr;         // half-step field rows (materialising calls): 2 x kFieldChunk x row_len
    size_t ftab_h_cap = 0;
    double *fvh = nullptr;          // their field vectors, 2 x (n+1) x ndim
    int64_t fvh_cap = 0;
    int64_t row_len = 0;
    int64_t foff[3] = {0, 0, 0};
    double *fvec = nullptr;         // device field vectors, (n+1) x ndim
    int64_t fvec_cap = 0;
    // pinned staging ring for host -> device uploads: kStageSlots slots of
    // host_stage_cap doubles; a slot is reused once its previous copy is done
    double *host_stage = nullptr;
    int64_t host_stage_cap = 0;
    cudaEvent_t stage_done[kStageSlots] = {};
    int stage_next = 0, stage_cur = 0;

    double *partial = nullptr;
    double *result = nullptr;
    double *host_result = nullptr;  // pinned, 4 doubles
    double *pgrid = nullptr;
    void *scratch = nullptr;

    int *errflag = nullptr;         // device word set by kernels whose bounded waits gave up
    unsigned long long *tile_ctr = nullptr;   // tile counters of the persistent passes (one per pair)
    unsigned long long tile_base[2] = {0, 0};   // their values at the start of the next launch
    bool async_passes = true;       // persistent passes with bulk / TMA prefetch
    int pass_var[2][2] = {{0, 0}, {0, 0}};   // launch-shape variant per axis kind (contig, strided) and nc - 1
    uint64_t wait_ns = 0;           // limit of the passes' tile-copy waits (0: the kernels' default)
    struct MapEntry {
        void *ptr;
        int axis, nc;
        TensorMapBytes map;
    };
    std::vector<MapEntry> maps;     // tensor maps of psi / scratch per strided axis

    int prof_every = 0;             // 0: off; 1: every kernel; k > 1: the passes of one split step in k
    std::vector<EventPair> events;
    std::vector<cudaEvent_t> event_pool;
    int64_t launches = 0;
};

namespace {

bool is_finite(double x) { return std::isfinite(x); }

#ifndef SOP_CHECK
#define SOP_CHECK 0
#endif
constexpr size_t kCanaryPad = 256;   // bytes after each device buffer in check builds

// Allocation-failure injection (sop_debug_fail_alloc): the number of
// device allocations still to succeed before one fails, or -1 (off).
std::atomic<int64_t> g_fail_alloc{-1};

#if SOP_CHECK
// Check builds: every device allocation carries kCanary bytes of a fixed
// pattern after its end, verified when the buffer is freed and by
// sop_debug_check_canaries; a write past the end of a buffer shows there.
constexpr size_t kCanary = kCanaryPad;
constexpr unsigned char kCanaryByte = 0xA5;
std::mutex g_canary_mu;
std::map<void *, size_t> g_canary;   // buffer -> requested bytes
std::atomic<int64_t> g_canary_bad{0};
bool canary_intact(void *p, size_t bytes) {
    unsigned char tail[kCanary];
    if (cudaMemcpy(tail, static_cast<char *>(p) + bytes, kCanary, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    for (size_t i = 0; i < kCanary; ++i)
        if (tail[i] != kCanaryByte) return false;
    return true;
}
#endif

template <typename T> int dalloc(T **p, size_t bytes, const char *what) {
    if (bytes == 0) bytes = 16;
    if (g_fail_alloc.load() >= 0 && g_fail_alloc.fetch_sub(1) == 0) {
        *p = nullptr;
        return fail(SOP_ENOMEM, std::string("cudaMalloc(") + what + "): injected allocation failure");
    }
    const size_t total = bytes + (SOP_CHECK ? kCanaryPad : 0);
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), total);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? SOP_ENOMEM : SOP_ECUDA,
                    std::string("cudaMalloc(") + what + ", " + std::to_string(bytes) + " bytes): " + cudaGetErrorString(e));
    }
#if SOP_CHECK
    e = cudaMemset(reinterpret_cast<char *>(*p) + bytes, kCanaryByte, kCanary);
    if (e != cudaSuccess) return fail(SOP_ECUDA, std::string("cudaMemset(canary of ") + what + ")");
    std::lock_guard<std::mutex> lock(g_canary_mu);
    g_canary[reinterpret_cast<void *>(*p)] = bytes;
#endif
    return SOP_OK;
}

void dfree(void *p) {
    if (!p) return;
#if SOP_CHECK
    {
        std::lock_guard<std::mutex> lock(g_canary_mu);
        auto it = g_canary.find(p);
        if (it != g_canary.end()) {
            if (!canary_intact(p, it->second)) {
                g_canary_bad.fetch_add(1);
                std::fprintf(stderr, "sop check: canary after a %zu-byte buffer overwritten\n", it->second);
            }
            g_canary.erase(it);
        }
    }
#endif
    cudaFree(p);
}

double lattice_p(int64_t n, double h, int64_t k, double hbar) {
    const int64_t kap = (2 * k < n) ? k : k - n;
    return hbar * kTwoPi * (double)kap / ((double)n * h);
}

cudaEvent_t take_event(sop_plan p) {
    if (!p->event_pool.empty()) {
        cudaEvent_t e = p->event_pool.back();
        p->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch bracket: counts launches and, when profiling and `sampled`, records events.
struct Bracket {
    sop_plan p;
    int cls;
    bool on;
    cudaEvent_t a = nullptr;
    Bracket(sop_plan pp, int c, bool sampled = true) : p(pp), cls(c), on(pp->prof_every != 0 && sampled) {
        if (on) {
            a = take_event(p);
            cudaEventRecord(a, p->stream);
        }
    }
    void done(int nlaunch = 1) {
        p->launches += nlaunch;
        if (on) {
            cudaEvent_t b = take_event(p);
            cudaEventRecord(b, p->stream);
            p->events.push_back({a, b, cls});
        }
    }
};

// A free staging slot of at least `doubles` entries; returns its address.
int ensure_stage(sop_plan p, int64_t doubles, double **slot_out) {
    if (p->host_stage_cap < doubles) {
        if (p->host_stage) {
            for (int k = 0; k < kStageSlots; ++k) cudaEventSynchronize(p->stage_done[k]);
            cudaFreeHost(p->host_stage);
            p->host_stage = nullptr;
            p->host_stage_cap = 0;
        }
        const int64_t cap = doubles < 4096 ? 4096 : doubles;
        cudaError_t e = cudaHostAlloc(reinterpret_cast<void **>(&p->host_stage),
                                      (size_t)cap * kStageSlots * sizeof(double), cudaHostAllocDefault);
        if (e != cudaSuccess) return cuda_fail(e, "cudaHostAlloc");
        p->host_stage_cap = cap;
    }
    const int k = p->stage_next;
    p->stage_next = (k + 1) % kStageSlots;
    // the copy that last read this slot (kStageSlots uploads ago) has finished
    cudaError_t e = cudaEventSynchronize(p->stage_done[k]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    *slot_out = p->host_stage + (size_t)k * p->host_stage_cap;
    p->stage_cur = k;
    return SOP_OK;
}

// Upload n doubles through the pinned staging ring to dst (async).
int upload(sop_plan p, double *dst, const double *src, int64_t n) {
    double *slot = nullptr;
    int rc = ensure_stage(p, n, &slot);
    if (rc) return rc;
    std::memcpy(slot, src, (size_t)n * sizeof(double));
    cudaError_t e = cudaMemcpyAsync(dst, slot, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(upload)");
    cudaEventRecord(p->stage_done[p->stage_cur], p->stream);
    return SOP_OK;
}

int plan_free(sop_plan p) {
    if (!p) return SOP_OK;
    cudaStreamSynchronize(p->stream);
    if (p->rev) plan_free(p->rev);
    for (int a = 0; a < 3; ++a) {
        dfree(p->tw[a]);
        dfree(p->stw[a][0]);
        dfree(p->stw[a][1]);
        dfree(p->kin[a]);
    }
    dfree(p->V);
    dfree(p->vhalf);
    dfree(p->vfull);
    dfree(p->dtab);
    dfree(p->mtab);
    dfree(p->theta);
    dfree(p->ftab);
    dfree(p->ftab_h);
    dfree(p->vbad);
    dfree(p->fvh);
    dfree(p->fvec);
    dfree(p->partial);
    dfree(p->result);
    dfree(p->pgrid);
    dfree(p->scratch);
    dfree(p->adj);
    dfree(p->errflag);
    dfree(p->tile_ctr);
    if (p->host_stage) cudaFreeHost(p->host_stage);
    if (p->host_result) cudaFreeHost(p->host_result);
    for (int k = 0; k < kStageSlots; ++k)
        if (p->stage_done[k]) cudaEventDestroy(p->stage_done[k]);
    for (auto &ep : p->events) {
        cudaEventDestroy(ep.a);
        cudaEventDestroy(ep.b);
    }
    for (auto e : p->event_pool) cudaEventDestroy(e);
    delete p;
    return SOP_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

int largest_divisor_le_host(int n, int cap) {
    int d = n < cap ? n : cap;
    while (n % d != 0) --d;
    return d;
}

// 4D (3D for 2D lattices) tensor map of an array of p->comps components over
// the lattice, in 8-byte elements (a c64 value or half a c128 value), with a
// box of the async pass's pencils-per-CTA along x, up to 256 points along the
// pass axis and one along the rest.
int tensor_map(sop_plan p, void *base, int axis, int nc, TensorMapBytes *out) {
    for (auto &m : p->maps)
        if (m.ptr == base && m.axis == axis && m.nc == nc) {
            *out = m.map;
            return SOP_OK;
        }
    auto enc = tensor_map_encoder();
    if (!enc) return fail(SOP_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const int k = p->f64 ? 2 : 1;
    const int n = (int)p->dims[axis];
    const int wp = async_pencils_per_cta(p->f64, n, nc, false);
    if (wp <= 0) return fail(SOP_EUNSUPPORTED, "no asynchronous pass for this size");
    const int rank = p->ndim + 1;
    cuuint64_t gdim[5] = {1, 1, 1, 1, 1}, gstride[4] = {0, 0, 0, 0};
    cuuint32_t box[5] = {1, 1, 1, 1, 1}, estr[5] = {1, 1, 1, 1, 1};
    gdim[0] = (cuuint64_t)p->dims[0] * k;
    box[0] = (cuuint32_t)(wp * k);
    uint64_t bytes = (uint64_t)p->dims[0] * p->csz;
    for (int d = 1; d < p->ndim; ++d) {
        gdim[d] = (cuuint64_t)p->dims[d];
        box[d] = d == axis ? (cuuint32_t)largest_divisor_le_host(n, 256) : 1;
        gstride[d - 1] = bytes;
        bytes *= (uint64_t)p->dims[d];
    }
    gdim[p->ndim] = (cuuint64_t)p->comps;
    gstride[p->ndim - 1] = bytes;
    CUtensorMap map;
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, (cuuint32_t)rank, base, gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SOP_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    sop_plan_s::MapEntry ent;
    ent.ptr = base;
    ent.axis = axis;
    ent.nc = nc;
    std::memcpy(ent.map.b, &map, sizeof(map));
    if (p->maps.size() >= 16) p->maps.erase(p->maps.begin());
    p->maps.push_back(ent);
    *out = ent.map;
    return SOP_OK;
}

// Launch one pass: the persistent asynchronous kernel when it exists for the
// size, else the one-shot kernel.  Returns a sop_status.
int launch_pass(sop_plan p, const PassArgs &a0, int nc, const char *what) {
    const bool contig = a0.axis == 0;
    if (p->async_passes) {
        PassArgs a = a0;
        a.errflag = p->errflag;
        a.wait_ns = p->wait_ns;
        a.tile_ctr = p->tile_ctr;
        a.stw = p->stw[a.axis][nc - 1];
        a.tile_base[0] = p->tile_base[0];
        a.tile_base[1] = p->tile_base[1];
        a.n_comp_total = p->comps;
        TensorMapBytes tm;
        std::memset(&tm, 0, sizeof(tm));
        const int wp = async_pencils_per_cta(p->f64, (int)p->dims[a.axis], nc, contig);
        if (wp > 0) {
            if (!contig) {
                int rc = tensor_map(p, a.psi, a.axis, nc, &tm);
                if (rc) return rc;
            }
            cudaError_t e = cudaErrorInvalidValue;
            int64_t adv = 0;
            const int var = p->pass_var[contig ? 0 : 1][nc - 1];
            if (nc == 4) {
                e = p->f64 ? (contig ? launch_async4_f64_contig(a, tm, p->stream, &adv)
                                     : launch_async4_f64_strided(a, tm, p->stream, &adv))
                           : (contig ? launch_async4_f32_contig(a, tm, p->stream, &adv)
                                     : launch_async4_f32_strided(a, tm, p->stream, &adv));
                if (e == cudaSuccess) {
                    p->tile_base[0] += (unsigned long long)adv;
                    return SOP_OK;
                }
                return cuda_fail(e, what);   // callers check fused_dirac3_ok first
            } else if (var > 0 && var < kPassVariants) {
                e = launch_async_variant(p->f64, contig, var, a, nc, tm, p->stream, &adv);
                if (e == cudaErrorInvalidValue) cudaGetLastError();   // no such variant for the size
            }
            if (e == cudaSuccess) {
            } else if (e != cudaErrorInvalidValue) {
                return cuda_fail(e, what);
            } else if (p->f64)
                e = contig ? launch_async_f64_contig(a, nc, tm, p->stream, &adv)
                           : launch_async_f64_strided(a, nc, tm, p->stream, &adv);
            else
                e = contig ? launch_async_f32_contig(a, nc, tm, p->stream, &adv)
                           : launch_async_f32_strided(a, nc, tm, p->stream, &adv);
            if (e == cudaSuccess) {
                p->tile_base[0] += (unsigned long long)adv;
                if (nc == 2) p->tile_base[1] += (unsigned long long)adv;
                return SOP_OK;
            }
            if (e != cudaErrorInvalidValue) return cuda_fail(e, what);
            cudaGetLastError();   // size without an asynchronous kernel: use the one-shot pass
        }
    }
    cudaError_t e;
    PassArgs a1 = a0;
    a1.errflag = p->errflag;   // check builds record failed index tests here
    if (p->f64) e = contig ? launch_pass_f64_contig(a1, nc, p->stream) : launch_pass_f64_strided(a1, nc, p->stream);
    else e = contig ? launch_pass_f32_contig(a1, nc, p->stream) : launch_pass_f32_strided(a1, nc, p->stream);
    return e == cudaSuccess ? SOP_OK : cuda_fail(e, what);
}

void base_args(sop_plan p, PassArgs &a, void *psi, int axis) {
    std::memset(&a, 0, sizeof(a));
    a.psi = psi;
    a.comp_stride = p->npts;
    a.n_pencils = p->npts / p->dims[axis];
    a.n_batch = 1;
    int64_t stride = 1;
    for (int b = 0; b < axis; ++b) stride *= p->dims[b];
    a.stride = stride;
    a.ndim = p->ndim;
    a.axis = axis;
    for (int b = 0; b < 3; ++b) a.dims[b] = b < p->ndim ? p->dims[b] : 1;
    a.tw = p->tw[axis];
    // strided tiles: element stride of the coordinate that is neither x nor the axis
    a.o_stride = 0;
    if (p->ndim == 3 && axis == 1) a.o_stride = p->dims[0] * p->dims[1];
    if (p->ndim == 3 && axis == 2) a.o_stride = p->dims[0];
    a.scale_hi = p->scale_hi;
    a.scale_lo = p->scale_lo;
    a.pair_comp[0][0] = 0;
    a.pair_comp[0][1] = 3;
    a.pair_comp[1][0] = 1;
    a.pair_comp[1][1] = 2;
}

// Whether the passes of split step P (index within one sop_step call) are
// timed: all of them, or with sampling every k-th one, P = k/2 mod k.
bool step_sampled(const sop_plan p, int64_t P) {
    if (p->prof_every <= 1) return true;
    return P % p->prof_every == p->prof_every / 2;
}

int run_pass(sop_plan p, const PassArgs &a, int nc, int cls, const char *what, bool sampled = true) {
    Bracket br(p, cls, sampled);
    int rc = launch_pass(p, a, nc, what);
    if (rc) return rc;
    br.done();
    return SOP_OK;
}

// SOP_ETIMEOUT if a kernel's bounded wait gave up since the last check
// (call only after synchronising the plan stream).
int check_errflag(sop_plan p) {
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, p->errflag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(error flag)");
    if (h != 0) {
        // CTAs that gave up left their tile claims unfinished: restart the counters.
        cudaMemset(p->errflag, 0, sizeof(int));
        cudaMemset(p->tile_ctr, 0, 2 * sizeof(unsigned long long));
        p->tile_base[0] = p->tile_base[1] = 0;
        if (h & 4)   // check builds only
            return fail(SOP_ECUDA, "a pass kernel's bounds or alignment check failed (access skipped; SOP_CHECK build)");
        return fail(SOP_ETIMEOUT, "a pass kernel gave up waiting for its tile copies (bounded wait)");
    }
    return SOP_OK;
}

// Rebuild the tables that depend on the time step (and V).
int ensure_tables(sop_plan p, double dt) {
    if (p->tables_valid && p->tables_dt == dt) return SOP_OK;
    const double hbar = p->prm.hbar;
    cudaError_t e;
    if (p->v_set) {
        Bracket br(p, 4);
        e = build_vphase(p->vhalf, p->V, p->npts, 0.5 * dt / hbar, p->f64, p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "build_vphase(half)");
        e = build_vphase(p->vfull, p->V, p->npts, dt / hbar, p->f64, p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "build_vphase(full)");
        br.done(2);
    }
    if (p->comps == 1) {
        // Separable kinetic factor exp(-i tau p_a^2 / (2 m hbar)) per axis (Eq. 13, A = 0).
        std::vector<double> th;
        for (int a = 0; a < p->ndim; ++a)
            for (int64_t k = 0; k < p->dims[a]; ++k) {
                const double pk = lattice_p(p->dims[a], p->h[a], k, hbar);
                th.push_back(dt * pk * pk / (2.0 * p->prm.mass * hbar));
            }
        int rc = upload(p, p->theta, th.data(), (int64_t)th.size());
        if (rc) return rc;
        Bracket br(p, 4);
        int64_t off = 0;
        for (int a = 0; a < p->ndim; ++a) {
            e = build_axis_phase(p->kin[a], p->theta + off, (int)p->dims[a], p->f64, p->stream);
            if (e != cudaSuccess) return cuda_fail(e, "build_axis_phase");
            off += p->dims[a];
        }
        br.done(p->ndim);
    } else {
        Bracket br(p, 4);
        e = p->ndim == 3 ? build_dirac3_table(p->dtab, p->dims, p->h, p->prm.mass, p->prm.c, hbar, dt, p->f64,
                                              p->stream)
                         : build_dirac_table(p->dtab, p->dims, p->h, p->prm.mass, p->prm.c, hbar, dt, p->f64,
                                             p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "build_dirac_table");
        br.done();
    }
    p->tables_dt = dt;
    p->tables_valid = true;
    return SOP_OK;
}

// 2x2 blocks of the half-step spinor-mixing factor (Eq. 26 with delta = 1/2,
// Abar = A tau) on the component pairs (1,4) and (2,3) of a 2D spinor:
//   R = cos(theta) + i sin(theta) sum_i n_i alpha_i,  theta = q c |A| tau / (2 hbar),
// where sum_i n_i alpha_i is [[0, n_x - i n_y],[n_x + i n_y, 0]] on (1,4) and
// [[0, n_x + i n_y],[n_x - i n_y, 0]] on (2,3).
void mixing_blocks(const sop_plan p, const double *A, double dt, cd R[2][2][2]) {
    double ax = 0, ay = 0;
    if (A) {
        ax = A[0] * dt;
        ay = A[1] * dt;
    }
    const double amag = std::sqrt(ax * ax + ay * ay);
    const double theta = 0.5 * p->prm.charge * p->prm.c * amag / p->prm.hbar;
    const double co = std::cos(theta), si = std::sin(theta);
    const double nx = amag > 0 ? ax / amag : 0.0, ny = amag > 0 ? ay / amag : 0.0;
    const cd I(0, 1);
    for (int pr = 0; pr < 2; ++pr) {
        const cd up = pr == 0 ? cd(nx, -ny) : cd(nx, ny);
        const cd lo = pr == 0 ? cd(nx, ny) : cd(nx, -ny);
        R[pr][0][0] = co;
        R[pr][0][1] = I * si * up;
        R[pr][1][0] = I * si * lo;
        R[pr][1][1] = co;
    }
}

// Laser rows of a Schroedinger call: which axes carry a field, where each
// axis starts in a row of the field tables, the row length.
struct FieldRows {
    int active[3] = {0, 0, 0};
    bool any = false;
    int64_t offs[3] = {0, 0, 0};
    int64_t row_len = 0;
};

// Field vectors of n steps, uploaded to p->fvec and turned into rows per
// chunk.  Length gauge: the real-space factors' f_P = -q tau/(2 hbar)
// (E_{P-1} + E_P) for P = 0..n (the laser part of exp(-i tau W/(2 hbar)) of
// both adjacent half steps; build_field_tables).  Velocity gauge: the
// kinetic factors' momentum shifts s_P = q A_P for P = 0..n-1
// (build_kin_field_tables).
int prepare_fields(sop_plan p, int64_t n, double dt, const double *field, FieldRows &fr) {
    const int nd = p->ndim;
    auto sample = [&](int64_t s, int a) -> double {
        return (field && s >= 0 && s < n) ? field[s * nd + a] : 0.0;
    };
    if (field)
        for (int64_t s = 0; s < n; ++s)
            for (int a = 0; a < nd; ++a)
                if (field[s * nd + a] != 0.0) fr.active[a] = 1;
    fr.any = fr.active[0] || fr.active[1] || fr.active[2];
    if (fr.any) {
        if (p->fvec_cap < (n + 1) * nd) {
            cudaStreamSynchronize(p->stream);
            dfree(p->fvec);
            p->fvec = nullptr;
            p->fvec_cap = 0;
            int rc = dalloc(&p->fvec, (size_t)(n + 1) * nd * sizeof(double), "field vectors");
            if (rc) return rc;
            p->fvec_cap = (n + 1) * nd;
        }
        std::vector<double> fv((size_t)(n + 1) * nd);
        if (p->gauge == SOP_GAUGE_VELOCITY) {
            // momentum shifts s_P = q A_P of the kinetic factors, P = 0..n-1
            for (int64_t P = 0; P <= n; ++P)
                for (int a = 0; a < nd; ++a) fv[P * nd + a] = p->prm.charge * sample(P, a);
        } else {
            const double k = -p->prm.charge * dt / (2.0 * p->prm.hbar);
            for (int64_t P = 0; P <= n; ++P)
                for (int a = 0; a < nd; ++a) fv[P * nd + a] = k * (sample(P - 1, a) + sample(P, a));
        }
        int rc = upload(p, p->fvec, fv.data(), (int64_t)fv.size());
        if (rc) return rc;
    }
    for (int a = 0; a < nd; ++a)
        if (fr.active[a]) {
            fr.offs[a] = fr.row_len;
            fr.row_len += p->dims[a];
        }
    return SOP_OK;
}

// Field sample a of step s of a call of n steps (0 outside the call or
// without a field).
double field_sample(const double *field, int64_t n, int nd, int64_t s, int a) {
    return (field && s >= 0 && s < n) ? field[s * nd + a] : 0.0;
}

// Dirac with a vector potential that varies along x_1: the call's samples
// (n x dims[0] x ndim) go to the device once, and room for kProfileChunk rows
// of per-column mixing is reserved.
int prepare_profile(sop_plan p, int64_t n, const double *field) {
    const int64_t nx = p->dims[0];
    const int64_t cnt = n * nx * p->ndim;
    int rc = SOP_OK;
    if (p->fvec_cap < cnt) {
        cudaStreamSynchronize(p->stream);
        dfree(p->fvec);
        p->fvec = nullptr;
        p->fvec_cap = 0;
        rc = dalloc(&p->fvec, (size_t)cnt * sizeof(double), "field samples");
        if (rc) return rc;
        p->fvec_cap = cnt;
    }
    rc = upload(p, p->fvec, field, cnt);
    if (rc) return rc;
    const size_t need = (size_t)kProfileChunk * nx * 4 * p->csz;   // 8 reals per column
    if (p->mtab_cap < need) {
        cudaStreamSynchronize(p->stream);
        dfree(p->mtab);
        p->mtab = nullptr;
        p->mtab_cap = 0;
        rc = dalloc(&p->mtab, need, "mixing matrices");
        if (rc) return rc;
        p->mtab_cap = need;
    }
    return SOP_OK;
}

// Per-column merged mixing of rows P0 .. P1-1 into p->mtab (profile_row reads it).
int profile_rows(sop_plan p, int64_t n, double dt, int64_t P0, int64_t P1) {
    const int64_t nx = p->dims[0];
    const int nd = p->ndim;
    const double hbar = p->prm.hbar;
    Bracket br(p, 4);
    cudaError_t e = build_mix_rows(p->mtab, p->fvec, P0, P1 - P0, nx, nd, n, p->prm.charge, p->prm.c, hbar, dt,
                                   p->f64, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "mixing matrices");
    br.done();
    return SOP_OK;
}

const void *profile_row(sop_plan p, int64_t P, int64_t P0) {
    return static_cast<const char *>(p->mtab) + (size_t)(P - P0) * p->dims[0] * 4 * p->csz;
}

// Dirac, 2D, vector potential varying along x_1.
int step_dirac2d_profile(sop_plan p, int64_t n, double dt) {
    const int64_t nx = p->dims[0];
    int rc = SOP_OK;
    if (p->async_passes && async_pencils_per_cta(p->f64, (int)nx, 2, true) > 0) {
        // A in the lattice plane keeps the component pairs (1,4) and (2,3)
        // (b_3 = d_1 = d_2 = 0 in every merged mixing), so the per-column
        // mixing runs inside the x pass of the pairs, as the uniform mixing
        // does: two passes per step.
        for (int64_t P0 = 0; P0 <= n; P0 += kProfileChunk) {
            const int64_t P1 = std::min<int64_t>(n + 1, P0 + kProfileChunk);
            if ((rc = profile_rows(p, n, dt, P0, P1))) return rc;
            for (int64_t P = P0; P < P1; ++P) {
                const bool smp = step_sampled(p, P);
                PassArgs a;
                base_args(p, a, p->psi, 0);
                a.pre = P > 0 ? +1 : 0;
                a.post = P < n ? -1 : 0;
                a.op = OP_DV;
                a.vtab = p->v_set ? ((P == 0 || P == n) ? p->vhalf : p->vfull) : nullptr;
                a.rows4 = profile_row(p, P, P0);
                if ((rc = run_pass(p, a, 2, 0, "Dirac real-space pass", smp))) return rc;
                if (P == n) break;
                PassArgs k;
                base_args(p, k, p->psi, 1);
                k.pre = -1;
                k.post = +1;
                k.op = OP_DT;
                k.dtab = p->dtab;
                if ((rc = run_pass(p, k, 2, 1, "Dirac momentum-space pass", smp))) return rc;
            }
        }
        return SOP_OK;
    }
    // ---- Dirac, 2D, column-dependent A: the mixing runs as its own
    // streaming pass between the x transforms of the four components;
    // the momentum-space factor stays fused in the y pass of the pairs.
    for (int64_t P0 = 0; P0 <= n; P0 += kProfileChunk) {
        const int64_t P1 = std::min<int64_t>(n + 1, P0 + kProfileChunk);
        if ((rc = profile_rows(p, n, dt, P0, P1))) return rc;
        for (int64_t P = P0; P < P1; ++P) {
            const bool smp = step_sampled(p, P);
            if (P > 0) {
                PassArgs a;
                base_args(p, a, p->psi, 0);
                a.n_batch = 4;
                a.pre = +1;
                a.op = OP_NONE;
                if ((rc = run_pass(p, a, 1, 2, "Dirac inverse x transform", smp))) return rc;
            }
            {
                Bracket br(p, 0, smp);
                cudaError_t e = launch_dirac3_real(p->psi, p->npts,
                                                   p->v_set ? ((P == 0 || P == n) ? p->vhalf : p->vfull) : nullptr,
                                                   nullptr, profile_row(p, P, P0), nx, p->f64, p->stream);
                if (e != cudaSuccess) return cuda_fail(e, "Dirac real-space factor");
                br.done();
            }
            if (P == n) break;
            PassArgs a;
            base_args(p, a, p->psi, 0);
            a.n_batch = 4;
            a.pre = -1;
            a.op = OP_NONE;
            if ((rc = run_pass(p, a, 1, 2, "Dirac forward x transform", smp))) return rc;
            PassArgs k;
            base_args(p, k, p->psi, 1);
            k.pre = -1;
            k.post = +1;
            k.op = OP_DT;
            k.dtab = p->dtab;
            if ((rc = run_pass(p, k, 2, 1, "Dirac momentum-space pass", smp))) return rc;
        }
    }
    return SOP_OK;
}

// Dirac, 1D, two components.
int step_dirac1d(sop_plan p, int64_t n, double dt, const double *field) {
    const double hbar = p->prm.hbar;
    int rc = SOP_OK;
    // ---- Dirac, 1D, two components: whole steps on chip ----------------
    // merged mixing M_P = R(A_P) R(A_{P-1}), R(A) = cos th + i sin th sigma_x,
    // th = q c A tau / (2 hbar) (the half-step factor; A = 0 beyond the call)
    auto R = [&](int64_t s, cd M[2][2]) {
        const double th = (field && s >= 0 && s < n) ? 0.5 * p->prm.charge * p->prm.c * field[s] * dt / hbar : 0.0;
        M[0][0] = M[1][1] = std::cos(th);
        M[0][1] = M[1][0] = cd(0.0, std::sin(th));
    };
    const size_t row_bytes = 4 * p->csz;
    const size_t bytes = (size_t)(n + 1) * row_bytes;
    if (p->mtab_cap < bytes) {
        cudaStreamSynchronize(p->stream);
        dfree(p->mtab);
        p->mtab = nullptr;
        p->mtab_cap = 0;
        rc = dalloc(&p->mtab, bytes, "Dirac mixing rows");
        if (rc) return rc;
        p->mtab_cap = bytes;
    }
    std::vector<double> packed(bytes / sizeof(double));
    for (int64_t P = 0; P <= n; ++P) {
        cd Rn[2][2], Rp[2][2];
        R(P, Rn);
        R(P - 1, Rp);
        cd M[4];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) M[2 * i + j] = Rn[i][0] * Rp[0][j] + Rn[i][1] * Rp[1][j];
        for (int q = 0; q < 4; ++q) {
            if (p->f64) {
                packed[(size_t)P * 8 + 2 * q] = M[q].real();
                packed[(size_t)P * 8 + 2 * q + 1] = M[q].imag();
            } else {
                float *f = reinterpret_cast<float *>(packed.data() + (size_t)P * 4);
                f[2 * q] = (float)M[q].real();
                f[2 * q + 1] = (float)M[q].imag();
            }
        }
    }
    rc = upload(p, static_cast<double *>(p->mtab), packed.data(), (int64_t)packed.size());
    if (rc) return rc;
    Args1D a1{};
    a1.psi = p->psi;
    a1.n_rows = 1;
    a1.n_steps = n;
    a1.p_begin = 0;
    a1.p_end = n + 1;
    a1.p_table0 = 0;
    a1.tw = p->tw[0];
    a1.vhalf = p->v_set ? p->vhalf : nullptr;
    a1.vfull = p->v_set ? p->vfull : nullptr;
    a1.mtab = p->mtab;
    a1.dtab = p->dtab;
    a1.scale_hi = p->scale_hi;
    a1.scale_lo = p->scale_lo;
    Bracket br(p, 3);
    cudaError_t e = p->f64 ? launch_1d_dirac_f64(a1, (int)p->dims[0], p->stream)
                           : launch_1d_dirac_f32(a1, (int)p->dims[0], p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "1D Dirac step kernel");
    br.done();
    return SOP_OK;
}

// Dirac, 3D, four components; prof: per-column mixing rows instead of a uniform A.
int step_dirac3d(sop_plan p, int64_t n, double dt, const double *field, bool prof) {
    const int64_t nx = p->dims[0];
    const double hbar = p->prm.hbar;
    int rc = SOP_OK;
    // ---- Dirac, 3D: the 4x4 factors couple all components ---------------
    // Per real-space index P: exp(-i V tau') M_P with M_P = R(A_P) R(A_{P-1}),
    // then (P < n) the forward transforms of all four components along x,
    // y, z, the momentum-space factor, the inverse transforms.
    cd al[3][4][4];
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) al[a][i][j] = 0.0;
    al[0][0][3] = al[0][1][2] = al[0][2][1] = al[0][3][0] = 1.0;   // alpha_1 (Dirac representation)
    al[1][0][3] = cd(0, -1);                                        // alpha_2
    al[1][1][2] = cd(0, 1);
    al[1][2][1] = cd(0, -1);
    al[1][3][0] = cd(0, 1);
    al[2][0][2] = 1.0;                                              // alpha_3
    al[2][1][3] = -1.0;
    al[2][2][0] = 1.0;
    al[2][3][1] = -1.0;
    // R(A) = cos th + i sin th sum_a (Abar_a/Abar) alpha_a with Abar_a = A_a tau and
    // th = q c Abar / (2 hbar) (Eq. 26 with delta = 1/2; identity for A = 0)
    auto R = [&](int64_t s, cd M[4][4]) {
        double Ab[3] = {0, 0, 0}, mag = 0.0;
        for (int a = 0; a < 3; ++a) {
            Ab[a] = prof ? 0.0 : field_sample(field, n, 3, s, a) * dt;   // (per-column: profile_rows)
            mag += Ab[a] * Ab[a];
        }
        mag = std::sqrt(mag);
        const double th = 0.5 * p->prm.charge * p->prm.c * mag / hbar;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                cd v = (i == j) ? cd(std::cos(th), 0.0) : cd(0.0, 0.0);
                if (mag > 0)
                    for (int a = 0; a < 3; ++a) v += cd(0.0, std::sin(th)) * (Ab[a] / mag) * al[a][i][j];
                M[i][j] = v;
            }
    };
    // Fused form (four passes per step, 4x4 factors inside the x and z passes)
    // where the four-component passes exist for the x and z sides; else the
    // transforms run as batched passes with the factors as streaming passes.
    const bool fused = p->async_passes && async_pencils_per_cta(p->f64, (int)p->dims[0], 4, true) > 0 &&
                       async_pencils_per_cta(p->f64, (int)p->dims[2], 4, false) > 0;
    int64_t P0 = 0;
    for (int64_t P = 0; P <= n; ++P) {
        if (prof && (P - P0 == kProfileChunk || P == 0)) {
            P0 = P;
            if ((rc = profile_rows(p, n, dt, P0, std::min<int64_t>(n + 1, P0 + kProfileChunk)))) return rc;
        }
        cd Rn[4][4], Rp[4][4];
        R(P, Rn);
        R(P - 1, Rp);
        double Md[32];
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                cd v = 0.0;
                for (int k = 0; k < 4; ++k) v += Rn[i][k] * Rp[k][j];
                Md[2 * (4 * i + j)] = v.real();
                Md[2 * (4 * i + j) + 1] = v.imag();
            }
        const bool smp = step_sampled(p, P);
        if (fused) {
            // x pass with all four components: [inverse FFT_x] -> exp(-i V tau') M_P -> [FFT_x]
            PassArgs a;
            base_args(p, a, p->psi, 0);
            a.pre = P > 0 ? +1 : 0;
            a.post = P < n ? -1 : 0;
            a.op = OP_D3V;
            a.vtab = p->v_set ? ((P == 0 || P == n) ? p->vhalf : p->vfull) : nullptr;
            if (prof) a.rows4 = profile_row(p, P, P0);
            else std::memcpy(a.mix4, Md, sizeof(Md));
            rc = run_pass(p, a, 4, 0, "3D Dirac real-space pass", smp);
            if (rc) return rc;
            if (P == n) break;
            // y: forward transforms of the four components (a batch)
            base_args(p, a, p->psi, 1);
            a.n_batch = 4;
            a.pre = -1;
            a.op = OP_NONE;
            rc = run_pass(p, a, 1, 2, "3D Dirac forward transform", smp);
            if (rc) return rc;
            // z pass with all four components: FFT_z -> U~ and 1/N -> inverse FFT_z
            base_args(p, a, p->psi, 2);
            a.pre = -1;
            a.post = +1;
            a.op = OP_D3T;
            a.dtab = p->dtab;
            rc = run_pass(p, a, 4, 1, "3D Dirac momentum-space pass", smp);
            if (rc) return rc;
            // y: inverse transforms
            base_args(p, a, p->psi, 1);
            a.n_batch = 4;
            a.pre = +1;
            a.op = OP_NONE;
            rc = run_pass(p, a, 1, 2, "3D Dirac inverse transform", smp);
            if (rc) return rc;
            continue;
        }
        {
            Bracket br(p, 0, smp);
            cudaError_t e = launch_dirac3_real(p->psi, p->npts, p->v_set ? ((P == 0 || P == n) ? p->vhalf : p->vfull)
                                                                         : nullptr,
                                               prof ? nullptr : Md, prof ? profile_row(p, P, P0) : nullptr, nx, p->f64,
                                               p->stream);
            if (e != cudaSuccess) return cuda_fail(e, "3D Dirac real-space factor");
            br.done();
        }
        if (P == n) break;
        for (int ax = 0; ax < 3; ++ax) {
            PassArgs a;
            base_args(p, a, p->psi, ax);
            a.n_batch = 4;
            a.pre = -1;
            a.op = OP_NONE;
            rc = run_pass(p, a, 1, 2, "3D Dirac forward transform", smp);
            if (rc) return rc;
        }
        {
            Bracket br(p, 1, smp);
            cudaError_t e = launch_dirac3_kinetic(p->psi, p->npts, p->dtab, p->scale_hi, p->scale_lo, p->f64,
                                                  p->stream);
            if (e != cudaSuccess) return cuda_fail(e, "3D Dirac momentum-space factor");
            br.done();
        }
        for (int ax = 2; ax >= 0; --ax) {
            PassArgs a;
            base_args(p, a, p->psi, ax);
            a.n_batch = 4;
            a.pre = +1;
            a.op = OP_NONE;
            rc = run_pass(p, a, 1, 2, "3D Dirac inverse transform", smp);
            if (rc) return rc;
        }
    }
    return SOP_OK;
}

// Dirac, 2D, four components as the component pairs (1,4) and (2,3).
int step_dirac2d(sop_plan p, int64_t n, double dt, const double *field) {
    int rc = SOP_OK;
    // ---- Dirac, 2D, component pairs ------------------------------------
    for (int64_t P = 0; P <= n; ++P) {
        PassArgs a;
        base_args(p, a, p->psi, 0);
        a.pre = P > 0 ? +1 : 0;
        a.post = P < n ? -1 : 0;
        a.op = OP_DV;
        a.vtab = p->v_set ? ((P == 0 || P == n) ? p->vhalf : p->vfull) : nullptr;
        cd Rn[2][2][2], Rp[2][2][2];
        double An[2] = {field_sample(field, n, 2, P, 0), field_sample(field, n, 2, P, 1)};
        double Ap[2] = {field_sample(field, n, 2, P - 1, 0), field_sample(field, n, 2, P - 1, 1)};
        mixing_blocks(p, (field && P < n) ? An : nullptr, dt, Rn);
        mixing_blocks(p, (field && P > 0) ? Ap : nullptr, dt, Rp);
        for (int pr = 0; pr < 2; ++pr) {
            // M = R(A_P) R(A_{P-1}): trailing half of step P-1 first.
            cd M[2][2];
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) M[i][j] = Rn[pr][i][0] * Rp[pr][0][j] + Rn[pr][i][1] * Rp[pr][1][j];
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    a.mix[pr][2 * (2 * i + j)] = M[i][j].real();
                    a.mix[pr][2 * (2 * i + j) + 1] = M[i][j].imag();
                }
        }
        rc = run_pass(p, a, 2, 0, "Dirac real-space pass", step_sampled(p, P));
        if (rc) return rc;
        if (P < n) {
            PassArgs k;
            base_args(p, k, p->psi, 1);
            k.pre = -1;
            k.post = +1;
            k.op = OP_DT;
            k.dtab = p->dtab;
            rc = run_pass(p, k, 2, 1, "Dirac momentum-space pass", step_sampled(p, P));
            if (rc) return rc;
        }
    }
    return SOP_OK;
}

// Schroedinger, 1D/2D/3D, length or velocity gauge.
// mat_base != null (length gauge, ndim >= 2): the state after each step P of
// 1 .. n-1 is also written to mat_base + P mat_stride bytes (the real-space
// pass of index P applies the two half factors separately and stores the
// state between them).
int step_schrodinger(sop_plan p, int64_t n, double dt, const double *field, void *mat_base = nullptr,
                     int64_t mat_stride = 0) {
    const int nd = p->ndim;
    int rc = SOP_OK;
    FieldRows fr;
    rc = prepare_fields(p, n, dt, field, fr);
    if (rc) return rc;
    const bool mat = mat_base != nullptr && nd >= 2 && p->gauge == SOP_GAUGE_LENGTH;
    if (mat && fr.any) {
        // field vectors of the two halves met at P: k f_{P-1} and k f_P
        const double kf = -p->prm.charge * dt / (2.0 * p->prm.hbar);
        const int64_t need = 2 * (n + 1) * nd;
        if (p->fvh_cap < need) {
            cudaStreamSynchronize(p->stream);
            dfree(p->fvh);
            p->fvh = nullptr;
            p->fvh_cap = 0;
            if ((rc = dalloc(&p->fvh, (size_t)need * sizeof(double), "half-step field vectors"))) return rc;
            p->fvh_cap = need;
        }
        std::vector<double> fv((size_t)need);
        for (int64_t P = 0; P <= n; ++P)
            for (int a = 0; a < nd; ++a) {
                fv[P * nd + a] = kf * field_sample(field, n, nd, P - 1, a);
                fv[(n + 1) * nd + P * nd + a] = kf * field_sample(field, n, nd, P, a);
            }
        if ((rc = upload(p, p->fvh, fv.data(), need))) return rc;
        const size_t bytes = (size_t)2 * kFieldChunk * fr.row_len * p->csz;
        if (p->ftab_h_cap < bytes) {
            cudaStreamSynchronize(p->stream);
            dfree(p->ftab_h);
            p->ftab_h = nullptr;
            p->ftab_h_cap = 0;
            if ((rc = dalloc(&p->ftab_h, bytes, "half-step field tables"))) return rc;
            p->ftab_h_cap = bytes;
        }
    }
    const int *active = fr.active;
    const bool any_field = fr.any;
    const int64_t *offs = fr.offs;
    const int64_t row_len = fr.row_len;

    // the field enters the real-space factors (length gauge) or the kinetic
    // factors (velocity gauge)
    const bool vel = p->gauge == SOP_GAUGE_VELOCITY;
    const bool rfield = any_field && !vel, kfield = any_field && vel;
    for (int64_t P0 = 0; P0 <= n; P0 += kFieldChunk) {
        const int64_t P1 = std::min<int64_t>(n + 1, P0 + kFieldChunk);
        if (any_field) {
            Bracket br(p, 4);
            cudaError_t e = vel ? build_kin_field_tables(p->ftab, p->fvec + P0 * nd, std::min(P1, n) - P0, nd, p->dims,
                                                         p->h, active, offs, row_len,
                                                         dt / (2.0 * p->prm.mass * p->prm.hbar), p->prm.hbar, p->f64,
                                                         p->stream)
                                : build_field_tables(p->ftab, p->fvec + P0 * nd, P1 - P0, nd, p->dims, p->h, active,
                                                     offs, row_len, p->f64, p->stream);
            if (e != cudaSuccess) return cuda_fail(e, "field tables");
            if (mat) {
                char *h = static_cast<char *>(p->ftab_h);
                e = build_field_tables(h, p->fvh + P0 * nd, P1 - P0, nd, p->dims, p->h, active, offs, row_len, p->f64,
                                       p->stream);
                if (e == cudaSuccess)
                    e = build_field_tables(h + (size_t)kFieldChunk * row_len * p->csz, p->fvh + (n + 1 + P0) * nd,
                                           P1 - P0, nd, p->dims, p->h, active, offs, row_len, p->f64, p->stream);
                if (e != cudaSuccess) return cuda_fail(e, "half-step field tables");
            }
            br.done();
        }
        auto frow = [&](int64_t P, int a) -> const void * {
            if (!rfield || !active[a]) return nullptr;
            return static_cast<const char *>(p->ftab) + ((P - P0) * row_len + offs[a]) * p->csz;
        };
        auto hrow = [&](int half, int64_t P, int a) -> const void * {   // half 0: k f_{P-1}, 1: k f_P
            if (!rfield || !active[a]) return nullptr;
            return static_cast<const char *>(p->ftab_h) +
                   (((size_t)half * kFieldChunk + (P - P0)) * row_len + offs[a]) * p->csz;
        };
        auto krow = [&](int64_t P, int a) -> const void * {
            if (!kfield || !active[a]) return p->kin[a];
            return static_cast<const char *>(p->ftab) + ((P - P0) * row_len + offs[a]) * p->csz;
        };
        if (nd == 1) {
            Args1D a1{};
            a1.psi = p->psi;
            a1.n_rows = 1;
            a1.n_steps = n;
            a1.p_begin = P0;
            a1.p_end = P1;
            a1.p_table0 = P0;
            a1.tw = p->tw[0];
            a1.vhalf = p->v_set ? p->vhalf : nullptr;
            a1.vfull = p->v_set ? p->vfull : nullptr;
            a1.ftab = rfield ? p->ftab : nullptr;
            a1.ttab = kfield ? p->ftab : p->kin[0];
            a1.ttab_stride = kfield ? row_len : 0;
            a1.scale_hi = p->scale_hi;
            a1.scale_lo = p->scale_lo;
            Bracket br(p, 3);
            cudaError_t e = p->f64 ? launch_1d_f64(a1, (int)p->dims[0], p->stream)
                                   : launch_1d_f32(a1, (int)p->dims[0], p->stream);
            if (e != cudaSuccess) return cuda_fail(e, "1D step kernel");
            br.done();
            continue;
        }
        for (int64_t P = P0; P < P1; ++P) {
            PassArgs a;
            base_args(p, a, p->psi, 0);
            a.pre = P > 0 ? +1 : 0;
            a.post = P < n ? -1 : 0;
            a.op = OP_V;
            a.vtab = p->v_set ? ((P == 0 || P == n) ? p->vhalf : p->vfull) : nullptr;
            for (int ax = 0; ax < nd; ++ax) a.ftab[ax] = frow(P, ax);
            if (mat && P > 0 && P < n) {
                a.mat_out = static_cast<char *>(mat_base) + P * mat_stride;
                a.vtab = p->v_set ? p->vhalf : nullptr;
                for (int ax = 0; ax < nd; ++ax) {
                    a.ftab[ax] = hrow(0, P, ax);
                    a.fh2[ax] = hrow(1, P, ax);
                }
            }
            const bool smp = step_sampled(p, P);
            rc = run_pass(p, a, 1, 0, "real-space pass", smp);
            if (rc) return rc;
            if (P == n) break;
            if (nd == 2) {
                PassArgs k;
                base_args(p, k, p->psi, 1);
                k.pre = -1;
                k.post = +1;
                k.op = OP_T;
                for (int ax = 0; ax < nd; ++ax) k.ttab[ax] = krow(P, ax);
                rc = run_pass(p, k, 1, 1, "momentum-space pass", smp);
                if (rc) return rc;
            } else {
                PassArgs y;
                base_args(p, y, p->psi, 1);
                y.pre = -1;
                y.op = OP_NONE;
                rc = run_pass(p, y, 1, 2, "forward middle-axis pass", smp);
                if (rc) return rc;
                PassArgs k;
                base_args(p, k, p->psi, 2);
                k.pre = -1;
                k.post = +1;
                k.op = OP_T;
                for (int ax = 0; ax < nd; ++ax) k.ttab[ax] = krow(P, ax);
                rc = run_pass(p, k, 1, 1, "momentum-space pass", smp);
                if (rc) return rc;
                y.pre = +1;
                rc = run_pass(p, y, 1, 2, "inverse middle-axis pass", smp);
                if (rc) return rc;
            }
        }
    }
    return SOP_OK;
}

int step_impl(sop_plan p, int64_t n, double dt, const double *field) {
    if (!p) return fail(SOP_EINVAL, "sop_step: null plan");
    if (!p->psi) return fail(SOP_ESTATE, "sop_step: no state bound (call sop_bind_state first)");
    if (n < 0) return fail(SOP_EINVAL, "sop_step: n_steps < 0");
    if (!is_finite(dt)) return fail(SOP_EINVAL, "sop_step: dt is not finite");
    if (n == 0) return SOP_OK;
    const int64_t per_step = (int64_t)p->ndim * (p->profile ? p->dims[0] : 1);   // samples per step
    if (field)
        for (int64_t i = 0; i < n * per_step; ++i)
            if (!is_finite(field[i])) return fail(SOP_EINVAL, "sop_step: field sample is not finite");
    int rc = ensure_tables(p, dt);
    if (rc) return rc;
    const bool prof = p->comps == 4 && p->profile && field;
    if (prof && (rc = prepare_profile(p, n, field))) return rc;
    if (p->comps == 2) return step_dirac1d(p, n, dt, field);
    if (p->comps == 4 && p->ndim == 3) return step_dirac3d(p, n, dt, field, prof);
    if (p->comps == 4) return prof ? step_dirac2d_profile(p, n, dt) : step_dirac2d(p, n, dt, field);
    return step_schrodinger(p, n, dt, field);
}

// A Schroedinger step sequence (length gauge, ndim >= 2) that also writes the
// state after each step P = 1 .. n-1 to mat_base + P mat_stride bytes.
int step_impl_mat(sop_plan p, int64_t n, double dt, const double *field, void *mat_base, int64_t mat_stride) {
    if (n <= 0) return SOP_OK;
    int rc = ensure_tables(p, dt);
    if (rc) return rc;
    return step_schrodinger(p, n, dt, field, mat_base, mat_stride);
}

int read_result(sop_plan p, int count, double *out) {
    cudaError_t e = cudaMemcpyAsync(p->host_result, p->result, count * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(result)");
    e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    for (int i = 0; i < count; ++i) out[i] = p->host_result[i];
    return check_errflag(p);
}

}  // namespace

namespace sop {
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace sop

extern "C" {

int sop_version(void) { return 1; }

const char *sop_last_error(void) { return g_err.c_str(); }

int sop_plan_create(sop_plan *out, int ndim, const int64_t *dims, const double *spacing, int components, int dtype,
                    const sop_params *params, void *cuda_stream) {
    if (!out) return fail(SOP_EINVAL, "sop_plan_create: out is NULL");
    *out = nullptr;
    if (!dims || !spacing) return fail(SOP_EINVAL, "sop_plan_create: dims or spacing is NULL");
    if (ndim < 1 || ndim > 3) return fail(SOP_EINVAL, "sop_plan_create: ndim must be 1, 2 or 3");
    if (dtype != SOP_C64 && dtype != SOP_C128) return fail(SOP_EINVAL, "sop_plan_create: dtype must be SOP_C64 or SOP_C128");
    if (components != 1 && components != 2 && components != 4)
        return fail(SOP_EINVAL, "sop_plan_create: components must be 1, 2 or 4");
    for (int a = 0; a < ndim; ++a) {
        if (dims[a] <= 0) return fail(SOP_EINVAL, "sop_plan_create: dims must be positive");
        if (!(spacing[a] > 0) || !is_finite(spacing[a])) return fail(SOP_EINVAL, "sop_plan_create: spacing must be finite and > 0");
        if (!size_supported(dims[a]))
            return fail(SOP_EUNSUPPORTED, "sop_plan_create: side " + std::to_string(dims[a]) +
                                              " is not 2^a*3^b with a>=2, b<=1, 8<=n<=4096");
    }
    if (components == 4 && ndim == 1)
        return fail(SOP_EUNSUPPORTED, "sop_plan_create: the four-component Dirac path needs ndim = 2 or 3");
    if (components == 2 && ndim != 1)
        return fail(SOP_EUNSUPPORTED, "sop_plan_create: the two-component Dirac path is one-dimensional");
    sop_params prm{1.0, -1.0, 1.0, 137.036};
    if (params) prm = *params;
    if (!(prm.mass > 0) || !(prm.hbar > 0) || !(prm.c > 0) || !is_finite(prm.charge))
        return fail(SOP_EINVAL, "sop_plan_create: mass, hbar and c must be > 0 and charge finite");

    sop_plan p = new sop_plan_s();
    p->ndim = ndim;
    for (int a = 0; a < ndim; ++a) {
        p->dims[a] = dims[a];
        p->h[a] = spacing[a];
    }
    p->comps = components;
    p->f64 = dtype == SOP_C128;
    p->prm = prm;
    p->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    p->csz = p->f64 ? 16 : 8;
    {
        // "C,S": launch-shape variants of the contiguous and strided passes
        // (both component counts) instead of the default shape
        const char *env = std::getenv("SOP_PASS_SHAPE");
        int vc = 0, vs = 0;
        if (env && std::sscanf(env, "%d,%d", &vc, &vs) == 2 && vc >= 0 && vc < kPassVariants && vs >= 0 &&
            vs < kPassVariants)
            for (int nc = 0; nc < 2; ++nc) {
                p->pass_var[0][nc] = vc;
                p->pass_var[1][nc] = vs;
            }
    }
    {
        const char *env = std::getenv("SOP_PASSES");   // "sync": one-shot passes (for comparisons)
        p->async_passes = !(env && std::string(env) == "sync");
    }
    p->npts = 1;
    for (int a = 0; a < ndim; ++a) p->npts *= dims[a];
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        plan_free(p);
        return cuda_fail(e, "cudaGetDevice");
    }
    // 1/N as hi + lo in the working precision.
    {
        const double inv = 1.0 / (double)p->npts;
        if (p->f64) {
            p->scale_hi = inv;
            p->scale_lo = 0.0;
        } else {
            const float hi = (float)inv;
            p->scale_hi = hi;
            p->scale_lo = (double)(float)(inv - (double)hi);
        }
    }
    int rc = SOP_OK;
    int64_t sum_n = 0;
    for (int a = 0; a < ndim; ++a) sum_n += dims[a];
    for (int k = 0; k < kStageSlots && e == cudaSuccess; ++k)
        e = cudaEventCreateWithFlags(&p->stage_done[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        plan_free(p);
        return cuda_fail(e, "cudaEventCreate");
    }
    for (int a = 0; a < ndim && !rc; ++a) {
        rc = dalloc(&p->tw[a], (size_t)dims[a] * 16, "twiddles");   // float4 hi/lo or double2
        if (!rc && components == 1) rc = dalloc(&p->kin[a], (size_t)dims[a] * p->csz, "kinetic table");
    }
    if (!rc && components > 1)   // per momentum: 4 reals (1D, 2D) or 8 (3D)
        rc = dalloc(&p->dtab, (size_t)p->npts * (ndim == 3 ? 4 : 2) * p->csz, "Dirac table");
    if (!rc) rc = dalloc(&p->theta, (size_t)sum_n * sizeof(double), "angles");
    if (!rc) rc = dalloc(&p->partial, (size_t)reduce_blocks() * sizeof(double), "partials");
    if (!rc) rc = dalloc(&p->result, 4 * sizeof(double), "result");
    if (!rc) rc = dalloc(&p->pgrid, (size_t)sum_n * sizeof(double), "momenta");
    if (!rc) rc = dalloc(&p->errflag, sizeof(int), "error flag");
    if (!rc) rc = dalloc(&p->tile_ctr, 2 * sizeof(unsigned long long), "tile counters");
    if (!rc) {
        e = cudaMemsetAsync(p->errflag, 0, sizeof(int), p->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(p->tile_ctr, 0, 2 * sizeof(unsigned long long), p->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemsetAsync(error flag, tile counters)");
    }
    if (!rc) {
        p->row_len = sum_n;
        rc = dalloc(&p->ftab, (size_t)kFieldChunk * sum_n * p->csz, "field tables");
    }
    if (!rc) {
        e = cudaHostAlloc(reinterpret_cast<void **>(&p->host_result), 4 * sizeof(double), cudaHostAllocDefault);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaHostAlloc(result)");
    }
    if (rc) {
        plan_free(p);
        return rc;
    }
    for (int a = 0; a < ndim; ++a) {
        e = build_twiddles(p->tw[a], (int)dims[a], p->f64, p->stream);
        if (e != cudaSuccess) {
            plan_free(p);
            return cuda_fail(e, "build_twiddles");
        }
        p->launches++;
        // per-stage tables of the persistent passes (nc = 2 only for the Dirac pairs)
        for (int nc = 1; nc <= (components == 4 ? 2 : 1); ++nc) {
            auto st = p->f64 ? stage_table_f64 : stage_table_f32;
            const int entries = st((int)dims[a], nc, nullptr, nullptr, p->stream);
            if (entries < 0) continue;
            rc = dalloc(&p->stw[a][nc - 1], (size_t)(entries > 0 ? entries : 1) * p->csz, "stage twiddles");
            if (rc) {
                plan_free(p);
                return rc;
            }
            if (entries > 0) {
                st((int)dims[a], nc, p->stw[a][nc - 1], p->tw[a], p->stream);
                p->launches++;
            }
        }

    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        plan_free(p);
        return cuda_fail(e, "stage twiddle tables");
    }
    std::vector<double> pg;
    for (int a = 0; a < ndim; ++a)
        for (int64_t k = 0; k < dims[a]; ++k) pg.push_back(lattice_p(dims[a], spacing[a], k, prm.hbar));
    rc = upload(p, p->pgrid, pg.data(), (int64_t)pg.size());
    if (rc) {
        plan_free(p);
        return rc;
    }
    e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        plan_free(p);
        return cuda_fail(e, "cudaStreamSynchronize(create)");
    }
    *out = p;
    return SOP_OK;
}

int sop_plan_destroy(sop_plan plan) { return plan_free(plan); }

int sop_bind_state(sop_plan p, void *psi_dev) {
    if (!p) return fail(SOP_EINVAL, "sop_bind_state: null plan");
    if (!psi_dev) return fail(SOP_EINVAL, "sop_bind_state: psi is NULL");
    if (reinterpret_cast<uintptr_t>(psi_dev) % 16 != 0)
        return fail(SOP_EINVAL, "sop_bind_state: psi must be 16-byte aligned");
    p->psi = psi_dev;
    return SOP_OK;
}

int sop_set_potential(sop_plan p, const void *V_dev, int v_is_fp64) {
    if (!p) return fail(SOP_EINVAL, "sop_set_potential: null plan");
    if (!V_dev) return fail(SOP_EINVAL, "sop_set_potential: V is NULL");
    if (reinterpret_cast<uintptr_t>(V_dev) % (v_is_fp64 ? 8 : 4) != 0)
        return fail(SOP_EINVAL, "sop_set_potential: V is misaligned");
    int rc = SOP_OK;
    if (!p->V) rc = dalloc(&p->V, (size_t)p->npts * sizeof(double), "potential");
    if (!rc && !p->vhalf) rc = dalloc(&p->vhalf, (size_t)p->npts * p->csz, "half phase table");
    if (!rc && !p->vfull) rc = dalloc(&p->vfull, (size_t)p->npts * p->csz, "full phase table");
    if (!rc && !p->vbad) rc = dalloc(&p->vbad, sizeof(int), "potential check");
    if (rc) return rc;
    Bracket br(p, 4);
    cudaError_t e = cudaMemsetAsync(p->vbad, 0, sizeof(int), p->stream);
    if (e == cudaSuccess) e = convert_potential(p->V, V_dev, p->npts, v_is_fp64 != 0, p->vbad, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "convert_potential");
    br.done();
    int bad = 0;
    e = cudaMemcpyAsync(&bad, p->vbad, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sop_set_potential: reading the potential check");
    if (bad) {
        p->v_set = false;
        p->tables_valid = false;
        return fail(SOP_EINVAL, "sop_set_potential: V holds a value that is not finite (NaN or Inf)");
    }
    p->v_set = true;
    p->tables_valid = false;
    ++p->v_version;
    return SOP_OK;
}

int sop_set_field_profile(sop_plan p, int along_x1) {
    if (!p) return fail(SOP_EINVAL, "sop_set_field_profile: null plan");
    if (p->comps != 4) return fail(SOP_EUNSUPPORTED, "sop_set_field_profile: four-component Dirac plans only");
    if (along_x1 != 0 && along_x1 != 1) return fail(SOP_EINVAL, "sop_set_field_profile: along_x1 must be 0 or 1");
    p->profile = along_x1 == 1;
    return SOP_OK;
}

int sop_set_gauge(sop_plan p, int gauge) {
    if (!p) return fail(SOP_EINVAL, "sop_set_gauge: null plan");
    if (gauge != SOP_GAUGE_LENGTH && gauge != SOP_GAUGE_VELOCITY)
        return fail(SOP_EINVAL, "sop_set_gauge: gauge must be SOP_GAUGE_LENGTH or SOP_GAUGE_VELOCITY");
    if (p->comps != 1) return fail(SOP_EUNSUPPORTED, "sop_set_gauge: Schroedinger plans only (Dirac takes A)");
    p->gauge = gauge;
    return SOP_OK;
}

int sop_step(sop_plan p, int64_t n_steps, double dt, const double *field_samples) {
    return step_impl(p, n_steps, dt, field_samples);
}

int sop_step_host(sop_plan p, void *psi_host, int64_t n_steps, double dt, const double *field_samples) {
    if (!p) return fail(SOP_EINVAL, "sop_step_host: null plan");
    if (!psi_host) return fail(SOP_EINVAL, "sop_step_host: psi_host is NULL");
    if (!p->psi) return fail(SOP_ESTATE, "sop_step_host: no device state bound");
    const size_t bytes = (size_t)p->npts * p->comps * p->csz;
    cudaError_t e = cudaMemcpyAsync(p->psi, psi_host, bytes, cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(H2D)");
    int rc = step_impl(p, n_steps, dt, field_samples);
    if (rc) return rc;
    e = cudaMemcpyAsync(psi_host, p->psi, bytes, cudaMemcpyDeviceToHost, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(D2H)");
    e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return check_errflag(p);
}

int sop_norm(sop_plan p, double *out) {
    if (!p || !out) return fail(SOP_EINVAL, "sop_norm: null argument");
    if (!p->psi) return fail(SOP_ESTATE, "sop_norm: no state bound");
    double dV = 1.0;
    for (int a = 0; a < p->ndim; ++a) dV *= p->h[a];
    Bracket br(p, 4);
    cudaError_t e = reduce_norm(p->psi, p->npts * p->comps, p->f64, p->partial, p->result, dV, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reduce_norm");
    br.done(2);
    return read_result(p, 1, out);
}

int sop_energy(sop_plan p, double *out) {
    if (!p || !out) return fail(SOP_EINVAL, "sop_energy: null argument");
    if (!p->psi) return fail(SOP_ESTATE, "sop_energy: no state bound");
    const size_t bytes = (size_t)p->npts * p->comps * p->csz;
    int rc = SOP_OK;
    if (!p->scratch) rc = dalloc(&p->scratch, bytes, "energy scratch");
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(p->scratch, p->psi, bytes, cudaMemcpyDeviceToDevice, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(D2D)");
    for (int ax = 0; ax < p->ndim; ++ax) {
        PassArgs a;
        base_args(p, a, p->scratch, ax);
        a.n_batch = p->comps;
        a.pre = -1;
        a.op = OP_NONE;
        rc = run_pass(p, a, 1, 2, "energy forward transform");
        if (rc) return rc;
    }
    double dV = 1.0;
    for (int a = 0; a < p->ndim; ++a) dV *= p->h[a];
    Bracket br(p, 4);
    e = reduce_energy_t(p->scratch, p->ndim, p->dims, p->pgrid, p->comps, p->prm.mass, p->prm.c, p->f64, p->partial,
                        p->result, dV / (double)p->npts, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reduce_energy_t");
    int nl = 2;
    if (p->v_set) {
        e = reduce_energy_v(p->psi, p->V, p->npts, p->comps, p->f64, p->partial, p->result + 1, dV, p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "reduce_energy_v");
        nl += 2;
    } else {
        cudaMemsetAsync(p->result + 1, 0, sizeof(double), p->stream);
    }
    br.done(nl);
    double r[2];
    rc = read_result(p, 2, r);
    if (rc) return rc;
    *out = r[0] + r[1];
    return SOP_OK;
}

int sop_profile_enable(sop_plan p, int every) {
    if (!p) return fail(SOP_EINVAL, "sop_profile_enable: null plan");
    if (every < 0) return fail(SOP_EINVAL, "sop_profile_enable: every < 0");
    p->prof_every = every;
    return SOP_OK;
}

int sop_profile_read(sop_plan p, double *ms, int64_t *launches, int max_classes) {
    if (!p || !ms || !launches || max_classes <= 0) return fail(SOP_EINVAL, "sop_profile_read: bad argument");
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    for (int c = 0; c < max_classes; ++c) {
        ms[c] = 0.0;
        launches[c] = 0;
    }
    for (auto &ep : p->events) {
        float t = 0.f;
        cudaEventElapsedTime(&t, ep.a, ep.b);
        if (ep.cls < max_classes) {
            ms[ep.cls] += t;
            launches[ep.cls] += 1;
        }
        p->event_pool.push_back(ep.a);
        p->event_pool.push_back(ep.b);
    }
    p->events.clear();
    return check_errflag(p);
}

int64_t sop_launch_counter(sop_plan p) { return p ? p->launches : 0; }

int sop_debug_check_canaries(int64_t *bad) {
    if (!bad) return fail(SOP_EINVAL, "sop_debug_check_canaries: null output");
#if SOP_CHECK
    std::lock_guard<std::mutex> lock(g_canary_mu);
    int64_t n = g_canary_bad.load();
    for (auto &kv : g_canary)
        if (!canary_intact(kv.first, kv.second)) ++n;
    *bad = n;
    return SOP_OK;
#else
    *bad = 0;
    return fail(SOP_EUNSUPPORTED, "sop_debug_check_canaries: the library was built without SOP_CHECK");
#endif
}

int sop_debug_fail_alloc(int64_t after) {
    g_fail_alloc.store(after < 0 ? -1 : after);
    return SOP_OK;
}

int sop_set_wait_limit(sop_plan p, uint64_t wait_ns) {
    if (!p) return fail(SOP_EINVAL, "sop_set_wait_limit: null plan");
    p->wait_ns = wait_ns;
    return SOP_OK;
}

int sop_set_pass_shape(sop_plan p, int axis_kind, int shape) {
    if (!p) return fail(SOP_EINVAL, "sop_set_pass_shape: null plan");
    if (axis_kind != 0 && axis_kind != 1) return fail(SOP_EINVAL, "sop_set_pass_shape: axis_kind must be 0 or 1");
    if (shape < 0 || shape >= kPassVariants) return fail(SOP_EINVAL, "sop_set_pass_shape: shape out of range");
    p->pass_var[axis_kind][0] = p->pass_var[axis_kind][1] = shape;
    return SOP_OK;
}

int sop_autotune(sop_plan p, double dt, int trial_steps, int *chosen) {
    if (!p) return fail(SOP_EINVAL, "sop_autotune: null plan");
    if (!p->psi) return fail(SOP_ESTATE, "sop_autotune: no state bound");
    if (!is_finite(dt)) return fail(SOP_EINVAL, "sop_autotune: dt is not finite");
    if (trial_steps <= 0) trial_steps = 16;
    if (chosen) chosen[0] = chosen[1] = 0;
    if (p->ndim == 1 || !p->async_passes) return SOP_OK;   // no pencil passes to shape
    static_assert(SOP_PASS_SHAPES == kPassVariants, "shape count");
    // per-process cache: lattice shape, components, dtype, device -> shapes
    static std::mutex mu;
    static std::map<std::vector<int64_t>, std::pair<int, int>> cache;
    const std::vector<int64_t> key = {p->device, p->ndim, p->dims[0], p->dims[1], p->dims[2], p->comps, p->f64 ? 1 : 0};
    // SOP_AUTOTUNE_CACHE=<file>: choices persist across processes, one line
    // per device model and shape ("<model> ndim n0 n1 n2 comps f64 C S")
    const char *cache_file = std::getenv("SOP_AUTOTUNE_CACHE");
    std::string model;
    if (cache_file && *cache_file) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) model = prop.name;
        for (char &ch : model)
            if (ch == ' ') ch = '_';
    }
    {
        std::lock_guard<std::mutex> lock(mu);
        static std::set<std::string> loaded;   // (file, device) pairs read once
        const std::string once = model.empty() ? std::string() : std::string(cache_file) + "#" + std::to_string(p->device);
        if (!model.empty() && !loaded.count(once)) {
            loaded.insert(once);
            if (FILE *f = std::fopen(cache_file, "r")) {
                char line[512], name[256];
                long long v[7];
                int c0, c1;
                while (std::fgets(line, sizeof(line), f)) {   // malformed lines are skipped
                    if (std::sscanf(line, "%255s %lld %lld %lld %lld %lld %lld %d %d", name, &v[0], &v[1], &v[2],
                                    &v[3], &v[4], &v[5], &c0, &c1) != 9)
                        continue;
                    if (model == name && c0 >= 0 && c0 < kPassVariants && c1 >= 0 && c1 < kPassVariants &&
                        (v[5] == 0 || (c0 == 0 && c1 == 0)))   // complex128 has shape 0 only
                        cache[{p->device, v[0], v[1], v[2], v[3], v[4], v[5]}] = {c0, c1};
                }
                std::fclose(f);
            }
        }
        auto it = cache.find(key);
        if (it != cache.end()) {
            p->pass_var[0][0] = p->pass_var[0][1] = it->second.first;
            p->pass_var[1][0] = p->pass_var[1][1] = it->second.second;
            if (chosen) {
                chosen[0] = it->second.first;
                chosen[1] = it->second.second;
            }
            return SOP_OK;
        }
    }
    const size_t bytes = (size_t)p->npts * p->comps * p->csz;
    int rc = SOP_OK;
    if (!p->scratch) rc = dalloc(&p->scratch, bytes, "autotune scratch");
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(p->scratch, p->psi, bytes, cudaMemcpyDeviceToDevice, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(D2D)");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    void *const saved_psi = p->psi;
    const int saved_prof = p->prof_every;
    p->psi = p->scratch;
    p->prof_every = 0;
    int best[2] = {0, 0};
    // coordinate descent over the two pass kinds, twice (the step time of a
    // shape depends on the other kind's shape through the launch overlap);
    // each shape is timed as the best of five trials of whole split steps
    for (int sweep = 0; sweep < 4 && !rc; ++sweep) {
        const int kind = sweep & 1;
        float best_ms = 0.f;
        const int nshapes = p->f64 ? 1 : kPassVariants;   // shapes 1.. exist for complex64 only
        if (nshapes == 1) continue;
        for (int v = 0; v < nshapes && !rc; ++v) {
            p->pass_var[kind][0] = p->pass_var[kind][1] = v;
            rc = step_impl(p, 2, dt, nullptr);   // warm-up (tables, tensor maps, attributes)
            if (rc) break;
            float ms = 0.f;
            for (int rep = 0; rep < 5 && !rc; ++rep) {   // best of five trials
                cudaEventRecord(e0, p->stream);
                rc = step_impl(p, trial_steps, dt, nullptr);
                if (rc) break;
                cudaEventRecord(e1, p->stream);
                if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
                    rc = cuda_fail(e, "cudaEventSynchronize");
                    break;
                }
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep == 0 || t < ms) ms = t;
            }
            if (rc) break;
            if (v == 0 || ms < best_ms) {
                best_ms = ms;
                best[kind] = v;
            }
        }
        p->pass_var[kind][0] = p->pass_var[kind][1] = best[kind];
    }
    for (int kind = 0; kind < 2; ++kind) p->pass_var[kind][0] = p->pass_var[kind][1] = best[kind];
    p->psi = saved_psi;
    p->prof_every = saved_prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc) rc = check_errflag(p);
    if (rc) {
        p->pass_var[0][0] = p->pass_var[0][1] = p->pass_var[1][0] = p->pass_var[1][1] = 0;
        return rc;
    }
    {
        std::lock_guard<std::mutex> lock(mu);
        cache[key] = {best[0], best[1]};
        if (!model.empty())
            if (FILE *f = std::fopen(cache_file, "a")) {
                std::fprintf(f, "%s %d %lld %lld %lld %d %d %d %d\n", model.c_str(), p->ndim, (long long)p->dims[0],
                             (long long)p->dims[1], (long long)p->dims[2], p->comps, p->f64 ? 1 : 0, best[0], best[1]);
                std::fclose(f);
            }
    }
    if (chosen) {
        chosen[0] = best[0];
        chosen[1] = best[1];
    }
    return SOP_OK;
}

// ---------------------------------------------------------------------------
// Batched propagation: independent 2D Schroedinger lattices of uneven sizes
// advanced in lockstep, one multi-instance launch per pass kind and per
// pass-axis size (lattices sharing that size share the launch's tiles).
// ---------------------------------------------------------------------------

}  // extern "C"

struct sop_batch_s {
    std::vector<sop_plan> plans;
    cudaStream_t stream = nullptr;
    bool f64 = false;
    unsigned long long *tile_ctr = nullptr;
    unsigned long long tile_base = 0;
    InstDesc *desc = nullptr;
    size_t desc_cap = 0;   // descriptors
    // One merged middle step as a CUDA graph: the size groups of each pass kind
    // run concurrently on side streams, each on its own tile counter (reset at
    // the start of every replay); the field row is a device word the graph
    // advances.  Captured once per descriptor buffer and replayed per step.
    cudaGraphExec_t step_exec = nullptr;
    const InstDesc *exec_desc = nullptr;
    std::vector<int> exec_shapes;   // launch shapes of the groups the graph was captured with
    int exec_kernels = 0;
    std::vector<cudaStream_t> side;
    cudaStream_t cap = nullptr;   // capture stream
    std::vector<cudaEvent_t> evs;
    unsigned long long *gctr = nullptr;
    size_t gctr_cap = 0;
    int64_t *row_dev = nullptr;
    bool graphs = true;   // SOP_BATCH_GRAPH=0 turns the replayed graph off (direct launches)
};

namespace {

int batch_free(sop_batch b) {
    if (!b) return SOP_OK;
    cudaStreamSynchronize(b->stream);
    if (b->step_exec) cudaGraphExecDestroy(b->step_exec);
    for (cudaStream_t st : b->side) cudaStreamDestroy(st);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaEvent_t ev : b->evs) cudaEventDestroy(ev);
    dfree(b->tile_ctr);
    dfree(b->desc);
    dfree(b->gctr);
    dfree(b->row_dev);
    delete b;
    return SOP_OK;
}

// One multi-instance pass of a replayed step on stream st with its own counter.
cudaError_t batch_launch_shape(sop_batch b, PassArgs &a, bool contig, int shape, cudaStream_t st, int64_t *adv);

cudaError_t batch_launch_on(sop_batch b, PassArgs &a, bool contig, cudaStream_t st, unsigned long long *ctr,
                            int shape) {
    sop_plan p0 = b->plans[0];
    a.errflag = p0->errflag;
    a.wait_ns = p0->wait_ns;
    a.tile_ctr = ctr;
    a.tile_base[0] = a.tile_base[1] = 0;
    a.n_comp_total = 1;
    int64_t adv = 0;
    return batch_launch_shape(b, a, contig, shape, st, &adv);
}

// One multi-instance pass over the lattices of a group.
// shape: launch shape of the group (0: default); shapes without a kernel
// for the size fall back to shape 0.
cudaError_t batch_launch_shape(sop_batch b, PassArgs &a, bool contig, int shape, cudaStream_t st, int64_t *adv) {
    TensorMapBytes tm;
    std::memset(&tm, 0, sizeof(tm));
    cudaError_t e = cudaErrorInvalidValue;
    if (shape > 0 && shape < kPassVariants && !b->f64) {
        e = launch_async_variant(false, contig, shape, a, 1, tm, st, adv);
        if (e == cudaErrorInvalidValue) cudaGetLastError();
    }
    if (e != cudaErrorInvalidValue) return e;
    if (b->f64)
        return contig ? launch_async_f64_contig(a, 1, tm, st, adv) : launch_async_f64_strided(a, 1, tm, st, adv);
    return contig ? launch_async_f32_contig(a, 1, tm, st, adv) : launch_async_f32_strided(a, 1, tm, st, adv);
}

int batch_launch(sop_batch b, PassArgs &a, bool contig, const char *what, int shape = 0) {
    sop_plan p0 = b->plans[0];
    a.errflag = p0->errflag;
    a.wait_ns = p0->wait_ns;
    a.tile_ctr = b->tile_ctr;
    a.tile_base[0] = a.tile_base[1] = b->tile_base;
    a.n_comp_total = 1;
    int64_t adv = 0;
    cudaError_t e = batch_launch_shape(b, a, contig, shape, b->stream, &adv);
    if (e != cudaSuccess) return cuda_fail(e, what);
    b->tile_base += (unsigned long long)adv;
    p0->launches += 1;
    return SOP_OK;
}

}  // namespace

extern "C" {

int sop_batch_create(sop_batch *out, int n_plans, const sop_plan *plans) {
    if (!out) return fail(SOP_EINVAL, "sop_batch_create: out is NULL");
    *out = nullptr;
    if (n_plans < 1 || !plans) return fail(SOP_EINVAL, "sop_batch_create: no plans");
    for (int i = 0; i < n_plans; ++i) {
        const sop_plan p = plans[i];
        if (!p) return fail(SOP_EINVAL, "sop_batch_create: null plan");
        if (p->comps != 1 || p->ndim != 2)
            return fail(SOP_EUNSUPPORTED, "sop_batch_create: two-dimensional Schroedinger plans only");
        if (p->gauge != SOP_GAUGE_LENGTH) return fail(SOP_EUNSUPPORTED, "sop_batch_create: length-gauge plans only");
        if (p->f64 != plans[0]->f64 || p->stream != plans[0]->stream)
            return fail(SOP_EINVAL, "sop_batch_create: plans differ in dtype or stream");

        for (int j = 0; j < i; ++j)
            if (plans[j] == p) return fail(SOP_EINVAL, "sop_batch_create: a plan appears twice");
    }
    sop_batch b = new sop_batch_s();
    b->plans.assign(plans, plans + n_plans);
    b->stream = plans[0]->stream;
    b->f64 = plans[0]->f64;
    {
        const char *env = std::getenv("SOP_BATCH_GRAPH");
        b->graphs = !(env && std::string(env) == "0");
    }
    int rc = dalloc(&b->tile_ctr, 2 * sizeof(unsigned long long), "batch tile counters");
    if (!rc) {
        cudaError_t e = cudaMemsetAsync(b->tile_ctr, 0, 2 * sizeof(unsigned long long), b->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemsetAsync(batch tile counters)");
    }
    if (rc) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return SOP_OK;
}

int sop_batch_destroy(sop_batch b) { return batch_free(b); }

int sop_batch_step(sop_batch b, int64_t n, double dt, const double *const *fields) {
    if (!b) return fail(SOP_EINVAL, "sop_batch_step: null batch");
    if (n < 0) return fail(SOP_EINVAL, "sop_batch_step: n_steps < 0");
    if (!is_finite(dt)) return fail(SOP_EINVAL, "sop_batch_step: dt is not finite");
    if (n == 0) return SOP_OK;
    const int np = (int)b->plans.size();
    std::vector<FieldRows> fr((size_t)np);
    for (int i = 0; i < np; ++i) {
        sop_plan p = b->plans[i];
        if (!p->psi) return fail(SOP_ESTATE, "sop_batch_step: a plan has no state bound");
        if (p->gauge != SOP_GAUGE_LENGTH) return fail(SOP_EUNSUPPORTED, "sop_batch_step: length-gauge plans only");
        const double *f = fields ? fields[i] : nullptr;
        if (f)
            for (int64_t k = 0; k < n * 2; ++k)
                if (!is_finite(f[k])) return fail(SOP_EINVAL, "sop_batch_step: field sample is not finite");
        int rc = ensure_tables(p, dt);
        if (rc) return rc;
        rc = prepare_fields(p, n, dt, f, fr[(size_t)i]);
        if (rc) return rc;
    }
    // groups by pass-axis size: the x passes by n_x, the y passes by n_y
    struct Group {
        int axis;
        bool multi = false;   // one multi-instance launch (else one-shot passes per lattice)
        int shape = 0;        // launch shape: the first member's (sop_autotune / sop_set_pass_shape)
        std::vector<int> members;
        int64_t first = 0, tiles = 0;
    };
    std::map<int64_t, Group> gx, gy;
    for (int i = 0; i < np; ++i) {
        gx[b->plans[i]->dims[0]].members.push_back(i);
        gy[b->plans[i]->dims[1]].members.push_back(i);
    }
    for (auto &kv : gx) kv.second.axis = 0;
    for (auto &kv : gy) kv.second.axis = 1;
    std::vector<InstDesc> hd;
    for (auto *gm : {&gx, &gy})
        for (auto &kv : *gm) {
            Group &g = kv.second;
            g.first = (int64_t)hd.size();
            const int axis = g.axis;
            g.shape = b->plans[g.members[0]]->pass_var[axis == 0 ? 0 : 1][0];
            if (b->f64) g.shape = 0;   // shapes other than 0 exist for complex64 only
            // pencils per CTA of the group's launch shape: the tiles of every
            // lattice are laid out for it
            int wp = async_pencils_per_cta_shape(b->f64, (int)kv.first, axis == 0, g.shape);
            if (wp <= 0) {
                g.shape = 0;
                wp = async_pencils_per_cta(b->f64, (int)kv.first, 1, axis == 0);
            }
            g.multi = wp > 0 && b->plans[g.members[0]]->async_passes;
            if (!g.multi) continue;
            int64_t tiles = 0;
            for (int i : g.members) {
                sop_plan p = b->plans[i];
                InstDesc d;
                std::memset(&d, 0, sizeof(d));
                d.psi = p->psi;
                d.vhalf = p->v_set ? p->vhalf : nullptr;
                d.vfull = p->v_set ? p->vfull : nullptr;
                const FieldRows &f = fr[(size_t)i];
                d.ftab = f.any ? p->ftab : nullptr;
                d.frow_len = f.row_len;
                for (int a = 0; a < 3; ++a) {
                    d.foff[a] = (a < 2 && f.active[a]) ? f.offs[a] : -1;
                    d.ttab[a] = a < 2 ? p->kin[a] : nullptr;
                    d.dims[a] = p->dims[a];
                }
                d.n_pencils = p->npts / p->dims[axis];
                if (axis == 0) {
                    d.n_xgroups = 0;
                    d.tile_begin = tiles;
                    tiles += (d.n_pencils + wp - 1) / wp;
                } else {
                    d.n_xgroups = (p->dims[0] + wp - 1) / wp;
                    d.o_stride = 0;
                    d.tiles_per_batch = d.n_xgroups * (d.n_pencils / p->dims[0]);
                    d.tile_begin = tiles;
                    tiles += d.n_xgroups;
                    TensorMapBytes tm;
                    int rc = tensor_map(p, p->psi, 1, 1, &tm);
                    if (rc) return rc;
                    std::memcpy(d.tmap, tm.b, sizeof(d.tmap));
                }
                d.scale_hi = p->scale_hi;
                d.scale_lo = p->scale_lo;
                hd.push_back(d);
            }
            g.tiles = tiles;
        }
    if (!hd.empty() && b->desc_cap < hd.size()) {
        cudaStreamSynchronize(b->stream);
        dfree(b->desc);
        b->desc = nullptr;
        b->desc_cap = 0;
        int rc = dalloc(&b->desc, hd.size() * sizeof(InstDesc), "batch descriptors");
        if (rc) return rc;
        b->desc_cap = hd.size();
    }
    static_assert(sizeof(InstDesc) % sizeof(double) == 0, "descriptor size");
    int rc = SOP_OK;
    if (!hd.empty()) {
        rc = upload(b->plans[0], reinterpret_cast<double *>(b->desc), reinterpret_cast<const double *>(hd.data()),
                    (int64_t)(hd.size() * sizeof(InstDesc) / sizeof(double)));
        if (rc) return rc;
    }
    // one-shot pass of one lattice (groups without a persistent kernel)
    auto single = [&](int i, int axis, int pre, int post, int op, int64_t P, int64_t P0, const char *what) -> int {
        sop_plan p = b->plans[i];
        const FieldRows &f = fr[(size_t)i];
        PassArgs a;
        base_args(p, a, p->psi, axis);
        a.pre = pre;
        a.post = post;
        a.op = op;
        if (op == OP_V) {
            a.vtab = p->v_set ? ((P == 0 || P == n) ? p->vhalf : p->vfull) : nullptr;
            for (int ax = 0; ax < 2; ++ax)
                a.ftab[ax] = f.active[ax] ? static_cast<const char *>(p->ftab) + ((P - P0) * f.row_len + f.offs[ax]) * p->csz
                                          : nullptr;
        } else {
            for (int ax = 0; ax < 2; ++ax) a.ttab[ax] = p->kin[ax];
        }
        return launch_pass(p, a, 1, what);
    };
    // One real-space index P launched directly on the batch stream: the x
    // passes of every size group, then (P < n) the y passes.
    auto direct_step = [&](int64_t P, int64_t P0) -> int {
        int rc2 = SOP_OK;
        for (auto &kv : gx) {
            Group &g = kv.second;
            if (!g.multi) {
                for (int i : g.members)
                    if ((rc2 = single(i, 0, P > 0 ? +1 : 0, P < n ? -1 : 0, OP_V, P, P0, "real-space pass"))) return rc2;
                continue;
            }
            sop_plan p0 = b->plans[g.members[0]];
            PassArgs a;
            base_args(p0, a, p0->psi, 0);
            a.pre = P > 0 ? +1 : 0;
            a.post = P < n ? -1 : 0;
            a.op = OP_V;
            a.inst = b->desc + g.first;
            a.n_inst = (int)g.members.size();
            a.P = P;
            a.p_table0 = P0;
            a.n_total = n;
            a.n_tiles = g.tiles;
            a.stw = p0->stw[0][0];   // per-stage twiddles of this x size (shapes reading them through L1)
            if ((rc2 = batch_launch(b, a, true, "batched real-space pass", g.shape))) return rc2;
        }
        if (P == n) return SOP_OK;
        for (auto &kv : gy) {
            Group &g = kv.second;
            if (!g.multi) {
                for (int i : g.members)
                    if ((rc2 = single(i, 1, -1, +1, OP_T, P, P0, "momentum-space pass"))) return rc2;
                continue;
            }
            sop_plan p0 = b->plans[g.members[0]];
            PassArgs a;
            base_args(p0, a, p0->psi, 1);
            a.pre = -1;
            a.post = +1;
            a.op = OP_T;
            a.inst = b->desc + g.first;
            a.n_inst = (int)g.members.size();
            a.P = P;
            a.p_table0 = P0;
            a.n_total = n;
            a.n_tiles = g.tiles;
            a.stw = p0->stw[1][0];
            if ((rc2 = batch_launch(b, a, false, "batched momentum-space pass", g.shape))) return rc2;
        }
        return SOP_OK;
    };

    // The merged middle step (0 < P < n) as a replayed graph: every group is a
    // multi-instance launch, so its arguments do not depend on P; the field
    // row comes from b->row_dev.
    bool all_multi = !hd.empty();
    for (auto *gm : {&gx, &gy})
        for (auto &kv : *gm) all_multi = all_multi && kv.second.multi;
    const size_t ngroups = gx.size() + gy.size();
    std::vector<int> shapes_now;
    for (auto *gm : {&gx, &gy})
        for (auto &kv : *gm) shapes_now.push_back(kv.second.shape);
    auto ensure_graph = [&]() -> int {
        if (b->step_exec && b->exec_desc == b->desc && b->exec_shapes == shapes_now) return SOP_OK;
        if (b->step_exec) {
            cudaGraphExecDestroy(b->step_exec);
            b->step_exec = nullptr;
        }
        int rc2 = SOP_OK;
        if (b->gctr_cap < ngroups) {
            dfree(b->gctr);
            b->gctr = nullptr;
            b->gctr_cap = 0;
            if ((rc2 = dalloc(&b->gctr, ngroups * 2 * sizeof(unsigned long long), "batch group counters"))) return rc2;
            b->gctr_cap = ngroups;
        }
        if (!b->row_dev && (rc2 = dalloc(&b->row_dev, sizeof(int64_t), "batch step row"))) return rc2;
        const size_t nside = std::max(gx.size(), gy.size());
        while (b->side.size() < nside) {
            cudaStream_t st;
            cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
            b->side.push_back(st);
        }
        while (b->evs.size() < 2 * nside + 2) {
            cudaEvent_t ev;
            cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreateWithFlags");
            b->evs.push_back(ev);
        }
        // captured on a stream of its own (the batch stream may be the legacy
        // default stream, which cannot be captured); launched on the batch stream
        if (!b->cap) {
            cudaError_t e0 = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
            if (e0 != cudaSuccess) return cuda_fail(e0, "cudaStreamCreateWithFlags");
        }
        cudaStream_t cs = b->cap;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        int kernels = 0;
        auto phase = [&](std::map<int64_t, Group> &gm, bool contig, size_t ctr0, cudaEvent_t fork) -> cudaError_t {
            cudaError_t e2 = cudaEventRecord(fork, cs);
            size_t k = 0;
            for (auto &kv : gm) {
                Group &g = kv.second;
                cudaStream_t st = b->side[k];
                if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(st, fork, 0);
                sop_plan p0 = b->plans[g.members[0]];
                PassArgs a;
                base_args(p0, a, p0->psi, contig ? 0 : 1);
                a.pre = contig ? +1 : -1;
                a.post = contig ? -1 : +1;
                a.op = contig ? OP_V : OP_T;
                a.inst = b->desc + g.first;
                a.n_inst = (int)g.members.size();
                a.P = 1;
                a.p_table0 = 0;
                a.n_total = n;
                a.n_tiles = g.tiles;
                a.row_dev = b->row_dev;
                a.stw = p0->stw[contig ? 0 : 1][0];
                if (e2 == cudaSuccess) e2 = batch_launch_on(b, a, contig, st, b->gctr + 2 * (ctr0 + k), g.shape);
                ++kernels;
                cudaEvent_t join = b->evs[2 + 2 * k + (contig ? 0 : 1)];
                if (e2 == cudaSuccess) e2 = cudaEventRecord(join, st);
                if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(cs, join, 0);
                ++k;
            }
            return e2;
        };
        e = cudaMemsetAsync(b->gctr, 0, ngroups * 2 * sizeof(unsigned long long), cs);
        if (e == cudaSuccess) e = phase(gx, true, 0, b->evs[0]);
        if (e == cudaSuccess) e = phase(gy, false, gx.size(), b->evs[1]);
        if (e == cudaSuccess) e = advance_counter(b->row_dev, cs);
        cudaGraph_t graph = nullptr;
        cudaError_t ee = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = ee;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->step_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->step_exec = nullptr;
            return cuda_fail(e, "capturing the batched step graph");
        }
        b->exec_desc = b->desc;
        b->exec_shapes = shapes_now;
        b->exec_kernels = kernels + 1;
        return SOP_OK;
    };
    const bool use_graph = b->graphs && all_multi;

    for (int64_t P0 = 0; P0 <= n; P0 += kFieldChunk) {
        const int64_t P1 = std::min<int64_t>(n + 1, P0 + kFieldChunk);
        for (int i = 0; i < np; ++i) {
            sop_plan p = b->plans[i];
            const FieldRows &f = fr[(size_t)i];
            if (!f.any) continue;
            cudaError_t e = build_field_tables(p->ftab, p->fvec + P0 * 2, P1 - P0, 2, p->dims, p->h, f.active,
                                               f.offs, f.row_len, p->f64, p->stream);
            if (e != cudaSuccess) return cuda_fail(e, "build_field_tables");
            p->launches += 1;
        }
        int64_t P = P0;
        if (P == 0) {
            if ((rc = direct_step(0, P0))) return rc;
            P = 1;
        }
        const int64_t mid_end = std::min<int64_t>(P1, n);   // middle indices P < n of this chunk
        if (use_graph && mid_end - P >= 2) {
            if ((rc = ensure_graph())) return rc;
            const int64_t Pstart = P;
            cudaError_t e = set_counter(b->row_dev, P - P0, b->stream);
            for (; e == cudaSuccess && P < mid_end; ++P) e = cudaGraphLaunch(b->step_exec, b->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch(batched step)");
            b->plans[0]->launches += (int64_t)b->exec_kernels * (mid_end - Pstart) + 1;
        }
        for (; P < P1; ++P)
            if ((rc = direct_step(P, P0))) return rc;
    }
    return SOP_OK;
}

int sop_adjoint_gradient(sop_plan p, const void *phi_dev, int64_t n_steps, double dt, const double *field,
                         int64_t every, double *J, double *grad_field, double *grad_V_dev) {
    if (!p) return fail(SOP_EINVAL, "sop_adjoint_gradient: null plan");
    if (p->comps != 1) return fail(SOP_EUNSUPPORTED, "sop_adjoint_gradient: Schroedinger plans only");
    if (p->gauge != SOP_GAUGE_LENGTH)
        return fail(SOP_EUNSUPPORTED, "sop_adjoint_gradient: length-gauge plans only");
    if (!p->psi) return fail(SOP_ESTATE, "sop_adjoint_gradient: no state bound (psi_0)");
    if (!phi_dev || !J) return fail(SOP_EINVAL, "sop_adjoint_gradient: phi or J is NULL");
    if (n_steps < 1 || every < 1) return fail(SOP_EINVAL, "sop_adjoint_gradient: n_steps and every must be >= 1");
    if (!std::isfinite(dt) || dt == 0.0) return fail(SOP_EINVAL, "sop_adjoint_gradient: dt must be finite and nonzero");
    if (reinterpret_cast<uintptr_t>(phi_dev) % 16 != 0)
        return fail(SOP_EINVAL, "sop_adjoint_gradient: phi must be 16-byte aligned");
    if (p->npts >= ((int64_t)1 << 31))
        return fail(SOP_EUNSUPPORTED, "sop_adjoint_gradient: lattices of 2^31 points or more");
    const int nd = p->ndim;
    const int64_t N = n_steps;
    if (field)
        for (int64_t k = 0; k < N * nd; ++k)
            if (!std::isfinite(field[k])) return fail(SOP_EINVAL, "sop_adjoint_gradient: non-finite field sample");
    int rc = SOP_OK;
    // the costate plan: same lattice and potential, its own tables for -dt
    if (!p->rev) {
        sop_plan r = nullptr;
        rc = sop_plan_create(&r, nd, p->dims, p->h, 1, p->f64 ? SOP_C128 : SOP_C64, &p->prm, p->stream);
        if (rc) return rc;
        r->async_passes = p->async_passes;
        p->rev = r;
    }
    // the costate plan takes this plan's launch shapes and, once per potential
    // version, its potential
    for (int k = 0; k < 2; ++k)
        for (int c = 0; c < 2; ++c) p->rev->pass_var[k][c] = p->pass_var[k][c];
    if (!p->v_set) {
        p->rev->v_set = false;
        p->rev->tables_valid = false;
        p->rev_v_version = 0;
    } else if (p->rev_v_version != p->v_version || !p->rev->v_set) {
        rc = sop_set_potential(p->rev, p->V, 1);
        if (rc) return rc;
        p->rev_v_version = p->v_version;
    }
    const size_t sb = (size_t)p->npts * p->csz;
    const int64_t K = (N + every - 1) / every;           // checkpoints at 0, every, 2 every, ...
    const int64_t S = std::min<int64_t>(every, N) + 1;   // states of one recomputed segment
    // one device block, carved into the buffers below (256-byte aligned) and
    // kept in the plan for the next call of the same or a smaller size
    const size_t npart = (size_t)std::max(inner_partials(), seg_partials((int)std::min<int64_t>(every, N)));
    const size_t sizes[8] = {(size_t)K * sb, (size_t)S * sb, sb, (size_t)S * sb, (size_t)(N + 1) * 8 * sizeof(double),
                             8 * sizeof(double), (size_t)p->npts * 2 * sizeof(double), npart * sizeof(double)};
    size_t offs[8], total = 0;
    for (int k = 0; k < 8; ++k) {
        offs[k] = total;
        total += (sizes[k] + 255) & ~size_t(255);
    }
    if (p->adj_cap < total) {
        cudaStreamSynchronize(p->stream);
        dfree(p->adj);
        p->adj = nullptr;
        p->adj_cap = 0;
        if ((rc = dalloc(&p->adj, total, "adjoint buffers"))) return rc;
        p->adj_cap = total;
    }
    char *const ck = p->adj + offs[0], *const seg = p->adj + offs[1], *const lam = p->adj + offs[2],
               *const lseg = p->adj + offs[3];
    double *const sdev = reinterpret_cast<double *>(p->adj + offs[4]);
    double *const cdev = reinterpret_cast<double *>(p->adj + offs[5]);
    double *const acc = reinterpret_cast<double *>(p->adj + offs[6]);
    double *const part = reinterpret_cast<double *>(p->adj + offs[7]);
    auto cleanup = [&]() { cudaStreamSynchronize(p->stream); };
    void *const psi_user = p->psi;
    const double dV = p->h[0] * (nd > 1 ? p->h[1] : 1.0) * (nd > 2 ? p->h[2] : 1.0);
    const double *F = field;
    std::vector<double> zero((size_t)nd, 0.0);
    auto frow = [&](int64_t n) -> const double * { return F ? F + n * nd : zero.data(); };
    auto slot = [&](char *base, int64_t k) -> void * { return base + (size_t)k * sb; };
    auto copy = [&](void *dst, const void *src) -> int {
        cudaError_t e = cudaMemcpyAsync(dst, src, sb, cudaMemcpyDeviceToDevice, p->stream);
        return e == cudaSuccess ? SOP_OK : cuda_fail(e, "cudaMemcpyAsync(adjoint state)");
    };
    auto inner = [&](const void *a, const void *b, double *out) -> int {
        cudaError_t e = launch_inner(a, b, p->f64, nd, p->dims, p->h, dV, part, out, p->stream);
        p->launches += 2;
        return e == cudaSuccess ? SOP_OK : cuda_fail(e, "adjoint inner product");
    };
    auto accum = [&](const void *a, const void *b, double w) -> int {
        cudaError_t e = launch_accum(a, b, p->f64, p->npts, w, acc, p->stream);
        p->launches += 1;
        return e == cudaSuccess ? SOP_OK : cuda_fail(e, "adjoint accumulation");
    };
    auto step_on = [&](sop_plan q, void *state, double h, int64_t n, int64_t count = 1) -> int {
        q->psi = state;
        return step_impl(q, count, h, F ? frow(n) : nullptr);
    };
    auto body = [&]() -> int {
        int r = cudaMemsetAsync(acc, 0, (size_t)p->npts * 2 * sizeof(double), p->stream) == cudaSuccess
                    ? SOP_OK : cuda_fail(cudaGetLastError(), "cudaMemsetAsync(accumulator)");
        if (r) return r;
        // forward sweep to psi_N, checkpoints every `every` steps (a segment is
        // one sop_step call, with its half steps merged)
        void *work = slot(seg, 0);
        if ((r = copy(work, psi_user))) return r;
        for (int64_t s = 0; s < K; ++s) {
            const int64_t n0 = s * every, n1 = std::min<int64_t>(N, n0 + every);
            if ((r = copy(slot(ck, s), work))) return r;
            if ((r = step_on(p, work, dt, n0, n1 - n0))) return r;
        }
        // c = <phi|psi_N>; s_N = <lambda_N|X|psi_N> with lambda_N = phi
        if ((r = inner(phi_dev, work, cdev))) return r;
        if ((r = inner(phi_dev, work, sdev + N * 8))) return r;
        if ((r = copy(lam, phi_dev))) return r;
        if ((r = accum(lam, work, 1.0))) return r;
        // backward sweep, one checkpoint segment at a time
        std::vector<double> frev((size_t)std::min<int64_t>(every, N) * nd);
        for (int64_t s = K - 1; s >= 0; --s) {
            const int64_t n0 = s * every, n1 = std::min<int64_t>(N, n0 + every);
            const int64_t L = n1 - n0;
            if ((r = copy(slot(seg, 0), slot(ck, s)))) return r;
            if (nd >= 2) {
                // states n0 .. n1 - 1 from one merged call of L - 1 steps on slot
                // L - 1 that writes the states in between into slots 1 .. L - 2
                if (L > 1) {
                    if ((r = copy(slot(seg, L - 1), slot(ck, s)))) return r;
                    p->psi = slot(seg, L - 1);
                    if ((r = step_impl_mat(p, L - 1, dt, F ? F + n0 * nd : nullptr, seg, (int64_t)sb))) return r;
                }
                // costates lambda_{n1-1} .. lambda_{n0} from one merged call of L
                // steps with -dt and the field rows reversed (U_m^dagger is the
                // step with -dt); the state after P steps, lambda_{n1-P}, lands
                // in slot L - P
                if ((r = copy(slot(lseg, 0), lam))) return r;
                if (F)
                    for (int64_t k = 0; k < L; ++k)
                        for (int a = 0; a < nd; ++a) frev[(size_t)(k * nd + a)] = F[(n1 - 1 - k) * nd + a];
                p->rev->psi = slot(lseg, 0);
                if ((r = step_impl_mat(p->rev, L, -dt, F ? frev.data() : nullptr, slot(lseg, L), -(int64_t)sb)))
                    return r;
            } else {
                for (int64_t k = 0; k + 1 < L; ++k) {   // states n0 .. n1 - 1 (psi_{n1} is not needed again)
                    if ((r = copy(slot(seg, k + 1), slot(seg, k)))) return r;
                    if ((r = step_on(p, slot(seg, k + 1), dt, n0 + k))) return r;
                }
                // costates lambda_{m-1} = U_{m-1}^dagger lambda_m (the step with -dt)
                if ((r = copy(slot(lseg, L - 1), lam))) return r;
                if ((r = step_on(p->rev, slot(lseg, L - 1), -dt, n1 - 1))) return r;
                for (int64_t k = L - 2; k >= 0; --k) {
                    if ((r = copy(slot(lseg, k), slot(lseg, k + 1)))) return r;
                    if ((r = step_on(p->rev, slot(lseg, k), -dt, n0 + k))) return r;
                }
            }
            // the whole segment's overlaps and potential-gradient accumulation in one reduction
            cudaError_t e = launch_seg_reduce(lseg, seg, p->f64, (int)L, n0, nd, p->dims, p->h, dV, acc, part, sdev,
                                              p->stream);
            p->launches += 2;
            if (e != cudaSuccess) return cuda_fail(e, "adjoint segment reduction");
            if ((r = copy(lam, slot(lseg, 0)))) return r;
        }
        return SOP_OK;
    };
    rc = body();
    p->psi = psi_user;
    if (p->rev) p->rev->psi = nullptr;
    if (rc) {
        cleanup();
        return rc;
    }
    // gradients: k_E = (-i dt / (2 hbar)) (-q), k_V = -i dt / (2 hbar)
    std::vector<double> sh((size_t)(N + 1) * 8), ch(8);
    cudaError_t e = cudaMemcpyAsync(sh.data(), sdev, sh.size() * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ch.data(), cdev, 8 * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "adjoint results");
    }
    const cd c(ch[0], ch[1]);
    *J = std::norm(c);
    const double hbar = p->prm.hbar;
    const cd kE = cd(0.0, -dt / (2.0 * hbar)) * (-p->prm.charge);
    const cd kV = cd(0.0, -dt / (2.0 * hbar));
    if (grad_field)
        for (int64_t n = 0; n < N; ++n)
            for (int a = 0; a < nd; ++a) {
                const cd s1(sh[(n + 1) * 8 + 2 + 2 * a], sh[(n + 1) * 8 + 3 + 2 * a]);
                const cd s0(sh[n * 8 + 2 + 2 * a], sh[n * 8 + 3 + 2 * a]);
                grad_field[n * nd + a] = 2.0 * std::real(std::conj(c) * kE * (s1 + s0));
            }
    if (grad_V_dev) {
        const cd z = std::conj(c) * kV * dV;
        e = launch_grad_v(acc, p->f64, p->npts, z.real(), z.imag(), grad_V_dev, p->stream);
        p->launches += 1;
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "adjoint potential gradient");
        }
    }
    cleanup();
    return check_errflag(p);
}

int sop_spectral(sop_plan p, int64_t n_steps, double dt, int n_energies, const double *energies, double *chi_out,
                 double *spectrum_out, void *psiE_dev) {
    static_assert(SOP_SPECTRAL_MAX_EIGEN == SOP_SPECTRAL_MAX_ENERGIES, "eigenfunction slots");
    if (!p) return fail(SOP_EINVAL, "sop_spectral: null plan");
    if (!p->psi) return fail(SOP_ESTATE, "sop_spectral: no state bound (the trial state psi_0)");
    if (n_steps < 1) return fail(SOP_EINVAL, "sop_spectral: n_steps must be >= 1");
    if (!std::isfinite(dt) || dt == 0.0) return fail(SOP_EINVAL, "sop_spectral: dt must be finite and nonzero");
    if (n_energies < 0 || (n_energies > 0 && !energies))
        return fail(SOP_EINVAL, "sop_spectral: n_energies < 0 or energies is NULL");
    for (int k = 0; k < n_energies; ++k)
        if (!std::isfinite(energies[k])) return fail(SOP_EINVAL, "sop_spectral: non-finite energy");
    if (psiE_dev && n_energies > SOP_SPECTRAL_MAX_EIGEN)
        return fail(SOP_EINVAL, "sop_spectral: more than SOP_SPECTRAL_MAX_EIGEN eigenfunction energies");
    if (psiE_dev && reinterpret_cast<uintptr_t>(psiE_dev) % 16 != 0)
        return fail(SOP_EINVAL, "sop_spectral: psiE must be 16-byte aligned");
    const int64_t N = n_steps;
    const int64_t len = p->npts * p->comps;
    const size_t sb = (size_t)len * p->csz;
    const int K = n_energies;
    const bool want_psi = psiE_dev && K > 0;
    double dV = 1.0;
    for (int a = 0; a < p->ndim; ++a) dV *= p->h[a];
    char *psi0 = nullptr, *ring = nullptr;
    double *chi = nullptr, *part = nullptr, *Ed = nullptr, *spec = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(p->stream);
        dfree(psi0);
        dfree(ring);
        dfree(chi);
        dfree(part);
        dfree(Ed);
        dfree(spec);
    };
    int rc = dalloc(&psi0, sb, "spectral trial state");
    if (!rc) rc = dalloc(&chi, (size_t)(N + 1) * 2 * sizeof(double), "spectral autocorrelation");
    if (!rc) rc = dalloc(&part, (size_t)(inner_partials() + 1) * sizeof(double), "spectral partials");
    if (!rc && K > 0) rc = dalloc(&Ed, (size_t)K * sizeof(double), "spectral energies");
    if (!rc && K > 0) rc = dalloc(&spec, (size_t)K * 2 * sizeof(double), "spectral values");
    if (rc) {
        cleanup();
        return rc;
    }
    // eigenfunctions: a ring of B states so that the K accumulators are read
    // and written once per B steps; without room for it, B = 1 straight from psi
    int B = 1;
    if (want_psi)
        for (int b = SOP_SPECTRAL_RING; b > 1 && !ring; b /= 2)
            if (cudaMalloc(reinterpret_cast<void **>(&ring), (size_t)b * sb) == cudaSuccess)
                B = b;
            else {
                ring = nullptr;
                cudaGetLastError();   // clear the allocation error; try fewer slots
            }
    auto body = [&]() -> int {
        // the block counter of the sample reduction sits after the partials
        unsigned *done = reinterpret_cast<unsigned *>(part + inner_partials());
        cudaError_t e = cudaMemcpyAsync(psi0, p->psi, sb, cudaMemcpyDeviceToDevice, p->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(done, 0, sizeof(unsigned), p->stream);
        if (e == cudaSuccess && want_psi)
            e = cudaMemsetAsync(psiE_dev, 0, (size_t)K * len * 2 * sizeof(double), p->stream);
        if (e == cudaSuccess && K > 0)
            e = cudaMemcpyAsync(Ed, energies, (size_t)K * sizeof(double), cudaMemcpyHostToDevice, p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "spectral set-up copies");
        std::vector<double> wre((size_t)B * K), wim((size_t)B * K);
        const double hbar = p->prm.hbar;
        int fill = 0;
        for (int64_t n = 0; n <= N; ++n) {
            if (n > 0) {
                const int r = step_impl(p, 1, dt, nullptr);
                if (r) return r;
            }
            // the window 1 - cos(2 pi t_n / T) vanishes at n = 0 and n = N
            const bool acc = want_psi && n > 0 && n < N;
            e = launch_spectral_sample(psi0, p->psi, p->f64, len, acc && ring ? ring + (size_t)fill * sb : nullptr,
                                       dV, part, done, chi + 2 * n, p->stream);
            p->launches += 1;
            if (e != cudaSuccess) return cuda_fail(e, "spectral sample");
            if (!acc) continue;
            const double t = (double)n * dt;
            const double win = dt * (1.0 - std::cos(2.0 * M_PI * (double)n / (double)N));
            for (int k = 0; k < K; ++k) {
                const double ph = t * energies[k] / hbar;
                wre[(size_t)fill * K + k] = win * std::cos(ph);
                wim[(size_t)fill * K + k] = win * std::sin(ph);
            }
            if (++fill == B || n == N - 1) {
                e = launch_spectral_accum(ring ? static_cast<const void *>(ring) : p->psi, p->f64, fill, len, K,
                                          wre.data(), wim.data(), static_cast<double *>(psiE_dev), p->stream);
                p->launches += 1;
                if (e != cudaSuccess) return cuda_fail(e, "spectral accumulation");
                fill = 0;
            }
        }
        if (want_psi) {
            e = launch_spectral_finish(static_cast<double *>(psiE_dev), p->f64, (int64_t)K * len, p->stream);
            p->launches += p->f64 ? 0 : 1;
            if (e != cudaSuccess) return cuda_fail(e, "spectral accumulator conversion");
        }
        if (K > 0) {
            e = launch_spectrum(chi, N, dt, hbar, Ed, K, spec, p->stream);
            p->launches += 1;
            if (e != cudaSuccess) return cuda_fail(e, "spectral transform");
        }
        if (chi_out) {
            e = cudaMemcpyAsync(chi_out, chi, (size_t)(N + 1) * 2 * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
            if (e != cudaSuccess) return cuda_fail(e, "spectral autocorrelation (D2H)");
        }
        if (spectrum_out && K > 0) {
            e = cudaMemcpyAsync(spectrum_out, spec, (size_t)K * 2 * sizeof(double), cudaMemcpyDeviceToHost, p->stream);
            if (e != cudaSuccess) return cuda_fail(e, "spectral values (D2H)");
        }
        e = cudaStreamSynchronize(p->stream);
        return e == cudaSuccess ? SOP_OK : cuda_fail(e, "spectral results");
    };
    rc = body();
    cleanup();
    if (rc) return rc;
    return check_errflag(p);
}

}  // extern "C"
