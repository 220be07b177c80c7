// sop_1d_inst.cu -- instantiates the one-dimensional whole-step kernels
// (Schroedinger and two-component Dirac) for one dtype (-DSOP_REAL=float|double, with -DSOP_IS_DOUBLE=1 for double); the
// double build also defines the pass-geometry query and the shared-memory
// attribute helper.
#include <map>
#include <mutex>
#include <set>
#include <utility>

#include "sop_async.cuh"

#ifndef SOP_REAL
#error "SOP_REAL must be defined"
#endif

#define SOP_SIZES(X) \
    X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) \
    X(1536) X(2048) X(3072) X(4096)

namespace sop {

#if SOP_IS_DOUBLE
cudaError_t launch_1d_f64(const Args1D &a, int n, cudaStream_t s) {
#else
cudaError_t launch_1d_f32(const Args1D &a, int n, cudaStream_t s) {
#endif
    switch (n) {
#define SOP_CASE(N) \
    case N:         \
        return launch_1d_t<SOP_REAL, N>(a, s);
        SOP_SIZES(SOP_CASE)
#undef SOP_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

#if SOP_IS_DOUBLE
cudaError_t launch_1d_dirac_f64(const Args1D &a, int n, cudaStream_t s) {
#else
cudaError_t launch_1d_dirac_f32(const Args1D &a, int n, cudaStream_t s) {
#endif
    switch (n) {
#define SOP_CASE(N) \
    case N:         \
        return launch_1d_dirac_t<SOP_REAL, N>(a, s);
        SOP_SIZES(SOP_CASE)
#undef SOP_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

#if SOP_IS_DOUBLE
namespace {
template <typename Real, int N> void geom_of(int nc, bool contig, int *th, int *wp, int *sm) {
    if (nc == 1) {
        if (contig) { using C = PassCfg<Real, N, 1, true>; *th = C::THREADS; *wp = C::WP; *sm = (int)C::SMEM; }
        else { using C = PassCfg<Real, N, 1, false>; *th = C::THREADS; *wp = C::WP; *sm = (int)C::SMEM; }
    } else {
        if (contig) { using C = PassCfg<Real, N, 2, true>; *th = C::THREADS; *wp = C::WP; *sm = (int)C::SMEM; }
        else { using C = PassCfg<Real, N, 2, false>; *th = C::THREADS; *wp = C::WP; *sm = (int)C::SMEM; }
    }
}
}  // namespace

bool pass_geometry(bool f64, int n, int nc, bool contig, int *threads, int *pencils_per_cta, int *smem) {
    switch (n) {
#define SOP_CASE(N)                                                                          \
    case N:                                                                                  \
        if (f64) geom_of<double, N>(nc, contig, threads, pencils_per_cta, smem);             \
        else geom_of<float, N>(nc, contig, threads, pencils_per_cta, smem);                  \
        return true;
        SOP_SIZES(SOP_CASE)
#undef SOP_CASE
        default:
            return false;
    }
}

namespace {
// Pencils per CTA of the persistent pass, 0 where it does not fit on an SM.
template <typename Real, int N, int NC, bool CONTIG> int async_wp_fit() {
    using Cfg = AsyncCfg<Real, N, NC, CONTIG>;
    return Cfg::FITS ? Cfg::WP : 0;
}
template <typename Real, int N> int async_wp_of(int nc, bool contig) {
    if (nc == 1) return contig ? async_wp_fit<Real, N, 1, true>() : async_wp_fit<Real, N, 1, false>();
    if (nc == 4) {
        if constexpr (N <= 1024) return contig ? async_wp_fit<Real, N, 4, true>() : async_wp_fit<Real, N, 4, false>();
        return 0;
    }
    return contig ? async_wp_fit<Real, N, 2, true>() : async_wp_fit<Real, N, 2, false>();
}
}  // namespace

namespace {
template <typename Real, int N, int VAR> int shape_wp(bool contig) {
    if (contig) {
        using Cfg = AsyncCfg<Real, N, 1, true, VAR>;
        return Cfg::FITS ? Cfg::WP : 0;
    }
    using Cfg = AsyncCfg<Real, N, 1, false, VAR>;
    return Cfg::FITS ? Cfg::WP : 0;
}
template <typename Real, int N> int shape_wp_of(int shape, bool contig) {
    switch (shape) {
        case 1: return shape_wp<Real, N, 1>(contig);
        case 2: return shape_wp<Real, N, 2>(contig);
        case 3: return shape_wp<Real, N, 3>(contig);
        case 4: return shape_wp<Real, N, 4>(contig);
        case 5: return shape_wp<Real, N, 5>(contig);
        case 6: return shape_wp<Real, N, 6>(contig);
        case 7: return shape_wp<Real, N, 7>(contig);
        default: return shape_wp<Real, N, 0>(contig);
    }
}
}  // namespace

int async_pencils_per_cta_shape(bool f64, int n, bool contig, int shape) {
    static_assert(kPassVariants == 8, "one case per launch shape");
    if (shape != 0 && (f64 || !shape_sizes_has(n))) return 0;   // no kernel of that shape
    switch (n) {
#define SOP_CASE(N) \
    case N:         \
        return f64 ? shape_wp_of<double, N>(shape, contig) : shape_wp_of<float, N>(shape, contig);
        SOP_SIZES(SOP_CASE)
#undef SOP_CASE
        default:
            return 0;
    }
}

int async_pencils_per_cta(bool f64, int n, int nc, bool contig) {
    switch (n) {
#define SOP_CASE(N) \
    case N:         \
        return f64 ? async_wp_of<double, N>(nc, contig) : async_wp_of<float, N>(nc, contig);
        SOP_SIZES(SOP_CASE)
#undef SOP_CASE
        default:
            return 0;
    }
}

cudaError_t persistent_grid(const void *kern, int threads, size_t smem, int *blocks_per_sm, int *sms) {
    // Resident CTAs per SM and SM count, cached per (kernel, device).
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, std::pair<int, int>> cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find({kern, dev});
    if (it != cache.end()) {
        *blocks_per_sm = it->second.first;
        *sms = it->second.second;
        return cudaSuccess;
    }
    int nb = 0, ns = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&ns, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (nb < 1) nb = 1;
    cache[{kern, dev}] = {nb, ns};
    *blocks_per_sm = nb;
    *sms = ns;
    return cudaSuccess;
}

cudaError_t ensure_smem_attr(const void *kern, int bytes) {
    // The attribute is per function and device; remember which pairs are set.
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({kern, dev})) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.insert({kern, dev});
    return e;
}
#endif

}  // namespace sop
