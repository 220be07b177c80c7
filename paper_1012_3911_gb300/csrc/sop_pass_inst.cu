// sop_pass_inst.cu -- instantiates the pencil-pass kernels for one dtype and
// one axis kind.  The build compiles this file four times:
//   -DSOP_REAL=float|double  -DSOP_CONTIG=1 (axis 0, contiguous) | 0 (strided)
#include "sop_async.cuh"

#ifndef SOP_REAL
#error "SOP_REAL must be defined"
#endif
#ifndef SOP_CONTIG
#error "SOP_CONTIG must be defined"
#endif

#define SOP_CAT2(a, b) a##b
#define SOP_CAT(a, b) SOP_CAT2(a, b)
#if SOP_CONTIG
#define SOP_KIND _contig
#else
#define SOP_KIND _strided
#endif
#define SOP_SUFFIX_float _f32
#define SOP_SUFFIX_double _f64
#define SOP_LAUNCH_NAME SOP_CAT(SOP_CAT(launch_pass, SOP_CAT(SOP_SUFFIX_, SOP_REAL)), SOP_KIND)
#define SOP_ASYNC_NAME SOP_CAT(SOP_CAT(launch_async, SOP_CAT(SOP_SUFFIX_, SOP_REAL)), SOP_KIND)

#define SOP_SIZES(X) \
    X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) \
    X(1536) X(2048) X(3072) X(4096)

namespace sop {

cudaError_t SOP_LAUNCH_NAME(const PassArgs &a, int nc, cudaStream_t s) {
    const int n = (int)a.dims[a.axis];
    switch (n) {
#define SOP_CASE(N)                                                                   \
    case N:                                                                           \
        return nc == 1 ? launch_pass_t<SOP_REAL, N, 1, (SOP_CONTIG != 0)>(a, s)       \
                       : launch_pass_t<SOP_REAL, N, 2, (SOP_CONTIG != 0)>(a, s);
        SOP_SIZES(SOP_CASE)
#undef SOP_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t SOP_ASYNC_NAME(const PassArgs &a, int nc, const TensorMapBytes &tmap, cudaStream_t s,
                           int64_t *ctr_advance) {
    const int n = (int)a.dims[a.axis];
    switch (n) {
#define SOP_CASE(N)                                                                           \
    case N:                                                                                   \
        return nc == 1 ? launch_async_t<SOP_REAL, N, 1, (SOP_CONTIG != 0)>(a, tmap, s, ctr_advance) \
                       : launch_async_t<SOP_REAL, N, 2, (SOP_CONTIG != 0)>(a, tmap, s, ctr_advance);
        SOP_SIZES(SOP_CASE)
#undef SOP_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

#if SOP_CONTIG
int SOP_CAT(stage_table, SOP_CAT(SOP_SUFFIX_, SOP_REAL))(int n, int nc, void *out, const void *tw, cudaStream_t s) {
    switch (n) {
#define SOP_CASE(N) \
    case N:         \
        return nc == 1 ? stage_table_t<SOP_REAL, N, 1>(out, tw, s) : stage_table_t<SOP_REAL, N, 2>(out, tw, s);
        SOP_SIZES(SOP_CASE)
#undef SOP_CASE
        default:
            return -1;
    }
}
#endif

}  // namespace sop
