// sop_pass4_inst.cu -- instantiates the four-component pencil passes of the
// three-dimensional Dirac step (all four spinor components of a pencil in one
// CTA, the 4x4 factors fused between the transforms) for one dtype and axis
// kind.  The build compiles this file four times:
//   -DSOP_REAL=float|double  -DSOP_CONTIG=1 (axis 0) | 0 (strided axes)
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
#define SOP_ASYNC4_NAME SOP_CAT(SOP_CAT(launch_async4, SOP_CAT(SOP_SUFFIX_, SOP_REAL)), SOP_KIND)

#define SOP_SIZES4(X) \
    X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024)

namespace sop {

cudaError_t SOP_ASYNC4_NAME(const PassArgs &a, const TensorMapBytes &tmap, cudaStream_t s, int64_t *ctr_advance) {
    const int n = (int)a.dims[a.axis];
    switch (n) {
#define SOP_CASE(N) \
    case N:         \
        return launch_async_t<SOP_REAL, N, 4, (SOP_CONTIG != 0)>(a, tmap, s, ctr_advance);
        SOP_SIZES4(SOP_CASE)
#undef SOP_CASE
        default:
            *ctr_advance = 0;
            return cudaErrorInvalidValue;
    }
}

}  // namespace sop
