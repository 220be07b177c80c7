// sop_pass_var.cu -- launch-shape variants of the persistent pencil pass for
// the sizes of the paper-shaped lattices.  The build compiles this file once
// per dtype, axis kind and variant:
//   -DSOP_REAL=float|double  -DSOP_CONTIG=1|0  -DSOP_VAR=1..kPassVariants-1
// Each unit defines launch_async_var_<dtype>_<kind>_<VAR>; sizes it does not
// instantiate return cudaErrorInvalidValue (the caller then uses variant 0).
#include "sop_async.cuh"

#ifndef SOP_REAL
#error "SOP_REAL must be defined"
#endif
#ifndef SOP_CONTIG
#error "SOP_CONTIG must be defined"
#endif
#ifndef SOP_VAR
#error "SOP_VAR must be defined"
#endif

#define SOP_CAT2(a, b) a##b
#define SOP_CAT(a, b) SOP_CAT2(a, b)
#if SOP_CONTIG
#define SOP_KIND _contig_
#else
#define SOP_KIND _strided_
#endif
#define SOP_SUFFIX_float _f32
#define SOP_SUFFIX_double _f64
#define SOP_VAR_NAME SOP_CAT(SOP_CAT(SOP_CAT(launch_async_var, SOP_CAT(SOP_SUFFIX_, SOP_REAL)), SOP_KIND), SOP_VAR)


namespace sop {

cudaError_t SOP_VAR_NAME(const PassArgs &a, int nc, const TensorMapBytes &tmap, cudaStream_t s,
                         int64_t *ctr_advance) {
    const int n = (int)a.dims[a.axis];
    switch (n) {
#define SOP_CASE(N)                                                                                               \
    case N:                                                                                                       \
        return nc == 1 ? launch_async_t<SOP_REAL, N, 1, (SOP_CONTIG != 0), SOP_VAR>(a, tmap, s, ctr_advance)     \
                       : launch_async_t<SOP_REAL, N, 2, (SOP_CONTIG != 0), SOP_VAR>(a, tmap, s, ctr_advance);
        SOP_VAR_SIZES(SOP_CASE)
#undef SOP_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace sop
