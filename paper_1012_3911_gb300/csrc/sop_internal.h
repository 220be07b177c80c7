// sop_internal.h -- declarations shared by the host driver and the kernel
// translation units of libsop.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sop {

// Pointwise operator applied between the two transforms of a pass.
enum PassOp : int {
    OP_NONE = 0,  // transforms only
    OP_V = 1,     // Schroedinger real-space factor (Eq. 11, length-gauge field)
    OP_T = 2,     // Schroedinger momentum-space factor (Eq. 13) and 1/N
    OP_DV = 3,    // Dirac real-space factor (Eqs. 21-26), one component pair
    OP_DT = 4,    // Dirac momentum-space factor (Eq. 33 in closed form) and 1/N
    OP_D3V = 5,   // 3D Dirac real-space factor on all four components (Eqs. 21-26, 4x4)
    OP_D3T = 6,   // 3D Dirac momentum-space factor on all four components and 1/N
};

// Arguments of one pencil pass along one axis.  A "pencil" is the set of
// n = dims[axis] points that differ only in the axis index.
struct InstDesc;

struct PassArgs {
    void *psi;               // complex array of the plan's dtype
    int64_t comp_stride;     // points per component (prod dims)
    int64_t n_pencils;       // pencils per batch entry (prod of the other dims)
    int n_batch;             // independent copies (components treated as a batch)
    int64_t stride;          // element stride along the axis = prod(dims[0..axis-1])
    int ndim;
    int axis;
    int64_t dims[3];
    int pre;                 // transform before the operator: 0 none, -1 forward, +1 inverse
    int post;                // transform after the operator
    int op;                  // PassOp
    const void *tw;          // twiddles exp(-2 pi i e / n), e < n, plan dtype
    const void *stw;         // the per-stage twiddle table of the pass axis (persistent passes)
    // OP_V / OP_DV: per-point phase table (z-form for FP32, factor for FP64), may be null
    const void *vtab;
    // OP_V: per-axis field phase tables of this pass (null = axis has no field)
    const void *ftab[3];
    // OP_V with mat_out set (contiguous single-lattice passes): the state
    // between the two half factors is written to mat_out.  vtab is then the
    // half-step phase table, ftab the field rows of the trailing half of the
    // previous step and fh2 those of the leading half of this one.
    void *mat_out;
    const void *fh2[3];
    // OP_T: per-axis kinetic tables
    const void *ttab[3];
    // OP_DT: per-momentum table (cos, sin*mc^2/E, sin*c p_x/E, sin*c p_y/E)
    const void *dtab;
    double scale_hi, scale_lo;   // 1/N as an unevaluated sum hi + lo
    // OP_DV: 2x2 complex block per component pair (re, im of m00, m01, m10, m11)
    double mix[2][8];
    int pair_comp[2][2];     // component indices of each pair
    // OP_D3V: the merged 4x4 mixing (row-major re, im) or, with rows4 set, the
    // compact mixing row (8 reals, plan precision) of each x_1 column
    double mix4[32];
    const void *rows4;
    // Persistent asynchronous passes (filled by the launcher)
    int *errflag;            // device word; bit 1 set when a bounded wait gave up
    uint64_t wait_ns;        // limit of the tile-copy waits (0: kWaitLimitNs)
    // Dynamic tile scheduling: CTAs claim tiles with atomicAdd on
    // tile_ctr[pz] (pz: component pair); claim - tile_base[pz] is the tile
    // index.  A launch advances each counter it uses by n_tiles + gridDim.x
    // (every CTA ends with one claim past the last tile).
    unsigned long long *tile_ctr;
    unsigned long long tile_base[2];
    // Multi-instance passes (inst != null): tiles of n_inst lattices that
    // share the pass-axis size; P is the real-space index of the launch
    // (its row in each instance's field table is P - p_table0) and n_total
    // the step count of the call (P = 0 and P = n_total take the half factor).
    const InstDesc *inst;
    int n_inst;
    int64_t P, p_table0, n_total;
    // Graph-replayed steps: when set, the launch is a merged middle step
    // (full real-space factor) whose field row P - p_table0 is read from this
    // device word (advanced by the replayed graph itself) instead of P.
    const int64_t *row_dev;
    int64_t n_tiles;         // tiles of the pass (per component pair for nc == 2)
    int64_t n_xgroups;       // strided: tiles along x
    int64_t o_stride;        // strided: element stride of the remaining coordinate
    int n_comp_total;        // components in the array (tensor-map outer extent)
};

// One lattice of a multi-instance pass (device memory; a batch of
// independent Schroedinger problems advanced in lockstep).  The tensor map
// comes first so that it is 64-byte aligned.
struct alignas(64) InstDesc {
    unsigned char tmap[128];   // CUtensorMap of psi for the strided axis of the pass
    void *psi;
    const void *vhalf, *vfull; // per-point phase tables (half and merged real-space factor), may be null
    const void *ftab;          // field tables of the launch's chunk: rows of frow_len, or null
    const void *ttab[3];       // kinetic rows per axis
    int64_t foff[3];           // offset of axis a in a field row; -1: no field along a
    int64_t frow_len;
    int64_t dims[3];
    int64_t n_pencils, n_xgroups, o_stride;
    int64_t tiles_per_batch;   // strided axes: n_xgroups x (pencils / n_x)
    int64_t tile_begin;        // first global tile of this instance
    double scale_hi, scale_lo; // 1/N of this lattice
};

// Arguments of the one-dimensional whole-step kernel.
struct Args1D {
    void *psi;
    int64_t n_rows;          // independent 1D problems
    int64_t n_steps;         // steps of the whole sop_step call
    int64_t p_begin, p_end;  // real-space factor indices handled by this launch
    int64_t p_table0;        // index of the first field-table row in ftab
    const void *tw;
    const void *vhalf, *vfull;   // phase tables (may be null)
    const void *ftab;            // field tables, row per real-space index, n entries (may be null)
    const void *ttab;            // kinetic table, or rows of ttab_stride entries per step (velocity gauge)
    int64_t ttab_stride;         // 0: one table for every step; else row (P - p_table0) for step P
    double scale_hi, scale_lo;
    // Two-component Dirac (1D): mixing rows of 4 complex values (m00, m01,
    // m10, m11) in the plan's precision per real-space index, row P - p_table0,
    // and the per-momentum table (cos, sin mc^2/E, sin c p/E, 0) of the
    // momentum-space factor
    const void *mtab;
    const void *dtab;
};

// Launchers, one translation unit per dtype and axis kind (sop_pass_inst.cu
// compiled four times, sop_1d_inst.cu twice).  nc: coupled components per
// pencil (1 or 2).  They return cudaErrorInvalidValue for a size without a
// kernel.
// Three-dimensional four-component Dirac (sop_dirac3d.cu): the per-momentum
// table (8 reals per momentum in the plan's precision), the real-space factor
// exp(-i V tau') M (M: 16 complex FP64 values, row-major; vtab may be null) and
// the momentum-space factor with 1/N, each one pass over the four components.
cudaError_t build_dirac3_table(void *out, const int64_t *dims, const double *h, double mass, double c, double hbar,
                               double dt, bool f64, cudaStream_t s);
cudaError_t launch_dirac3_real(void *psi, int64_t npts, const void *vtab, const double *M, const void *rows,
                               int64_t nx, bool f64, cudaStream_t s);
// Merged mixing per column for rows P0 .. P0 + n_rows - 1 (8 reals of the
// plan's precision each, [row][column][8]: a, b, d, 0 of a + i b.alpha +
// i d.Sigma) from the device samples avec (n_steps x nx x ndim doubles);
// with M = null, launch_dirac3_real uses these rows instead of the uniform M.
cudaError_t build_mix_rows(void *out, const double *avec, int64_t P0, int64_t n_rows, int64_t nx, int ndim,
                           int64_t n_steps, double charge, double c, double hbar, double tau, bool f64,
                           cudaStream_t s);
cudaError_t launch_dirac3_kinetic(void *psi, int64_t npts, const void *tab, double shi, double slo, bool f64,
                                  cudaStream_t s);
// One-dimensional two-component Dirac whole-step kernel (sop_1d_inst.cu).
cudaError_t launch_1d_dirac_f32(const Args1D &a, int n, cudaStream_t s);
cudaError_t launch_1d_dirac_f64(const Args1D &a, int n, cudaStream_t s);
cudaError_t launch_pass_f32_contig(const PassArgs &a, int nc, cudaStream_t s);
cudaError_t launch_pass_f32_strided(const PassArgs &a, int nc, cudaStream_t s);
cudaError_t launch_pass_f64_contig(const PassArgs &a, int nc, cudaStream_t s);
cudaError_t launch_pass_f64_strided(const PassArgs &a, int nc, cudaStream_t s);
// Persistent passes with asynchronous (bulk / TMA) prefetch of the next tile.
// tmap: the 4D tensor map of psi for strided axes (ignored for axis 0).
// *ctr_advance: how far the launch moves the tile counters.
struct TensorMapBytes {
    alignas(64) unsigned char b[128];
};
cudaError_t launch_async_f32_contig(const PassArgs &a, int nc, const TensorMapBytes &tmap, cudaStream_t s,
                                 int64_t *ctr_advance);
cudaError_t launch_async_f32_strided(const PassArgs &a, int nc, const TensorMapBytes &tmap, cudaStream_t s,
                                 int64_t *ctr_advance);
cudaError_t launch_async_f64_contig(const PassArgs &a, int nc, const TensorMapBytes &tmap, cudaStream_t s,
                                 int64_t *ctr_advance);
cudaError_t launch_async_f64_strided(const PassArgs &a, int nc, const TensorMapBytes &tmap, cudaStream_t s,
                                 int64_t *ctr_advance);
// Four-component passes of the 3D Dirac step (sop_pass4_inst.cu, sides up to
// 1024); cudaErrorInvalidValue for a side without a kernel that fits an SM.
cudaError_t launch_async4_f32_contig(const PassArgs &a, const TensorMapBytes &tmap, cudaStream_t s,
                                     int64_t *ctr_advance);
cudaError_t launch_async4_f32_strided(const PassArgs &a, const TensorMapBytes &tmap, cudaStream_t s,
                                      int64_t *ctr_advance);
cudaError_t launch_async4_f64_contig(const PassArgs &a, const TensorMapBytes &tmap, cudaStream_t s,
                                     int64_t *ctr_advance);
cudaError_t launch_async4_f64_strided(const PassArgs &a, const TensorMapBytes &tmap, cudaStream_t s,
                                      int64_t *ctr_advance);
// Launch-shape variants 1 .. kPassVariants - 1 of the persistent pass
// (sop_pass_var.cu, complex64 only); cudaErrorInvalidValue for a size, dtype
// or variant without a kernel.
constexpr int kPassVariants = 8;
cudaError_t launch_async_variant(bool f64, bool contig, int var, const PassArgs &a, int nc, const TensorMapBytes &tmap,
                                 cudaStream_t s, int64_t *ctr_advance);
// Adjoint-gradient reductions (sop_adjoint.cu).  launch_inner writes 8
// doubles to out: dV (<a|b>, <a|X_0|b>, <a|X_1|b>, <a|X_2|b>) as re, im
// pairs (axes beyond ndim are zero); partial holds inner_partials() doubles.
int inner_partials();
cudaError_t launch_inner(const void *a, const void *b, bool f64, int ndim, const int64_t *dims, const double *h,
                         double dV, double *partial, double *out, cudaStream_t s);
// A whole checkpoint segment: for k < count, slots k of lam and psi (count
// consecutive lattices each) hold the costate and the state of step m0 + k;
// writes the 8 values of launch_inner for each step into out + (m0 + k) 8 and
// adds sum_k w_k conj(lam_k) psi_k to acc (w = 1 for step 0, else 2).
// partial holds seg_partials(count) doubles.
int seg_partials(int count);
cudaError_t launch_seg_reduce(const void *lam, const void *psi, bool f64, int count, int64_t m0, int ndim,
                              const int64_t *dims, const double *h, double dV, double *acc, double *partial,
                              double *out, cudaStream_t s);
// acc_j += w conj(a_j) b_j, 16 bytes per point: complex128 (f64) or, for
// complex64 states, the float pair (hi.re, hi.im, lo.re, lo.im) that
// launch_grad_v reads back
cudaError_t launch_accum(const void *a, const void *b, bool f64, int64_t npts, double w, double *acc,
                         cudaStream_t s);
// Spectral method.  launch_spectral_sample: chi[0..1] = dV <psi0|psi> and,
// if slot is not NULL, a copy of psi into slot (len values); partial holds
// inner_partials() doubles, *done is a zeroed counter (left zeroed).  launch_spectral_accum: acc[k][j] += sum_{b<B}
// (wre[b K + k] + i wim[b K + k]) ring[b len + j] for B <= SOP_SPECTRAL_RING
// states and K <= SOP_SPECTRAL_MAX_ENERGIES energies (acc: K x len double2).
// For complex64 states the accumulator holds float pairs until
// launch_spectral_finish (n = K x len values) turns them into complex128; a
// no-op for complex128.
// launch_spectrum: the windowed transform of chi (N + 1 pairs) at K energies
// (device array E) into spec (2 K doubles).
#define SOP_SPECTRAL_MAX_ENERGIES 16
#define SOP_SPECTRAL_RING 8
cudaError_t launch_spectral_sample(const void *psi0, const void *psi, bool f64, int64_t len, void *slot, double dV,
                                   double *partial, unsigned *done, double *chi, cudaStream_t s);
cudaError_t launch_spectral_accum(const void *ring, bool f64, int B, int64_t len, int K, const double *wre,
                                  const double *wim, double *acc, cudaStream_t s);
cudaError_t launch_spectral_finish(double *acc, bool f64, int64_t n, cudaStream_t s);
cudaError_t launch_spectrum(const double *chi, int64_t N, double dt, double hbar, const double *E, int K,
                            double *spec, cudaStream_t s);
// g_j = 2 Re((zr + i zi) acc_j), acc as launch_accum left it
cudaError_t launch_grad_v(const double *acc, bool f64, int64_t npts, double zr, double zi, double *g,
                          cudaStream_t s);

// Per-stage twiddle table of an n-point axis for the persistent passes:
// out == nullptr returns its entry count, else fills out from tw (async);
// -1 for a size without persistent passes.
int stage_table_f32(int n, int nc, void *out, const void *tw, cudaStream_t s);
// *p = v, and *p += 1, each one single-thread kernel on s (the step row of
// graph-replayed batched steps).
cudaError_t set_counter(int64_t *p, int64_t v, cudaStream_t s);
cudaError_t advance_counter(int64_t *p, cudaStream_t s);
int stage_table_f64(int n, int nc, void *out, const void *tw, cudaStream_t s);
// Pencils per CTA of the asynchronous pass (the tensor-map box width for
// strided axes); 0 when that pass does not fit on an SM (one-shot passes).
int async_pencils_per_cta(bool f64, int n, int nc, bool contig);
// The same for one-component passes of launch shape `shape` (the pencils per
// CTA of the contiguous axis depend on the shape; those of strided axes,
// which set the tensor-map box, do not).
int async_pencils_per_cta_shape(bool f64, int n, bool contig, int shape);
// Sides with launch shapes other than 0 (sop_pass_var.cu instantiates these).
#define SOP_VAR_SIZES(X) X(256) X(384) X(512) X(768) X(1024) X(1536) X(2048)
inline bool shape_sizes_has(int64_t n) {
#define SOP_VAR_HAS(N) n == N ||
    return SOP_VAR_SIZES(SOP_VAR_HAS) false;
#undef SOP_VAR_HAS
}
cudaError_t launch_1d_f32(const Args1D &a, int n, cudaStream_t s);
cudaError_t launch_1d_f64(const Args1D &a, int n, cudaStream_t s);
// Threads and dynamic shared memory of the pass kernel for (dtype, n, nc, contig).
bool pass_geometry(bool f64, int n, int nc, bool contig, int *threads, int *pencils_per_cta, int *smem);

// Sides with a kernel: 2^a * 3^b, a >= 2, b <= 1, 8 <= n <= 4096.
inline bool size_supported(int64_t n) {
    if (n < 8 || n > 4096) return false;
    if (n % 3 == 0) n /= 3;
    if (n < 4) return false;
    return (n & (n - 1)) == 0;
}

// Table set-up kernels (sop_tables.cu).  All phases are formed in FP64.
cudaError_t build_twiddles(void *out, int n, bool f64, cudaStream_t s);
cudaError_t build_vphase(void *out, const double *V, int64_t npts, double factor, bool f64,
                         cudaStream_t s);
cudaError_t build_axis_phase(void *out, const double *coef, int n, bool f64, cudaStream_t s);
// Velocity-gauge kinetic rows (Eq. 13): row P (< n_rows) holds, for each
// active axis a at offsets[a], exp(-i c (p_{a,k} - svec[P ndim + a])^2).
cudaError_t build_kin_field_tables(void *out, const double *svec, int64_t n_rows, int ndim, const int64_t *dims,
                                   const double *spacing, const int *active, const int64_t *offsets, int64_t row_len,
                                   double c, double hbar, bool f64, cudaStream_t s);
cudaError_t build_field_tables(void *out, const double *fvec, int64_t n_rows, int ndim,
                               const int64_t *dims, const double *spacing, const int *active,
                               const int64_t *offsets, int64_t row_len, bool f64, cudaStream_t s);
cudaError_t build_dirac_table(void *out, const int64_t *dims, const double *spacing, double mass,
                              double c, double hbar, double dt, bool f64, cudaStream_t s);
// out = in in FP64; *bad (if not null) becomes nonzero for a non-finite value.
cudaError_t convert_potential(double *out, const void *in, int64_t n, bool in_f64, int *bad, cudaStream_t s);

// Reductions (sop_reduce.cu).  partial must hold reduce_blocks() doubles.
int reduce_blocks();
cudaError_t reduce_norm(const void *psi, int64_t n, bool f64, double *partial, double *out,
                        double scale, cudaStream_t s);
cudaError_t reduce_energy_v(const void *psi, const double *V, int64_t npts, int comps, bool f64,
                            double *partial, double *out, double scale, cudaStream_t s);
cudaError_t reduce_energy_t(const void *psit, int ndim, const int64_t *dims,
                            const double *pgrid /* concatenated per-axis momenta */, int comps,
                            double mass, double c, bool f64, double *partial, double *out,
                            double scale, cudaStream_t s);

}  // namespace sop
