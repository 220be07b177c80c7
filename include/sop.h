/*
 * sop.h -- C ABI of libsop.so, a GB300 (sm_103a) Fourier split-operator
 * propagator for the time-dependent Schroedinger equation (scalar psi) and
 * the Dirac equation (four-component spinor) on periodic 1D/2D/3D lattices.
 *
 * One time step of size tau is the second-order Strang factorisation of
 * Bauke & Keitel (arXiv:1012.3911), Eqs. 6-8:
 *     psi <- U_A1(1/2) F^-1 U~_A2(1) F U_A1(1/2) psi
 * with the Schroedinger split of Eqs. 10a/10b (real-space factor Eq. 11,
 * momentum-space factor Eq. 13) and the Dirac split of Eqs. 18a/18b
 * (real-space factor Eqs. 21-26, momentum-space factor Eqs. 27-33).
 *
 * Conventions (all calls):
 *   - Units are set by sop_params (default: atomic units, electron:
 *     mass 1, charge -1, hbar 1, c 137.036).
 *   - Lattice: axis a has dims[a] points with spacing spacing[a];
 *     x_{a,j} = -dims[a]*spacing[a]/2 + j*spacing[a] (the box [-L/2, L/2)).
 *     Momenta p_{a,k} = hbar*2*pi*kappa/(dims[a]*spacing[a]) with kappa = k
 *     for 2k < dims[a], else k - dims[a].
 *   - Layout: psi is interleaved complex (complex64 = 2 x float, or
 *     complex128 = 2 x double) in C order with axis 0 (x) fastest:
 *     psi[c][z][y][x]; components c are contiguous blocks of prod(dims)
 *     points.  dims[0] = n_x.
 *   - Fields: field_samples holds n_steps rows of ndim doubles, the field at
 *     the midpoint t_n + tau/2 of each step, components in axis order.  For
 *     Schroedinger it is by default the electric field E in the length gauge
 *     (the scalar potential gains -q x.E), or the vector potential A in the
 *     velocity gauge after sop_set_gauge; for Dirac it is the uniform vector
 *     potential A of Eq. 18a.  NULL means no field.
 *   - Every call returns a sop_status.  Nothing throws across the ABI.  On a
 *     non-zero status, sop_last_error() returns a thread-local message.
 *   - Ownership: the plan owns its tables and scratch (device memory it
 *     allocates at create time or on first use); the caller owns psi and V.
 *   - Streams: all device work of a plan is enqueued on the CUDA stream
 *     given at create time (NULL: the legacy default stream).  sop_step is
 *     asynchronous; sop_norm, sop_energy and sop_step_host synchronise that
 *     stream.
 */
#ifndef SOP_H
#define SOP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sop_plan_s *sop_plan;

typedef enum { SOP_C64 = 0, SOP_C128 = 1 } sop_dtype;

typedef enum {
    SOP_OK = 0,
    SOP_EINVAL = -1,          /* bad argument (null pointer, bad size, misaligned pointer) */
    SOP_EUNSUPPORTED = -2,    /* valid but not supported (side not 2^a*3^b in [8,4096], ...) */
    SOP_ENOMEM = -3,          /* device allocation failed */
    SOP_ECUDA = -4,           /* a CUDA call failed; the message names it */
    SOP_ETIMEOUT = -5,        /* reserved for bounded device-side waits */
    SOP_ESTATE = -6           /* call out of order (e.g. stepping before a state is bound) */
} sop_status;

/* Physical constants; pass NULL to sop_plan_create for atomic units and an
 * electron (mass 1, charge -1, hbar 1, c 137.036). */
typedef struct {
    double mass;
    double charge;
    double hbar;
    double c;
} sop_params;

/* Create a plan for one lattice (Sec. 2.1: a regular rectangular lattice
 * of N points on which the Fourier transform becomes a DFT).
 *   out        receives the plan handle.
 *   ndim       1, 2 or 3.
 *   dims       ndim sides in axis order (dims[0] = n_x, contiguous); each
 *              side must be 2^a * 3^b with a >= 2, b <= 1 and 8 <= side <= 4096.
 *   spacing    ndim lattice spacings (> 0).
 *   components 1 (Schroedinger, Sec. 2.2), 4 (Dirac, Sec. 2.3, ndim = 2 or 3;
 *              in 3D the 4x4 factors couple all components and run as
 *              separate streaming passes between the transforms) or
 *              2 (the one-dimensional two-component Dirac equation at the
 *              end of Sec. 2.3, ndim = 1, alpha_1 = sigma_x, beta = sigma_z;
 *              field_samples are A_1, one per step).
 *   dtype      SOP_C64 (FP32 arithmetic, phase and twiddle tables formed in
 *              FP64 and rounded) or SOP_C128 (FP64 throughout).
 *   params     NULL or the physical constants.
 *   cuda_stream  a cudaStream_t (as void*) or NULL.
 * Allocates the plan's twiddle tables, reduction scratch and field-table
 * buffers on the current device.  Returns SOP_EINVAL, SOP_EUNSUPPORTED,
 * SOP_ENOMEM or SOP_ECUDA on failure (then *out is NULL). */
int sop_plan_create(sop_plan *out, int ndim, const int64_t *dims, const double *spacing,
                    int components, int dtype, const sop_params *params, void *cuda_stream);

/* Free every device buffer the plan owns.  Waits for the plan's stream.
 * Accepts NULL. */
int sop_plan_destroy(sop_plan plan);

/* Bind the wave function: psi_dev is a device pointer to components *
 * prod(dims) complex values of the plan's dtype, 16-byte aligned (the pass
 * kernels copy rows and tiles of it with bulk asynchronous copies).  The
 * plan borrows it; the caller keeps it alive while the plan steps.  sop_step
 * updates it in place.  Returns SOP_EINVAL for a NULL or misaligned pointer. */
int sop_bind_state(sop_plan plan, void *psi_dev);

/* Set the potential energy V (= q*phi of Eqs. 10a/18a, without the laser
 * term) from a device array of prod(dims) reals, FP64 if v_is_fp64 else
 * FP32.  The plan copies it (FP64) and rebuilds the phase tables
 * exp(-i V tau/(2 hbar)) and exp(-i V tau/hbar) at the next sop_step.
 * A plan whose potential was never set uses V = 0.  The conversion checks
 * every value and the call synchronises the plan stream to read the check:
 * SOP_EINVAL for a value that is not finite (the plan is then left without a
 * potential), SOP_EINVAL for a NULL or misaligned pointer. */
int sop_set_potential(sop_plan plan, const void *V_dev, int v_is_fp64);

/* Meaning of the field samples of a Schroedinger plan (Sec. 2.2):
 * SOP_GAUGE_LENGTH (the default): field_samples are the electric field E
 * at each step's midpoint, entering the real-space factor (Eq. 11 with
 * q phi = V - q x.E, the length gauge).  SOP_GAUGE_VELOCITY: they are the
 * vector potential A at each step's midpoint, entering the momentum-space
 * factor of Eq. 13 as exp(-i tau |p - q A|^2 / (2 m hbar)) (the time integral
 * of Eq. 13 by the midpoint rule; per-step kinetic rows are built on the
 * device for every 512 steps).  Dirac plans always take A (SOP_EUNSUPPORTED
 * here).  The adjoint gradient and batches accept length-gauge plans only.
 * Returns SOP_EINVAL for another value. */
/* Dirac plans (components = 4, 2D or 3D): along_x1 = 1 makes the field
 * samples a vector potential that varies along x_1, A(x_1, t), as for a
 * plane-wave laser pulse travelling along x_1 (the paper's scattering
 * example): field_samples then holds n_steps x dims[0] x ndim doubles, A at
 * each step's midpoint and lattice column i of axis 0 ([step][i][component]).
 * The mixing of Eq. 26 is then formed per column (on the device, in FP64, for
 * every 64 steps) and applied as a streaming pass of its own between the x
 * transforms; along_x1 = 0 (the default) is the uniform A.  Returns
 * SOP_EUNSUPPORTED for other plans, SOP_EINVAL for another value. */
int sop_set_field_profile(sop_plan plan, int along_x1);

#define SOP_GAUGE_LENGTH 0
#define SOP_GAUGE_VELOCITY 1
int sop_set_gauge(sop_plan plan, int gauge);

/* Advance the bound state by n_steps Strang steps of size dt (Eq. 8).  The
 * real-space factors of adjacent steps are merged (exact algebra): the call
 * applies one half real-space factor at its start and one at its end.
 * field_samples: host array of n_steps*ndim doubles or NULL (see above);
 * n_steps*dims[0]*ndim for a Dirac plan after sop_set_field_profile(plan, 1).
 * Asynchronous on the plan stream.  n_steps = 0 is a no-op.  Returns
 * SOP_ESTATE if no state is bound. */
int sop_step(sop_plan plan, int64_t n_steps, double dt, const double *field_samples);

/* As sop_step, for a wave function in HOST memory: copies psi_host (same
 * layout and dtype as the bound state) to the bound device buffer, steps,
 * copies the result back into psi_host and synchronises the stream.  The
 * host->device and device->host copies are inside the call (the paper's
 * "overall time including transfers", Sec. 4.2).  psi_host may be pinned or
 * pageable. */
int sop_step_host(sop_plan plan, void *psi_host, int64_t n_steps, double dt,
                  const double *field_samples);

/* *out = dV * sum over points and components of |psi|^2, accumulated in
 * FP64 (dV = product of spacings).  Synchronises the plan stream. */
int sop_norm(sop_plan plan, double *out);

/* *out = field-free energy <T> + <V> of the bound state, accumulated in
 * FP64: <V> = dV sum_j V_j |psi_j|^2 and <T> = (dV/N) sum_k psi~_k^dag T(p_k) psi~_k
 * with T = |p|^2/(2m) (Schroedinger) or c alpha.p + m c^2 beta (Dirac, Eq. 28).
 * Uses a plan-owned scratch copy of psi (allocated on first use).
 * Synchronises the plan stream. */
int sop_energy(sop_plan plan, double *out);

/* Per-pass device timing with CUDA events on the plan stream.
 * every = 0 disables it.  every = 1: sop_step records an event pair around
 * every kernel it launches.  every = k > 1: only the passes of one split
 * step in k are bracketed (step indices P = k/2 mod k within each sop_step
 * call, P = 0..n_steps for the real-space passes) together with every
 * table set-up kernel; the event records then barely perturb the back-to-
 * back pass launches, and per-class averages stay unbiased samples.
 * every < 0 is SOP_EINVAL.
 * sop_profile_read synchronises the stream and returns, per pass class,
 * the summed device milliseconds and the launch count since profiling was
 * enabled (arrays of max_classes entries, SOP_PASS_CLASSES at most); it
 * also resets the counters.  Classes: 0 real-space axis pass, 1 momentum-
 * space (last axis) pass, 2 middle-axis transform pass, 3 one-dimensional
 * whole-step kernel, 4 table set-up kernels. */
#define SOP_PASS_CLASSES 5
int sop_profile_enable(sop_plan plan, int every);
int sop_profile_read(sop_plan plan, double *ms, int64_t *launches, int max_classes);

/* Total number of kernels this plan has launched since it was created
 * (passes, table set-up and reductions).  Host-side counter; no sync. */
int64_t sop_launch_counter(sop_plan plan);

/* Launch shapes of the pencil passes (an implementation choice, not part of
 * the paper's method: every shape computes the same transforms, Sec. 2.1, in
 * the same operation order, so results are bit-identical across shapes).
 * A shape fixes the pencils per CTA, the number of tile buffers, where the
 * stage twiddles and the pass-axis factor row live (shared memory or L1) and
 * the register budget; SOP_PASS_SHAPES shapes exist, 0 is the default.
 *
 * sop_autotune: times every shape of the contiguous-axis pass (x), then of
 * the strided-axis passes (y, z), then both again with the other kind's
 * choice in place (two rounds of coordinate descent), for this plan's
 * lattice, component count and dtype, over trial_steps split steps of size
 * dt (<= 0: 16) with no field (best of five trials of whole steps), and
 * keeps the fastest of each.  The trials run on a scratch copy of
 * the bound state (allocated like sop_energy's scratch if absent), so the
 * state is unchanged.  Results are cached per process for the lattice shape,
 * component count, dtype and device: a later plan of the same shape takes
 * them without timing; with the environment variable SOP_AUTOTUNE_CACHE
 * naming a file, choices are also read from it (lines for this device model)
 * and new ones appended, so they persist across processes.  chosen (may be
 * NULL) receives 2 ints: the shapes of
 * the contiguous and the strided passes.  Synchronises the plan stream.
 * One-dimensional plans have no pencil passes (chosen = {0, 0}).
 * Errors: SOP_EINVAL (null plan), SOP_ESTATE (no state bound), SOP_ECUDA,
 * SOP_ETIMEOUT.
 *
 * sop_set_pass_shape: forces shape `shape` (0 .. SOP_PASS_SHAPES - 1) for the
 * contiguous (axis_kind 0) or strided (axis_kind 1) passes of this plan.
 * Sizes without a kernel of that shape use shape 0.  SOP_EINVAL for a bad
 * argument. */
#define SOP_PASS_SHAPES 8
int sop_autotune(sop_plan plan, double dt, int trial_steps, int *chosen);
int sop_set_pass_shape(sop_plan plan, int axis_kind, int shape);

/* Failure detection of the persistent passes (not part of the paper's
 * method).  Every wait of a pass kernel for its tile copies is bounded in wall
 * time (2 s by default, far beyond any copy).  A CTA whose wait runs out
 * records it in the plan's error word, lets its own copies finish and leaves;
 * later passes of the stream see the word and do nothing; the next
 * synchronising call (sop_norm, sop_energy, sop_step_host, ...) returns
 * SOP_ETIMEOUT and clears the word and the tile counters, after which the
 * plan steps normally again (the state of the failed call is unfinished).
 * sop_set_wait_limit sets the limit of the tile-copy waits in ns (0: the
 * default); a limit of a few ns makes the waits give up while the copies
 * still complete normally, which is how the error path is tested.
 * SOP_EINVAL for a null plan. */
int sop_set_wait_limit(sop_plan plan, uint64_t wait_ns);

/* Allocation-failure injection for tests of the error paths (not part of the
 * paper's method): after `after` more successful device allocations by this
 * library, the next one fails as if the device were out of memory (the call
 * that needed it returns SOP_ENOMEM and releases what it had allocated); a
 * negative value turns the injection off.  Process-wide.  Returns SOP_OK. */
int sop_debug_fail_alloc(int64_t after);

/* Check builds (a debugging aid, not part of the paper's method): compiled
 * with -DSOP_CHECK=1 (build.py with SOP_CHECK=1 in the environment writes
 * _build_check/libsop.so), the pass kernels test their global-memory indices
 * against the lattice, their shared-memory offsets against the tile buffer
 * and every TMA x coordinate for 16-byte alignment; a failed test skips the
 * access and sets bit 2 of the plan's error word, which the next
 * synchronising call reports as SOP_ECUDA.  Every device buffer of the
 * library is followed by 256 canary bytes, verified when it is freed.
 * sop_debug_check_canaries stores in *bad the number of overwritten canaries
 * (freed and live buffers) and returns SOP_OK; in a normal build it returns
 * SOP_EUNSUPPORTED.  Synchronises the device. */
int sop_debug_check_canaries(int64_t *bad);

/* Measured FMA throughput of the current device (not part of the paper's
 * method: the denominator of the arithmetic roofline reported for the FP64
 * split step).  Runs 8 independent FMA chains per thread on 8 CTAs of 256
 * threads per SM, times the best of 3 launches after a warm-up with CUDA
 * events on cuda_stream (NULL: legacy default) and writes 2 x FMAs per second
 * to *flops_per_s, for FP64 (f64 != 0) or FP32.  Synchronous; allocates and
 * frees one word of device memory.  SOP_EINVAL for a null output, SOP_ECUDA
 * for a CUDA error. */
int sop_fma_peak(int f64, double *flops_per_s, void *cuda_stream);

/* Norm without any device allocation.  Not part of the paper's method (it
 * has no counterpart there); it serves callers that may not allocate device
 * memory: programs whose own pool allocator owns all of HBM and forbids
 * other allocations, and latency-bound loops where cudaMalloc/cudaFree, which
 * can synchronise the whole device, would stall other streams.  Unlike
 * sop_norm it needs no plan.
 *   psi_dev   device pointer to n_values complex values (dtype SOP_C64 or
 *             SOP_C128), aligned to the complex size.
 *   out_dev   device pointer to one double; receives scale * sum |psi|^2,
 *             accumulated in FP64 (scale = dV gives the norm of sop_norm).
 *   cuda_stream  the stream the work is enqueued on (NULL: legacy default).
 * Asynchronous; the result is ready when the stream reaches it.  Calls no
 * cudaMalloc, cudaFree or allocating library routine: the block partial sums
 * live in a fixed array inside the library (256 KB on every GPU that loads
 * it, held until the process exits), so n_values is limited to 2^29;
 * larger inputs return SOP_EUNSUPPORTED.  Every slot the reduction reads is
 * written earlier in the same call, so nothing needs clearing between calls,
 * but all calls share the array: calls that may overlap on the GPU (unordered
 * streams or several host threads) race and must be serialised.  The first
 * call on each device looks up the array's device address (with that device
 * current) and keeps it for the life of the process; make that first call
 * before any stream capture.  Resetting a device (cudaDeviceReset) after that
 * first call is not supported: the kept address would then be stale.  Returns
 * SOP_EINVAL for null or misaligned pointers, a bad dtype or n_values < 0. */
int sop_norm_noalloc(const void *psi_dev, int64_t n_values, int dtype, double scale, double *out_dev,
                     void *cuda_stream);

/* Adjoint gradient of a final-state overlap (a follow-on of the method; the
 * paper has no adjoint).  With psi_0 the bound state (left unchanged),
 * psi_{n+1} = U_n psi_0 the split steps of Eqs. 6-8 / 10a-b with field
 * samples E_n (as sop_step), c = <phi|psi_N> = dV sum conj(phi) psi_N and
 * J = |c|^2, it returns
 *   *J,
 *   grad_field[n ndim + a] = dJ/dE_{n,a}       (host, n_steps x ndim; may be NULL)
 *   grad_V_dev[j]         = dJ/dV_j           (device, prod(dims) doubles; may be NULL)
 * from costates lambda_N = phi, lambda_n = U_n^dagger lambda_{n+1} (the step
 * with -dt):  dc/dE_{n,a} = (-i dt/(2 hbar)) (-q) (<lambda_{n+1}|X_a|psi_{n+1}>
 * + <lambda_n|X_a|psi_n>),  dc/dV_j = (-i dt/(2 hbar)) dV sum_n w_n
 * conj(lambda_{n,j}) psi_{n,j} (w = 1 at n = 0, N, else 2),  dJ = 2 Re(conj(c) dc).
 * Forward states are checkpointed every `every` steps and recomputed per
 * segment.  phi_dev: device array of the plan's dtype and lattice, 16-byte
 * aligned.  field may be NULL (all zero).  Schroedinger plans with fewer
 * than 2^31 lattice points only (SOP_EUNSUPPORTED otherwise); SOP_ESTATE without a bound state; SOP_EINVAL
 * for n_steps < 1, every < 1, dt zero or not finite, non-finite samples or
 * bad pointers.  Its checkpoints (ceil(n_steps/every) + 2 every + 3 states
 * and per-step overlaps) live in one device block that the plan keeps for
 * later calls of the same or a smaller size (grown when a call needs more,
 * freed by sop_plan_destroy); a second plan for the -dt steps is made on
 * first use and takes this plan's launch shapes and potential; synchronises
 * the plan stream. */
int sop_adjoint_gradient(sop_plan plan, const void *phi_dev, int64_t n_steps, double dt,
                         const double *field_samples, int64_t every, double *J, double *grad_field,
                         double *grad_V_dev);

/* Batched propagation (a follow-on of the method: many independent
 * problems).  A batch groups existing two-dimensional Schroedinger plans of
 * one dtype and one stream (sides may differ; each plan keeps its lattice,
 * potential, bound state and tables).  sop_batch_step advances every plan by
 * n_steps Strang steps of size dt exactly as sop_step would (Eqs. 6-8 with
 * the split of Eqs. 10a-b), in lockstep: per half step one persistent launch
 * per pass kind and per pass-axis size, whose tiles are claimed from one
 * counter across all lattices of that size (the instance is found from the
 * tile index; sizes without a persistent kernel, e.g. some complex128 sides
 * with a factor 3, take one-shot passes per lattice).  field_samples[i]
 * holds plan i's samples as for sop_step
 * (n_steps x 2, host) or NULL; field_samples itself may be NULL.
 * Asynchronous on the plans' stream; errors of the persistent kernels are
 * reported by the next synchronising call on the first plan.  The batch
 * borrows the plans: destroy the batch before them.  sop_batch_create
 * returns SOP_EUNSUPPORTED for other plan kinds, SOP_EINVAL for mixed dtypes
 * or streams or a repeated plan; sop_batch_step SOP_ESTATE when a plan has
 * no bound state. */
typedef struct sop_batch_s *sop_batch;
int sop_batch_create(sop_batch *out, int n_plans, const sop_plan *plans);
int sop_batch_step(sop_batch batch, int64_t n_steps, double dt, const double *const *field_samples);
int sop_batch_destroy(sop_batch batch);

/* Spectral method for eigenstates (the paper's eigenstates subsection): the
 * bound state is the trial state psi_0; it is advanced n_steps steps of size
 * dt in the time-independent potential (no field; each step a complete
 * Strang step, Eqs. 6-8 with the split of Eqs. 10a-b, so that every psi_n is
 * in real space), leaving psi_N bound.  With t_n = n dt, T = N dt:
 *   chi_n   = dV sum_j conj(psi_0,j) psi_n,j                 (autocorrelation)
 *   chi~(E) = dt sum_n (1 - cos(2 pi t_n / T)) chi_n exp(i E t_n / hbar)
 *   Psi_E   = dt sum_n (1 - cos(2 pi t_n / T)) psi_n exp(i E t_n / hbar)
 * for n = 0..N (the window vanishes at both ends); peaks of |chi~| are the
 * eigenvalues the trial state overlaps with and Psi_E at such a peak is the
 * (unnormalised) eigenfunction.  Sums over j run over all components (the
 * state's flat layout), so Dirac plans work alike.
 *   chi_out       host, 2 (n_steps + 1) doubles (re, im pairs) or NULL;
 *   energies      host, n_energies finite values (may be 0 with NULL);
 *   spectrum_out  host, 2 n_energies doubles (chi~(E_k) pairs) or NULL;
 *   psiE_dev      device complex128 [n_energies][points x components] in the
 *                 state's layout, 16-byte aligned, or NULL; requires
 *                 n_energies <= SOP_SPECTRAL_MAX_EIGEN.
 * chi is summed to about 48 significant bits or more (products, and sums of
 * four of them, in the state's precision; then float pairs for complex64
 * states, FP64 for complex128 states; block sums in FP64).  Psi_E is accumulated from the states of up to 8 consecutive
 * steps at a time (kept in a ring of state copies on the device; fewer when
 * memory is short), in FP64 for complex128 states and as an unevaluated sum
 * of two floats (about 48 significant bits) for complex64 states.  Synchronous (returns when the results are
 * on the host).  Errors: SOP_EINVAL for bad arguments, SOP_ESTATE without a
 * bound state, SOP_ENOMEM for the scratch (one state copy and
 * 2 (n_steps + 1) doubles on the device). */
#define SOP_SPECTRAL_MAX_EIGEN 16
int sop_spectral(sop_plan plan, int64_t n_steps, double dt, int n_energies, const double *energies,
                 double *chi_out, double *spectrum_out, void *psiE_dev);

/* Message of the last failing call on this thread ("" if none). */
const char *sop_last_error(void);

/* ABI version (incremented on incompatible changes). */
int sop_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SOP_H */
