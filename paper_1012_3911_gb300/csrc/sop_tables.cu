// sop_tables.cu -- set-up kernels that form every phase table in FP64 and
// round it once to the plan's precision.  They run when a plan is created,
// when the time step or potential changes, and once per chunk of steps for
// the laser-field tables; none of them is on the per-step path.
//
// FP32 tables hold z = exp(-i theta) - 1 with the real part computed as
// -2 sin^2(theta/2) (no cancellation near theta = 0); FP64 tables hold
// exp(-i theta) itself (the representation the pass kernels expect).
#include <math.h>

#include "sop_internal.h"

namespace sop {

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

__device__ __forceinline__ void store_phase(void *out, int64_t idx, double theta, bool f64) {
    // exp(-i theta)
    double s, c;
    sincos(theta, &s, &c);
    if (f64) {
        reinterpret_cast<double2 *>(out)[idx] = make_double2(c, -s);
    } else {
        const double sh = sin(0.5 * theta);
        reinterpret_cast<float2 *>(out)[idx] = make_float2((float)(-2.0 * sh * sh), (float)(-s));
    }
}

__device__ __forceinline__ double lattice_x(int64_t n, double h, int64_t j) {
    return -0.5 * (double)n * h + (double)j * h;
}

__device__ __forceinline__ double lattice_p(int64_t n, double h, int64_t k, double hbar) {
    const int64_t kap = (2 * k < n) ? k : k - n;
    return hbar * kTwoPi * (double)kap / ((double)n * h);
}

__global__ void k_twiddles(void *out, int n, bool f64) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    // exp(-2 pi i e/n) = cospi(2e/n) - i sinpi(2e/n); reduce 2e/n to (-1, 1]
    double x = 2.0 * (double)e / (double)n;
    if (x > 1.0) x -= 2.0;
    double s, c;
    sincospi(x, &s, &c);
    if (f64) {
        reinterpret_cast<double2 *>(out)[e] = make_double2(c, -s);
    } else {
        // z = w - 1 with Re z = cos - 1 = -2 sin^2(pi x / 2) (no cancellation)
        double sh, chh;
        sincospi(0.5 * x, &sh, &chh);
        reinterpret_cast<float2 *>(out)[e] = make_float2((float)(-2.0 * sh * sh), (float)(-s));
    }
}

// exp(-i factor V_j), the merged or half real-space factor of Eq. 11 / 22
// without the laser term.  The FP64 sincos reduces its argument exactly, so
// the angle is passed unreduced.
__global__ void k_vphase(void *out, const double *V, int64_t npts, double factor, bool f64) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < npts;
         j += (int64_t)gridDim.x * blockDim.x) {
        store_phase(out, j, factor * V[j], f64);
    }
}

__global__ void k_axis_phase(void *out, const double *theta, int n, bool f64) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) store_phase(out, i, theta[i], f64);
}

struct FieldGeom {
    int ndim;
    int64_t dims[3];
    double spacing[3];
    int active[3];
    int64_t offsets[3];
};

// Row P, axis a, index i: exp(-i f_{P,a} x_{a,i}) (length-gauge laser term).
__global__ void k_field(void *out, const double *fvec, int64_t n_rows, int64_t row_len, FieldGeom g,
                        bool f64) {
    const int64_t total = n_rows * row_len;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t P = idx / row_len;
        const int64_t r = idx - P * row_len;
        int a = 0;
        while (a + 1 < g.ndim && (!g.active[a] || r >= g.offsets[a] + g.dims[a])) ++a;
        const int64_t i = r - g.offsets[a];
        const double theta = fvec[P * g.ndim + a] * lattice_x(g.dims[a], g.spacing[a], i);
        store_phase(out, idx, theta, f64);
    }
}

// Velocity gauge (Eq. 13 with the vector potential): row P, axis a, index k:
// exp(-i c (p_{a,k} - s_{P,a})^2) with s_P = q A_P and c = tau / (2 m hbar).
__global__ void k_kin_field(void *out, const double *svec, int64_t n_rows, int64_t row_len, FieldGeom g, double c,
                            double hbar, bool f64) {
    const int64_t total = n_rows * row_len;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t P = idx / row_len;
        const int64_t r = idx - P * row_len;
        int a = 0;
        while (a + 1 < g.ndim && (!g.active[a] || r >= g.offsets[a] + g.dims[a])) ++a;
        const int64_t k = r - g.offsets[a];
        const double d = lattice_p(g.dims[a], g.spacing[a], k, hbar) - svec[P * g.ndim + a];
        store_phase(out, idx, c * d * d, f64);
    }
}

// Dirac momentum-space factor (Eq. 33) in closed form per momentum:
//   U = cos(E tau/hbar) - i sin(E tau/hbar) H(p)/E,  H = c alpha.p + m c^2 beta,
// stored as (cos, sin*mc^2/E, sin*c p_x/E, sin*c p_y/E).
__global__ void k_dirac(void *out, int64_t nx, int64_t ny, double hx, double hy, double mass,
                        double c, double hbar, double tau, bool f64) {
    const int64_t total = nx * ny;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t kx = k % nx, ky = k / nx;
        const double px = lattice_p(nx, hx, kx, hbar), py = lattice_p(ny, hy, ky, hbar);
        const double mc2 = mass * c * c;
        const double E = sqrt(mc2 * mc2 + (px * px + py * py) * c * c);
        const double th = E * tau / hbar;
        double s, co;
        sincos(th, &s, &co);
        const double a = co, b = s * mc2 / E, cx = s * c * px / E, cy = s * c * py / E;
        if (f64) {
            double2 *o = reinterpret_cast<double2 *>(out);
            o[2 * k] = make_double2(a, b);
            o[2 * k + 1] = make_double2(cx, cy);
        } else {
            reinterpret_cast<float4 *>(out)[k] = make_float4((float)a, (float)b, (float)cx, (float)cy);
        }
    }
}

// out = in in FP64; *bad becomes nonzero if any value is not finite.
__global__ void k_convert(double *out, const void *in, int64_t n, bool in_f64, int *bad) {
    bool ok = true;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double v = in_f64 ? reinterpret_cast<const double *>(in)[j] : (double)reinterpret_cast<const float *>(in)[j];
        out[j] = v;
        ok = ok && isfinite(v);
    }
    if (!__all_sync(0xffffffffu, ok) && (threadIdx.x & 31) == 0 && bad) atomicOr(bad, 1);
}

unsigned grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

cudaError_t build_twiddles(void *out, int n, bool f64, cudaStream_t s) {
    k_twiddles<<<(n + 255) / 256, 256, 0, s>>>(out, n, f64);
    return cudaGetLastError();
}

cudaError_t build_vphase(void *out, const double *V, int64_t npts, double factor, bool f64, cudaStream_t s) {
    k_vphase<<<grid_for(npts, 256), 256, 0, s>>>(out, V, npts, factor, f64);
    return cudaGetLastError();
}

cudaError_t build_axis_phase(void *out, const double *theta, int n, bool f64, cudaStream_t s) {
    k_axis_phase<<<(n + 255) / 256, 256, 0, s>>>(out, theta, n, f64);
    return cudaGetLastError();
}

cudaError_t build_field_tables(void *out, const double *fvec, int64_t n_rows, int ndim, const int64_t *dims,
                               const double *spacing, const int *active, const int64_t *offsets,
                               int64_t row_len, bool f64, cudaStream_t s) {
    FieldGeom g{};
    g.ndim = ndim;
    for (int a = 0; a < 3; ++a) {
        g.dims[a] = a < ndim ? dims[a] : 1;
        g.spacing[a] = a < ndim ? spacing[a] : 1.0;
        g.active[a] = a < ndim ? active[a] : 0;
        g.offsets[a] = a < ndim ? offsets[a] : 0;
    }
    k_field<<<grid_for(n_rows * row_len, 256), 256, 0, s>>>(out, fvec, n_rows, row_len, g, f64);
    return cudaGetLastError();
}

cudaError_t build_kin_field_tables(void *out, const double *svec, int64_t n_rows, int ndim, const int64_t *dims,
                                   const double *spacing, const int *active, const int64_t *offsets, int64_t row_len,
                                   double c, double hbar, bool f64, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    FieldGeom g{};
    g.ndim = ndim;
    for (int a = 0; a < 3; ++a) {
        g.dims[a] = a < ndim ? dims[a] : 1;
        g.spacing[a] = a < ndim ? spacing[a] : 1.0;
        g.active[a] = a < ndim ? active[a] : 0;
        g.offsets[a] = a < ndim ? offsets[a] : 0;
    }
    k_kin_field<<<grid_for(n_rows * row_len, 256), 256, 0, s>>>(out, svec, n_rows, row_len, g, c, hbar, f64);
    return cudaGetLastError();
}

cudaError_t build_dirac_table(void *out, const int64_t *dims, const double *spacing, double mass, double c,
                              double hbar, double dt, bool f64, cudaStream_t s) {
    k_dirac<<<grid_for(dims[0] * dims[1], 256), 256, 0, s>>>(out, dims[0], dims[1], spacing[0], spacing[1],
                                                             mass, c, hbar, dt, f64);
    return cudaGetLastError();
}

cudaError_t convert_potential(double *out, const void *in, int64_t n, bool in_f64, int *bad, cudaStream_t s) {
    k_convert<<<grid_for(n, 256), 256, 0, s>>>(out, in, n, in_f64, bad);
    return cudaGetLastError();
}

namespace {
__global__ void k_set_counter(int64_t *p, int64_t v) { *p = v; }
__global__ void k_advance_counter(int64_t *p) { *p += 1; }
}  // namespace

cudaError_t set_counter(int64_t *p, int64_t v, cudaStream_t s) {
    k_set_counter<<<1, 1, 0, s>>>(p, v);
    return cudaGetLastError();
}

cudaError_t advance_counter(int64_t *p, cudaStream_t s) {
    k_advance_counter<<<1, 1, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace sop
