// sop_dirac3d.cu -- pointwise factors of the three-dimensional four-component
// Dirac step (Sec. 2.3 with d = 3).
//
// In three dimensions alpha_3 couples components (1,3) and (2,4) and
// alpha_1, alpha_2 couple (1,4) and (2,3), so neither factor splits into
// component pairs.  The step runs the three transforms of each component as
// separate pencil passes (components as a batch) and applies the two 4x4
// factors here, one streaming pass over the four components each:
//   real space:      psi <- exp(-i V tau') M psi, M the merged mixing of the
//                    adjacent half steps (Eqs. 21-26), uniform in space or,
//                    for a vector potential that varies along x_1, one
//                    compact matrix per lattice column (k_mix_rows);
//   momentum space:  psi~ <- (1/N) [cos(E tau) - i sin(E tau) H(p)/E] psi~,
//                    H = c alpha.p + m c^2 beta (the closed form of Eq. 33).
#include "sop_dirac4.cuh"
#include "sop_kernels.cuh"
#include "sop_internal.h"

namespace sop {

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 152 * 8;

__device__ __forceinline__ double lat_p(int64_t n, double h, int64_t k, double hbar) {
    const int64_t kap = (2 * k < n) ? k : k - n;
    return hbar * 6.283185307179586476925286766559 * (double)kap / ((double)n * h);
}

// Entry k (x fastest): (cos th, sin th mc^2/E, sin th c p_x/E, sin th c p_y/E,
// sin th c p_z/E, 0, 0, 0) with th = E tau / hbar, formed in FP64 and rounded
// to the plan's precision.
__global__ void k_dirac3_table(void *out, int64_t nx, int64_t ny, int64_t nz, double hx, double hy, double hz,
                               double mass, double c, double hbar, double tau, bool f64) {
    const int64_t total = nx * ny * nz;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t kx = k % nx, r = k / nx, ky = r % ny, kz = r / ny;
        const double px = lat_p(nx, hx, kx, hbar), py = lat_p(ny, hy, ky, hbar), pz = lat_p(nz, hz, kz, hbar);
        const double mc2 = mass * c * c;
        const double E = sqrt(mc2 * mc2 + (px * px + py * py + pz * pz) * c * c);
        double s, co;
        sincos(E * tau / hbar, &s, &co);
        const double q[5] = {co, s * mc2 / E, s * c * px / E, s * c * py / E, s * c * pz / E};
        if (f64) {
            double *o = reinterpret_cast<double *>(out) + 8 * k;
            for (int i = 0; i < 5; ++i) o[i] = q[i];
            o[5] = o[6] = o[7] = 0.0;
        } else {
            float4 *o = reinterpret_cast<float4 *>(out) + 2 * k;
            o[0] = make_float4((float)q[0], (float)q[1], (float)q[2], (float)q[3]);
            o[1] = make_float4((float)q[4], 0.f, 0.f, 0.f);
        }
    }
}

template <typename Real> struct Mix4 {
    cplx_t<Real> m[16];   // row-major 4x4
};

// psi <- exp(-i V tau') M psi on all points; M uniform (by value, a general
// 4x4) or, with rows != null, the merged mixing of the point's column x_1 in
// the compact form M = a + i b.alpha + i d.Sigma (8 reals per column:
// a, b_1..3, d_1..3, 0; Sigma_k = diag(sigma_k, sigma_k)), for a vector
// potential that varies along x_1.
template <typename Real>
__global__ void __launch_bounds__(kThreads) k_dirac3_real(cplx_t<Real> *psi, int64_t npts, const cplx_t<Real> *vtab,
                                                          Mix4<Real> M, const Real *rows, int64_t nx) {
    using C = cplx_t<Real>;
    using Ph = Phase<Real>;
    for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < npts; j += (int64_t)gridDim.x * kThreads) {
        C v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = __ldcg(psi + c * npts + j);
        const C f = vtab ? __ldcg(vtab + j) : Ph::one();
        C w[4];
        if (rows) {
            Real q[8];
            dirac4_load_row(rows + (j % nx) * 8, q);
            dirac4_mix_compact(q, v, w);
        } else {
            dirac4_mix(M.m, v, w);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) __stcg(psi + c * npts + j, vtab ? Ph::apply(w[c], f) : w[c]);
    }
}

// Half-step mixing of Eq. 26 for a vector potential Abar = A tau (ndim
// components), delta = 1/2: R = cos th + i sin th n.alpha with n = Abar/|Abar|
// and th = q c |Abar| / (2 hbar).
__device__ void mixing_params(const double *A, int ndim, double qc2h, double tau, double &c, double &s, double n[3]) {
    double Ab[3] = {0, 0, 0}, mag = 0.0;
    for (int a = 0; a < ndim; ++a) {
        Ab[a] = A ? A[a] * tau : 0.0;
        mag += Ab[a] * Ab[a];
    }
    mag = sqrt(mag);
    sincos(qc2h * mag, &s, &c);
    for (int a = 0; a < 3; ++a) n[a] = mag > 0 ? Ab[a] / mag : 0.0;
}

// Rows P0 .. P0 + n_rows - 1 of the merged mixing per column,
// R(A_P(i)) R(A_{P-1}(i)) = a + i b.alpha + i d.Sigma with
// (alpha_j alpha_k = delta_jk + i eps_jkl Sigma_l)
//   a = c_n c_p - s_n s_p n_n.n_p,  b = c_n s_p n_p + s_n c_p n_n,
//   d = -s_n s_p n_n x n_p,
// stored as 8 reals (a, b, d, 0) per column in the plan's precision; A_s(i) =
// avec[(s nx + i) ndim ...] for 0 <= s < n_steps and 0 (identity) otherwise.
__global__ void k_mix_rows(void *out, const double *avec, int64_t P0, int64_t n_rows, int64_t nx, int ndim,
                           int64_t n_steps, double qc2h, double tau, bool f64) {
    const int64_t total = n_rows * nx;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t P = P0 + e / nx, i = e % nx;
        double cn, sn, nn[3], cp, sp, np[3];
        mixing_params(P < n_steps ? avec + (P * nx + i) * ndim : nullptr, ndim, qc2h, tau, cn, sn, nn);
        mixing_params(P > 0 ? avec + ((P - 1) * nx + i) * ndim : nullptr, ndim, qc2h, tau, cp, sp, np);
        double q[8];
        q[0] = cn * cp - sn * sp * (nn[0] * np[0] + nn[1] * np[1] + nn[2] * np[2]);
        for (int k = 0; k < 3; ++k) q[1 + k] = cn * sp * np[k] + sn * cp * nn[k];
        q[4] = -sn * sp * (nn[1] * np[2] - nn[2] * np[1]);
        q[5] = -sn * sp * (nn[2] * np[0] - nn[0] * np[2]);
        q[6] = -sn * sp * (nn[0] * np[1] - nn[1] * np[0]);
        q[7] = 0.0;
        for (int k = 0; k < 8; ++k) {
            if (f64) reinterpret_cast<double *>(out)[e * 8 + k] = q[k];
            else reinterpret_cast<float *>(out)[e * 8 + k] = (float)q[k];
        }
    }
}

// U = cos - i sin H/E with H/E = [[mu, 0, kz, km], [0, mu, kp, -kz],
// [kz, km, -mu, 0], [kp, -kz, 0, -mu]], kp = c(p_x + i p_y)/E, km = conj(kp),
// kz = c p_z / E, mu = m c^2 / E; then 1/N.
template <typename Real>
__global__ void __launch_bounds__(kThreads) k_dirac3_kinetic(cplx_t<Real> *psi, int64_t npts, const Real *tab,
                                                             Real shi, Real slo) {
    using C = cplx_t<Real>;
    for (int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x; k < npts; k += (int64_t)gridDim.x * kThreads) {
        Real co, sm, sx, sy, sz;
        dirac4_load_kin(tab, k, co, sm, sx, sy, sz);
        C v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = __ldcg(psi + c * npts + k);
        C r[4];
        dirac4_kinetic(co, sm, sx, sy, sz, v, r);
#pragma unroll
        for (int c = 0; c < 4; ++c) __stcg(psi + c * npts + k, scale2(r[c], shi, slo));
    }
}

template <typename Real>
cudaError_t dirac3_real_t(void *psi, int64_t npts, const void *vtab, const double *Md, const void *rows, int64_t nx,
                          cudaStream_t s) {
    Mix4<Real> M{};   // (host code: no device helpers)
    if (Md)
        for (int q = 0; q < 16; ++q) {
            M.m[q].x = (Real)Md[2 * q];
            M.m[q].y = (Real)Md[2 * q + 1];
        }
    k_dirac3_real<Real><<<kBlocks, kThreads, 0, s>>>(static_cast<cplx_t<Real> *>(psi), npts,
                                                      static_cast<const cplx_t<Real> *>(vtab), M,
                                                      static_cast<const Real *>(rows), nx);
    return cudaGetLastError();
}

}  // namespace

cudaError_t build_dirac3_table(void *out, const int64_t *dims, const double *h, double mass, double c, double hbar,
                               double dt, bool f64, cudaStream_t s) {
    k_dirac3_table<<<kBlocks, kThreads, 0, s>>>(out, dims[0], dims[1], dims[2], h[0], h[1], h[2], mass, c, hbar, dt,
                                                f64);
    return cudaGetLastError();
}

cudaError_t launch_dirac3_real(void *psi, int64_t npts, const void *vtab, const double *M, const void *rows,
                               int64_t nx, bool f64, cudaStream_t s) {
    return f64 ? dirac3_real_t<double>(psi, npts, vtab, M, rows, nx, s)
               : dirac3_real_t<float>(psi, npts, vtab, M, rows, nx, s);
}

cudaError_t build_mix_rows(void *out, const double *avec, int64_t P0, int64_t n_rows, int64_t nx, int ndim,
                           int64_t n_steps, double charge, double c, double hbar, double tau, bool f64,
                           cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    k_mix_rows<<<kBlocks, kThreads, 0, s>>>(out, avec, P0, n_rows, nx, ndim, n_steps, 0.5 * charge * c / hbar, tau,
                                            f64);
    return cudaGetLastError();
}

cudaError_t launch_dirac3_kinetic(void *psi, int64_t npts, const void *tab, double shi, double slo, bool f64,
                                  cudaStream_t s) {
    if (f64)
        k_dirac3_kinetic<double><<<kBlocks, kThreads, 0, s>>>(static_cast<double2 *>(psi), npts,
                                                               static_cast<const double *>(tab), shi, slo);
    else
        k_dirac3_kinetic<float><<<kBlocks, kThreads, 0, s>>>(static_cast<float2 *>(psi), npts,
                                                              static_cast<const float *>(tab), (float)shi,
                                                              (float)slo);
    return cudaGetLastError();
}

}  // namespace sop
