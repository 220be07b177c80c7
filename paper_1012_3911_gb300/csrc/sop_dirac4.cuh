// sop_dirac4.cuh -- the pointwise 4x4 factors of the three-dimensional
// four-component Dirac step (Sec. 2.3 with d = 3) on one lattice point, shared
// by the streaming factor kernels (sop_dirac3d.cu) and the fused
// four-component pencil passes (sop_async.cuh, OP_D3V / OP_D3T).
//
//   real space:      psi <- M psi, M the merged mixing of adjacent half steps
//                    (Eqs. 21-26): a general 4x4 (uniform A) or, for A varying
//                    along x_1, the compact per-column form a + i b.alpha + i d.Sigma;
//   momentum space:  psi~ <- [cos(E tau) - i sin(E tau) H(p)/E] psi~ with
//                    H = c alpha.p + m c^2 beta (the closed form of Eq. 33).
#pragma once

#include "sop_fft.cuh"

namespace sop {

// w = M v, M row-major 4x4.
template <typename C> __device__ __forceinline__ void dirac4_mix(const C *M, const C (&v)[4], C (&w)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        C acc = cmul(M[4 * i], v[0]);
#pragma unroll
        for (int k = 1; k < 4; ++k) acc = cadd(acc, cmul(M[4 * i + k], v[k]));
        w[i] = acc;
    }
}

// w = (a + i b.alpha + i d.Sigma) v, q = (a, b_1, b_2, b_3, d_1, d_2, d_3, 0),
// Sigma_k = diag(sigma_k, sigma_k), Dirac representation of alpha.
template <typename C, typename Real>
__device__ __forceinline__ void dirac4_mix_compact(const Real (&q)[8], const C (&v)[4], C (&w)[4]) {
    const Real a = q[0], b1 = q[1], b2 = q[2], b3 = q[3], d1 = q[4], d2 = q[5], d3 = q[6];
    const C bm = mk<C>(b1, -b2), bp = mk<C>(b1, b2), dm = mk<C>(d1, -d2), dp = mk<C>(d1, d2);
    C u[4];
    u[0] = cadd(cadd(cmul(bm, v[3]), cscale(v[2], b3)), cadd(cscale(v[0], d3), cmul(dm, v[1])));
    u[1] = cadd(csub(cmul(bp, v[2]), cscale(v[3], b3)), csub(cmul(dp, v[0]), cscale(v[1], d3)));
    u[2] = cadd(cadd(cmul(bm, v[1]), cscale(v[0], b3)), cadd(cscale(v[2], d3), cmul(dm, v[3])));
    u[3] = cadd(csub(cmul(bp, v[0]), cscale(v[1], b3)), csub(cmul(dp, v[2]), cscale(v[3], d3)));
#pragma unroll
    for (int c = 0; c < 4; ++c) w[c] = cadd(cscale(v[c], a), mul_pi(u[c]));
}

// The 8 reals of a compact mixing row (plan precision) at r.
template <typename Real> __device__ __forceinline__ void dirac4_load_row(const Real *r, Real (&q)[8]) {
    if constexpr (sizeof(Real) == 4) {
        const float4 x0 = __ldg(reinterpret_cast<const float4 *>(r)), x1 = __ldg(reinterpret_cast<const float4 *>(r) + 1);
        q[0] = x0.x; q[1] = x0.y; q[2] = x0.z; q[3] = x0.w; q[4] = x1.x; q[5] = x1.y; q[6] = x1.z; q[7] = x1.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double2 x = __ldg(reinterpret_cast<const double2 *>(r) + k);
            q[2 * k] = x.x;
            q[2 * k + 1] = x.y;
        }
    }
}

// Table entry k of the momentum-space factor: (cos th, sin th mc^2/E,
// sin th c p_x/E, sin th c p_y/E, sin th c p_z/E) of 8 reals per momentum.
template <typename Real>
__device__ __forceinline__ void dirac4_load_kin(const Real *tab, int64_t k, Real &co, Real &sm, Real &sx, Real &sy,
                                                Real &sz) {
    if constexpr (sizeof(Real) == 4) {
        const float4 a = __ldcg(reinterpret_cast<const float4 *>(tab) + 2 * k);
        const float4 b = __ldcg(reinterpret_cast<const float4 *>(tab) + 2 * k + 1);
        co = a.x; sm = a.y; sx = a.z; sy = a.w; sz = b.x;
    } else {
        const double2 a = __ldcg(reinterpret_cast<const double2 *>(tab) + 4 * k);
        const double2 b = __ldcg(reinterpret_cast<const double2 *>(tab) + 4 * k + 1);
        const double2 d = __ldcg(reinterpret_cast<const double2 *>(tab) + 4 * k + 2);
        co = a.x; sm = a.y; sx = b.x; sy = b.y; sz = d.x;
    }
}

// r = [cos - i sin H/E] v with H/E = [[mu, 0, kz, km], [0, mu, kp, -kz],
// [kz, km, -mu, 0], [kp, -kz, 0, -mu]], kp = c(p_x + i p_y)/E, km = conj(kp),
// kz = c p_z / E, mu = m c^2 / E.
template <typename C, typename Real>
__device__ __forceinline__ void dirac4_kinetic(Real co, Real sm, Real sx, Real sy, Real sz, const C (&v)[4],
                                               C (&r)[4]) {
    const C dm = mk<C>(co, -sm), dp = mk<C>(co, sm);            // cos -+ i sin mu
    const C uz = mk<C>(Real(0), -sz), vz = mk<C>(Real(0), sz);   // -i sin kz, +i sin kz
    const C um = mk<C>(-sy, -sx);                                // -i sin km
    const C up = mk<C>(sy, -sx);                                 // -i sin kp
    r[0] = cadd(cmul(dm, v[0]), cadd(cmul(uz, v[2]), cmul(um, v[3])));
    r[1] = cadd(cmul(dm, v[1]), cadd(cmul(up, v[2]), cmul(vz, v[3])));
    r[2] = cadd(cmul(uz, v[0]), cadd(cmul(um, v[1]), cmul(dp, v[2])));
    r[3] = cadd(cmul(up, v[0]), cadd(cmul(vz, v[1]), cmul(dp, v[3])));
}

}  // namespace sop
