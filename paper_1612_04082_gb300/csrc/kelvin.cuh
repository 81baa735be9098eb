// kelvin.cuh -- device evaluators of the four Kelvin kernels of arXiv 1612.04082:
//   U (Eq. disp_1), P (Eq. disp_2), D (Eq. stress_2, textbook constant 1/(8 pi)),
//   S (Eq. stress_3, with the factor G).
// d = x_target - y_source.  Densities are passed pre-scaled so that the constant factors
// leave the inner loop:
//   t' = t / (16 pi (1-nu) G)           (single layer, displacement output)
//   u' = u / (8 pi (1-nu))              (double layer, displacement output)
//   nu' = (1-2nu) (n . u')              (per-source constant of the double layer)
// The stress evaluators take unscaled densities and apply their constants at the end.
#pragma once

#include <cuda_runtime.h>

namespace kfmm {

template <typename R> struct KelvinConst {
    R a34;   // 3 - 4 nu
    R b12;   // 1 - 2 nu
    R nu;
    R c_sl;  // 1 / (16 pi (1-nu) G)
    R c_dl;  // 1 / (8 pi (1-nu))
    R c_D;   // 1 / (8 pi (1-nu))          (D)
    R c_S;   // G / (4 pi (1-nu))          (S)
};

template <typename R> __host__ __device__ inline KelvinConst<R> make_kelvin(double G, double nu) {
    const double pi = 3.14159265358979323846;
    KelvinConst<R> k;
    k.a34 = R(3.0 - 4.0 * nu);
    k.b12 = R(1.0 - 2.0 * nu);
    k.nu = R(nu);
    k.c_sl = R(1.0 / (16.0 * pi * (1.0 - nu) * G));
    k.c_dl = R(1.0 / (8.0 * pi * (1.0 - nu)));
    k.c_D = R(1.0 / (8.0 * pi * (1.0 - nu)));
    k.c_S = R(G / (4.0 * pi * (1.0 - nu)));
    return k;
}

__device__ __forceinline__ float kf_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double kf_rsqrt(double x) { return rsqrt(x); }

// 1/r with the coincident-point convention (0 at r = 0).  CHK = false drops the test, for
// source sets known to hold no point coinciding with the target.
template <typename R, bool CHK = true> __device__ __forceinline__ R inv_r(R r2) {
    if (CHK) return r2 > R(0) ? kf_rsqrt(r2) : R(0);
    return kf_rsqrt(r2);
}

// Single layer, displacement: out += (3-4nu) t' / r + d (d . t') / r^3.
template <typename R, bool CHK = true>
__device__ __forceinline__ void acc_sl(R dx, R dy, R dz, R tx, R ty, R tz, R a34, R &ox, R &oy,
                                       R &oz) {
    R r2 = dx * dx + dy * dy + dz * dz;
    R ri = inv_r<R, CHK>(r2);
    R ri3 = ri * ri * ri;
    R dt = (dx * tx + dy * ty + dz * tz) * ri3;
    R a = a34 * ri;
    ox += a * tx + dt * dx;
    oy += a * ty + dt * dy;
    oz += a * tz + dt * dz;
}

// Single + double layer, displacement (pre-scaled t', u', nu' = (1-2nu) n.u'):
//   out += (3-4nu) t'/r + d (d.t')/r^3
//        + [(1-2nu)((d.n) u' + (d.u') n) + d (3 (d.n)(d.u')/r^2 - nu'... )] / r^3
// i.e. P u = 1/r^3 { (d.n)[(1-2nu) u + 3 d (d.u)/r^2] - (1-2nu)[d (n.u) - n (d.u)] }.
template <typename R, bool CHK = true>
__device__ __forceinline__ void acc_sl_dl(R dx, R dy, R dz, R tx, R ty, R tz, R ux, R uy, R uz, R nx,
                                          R ny, R nz, R nup, R a34, R b12, R &ox, R &oy, R &oz) {
    R r2 = dx * dx + dy * dy + dz * dz;
    R ri = inv_r<R, CHK>(r2);
    R ri2 = ri * ri;
    R ri3 = ri2 * ri;
    R dt = dx * tx + dy * ty + dz * tz;
    R dn = dx * nx + dy * ny + dz * nz;
    R du = dx * ux + dy * uy + dz * uz;
    R a = a34 * ri;
    R bd = ri3 * (dt + R(3) * dn * du * ri2 - nup);
    R cu = b12 * dn * ri3;
    R dn_ = b12 * du * ri3;
    ox += a * tx + bd * dx + cu * ux + dn_ * nx;
    oy += a * ty + bd * dy + cu * uy + dn_ * ny;
    oz += a * tz + bd * dz + cu * uz + dn_ * nz;
}

// acc_sl_dl with the double-layer density stored pre-multiplied by (1-2nu): u'' = (1-2nu) u'
// and c3 = 3 / (1-2nu) (nu < 1/2, so 1-2nu > 0).  The same sum with two multiplies fewer per
// pair: (1-2nu) (d.n) u' = (d.n) u'', (1-2nu) (d.u') n = (d.u'') n, 3 (d.u') = c3 (d.u'').
template <typename R, bool CHK = true>
__device__ __forceinline__ void acc_sl_dl_s(R dx, R dy, R dz, R tx, R ty, R tz, R ux, R uy, R uz, R nx,
                                            R ny, R nz, R nup, R a34, R c3, R &ox, R &oy, R &oz) {
    R r2 = dx * dx + dy * dy + dz * dz;
    R ri = inv_r<R, CHK>(r2);
    R ri2 = ri * ri;
    R ri3 = ri2 * ri;
    R dt = dx * tx + dy * ty + dz * tz;
    R dn = dx * nx + dy * ny + dz * nz;
    R du = dx * ux + dy * uy + dz * uz;
    R a = a34 * ri;
    R bd = ri3 * (dt + c3 * dn * du * ri2 - nup);
    R cu = dn * ri3;
    R dn_ = du * ri3;
    ox += a * tx + bd * dx + cu * ux + dn_ * nx;
    oy += a * ty + bd * dy + cu * uy + dn_ * ny;
    oz += a * tz + bd * dz + cu * uz + dn_ * nz;
}

// acc_dl with the pre-multiplied density of acc_sl_dl_s.
template <typename R, bool CHK = true>
__device__ __forceinline__ void acc_dl_s(R dx, R dy, R dz, R ux, R uy, R uz, R nx, R ny, R nz, R nup,
                                         R c3, R &ox, R &oy, R &oz) {
    R r2 = dx * dx + dy * dy + dz * dz;
    R ri = inv_r<R, CHK>(r2);
    R ri2 = ri * ri;
    R ri3 = ri2 * ri;
    R dn = dx * nx + dy * ny + dz * nz;
    R du = dx * ux + dy * uy + dz * uz;
    R bd = ri3 * (c3 * dn * du * ri2 - nup);
    R cu = dn * ri3;
    R dn_ = du * ri3;
    ox += bd * dx + cu * ux + dn_ * nx;
    oy += bd * dy + cu * uy + dn_ * ny;
    oz += bd * dz + cu * uz + dn_ * nz;
}

// Double layer only, displacement.
template <typename R, bool CHK = true>
__device__ __forceinline__ void acc_dl(R dx, R dy, R dz, R ux, R uy, R uz, R nx, R ny, R nz, R nup,
                                       R b12, R &ox, R &oy, R &oz) {
    R r2 = dx * dx + dy * dy + dz * dz;
    R ri = inv_r<R, CHK>(r2);
    R ri2 = ri * ri;
    R ri3 = ri2 * ri;
    R dn = dx * nx + dy * ny + dz * nz;
    R du = dx * ux + dy * uy + dz * uz;
    R bd = ri3 * (R(3) * dn * du * ri2 - nup);
    R cu = b12 * dn * ri3;
    R dn_ = b12 * du * ri3;
    ox += bd * dx + cu * ux + dn_ * nx;
    oy += bd * dy + cu * uy + dn_ * ny;
    oz += bd * dz + cu * uz + dn_ * nz;
}

// Stress of the single layer (Eq. stress_2, textbook constant), unscaled t:
//   sigma_ij += -c_D / r^3 [ (1-2nu)(t_i d_j + t_j d_i - delta_ij (d.t)) + 3 d_i d_j (d.t)/r^2 ]
// Accumulated without c_D (applied by the caller): s[6] in xx, yy, zz, yz, xz, xy.
template <typename R, bool CHK = true>
__device__ __forceinline__ void acc_D(R dx, R dy, R dz, R tx, R ty, R tz, R b12, R *s) {
    R r2 = dx * dx + dy * dy + dz * dz;
    R ri = inv_r<R, CHK>(r2);
    R ri2 = ri * ri;
    R ri3 = ri2 * ri;
    R dt = dx * tx + dy * ty + dz * tz;
    R b = b12 * ri3;       // (1-2nu)/r^3
    R c = R(3) * dt * ri3 * ri2;
    R e = b * dt;
    s[0] -= b * (R(2) * tx * dx) - e + c * dx * dx;
    s[1] -= b * (R(2) * ty * dy) - e + c * dy * dy;
    s[2] -= b * (R(2) * tz * dz) - e + c * dz * dz;
    s[3] -= b * (ty * dz + tz * dy) + c * dy * dz;
    s[4] -= b * (tx * dz + tz * dx) + c * dx * dz;
    s[5] -= b * (tx * dy + ty * dx) + c * dx * dy;
}

// Stress of the double layer (Eq. stress_3 with G), unscaled u, normal n:
//   sigma_ij += c_S / r^3 { 3 (d.n)(d.u)/r^2 (1-2nu) delta_ij + 3 nu (d.n)/r^2 (u_i d_j + u_j d_i)
//               - 15 (d.n)(d.u)/r^4 d_i d_j + 3 nu (d.u)/r^2 (n_i d_j + n_j d_i)
//               + (1-2nu)(3 (n.u)/r^2 d_i d_j + n_j u_i + n_i u_j) - (1-4nu)(n.u) delta_ij }
// Accumulated without c_S.
template <typename R, bool CHK = true>
__device__ __forceinline__ void acc_S(R dx, R dy, R dz, R ux, R uy, R uz, R nx, R ny, R nz, R nu_,
                                      R b12, R *s) {
    R r2 = dx * dx + dy * dy + dz * dz;
    R ri = inv_r<R, CHK>(r2);
    R ri2 = ri * ri;
    R ri3 = ri2 * ri;
    R dn = dx * nx + dy * ny + dz * nz;
    R du = dx * ux + dy * uy + dz * uz;
    R nuu = nx * ux + ny * uy + nz * uz;
    R diag = R(3) * dn * du * ri2 * b12 - (R(1) - R(4) * nu_) * nuu;   // * delta_ij
    R cud = R(3) * nu_ * dn * ri2;                                     // * (u_i d_j + u_j d_i)
    R cnd = R(3) * nu_ * du * ri2;                                     // * (n_i d_j + n_j d_i)
    R cdd = (R(3) * b12 * nuu - R(15) * dn * du * ri2) * ri2;          // * d_i d_j
    // (1-2nu)(n_j u_i + n_i u_j)
    s[0] += ri3 * (diag + R(2) * cud * ux * dx + R(2) * cnd * nx * dx + cdd * dx * dx + R(2) * b12 * nx * ux);
    s[1] += ri3 * (diag + R(2) * cud * uy * dy + R(2) * cnd * ny * dy + cdd * dy * dy + R(2) * b12 * ny * uy);
    s[2] += ri3 * (diag + R(2) * cud * uz * dz + R(2) * cnd * nz * dz + cdd * dz * dz + R(2) * b12 * nz * uz);
    s[3] += ri3 * (cud * (uy * dz + uz * dy) + cnd * (ny * dz + nz * dy) + cdd * dy * dz + b12 * (nz * uy + ny * uz));
    s[4] += ri3 * (cud * (ux * dz + uz * dx) + cnd * (nx * dz + nz * dx) + cdd * dx * dz + b12 * (nz * ux + nx * uz));
    s[5] += ri3 * (cud * (ux * dy + uy * dx) + cnd * (nx * dy + ny * dx) + cdd * dx * dy + b12 * (ny * ux + nx * uy));
}

}  // namespace kfmm
