// bem.cu -- piecewise-constant collocation BEM on the GPU (Eq. BIE, num, coef, num2), the
// two-pass matvec of Sec. "Matrix-vector products", restarted GMRES with FP64 vectors on
// the device, and the interior fields of Sec. "Computing topological derivatives"
// (Eq. stress_1, Eq. deriv, integrand of Eq. functional).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <memory>
#include <new>
#include <vector>

#include "common.cuh"
#include "kelvin.cuh"
#include "util.cuh"

using namespace kfmm;

// leaf cap of the interior (stress / topological derivative) context when the BEM picks its
// caps (the value timed fastest on a 400k-triangle cantilever with a 4.2M-point grid)
constexpr int BEM_INTERIOR_LEAF_CAP = 1024;

struct bem_ctx {
    kfmm_options opt;
    bool auto_cap = false;  // leaf caps chosen by the BEM (options absent or leaf_cap 0)
    int op = BEM_FMM;
    cudaStream_t stream = nullptr;
    double G = 1.0, nu = 0.3, K = 13.0 / 6.0;
    std::string err;
    int64_t n_launch = 0;
    int64_t nt = 0, nv = 0;
    kfmm_ctx *surf = nullptr;  // FMM over quadrature sources -> centroids
    kfmm_ctx *vol = nullptr;   // FMM over quadrature sources -> interior points
    bool surf_built = false, have_bc = false, have_sol = false;
    bool periodic = false;    // sums over the lattice of a cubic cell (bem_set_periodic)
    double cell_lo[3] = {0, 0, 0}, cell_side = 1.0;
    int macro_ncol = 0;       // uniform stress added before the TD (bem_set_macro_stress)
    DevBuf macro;             // double [macro_ncol][6]
    double setup_G = -1, setup_nu = -1;
    int matvecs = 0, matvecs_hi = 0;  // FMM and FP64-grade (direct) operator applications
    double near_radius = 0;           // FP64 pairs of the compensated direct sum: 4 x longest edge
    DevBuf d, rhs_hi;                 // GMRES-IR: correction, outer residual
    DevBuf verts, tris;
    DevBuf q32, qn32;        // float [16 nt][3]: quadrature points, element normals
    DevBuf q64, qn64;        // double [16 nt][3]
    DevBuf qw;               // double [16 nt]: weights (sum to the element area)
    DevBuf cen32, cen64;     // centroids float / double [nt][3]
    DevBuf corrU, corrT;     // double [nt][9]: analytic self block minus own quadrature terms
    int near_levels = 1;     // quadrature of the triangles sharing a vertex with the collocation
                             // triangle: the 4-node rule on 4^near_levels sub-triangles
    int near_ready = 0;      // near_levels the blocks below were made for (0 = none)
    int64_t n_near = 0;      // (collocation triangle, neighbour) pairs
    DevBuf nbr_off, nbr_idx; // int CSR: triangles sharing a vertex with each triangle
    DevBuf corrN;            // double [n_near][18]: upsampled minus 16-point blocks, U then P
    int ncol = 1;            // density columns of the boundary conditions (load cases)
    int sol_ncol = 1;        // columns of the stored boundary solution
    DevBuf mask, val;        // uint8 [3 nt] (shared by the columns), double [ncol][3 nt]
    DevBuf usol, tsol;       // double [sol_ncol][3 nt]
    DevBuf slq, dlq, fout;   // densities at quadrature points and summed field (FP32 or FP64)
    DevBuf basis;            // GMRES: (restart + 1) x n
    DevBuf w, r, x, b, part, hdev, av;  // [ncol][3 nt] vectors; reduction and coefficient scratch
    DevBuf stage[4], pts64, out64;
    kfmm_status fail(kfmm_status c, const std::string &m) {
        err = m;
        return c;
    }
};

namespace {

// ------------------------------------------------------------------------------------
// double3 helpers
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double3 ld3(const double *p) { return make_double3(p[0], p[1], p[2]); }
__device__ __forceinline__ double3 vsub(double3 a, double3 b) { return make_double3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ double3 vadd(double3 a, double3 b) { return make_double3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ double3 vmul(double s, double3 a) { return make_double3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double vdot(double3 a, double3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ double3 vcross(double3 a, double3 b)
{
    return make_double3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double vc(double3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

// Singular blocks at the centroid xi of a flat triangle with unit normal n.  Per edge, in
// polar coordinates about xi: u = unit direction to the foot of the perpendicular on the
// edge line (distance h), w = unit edge direction, e(phi) = cos(phi) u + sin(phi) w, the
// edge at R = h / cos(phi), phi in [pa, pb].  With F = asinh(tan phi):
//   int R = h F;  int cos^2 R = h sin;  int sin cos R = -h cos;  int sin^2 R = h (F - sin)
//   int cos ln R = ln h sin - (sin ln cos + F - sin);  int sin ln R = -ln h cos - (cos - cos ln cos)
// int_tri U dA = [(3-4nu) (int R) I + int e e^T R] / (16 pi (1-nu) G)   (radial part exact)
// PV int_tri P dA = (1-2nu)/(8 pi (1-nu)) (E n^T - n E^T), E = int e ln R  (in the element
// plane dr/dn = 0 and only the antisymmetric term of Eq. disp_2 remains).
__device__ void self_blocks(double3 A, double3 B, double3 C, double3 n, double G, double nu, double *Us, double *Ts)
{
    const double3 xi = vmul(1.0 / 3.0, vadd(vadd(A, B), C));
    const double3 V[3] = {A, B, C};
    double I0 = 0.0, Iee[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, E[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
        const double3 a = vsub(V[k], xi), bb = vsub(V[(k + 1) % 3], xi);
        const double3 edge = vsub(bb, a);
        const double L = sqrt(vdot(edge, edge));
        const double3 w = vmul(1.0 / L, edge);
        const double s_a = vdot(a, w);
        const double3 foot = vsub(a, vmul(s_a, w));
        const double h = sqrt(vdot(foot, foot));
        const double3 u = vmul(1.0 / h, foot);
        const double pa = atan2(s_a, h), pb = atan2(s_a + L, h);
        const double sa = sin(pa), sb = sin(pb), ca = cos(pa), cb = cos(pb);
        const double Fa = asinh(tan(pa)), Fb = asinh(tan(pb));
        const double lh = log(h), lca = log(ca), lcb = log(cb);
        I0 += h * (Fb - Fa);
        const double icc = h * (sb - sa);
        const double ics = -h * (cb - ca);
        const double iss = h * ((Fb - Fa) - (sb - sa));
        const double icl = lh * (sb - sa) - ((sb * lcb + Fb - sb) - (sa * lca + Fa - sa));
        const double isl = -lh * (cb - ca) - ((cb - cb * lcb) - (ca - ca * lca));
        for (int i = 0; i < 3; ++i) {
            const double ui = vc(u, i), wi = vc(w, i);
            for (int j = 0; j < 3; ++j) {
                const double uj = vc(u, j), wj = vc(w, j);
                Iee[3 * i + j] += icc * ui * uj + ics * (ui * wj + wi * uj) + iss * wi * wj;
            }
            E[i] += icl * ui + isl * wi;
        }
    }
    const double pi = 3.14159265358979323846;
    const double cu = 1.0 / (16.0 * pi * (1.0 - nu) * G);
    const double ct = (1.0 - 2.0 * nu) / (8.0 * pi * (1.0 - nu));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Us[3 * i + j] = cu * ((i == j ? (3.0 - 4.0 * nu) * I0 : 0.0) + Iee[3 * i + j]);
            Ts[3 * i + j] = ct * (E[i] * vc(n, j) - E[j] * vc(n, i));
        }
}

// One thread per triangle: geometry, the 16-point rule (4 midpoint sub-triangles, each
// with the degree-3 rule: centroid -27/48, points (3/5,1/5,1/5) 25/48), and the local-pass
// blocks corr = (analytic singular block) - (the element's own quadrature terms), FP64.
__global__ void bem_setup_kernel(int64_t nt, const double *__restrict__ verts, const int *__restrict__ tris,
                                 double G, double nu, float *__restrict__ q32, float *__restrict__ qn32,
                                 double *__restrict__ q64, double *__restrict__ qn64, double *__restrict__ qw,
                                 float *__restrict__ cen32, double *__restrict__ cen64, double *__restrict__ corrU,
                                 double *__restrict__ corrT, int *__restrict__ bad)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const double3 A = ld3(verts + 3 * tris[3 * k]), B = ld3(verts + 3 * tris[3 * k + 1]),
                  C = ld3(verts + 3 * tris[3 * k + 2]);
    const double3 cr = vcross(vsub(B, A), vsub(C, A));
    const double len = sqrt(vdot(cr, cr));
    const double3 xi = vmul(1.0 / 3.0, vadd(vadd(A, B), C));
    const double3 eab = vsub(B, A), ebc = vsub(C, B), eca = vsub(A, C);
    const double e2 = fmax(vdot(eab, eab), fmax(vdot(ebc, ebc), vdot(eca, eca)));
    if (!(len > 1e-12 * e2) || !isfinite(len)) {
        atomicExch(bad, 1);
        return;
    }
    const double3 n = vmul(1.0 / len, cr);
    const double area = 0.5 * len;
    for (int c = 0; c < 3; ++c) {
        cen64[3 * k + c] = vc(xi, c);
        cen32[3 * k + c] = (float)vc(xi, c);
    }
    const double3 mAB = vmul(0.5, vadd(A, B)), mBC = vmul(0.5, vadd(B, C)), mCA = vmul(0.5, vadd(C, A));
    const double3 sub[4][3] = {{A, mAB, mCA}, {mAB, B, mBC}, {mCA, mBC, C}, {mBC, mCA, mAB}};
    const double wt[4] = {-27.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0};
    const double lam[4][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {0.6, 0.2, 0.2}, {0.2, 0.6, 0.2}, {0.2, 0.2, 0.6}};
    // own quadrature terms of U and P at the centroid (kernel 0 at the coincident point)
    const auto kc = make_kelvin<double>(G, nu);
    double qU[9] = {0}, qT[9] = {0};
    int m = 0;
    for (int s = 0; s < 4; ++s)
        for (int g = 0; g < 4; ++g, ++m) {
            // the centre sub-triangle's centroid is the collocation point itself: use the same
            // bits, so every summation (FP32 FMM, FP64 direct, this local pass) sees r = 0
            // there and skips it; a barycentric recomputation lands ~1e-17 away instead
            const double3 y = (s == 3 && g == 0)
                                  ? xi
                                  : vadd(vadd(vmul(lam[g][0], sub[s][0]), vmul(lam[g][1], sub[s][1])),
                                         vmul(lam[g][2], sub[s][2]));
            const double wq = wt[g] * 0.25 * area;
            const int64_t j = 16 * k + m;
            for (int c = 0; c < 3; ++c) {
                q64[3 * j + c] = vc(y, c);
                q32[3 * j + c] = (float)vc(y, c);
                qn64[3 * j + c] = vc(n, c);
                qn32[3 * j + c] = (float)vc(n, c);
            }
            qw[j] = wq;
            const double3 d = vsub(xi, y);
            for (int col = 0; col < 3; ++col) {
                // column `col` of U and P: apply each kernel to the unit vector e_col
                double e[3] = {0, 0, 0};
                e[col] = 1.0;
                double ox = 0, oy = 0, oz = 0;
                acc_sl<double>(d.x, d.y, d.z, kc.c_sl * e[0], kc.c_sl * e[1], kc.c_sl * e[2], kc.a34, ox, oy, oz);
                qU[0 + col] += wq * ox;
                qU[3 + col] += wq * oy;
                qU[6 + col] += wq * oz;
                ox = oy = oz = 0;
                const double ue[3] = {kc.c_dl * e[0], kc.c_dl * e[1], kc.c_dl * e[2]};
                const double nup = kc.b12 * (n.x * ue[0] + n.y * ue[1] + n.z * ue[2]);
                acc_dl<double>(d.x, d.y, d.z, ue[0], ue[1], ue[2], n.x, n.y, n.z, nup, kc.b12, ox, oy, oz);
                qT[0 + col] += wq * ox;
                qT[3 + col] += wq * oy;
                qT[6 + col] += wq * oz;
            }
        }
    double Us[9], Ts[9];
    self_blocks(A, B, C, n, G, nu, Us, Ts);
    for (int a = 0; a < 9; ++a) {
        corrU[9 * k + a] = Us[a] - qU[a];
        corrT[9 * k + a] = Ts[a] - qT[a];
    }
}

// 3x3 blocks of U (Eq. disp_1) and P (Eq. disp_2, normal n) at offset d, times wq, added into
// U9, T9 (FP64, column `col` of each block is the kernel applied to e_col).
__device__ void add_kelvin_blocks(const double3 d, const double3 n, const KelvinConst<double> &kc, double wq,
                                  double *U9, double *T9)
{
    for (int col = 0; col < 3; ++col) {
        double e[3] = {0, 0, 0};
        e[col] = 1.0;
        double ox = 0, oy = 0, oz = 0;
        acc_sl<double>(d.x, d.y, d.z, kc.c_sl * e[0], kc.c_sl * e[1], kc.c_sl * e[2], kc.a34, ox, oy, oz);
        U9[0 + col] += wq * ox;
        U9[3 + col] += wq * oy;
        U9[6 + col] += wq * oz;
        ox = oy = oz = 0;
        const double ue[3] = {kc.c_dl * e[0], kc.c_dl * e[1], kc.c_dl * e[2]};
        const double nup = kc.b12 * (n.x * ue[0] + n.y * ue[1] + n.z * ue[2]);
        acc_dl<double>(d.x, d.y, d.z, ue[0], ue[1], ue[2], n.x, n.y, n.z, nup, kc.b12, ox, oy, oz);
        T9[0 + col] += wq * ox;
        T9[3 + col] += wq * oy;
        T9[6 + col] += wq * oz;
    }
}

// Upsampled quadrature of the near triangles (Sec. "Matrix-vector products": the sums over
// triangles next to the collocation point are the inaccurate ones): for each pair (l, k) of a
// collocation triangle l and a triangle k sharing a vertex with it, the blocks of U and P over
// k at xi_l by the 4-node rule on 4^levels sub-triangles (midpoint subdivision), minus the
// 16-point rule's blocks that the summation already holds.  One thread per pair, FP64.
__global__ void bem_near_kernel(int64_t n_pairs, const int *__restrict__ pair_l, const int *__restrict__ nbr_idx,
                                int levels, const double *__restrict__ verts, const int *__restrict__ tris,
                                const double *__restrict__ cen64, const double *__restrict__ q64,
                                const double *__restrict__ qn64, const double *__restrict__ qw, double G, double nu,
                                double *__restrict__ corrN)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_pairs) return;
    const int l = pair_l[e], k = nbr_idx[e];
    const auto kc = make_kelvin<double>(G, nu);
    const double3 xi = ld3(cen64 + 3 * (int64_t)l);
    const double3 n = ld3(qn64 + 3 * (16 * (int64_t)k));
    double U9[9] = {0}, T9[9] = {0}, U16[9] = {0}, T16[9] = {0};
    // the 16-point terms the summation holds for this pair
    for (int m = 0; m < 16; ++m) {
        const int64_t j = 16 * (int64_t)k + m;
        add_kelvin_blocks(vsub(xi, ld3(q64 + 3 * j)), n, kc, qw[j], U16, T16);
    }
    const double3 A = ld3(verts + 3 * tris[3 * k]), B = ld3(verts + 3 * tris[3 * k + 1]),
                  C = ld3(verts + 3 * tris[3 * k + 2]);
    const double3 cr = vcross(vsub(B, A), vsub(C, A));
    const double area = 0.5 * sqrt(vdot(cr, cr));
    const int nsub = 1 << (2 * levels);
    const double sub_area = area / nsub;
    const double wt[4] = {-27.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0};
    const double lam[4][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {0.6, 0.2, 0.2}, {0.2, 0.6, 0.2}, {0.2, 0.2, 0.6}};
    for (int s = 0; s < nsub; ++s) {
        // sub-triangle s: base-4 digits, most significant first, pick the midpoint children
        double3 a = A, bb = B, c = C;
        for (int lev = levels - 1; lev >= 0; --lev) {
            const int dgt = (s >> (2 * lev)) & 3;
            const double3 mab = vmul(0.5, vadd(a, bb)), mbc = vmul(0.5, vadd(bb, c)), mca = vmul(0.5, vadd(c, a));
            if (dgt == 0) { bb = mab; c = mca; }
            else if (dgt == 1) { a = mab; c = mbc; }
            else if (dgt == 2) { a = mca; bb = mbc; }
            else { a = mbc; bb = mca; c = mab; }
        }
        for (int g = 0; g < 4; ++g) {
            const double3 y = vadd(vadd(vmul(lam[g][0], a), vmul(lam[g][1], bb)), vmul(lam[g][2], c));
            add_kelvin_blocks(vsub(xi, y), n, kc, wt[g] * sub_area, U9, T9);
        }
    }
    for (int a = 0; a < 9; ++a) {
        corrN[18 * e + a] = U9[a] - U16[a];
        corrN[18 * e + 9 + a] = T9[a] - T16[a];
    }
}

// Densities at the quadrature points for columns c0 .. c0 + cn - 1 of M(u, t): sl = -t_k w,
// dl = u_k w, written [16 nt][3 cn].  mode 0: u, t given ([nt][3], one column; either may be
// NULL); mode 1: from the unknowns x [ncol][3 nt] and the mask (Eq. num2); mode 2: from the
// prescribed values [ncol][3 nt] and the mask (right-hand side, sign applied later).
template <typename R>
__global__ void bem_density_kernel(int64_t nt, int mode, int c0, int cn, const double *__restrict__ u,
                                   const double *__restrict__ t, const double *__restrict__ x,
                                   const uint8_t *__restrict__ mask, const double *__restrict__ qw,
                                   R *__restrict__ sl, R *__restrict__ dl)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 16 * nt * cn) return;
    const int64_t j = e / cn;
    const int cc = (int)(e % cn);
    const int64_t k = j / 16;
    const double w = qw[j];
    const double *xc = x ? x + (int64_t)(c0 + cc) * 3 * nt : nullptr;
    for (int c = 0; c < 3; ++c) {
        double uu = 0.0, tt = 0.0;
        const int64_t i = 3 * k + c;
        if (mode == 0) {
            uu = u ? u[i] : 0.0;
            tt = t ? t[i] : 0.0;
        } else if (mode == 1) {
            if (mask[i]) tt = xc[i];
            else uu = xc[i];
        } else {
            if (mask[i]) uu = xc[i];
            else tt = xc[i];
        }
        sl[j * 3 * cn + 3 * cc + c] = (R)(-tt * w);
        dl[j * 3 * cn + 3 * cc + c] = (R)(uu * w);
    }
}

// Local pass for columns c0 .. c0 + cn - 1: out_l = sign * (f_l + 1/2 u_l + corrT_l u_l -
// corrU_l t_l), with f [nt][3 cn] the summed field, FP64 output [ncol][3 nt] (mode 0: [nt][3]).
// Pair (k, comp) values of u and t of one column for the local pass.
__device__ __forceinline__ void local_ut(int mode, int64_t k, const double *u, const double *t, const double *xc,
                                         const uint8_t *mask, double *uu, double *tt)
{
    for (int c = 0; c < 3; ++c) {
        const int64_t i = 3 * k + c;
        uu[c] = tt[c] = 0.0;
        if (mode == 0) {
            uu[c] = u ? u[i] : 0.0;
            tt[c] = t ? t[i] : 0.0;
        } else if (mode == 1) {
            if (mask[i]) tt[c] = xc[i];
            else uu[c] = xc[i];
        } else {
            if (mask[i]) uu[c] = xc[i];
            else tt[c] = xc[i];
        }
    }
}

template <typename R>
__global__ void bem_post_kernel(int64_t nt, int mode, int c0, int cn, double sign, const R *__restrict__ f,
                                const double *__restrict__ u, const double *__restrict__ t,
                                const double *__restrict__ x, const uint8_t *__restrict__ mask,
                                const double *__restrict__ cU, const double *__restrict__ cT,
                                const int *__restrict__ nbr_off, const int *__restrict__ nbr_idx,
                                const double *__restrict__ corrN, double *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nt * cn) return;
    const int64_t k = e / cn;
    const int cc = (int)(e % cn);
    const int64_t col = (int64_t)(c0 + cc) * 3 * nt;
    const double *xc = x ? x + col : nullptr;
    double uu[3], tt[3];
    for (int c = 0; c < 3; ++c) {
        const int64_t i = 3 * k + c;
        uu[c] = tt[c] = 0.0;
        if (mode == 0) {
            uu[c] = u ? u[i] : 0.0;
            tt[c] = t ? t[i] : 0.0;
        } else if (mode == 1) {
            if (mask[i]) tt[c] = xc[i];
            else uu[c] = xc[i];
        } else {
            if (mask[i]) uu[c] = xc[i];
            else tt[c] = xc[i];
        }
    }
    double *o = out + (mode == 0 ? 0 : col);
    double v[3];
    for (int a = 0; a < 3; ++a) {
        v[a] = (double)f[k * 3 * cn + 3 * cc + a] + 0.5 * uu[a];
        for (int c = 0; c < 3; ++c) v[a] += cT[9 * k + 3 * a + c] * uu[c] - cU[9 * k + 3 * a + c] * tt[c];
    }
    if (corrN)  // upsampled quadrature of the neighbouring triangles
        for (int e = nbr_off[k]; e < nbr_off[k + 1]; ++e) {
            double un[3], tn[3];
            local_ut(mode, nbr_idx[e], u, t, xc, mask, un, tn);
            const double *dU = corrN + 18 * (int64_t)e, *dT = dU + 9;
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) v[a] += dT[3 * a + c] * un[c] - dU[3 * a + c] * tn[c];
        }
    for (int a = 0; a < 3; ++a) o[3 * k + a] = sign * v[a];
}

// ------------------------------------------------------------------------------------
// GMRES vector kernels (FP64).  Vectors of all density columns are stored one after the
// other ([ncol][n]); blockIdx.y is the column.
// ------------------------------------------------------------------------------------
constexpr int kVecBlocks = 2 * kNumSMs;
constexpr int kVecThreads = 256;

// part[(col * k + i) * gridDim.x + block] = partial sum of V_i[col] . w[col]; basis vector i
// starts at V + i * ldv, column col at + col * n
__global__ void mdot_kernel(const double *__restrict__ V, int64_t ldv, int k, const double *__restrict__ w, int64_t n,
                            double *__restrict__ part)
{
    __shared__ double red[kVecThreads / 32];
    const int col = blockIdx.y;
    const double *wc = w + (int64_t)col * n;
    for (int i = 0; i < k; ++i) {
        const double *v = V + (int64_t)i * ldv + (int64_t)col * n;
        double s = 0.0;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
            s += v[e] * wc[e];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < kVecThreads / 32; ++q) t += red[q];
            part[((int64_t)col * k + i) * gridDim.x + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

// out[e] = sum of part[e * nb .. e * nb + nb - 1], one warp per entry, FP64, in a fixed order
__global__ void reduce_parts_kernel(const double *__restrict__ part, int nb, int total, double *__restrict__ out)
{
    const int e = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (e >= total) return;
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int q = lane; q < nb; q += 32) s += part[(int64_t)e * nb + q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[e] = s;
}

// w[col] += sign * sum_i h[col * hld + i] V_i[col]
__global__ void maxpy_kernel(double *__restrict__ w, const double *__restrict__ V, int64_t ldv, int k,
                             const double *__restrict__ h, int hld, double sign, int64_t n)
{
    const int col = blockIdx.y;
    const double *hc = h + (int64_t)col * hld;
    double *wc = w + (int64_t)col * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += hc[i] * V[(int64_t)i * ldv + (int64_t)col * n + e];
        wc[e] += sign * s;
    }
}

// dst[col] = a[col] * src[col]
__global__ void scale_copy_kernel(double *__restrict__ dst, const double *__restrict__ src, const double *__restrict__ a,
                                  int64_t n)
{
    const int col = blockIdx.y;
    const double s = a[col];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[(int64_t)col * n + e] = s * src[(int64_t)col * n + e];
}

__global__ void sub_kernel(double *__restrict__ dst, const double *__restrict__ a, const double *__restrict__ b,
                           int64_t n)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = a[e] - b[e];
}

__global__ void add_kernel(double *__restrict__ dst, const double *__restrict__ a, int64_t n)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] += a[e];
}

// [nt][3 ncol] (the ABI's layout) <-> [ncol][3 nt] (the solver's): to_cols = 1 reads src in
// the ABI layout
__global__ void transpose_cols_kernel(int64_t nt, int ncol, int to_cols, const double *__restrict__ src,
                                      double *__restrict__ dst)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * nt * ncol) return;
    const int64_t k = e / (3 * ncol);
    const int r = (int)(e % (3 * ncol));
    const int col = r / 3, c = r % 3;
    const int64_t solver = (int64_t)col * 3 * nt + 3 * k + c;
    if (to_cols) dst[solver] = src[e];
    else dst[e] = src[solver];
}

// split the unknowns of every column into the boundary u and t (Eq. num2 back to Eq. num)
__global__ void split_kernel(int64_t n, int ncol, const double *__restrict__ x, const uint8_t *__restrict__ mask,
                             const double *__restrict__ val, double *__restrict__ u, double *__restrict__ t)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * ncol) return;
    const int64_t i = e % n;
    if (mask[i]) {
        u[e] = val[e];
        t[e] = x[e];
    } else {
        u[e] = x[e];
        t[e] = val[e];
    }
}

// interior sources of columns c0 .. c0 + cn - 1: sl = t_k w, dl = -u_k w, [16 nt][3 cn]
template <typename R>
__global__ void interior_density_kernel(int64_t nt, int c0, int cn, const double *__restrict__ u,
                                        const double *__restrict__ t, const double *__restrict__ qw, R *__restrict__ sl,
                                        R *__restrict__ dl)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 16 * nt * cn) return;
    const int64_t j = e / cn;
    const int cc = (int)(e % cn);
    const int64_t k = j / 16;
    const int64_t col = (int64_t)(c0 + cc) * 3 * nt;
    for (int c = 0; c < 3; ++c) {
        sl[j * 3 * cn + 3 * cc + c] = (R)(t[col + 3 * k + c] * qw[j]);
        dl[j * 3 * cn + 3 * cc + c] = (R)(-u[col + 3 * k + c] * qw[j]);
    }
}

__global__ void f2d_kernel(int64_t n, const float *__restrict__ a, double *__restrict__ b)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

// b[i][ld * ... ]: FP64 [n][no] into columns col of FP32 [n][no * ncol]
__global__ void d2f_cols_kernel(int64_t n, int no, int ncol, int col, const double *__restrict__ a,
                                float *__restrict__ b)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * no) return;
    const int64_t i = e / no;
    b[i * no * ncol + (int64_t)no * col + e % no] = (float)a[e];
}

// Eq. deriv: D^T = 3/(4E) (1-nu)/(7-5nu) [10 (1+nu) s:s - (1+5nu) (tr s)^2];
// energy density 1/2 s:eps with eps = ((1+nu) s - nu tr(s) I) / E.  s6 [n][6 ncol] ->
// td, energy [n][ncol].
// s [n][row] += m [row] for every point (row = 6 ncol: a uniform stress per column)
__global__ void add_macro_kernel(int64_t total, int row, const double *__restrict__ m, float *__restrict__ s)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) s[i] += (float)m[i % row];
}

__global__ void topo_kernel(int64_t n, int ncol, const float *__restrict__ s6, float E, float nu,
                            float *__restrict__ td, float *__restrict__ energy)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * ncol) return;
    const float *s = s6 + 6 * e;
    const float tr = s[0] + s[1] + s[2];
    const float ss = s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + 2.f * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]);
    if (td) td[e] = 0.75f / E * (1.f - nu) / (7.f - 5.f * nu) * (10.f * (1.f + nu) * ss - (1.f + 5.f * nu) * tr * tr);
    if (energy) energy[e] = 0.5f * ((1.f + nu) * ss - nu * tr * tr) / E;
}

unsigned g1(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------
#define BK_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return b->fail(KFMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
#define BK_LAUNCH()                                                                        \
    do {                                                                                   \
        ++b->n_launch;                                                                     \
        cudaError_t e_ = cudaGetLastError();                                               \
        if (e_ != cudaSuccess) return b->fail(KFMM_ERR_CUDA, std::string("bem kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)
#define BK_FMM(call)                                                                       \
    do {                                                                                   \
        kfmm_status s_ = (call);                                                           \
        if (s_ != KFMM_OK) return b->fail(s_, std::string("fmm: ") + kfmm_last_error(b->surf)); \
    } while (0)
#define BK_TRY(expr)                                                                       \
    do {                                                                                   \
        kfmm_status s_ = (expr);                                                           \
        if (s_ != KFMM_OK) return s_;                                                      \
    } while (0)

static kfmm_status bem_stage(bem_ctx *b, DevBuf &buf, const void *p, size_t bytes, const void **out)
{
    if (!p || is_device_ptr(p)) {
        *out = p;
        return KFMM_OK;
    }
    BK_CUDA(buf.ensure(bytes));
    BK_CUDA(cudaMemcpyAsync(buf.p, p, bytes, cudaMemcpyHostToDevice, b->stream));
    *out = buf.p;
    return KFMM_OK;
}

// Neighbour lists (triangles sharing a vertex) and the upsampled near blocks (bem_near_kernel).
static kfmm_status bem_near_setup(bem_ctx *b)
{
    const int64_t nt = b->nt;
    if (b->n_near == 0) {
        std::vector<int32_t> ht(3 * nt);
        BK_CUDA(cudaMemcpy(ht.data(), b->tris.p, sizeof(int32_t) * 3 * nt, cudaMemcpyDeviceToHost));
        std::vector<std::vector<int>> by_vertex(b->nv);
        for (int64_t k = 0; k < nt; ++k)
            for (int e = 0; e < 3; ++e) by_vertex[ht[3 * k + e]].push_back((int)k);
        std::vector<int> off(nt + 1, 0), idx, pl;
        std::vector<int> tmp;
        for (int64_t l = 0; l < nt; ++l) {
            tmp.clear();
            for (int e = 0; e < 3; ++e)
                for (int k : by_vertex[ht[3 * l + e]])
                    if (k != l) tmp.push_back(k);
            std::sort(tmp.begin(), tmp.end());
            tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
            for (int k : tmp) {
                idx.push_back(k);
                pl.push_back((int)l);
            }
            off[l + 1] = (int)idx.size();
        }
        b->n_near = (int64_t)idx.size();
        BK_CUDA(b->nbr_off.ensure(sizeof(int) * (nt + 1)));
        BK_CUDA(b->nbr_idx.ensure(sizeof(int) * std::max<int64_t>(1, 2 * b->n_near)));
        BK_CUDA(cudaMemcpy(b->nbr_off.p, off.data(), sizeof(int) * (nt + 1), cudaMemcpyHostToDevice));
        if (b->n_near) {
            BK_CUDA(cudaMemcpy(b->nbr_idx.p, idx.data(), sizeof(int) * b->n_near, cudaMemcpyHostToDevice));
            // the pair's collocation triangle, behind the neighbour indices
            BK_CUDA(cudaMemcpy(b->nbr_idx.as<int>() + b->n_near, pl.data(), sizeof(int) * b->n_near,
                               cudaMemcpyHostToDevice));
        }
    }
    BK_CUDA(b->corrN.ensure(sizeof(double) * 18 * std::max<int64_t>(1, b->n_near)));
    if (b->n_near) {
        bem_near_kernel<<<g1(b->n_near, 128), 128, 0, b->stream>>>(
            b->n_near, b->nbr_idx.as<int>() + b->n_near, b->nbr_idx.as<int>(), b->near_levels, b->verts.as<double>(),
            b->tris.as<int>(), b->cen64.as<double>(), b->q64.as<double>(), b->qn64.as<double>(), b->qw.as<double>(),
            b->G, b->nu, b->corrN.as<double>());
        BK_LAUNCH();
    }
    b->near_ready = b->near_levels;
    return KFMM_OK;
}

// Leaf cap of the boundary sums, timed on this surface: the cost of a matvec swings with how
// the tree levels fall on the geometry (the P2L of the X lists above all), by up to 1.7x
// between neighbouring caps (a cell with 16 voids, 208k triangles: 15.8, 16.2, 8.8, 13.7 and
// 7.9 ms at 64 ... 1024).  Each candidate is built and evaluated twice (one column of zero
// densities: the cost does not depend on the values); the second evaluation is timed.
static kfmm_status bem_tune_leaf_cap(bem_ctx *b)
{
    const int64_t nt = b->nt, nq = 16 * nt;
    BK_CUDA(b->slq.ensure(sizeof(float) * 3 * nq));
    BK_CUDA(b->dlq.ensure(sizeof(float) * 3 * nq));
    BK_CUDA(b->fout.ensure(sizeof(float) * 3 * nt));
    BK_CUDA(cudaMemsetAsync(b->slq.p, 0, sizeof(float) * 3 * nq, b->stream));
    BK_CUDA(cudaMemsetAsync(b->dlq.p, 0, sizeof(float) * 3 * nq, b->stream));
    cudaEvent_t e0, e1;
    BK_CUDA(cudaEventCreate(&e0));
    BK_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_cap = b->opt.leaf_cap;
    kfmm_status st = KFMM_OK;
    for (int cap : {128, 256, 512, 1024}) {
        b->surf->opt.leaf_cap = cap;
        st = kfmm_build(b->surf, b->q32.as<float>(), b->qn32.as<float>(), nq, b->cen32.as<float>(), nt);
        if (st == KFMM_OK)
            st = kfmm_eval(b->surf, b->slq.as<float>(), b->dlq.as<float>(), 1, KFMM_DISP, b->fout.as<float>());
        if (st != KFMM_OK) break;
        cudaEventRecord(e0, b->stream);
        st = kfmm_eval(b->surf, b->slq.as<float>(), b->dlq.as<float>(), 1, KFMM_DISP, b->fout.as<float>());
        cudaEventRecord(e1, b->stream);
        if (st != KFMM_OK) break;
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = KFMM_ERR_CUDA;
            break;
        }
        if (ms < best) best = ms, best_cap = cap;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != KFMM_OK) return b->fail(st, std::string("bem: leaf-cap tuning: ") + kfmm_last_error(b->surf));
    b->opt.leaf_cap = b->surf->opt.leaf_cap = best_cap;
    // the launch shapes were tuned on the first candidate's tree: tune them again on this one
    b->surf->tune.m2l_done = b->surf->tune.eval_done = false;
    return KFMM_OK;
}

static kfmm_status bem_setup(bem_ctx *b)
{
    const bool material = !(b->setup_G == b->G && b->setup_nu == b->nu);
    const int64_t nt = b->nt;
    if (material) {
        DevBuf bad;
        BK_CUDA(bad.ensure(sizeof(int)));
        BK_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), b->stream));
        bem_setup_kernel<<<g1(nt, 128), 128, 0, b->stream>>>(
            nt, b->verts.as<double>(), b->tris.as<int>(), b->G, b->nu, b->q32.as<float>(), b->qn32.as<float>(),
            b->q64.as<double>(), b->qn64.as<double>(), b->qw.as<double>(), b->cen32.as<float>(),
            b->cen64.as<double>(), b->corrU.as<double>(), b->corrT.as<double>(), bad.as<int>());
        BK_LAUNCH();
        int hb = 0;
        BK_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        BK_CUDA(cudaStreamSynchronize(b->stream));
        if (hb) return b->fail(KFMM_ERR_INVALID_ARG, "bem: zero-area or non-finite triangle");
        b->setup_G = b->G;
        b->setup_nu = b->nu;
        b->near_ready = 0;
    }
    if (b->op == BEM_FMM && !b->surf_built) {
        if (b->auto_cap && b->opt.autotune) BK_TRY(bem_tune_leaf_cap(b));
        BK_FMM(kfmm_build(b->surf, b->q32.as<float>(), b->qn32.as<float>(), 16 * nt, b->cen32.as<float>(), nt));
        b->surf_built = true;
    }
    if (b->near_levels > 1 && b->near_ready != b->near_levels) BK_TRY(bem_near_setup(b));
    return KFMM_OK;
}

// M(u, t) (mode 0, one column), A x (mode 1) or B y (mode 2; sign -1) for `nc` density
// columns into out (device, FP64 [nc][3 nt]; mode 0: [nt][3]), with the context's operator or
// the given one (a bem_operator).  The FMM sums all columns in one evaluation; the direct
// operators take one column at a time.
static kfmm_status bem_op_apply(bem_ctx *b, int mode, const double *u, const double *t, const double *x,
                                double *out, int which = -1, int nc = 1)
{
    BK_TRY(bem_setup(b));
    const int64_t nt = b->nt, nq = 16 * nt;
    const double sign = mode == 2 ? -1.0 : 1.0;
    const uint8_t *mask = b->mask.as<uint8_t>();
    if (which < 0) which = b->op;
    if (which == BEM_FMM) {
        ++b->matvecs;
        BK_CUDA(b->slq.ensure(sizeof(float) * 3 * nq * nc));
        BK_CUDA(b->dlq.ensure(sizeof(float) * 3 * nq * nc));
        BK_CUDA(b->fout.ensure(sizeof(float) * 3 * nt * nc));
        bem_density_kernel<float><<<g1(nq * nc), 256, 0, b->stream>>>(nt, mode, 0, nc, u, t, x, mask,
                                                                      b->qw.as<double>(), b->slq.as<float>(),
                                                                      b->dlq.as<float>());
        BK_LAUNCH();
        BK_FMM(kfmm_eval(b->surf, b->slq.as<float>(), b->dlq.as<float>(), nc, KFMM_DISP, b->fout.as<float>()));
        bem_post_kernel<float><<<g1(nt * nc), 256, 0, b->stream>>>(
            nt, mode, 0, nc, sign, b->fout.as<float>(), u, t, x, mask, b->corrU.as<double>(), b->corrT.as<double>(),
            b->nbr_off.as<int>(), b->nbr_idx.as<int>(), b->near_levels > 1 ? b->corrN.as<double>() : nullptr, out);
        BK_LAUNCH();
        return KFMM_OK;
    }
    BK_CUDA(b->slq.ensure(sizeof(double) * 3 * nq));
    BK_CUDA(b->dlq.ensure(sizeof(double) * 3 * nq));
    BK_CUDA(b->fout.ensure(sizeof(double) * 3 * nt));
    for (int c = 0; c < nc; ++c) {
        ++b->matvecs_hi;
        bem_density_kernel<double><<<g1(nq), 256, 0, b->stream>>>(nt, mode, c, 1, u, t, x, mask, b->qw.as<double>(),
                                                                  b->slq.as<double>(), b->dlq.as<double>());
        BK_LAUNCH();
        if (which == BEM_DIRECT_HI)
            BK_FMM(kfmm_direct_hi(b->surf, b->cen64.as<double>(), nt, b->q64.as<double>(), b->qn64.as<double>(), nq,
                                  b->slq.as<double>(), b->dlq.as<double>(), b->near_radius, b->fout.as<double>()));
        else
            BK_FMM(kfmm_direct(b->surf, KFMM_FP64, b->cen64.p, nt, b->q64.p, b->qn64.p, nq, b->slq.p, b->dlq.p,
                               KFMM_DISP, b->fout.p));
        bem_post_kernel<double><<<g1(nt), 256, 0, b->stream>>>(
            nt, mode, c, 1, sign, b->fout.as<double>(), u, t, x, mask, b->corrU.as<double>(), b->corrT.as<double>(),
            b->nbr_off.as<int>(), b->nbr_idx.as<int>(), b->near_levels > 1 ? b->corrN.as<double>() : nullptr, out);
        BK_LAUNCH();
    }
    return KFMM_OK;
}

// h[col * k + i] = V_i[col] . w[col] for i < k and every column (partial sums reduced on the
// device in a fixed order, one read-back)
static kfmm_status mdot(bem_ctx *b, const double *V, int64_t ldv, int k, const double *w, int nc, double *h)
{
    const int64_t n = 3 * b->nt;
    const int total = nc * k;
    BK_CUDA(b->part.ensure(sizeof(double) * ((size_t)kVecBlocks * total + total)));
    double *part = b->part.as<double>(), *red = part + (size_t)kVecBlocks * total;
    mdot_kernel<<<dim3(kVecBlocks, nc), kVecThreads, 0, b->stream>>>(V, ldv, k, w, n, part);
    BK_LAUNCH();
    reduce_parts_kernel<<<g1(total, 8), 256, 0, b->stream>>>(part, kVecBlocks, total, red);
    BK_LAUNCH();
    BK_CUDA(cudaMemcpyAsync(h, red, sizeof(double) * total, cudaMemcpyDeviceToHost, b->stream));
    BK_CUDA(cudaStreamSynchronize(b->stream));
    return KFMM_OK;
}

// w[col] += sign * sum_i h[col * hld + i] V_i[col] (h on the host)
static kfmm_status maxpy(bem_ctx *b, double *w, const double *V, int64_t ldv, int k, const double *h, int hld,
                         double sign, int nc)
{
    const int64_t n = 3 * b->nt;
    BK_CUDA(b->hdev.ensure(sizeof(double) * (size_t)nc * hld + 8));
    BK_CUDA(cudaMemcpyAsync(b->hdev.p, h, sizeof(double) * (size_t)nc * hld, cudaMemcpyHostToDevice, b->stream));
    maxpy_kernel<<<dim3(kVecBlocks, nc), kVecThreads, 0, b->stream>>>(w, V, ldv, k, b->hdev.as<double>(), hld, sign,
                                                                      n);
    BK_LAUNCH();
    BK_CUDA(cudaStreamSynchronize(b->stream));  // h lives on the host
    return KFMM_OK;
}

// dst[col] = a[col] * src[col] (a on the host)
static kfmm_status scale_copy(bem_ctx *b, double *dst, const double *src, const double *a, int nc)
{
    BK_CUDA(b->av.ensure(sizeof(double) * nc));
    BK_CUDA(cudaMemcpyAsync(b->av.p, a, sizeof(double) * nc, cudaMemcpyHostToDevice, b->stream));
    scale_copy_kernel<<<dim3(kVecBlocks, nc), kVecThreads, 0, b->stream>>>(dst, src, b->av.as<double>(), 3 * b->nt);
    BK_LAUNCH();
    BK_CUDA(cudaStreamSynchronize(b->stream));  // a lives on the host
    return KFMM_OK;
}

static kfmm_status vnorm(bem_ctx *b, const double *w, int nc, double *out)
{
    std::vector<double> s(nc);
    BK_TRY(mdot(b, w, 0, 1, w, nc, s.data()));
    for (int c = 0; c < nc; ++c) out[c] = std::sqrt(std::max(s[c], 0.0));
    return KFMM_OK;
}

// Restarted GMRES (classical Gram-Schmidt twice, FP64 vectors) for A x = rhs with operator
// `which`, for nc density columns in lockstep: every Arnoldi step applies the operator to all
// columns at once (one FMM evaluation), each column keeps its own Krylov basis, Hessenberg
// matrix and Givens rotations.  x (device, [nc][n]) holds the initial guess (zeroed when
// zero_x) and receives the iterate.  Column c stops extending its basis once its residual
// estimate reaches tol[c] * bn[c] (its next basis vectors are zero, so its products are zero);
// a restart cycle ends when no column extends; the true residual is formed at every restart.
// Stops when every column meets its tolerance or after maxit steps.  iters, rel[c] (true
// residual / bn[c]) and conv[c] are returned; x0_rel[c] (may be NULL) receives the initial
// guess's relative residual (an initial guess worse than zero is dropped for zero).
static kfmm_status gmres_core(bem_ctx *b, int which, int nc, const double *rhs, double *x, bool zero_x,
                              const double *bn, const double *tol, int m, int maxit, int *iters, double *rel,
                              bool *conv, double *x0_rel = nullptr)
{
    const int64_t n = 3 * b->nt, N = n * nc;
    BK_CUDA(b->basis.ensure(sizeof(double) * (size_t)(m + 1) * N));
    BK_CUDA(b->w.ensure(sizeof(double) * N));
    BK_CUDA(b->r.ensure(sizeof(double) * N));
    double *V = b->basis.as<double>(), *w = b->w.as<double>(), *r = b->r.as<double>();
    if (zero_x) BK_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * N, b->stream));
    std::vector<std::vector<double>> H(nc, std::vector<double>((size_t)(m + 1) * m, 0.0)), cs(nc, std::vector<double>(m)),
        sn(nc, std::vector<double>(m)), g(nc, std::vector<double>(m + 1));
    std::vector<double> beta(nc), h((size_t)nc * (m + 1)), h2((size_t)nc * (m + 1)), hn(nc), a(nc),
        ycoef((size_t)nc * (m + 1));
    std::vector<int> steps(nc);
    std::vector<char> extend(nc);
    int it = 0;
    bool first = true;
    while (true) {
        // true residual r = rhs - A x
        if (!zero_x || !first) {
            BK_TRY(bem_op_apply(b, 1, nullptr, nullptr, x, w, which, nc));
            sub_kernel<<<kVecBlocks, kVecThreads, 0, b->stream>>>(r, rhs, w, N);
            BK_LAUNCH();
        } else {
            BK_CUDA(cudaMemcpyAsync(r, rhs, sizeof(double) * N, cudaMemcpyDeviceToDevice, b->stream));
        }
        BK_TRY(vnorm(b, r, nc, beta.data()));
        if (first && !zero_x) {
            for (int c = 0; c < nc; ++c) {
                if (x0_rel) x0_rel[c] = beta[c] / bn[c];
                if (beta[c] > bn[c]) {
                    // an initial guess worse than zero is dropped: this column starts from zero
                    BK_CUDA(cudaMemsetAsync(x + c * n, 0, sizeof(double) * n, b->stream));
                    BK_CUDA(cudaMemcpyAsync(r + c * n, rhs + c * n, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                                            b->stream));
                    beta[c] = bn[c];
                }
            }
        }
        first = false;
        bool all = true;
        for (int c = 0; c < nc; ++c) {
            rel[c] = beta[c] / bn[c];
            conv[c] = rel[c] <= tol[c];
            all = all && conv[c];
        }
        if (all || it >= maxit) break;
        for (int c = 0; c < nc; ++c) {
            extend[c] = !conv[c] && beta[c] > 0.0;
            a[c] = extend[c] ? 1.0 / beta[c] : 0.0;
            std::fill(g[c].begin(), g[c].end(), 0.0);
            g[c][0] = beta[c];
            steps[c] = 0;
        }
        BK_TRY(scale_copy(b, V, r, a.data(), nc));
        for (int j = 0; j < m && it < maxit; ++j) {
            double *vj = V + (size_t)j * N, *vn = V + (size_t)(j + 1) * N;
            BK_TRY(bem_op_apply(b, 1, nullptr, nullptr, vj, w, which, nc));
            ++it;
            // classical Gram-Schmidt, twice (per column; columns that stopped have zero vectors)
            BK_TRY(mdot(b, V, N, j + 1, w, nc, h.data()));
            BK_TRY(maxpy(b, w, V, N, j + 1, h.data(), j + 1, -1.0, nc));
            BK_TRY(mdot(b, V, N, j + 1, w, nc, h2.data()));
            BK_TRY(maxpy(b, w, V, N, j + 1, h2.data(), j + 1, -1.0, nc));
            BK_TRY(vnorm(b, w, nc, hn.data()));
            bool any = false;
            for (int c = 0; c < nc; ++c) {
                a[c] = 0.0;
                if (!extend[c]) continue;
                double *hc = h.data() + (size_t)c * (j + 1), *h2c = h2.data() + (size_t)c * (j + 1);
                std::vector<double> col(j + 2);
                for (int i = 0; i <= j; ++i) col[i] = hc[i] + h2c[i];
                col[j + 1] = hn[c];
                a[c] = hn[c] > 0 ? 1.0 / hn[c] : 0.0;
                for (int i = 0; i < j; ++i) {
                    const double t0 = cs[c][i] * col[i] + sn[c][i] * col[i + 1];
                    col[i + 1] = -sn[c][i] * col[i] + cs[c][i] * col[i + 1];
                    col[i] = t0;
                }
                const double den = std::hypot(col[j], col[j + 1]);
                cs[c][j] = den > 0 ? col[j] / den : 1.0;
                sn[c][j] = den > 0 ? col[j + 1] / den : 0.0;
                col[j] = den;
                g[c][j + 1] = -sn[c][j] * g[c][j];
                g[c][j] = cs[c][j] * g[c][j];
                for (int i = 0; i <= j; ++i) H[c][(size_t)i * m + j] = col[i];
                steps[c] = j + 1;
                if (std::fabs(g[c][j + 1]) / bn[c] <= tol[c] || hn[c] == 0.0) {
                    extend[c] = 0;
                    a[c] = 0.0;  // its next basis vector is zero
                }
                any = any || extend[c];
            }
            BK_TRY(scale_copy(b, vn, w, a.data(), nc));
            if (!any) break;
        }
        // x += V y per column (columns that took no step add nothing)
        int kmax = 0;
        std::fill(ycoef.begin(), ycoef.end(), 0.0);
        for (int c = 0; c < nc; ++c) {
            const int jc = steps[c];
            kmax = std::max(kmax, jc);
            double *y = ycoef.data() + (size_t)c * (m + 1);
            for (int i = jc - 1; i >= 0; --i) {
                double s = g[c][i];
                for (int k2 = i + 1; k2 < jc; ++k2) s -= H[c][(size_t)i * m + k2] * y[k2];
                y[i] = s / H[c][(size_t)i * m + i];
            }
        }
        if (kmax > 0) BK_TRY(maxpy(b, x, V, N, kmax, ycoef.data(), m + 1, 1.0, nc));
    }
    *iters = it;
    return KFMM_OK;
}

static void fill_stats(int nc, const double *rel, const bool *conv, const double *x0, bem_stats *st)
{
    st->relres = 0.0;
    st->converged = 1;
    st->x0_relres = 0.0;
    for (int c = 0; c < nc; ++c) {
        st->relres = std::max(st->relres, rel[c]);
        st->converged = st->converged && conv[c];
        st->x0_relres = std::max(st->x0_relres, x0[c]);
    }
}

// right-hand sides B y of every column with operator `which`, their norms (0 -> 1)
static kfmm_status rhs_norms(bem_ctx *b, int which, double *rhs, std::vector<double> &bn)
{
    const int nc = b->ncol;
    BK_TRY(bem_op_apply(b, 2, nullptr, nullptr, b->val.as<double>(), rhs, which, nc));
    bn.assign(nc, 1.0);
    BK_TRY(vnorm(b, rhs, nc, bn.data()));
    for (double &v : bn)
        if (v == 0.0) v = 1.0;
    return KFMM_OK;
}

// the caller's initial guess [nt][3 ncol] (host or device) into x [ncol][3 nt]
static kfmm_status load_x0(bem_ctx *b, const double *x0, double *x)
{
    const int64_t N = 3 * b->nt * b->ncol;
    const void *dx0;
    BK_TRY(bem_stage(b, b->stage[0], x0, sizeof(double) * N, &dx0));
    transpose_cols_kernel<<<g1(N), 256, 0, b->stream>>>(b->nt, b->ncol, 1, (const double *)dx0, x);
    BK_LAUNCH();
    return KFMM_OK;
}

// Plain GMRES on the context's operator (FP64 direct, or FMM with FP64 Krylov vectors).
static kfmm_status gmres(bem_ctx *b, const bem_solve_opts &o, bem_stats *st)
{
    const int nc = b->ncol;
    const int64_t N = 3 * b->nt * nc;
    BK_CUDA(b->x.ensure(sizeof(double) * N));
    BK_CUDA(b->b.ensure(sizeof(double) * N));
    double *x = b->x.as<double>(), *rhs = b->b.as<double>();
    std::vector<double> bn;
    BK_TRY(rhs_norms(b, b->op, rhs, bn));
    if (o.x0) BK_TRY(load_x0(b, o.x0, x));
    int it = 0;
    std::vector<double> rel(nc, 1.0), x0_rel(nc, 1.0), tol(nc, o.tol);
    std::unique_ptr<bool[]> conv(new bool[nc]);
    BK_TRY(gmres_core(b, b->op, nc, rhs, x, o.x0 == nullptr, bn.data(), tol.data(), o.restart, o.maxit, &it,
                      rel.data(), conv.get(), x0_rel.data()));
    fill_stats(nc, rel.data(), conv.get(), x0_rel.data(), st);
    st->iters = it;
    st->outer = 1;
    return KFMM_OK;
}

// Mixed-precision GMRES with iterative refinement: the right-hand side, every outer residual
// r = b - A x and the update x += d are FP64, with an FP64-grade all-pairs operator (the exact
// discrete operator: the compensated direct sum for refine = 1, the FP64 direct sum for
// refine = 2); each correction solves A d = r by GMRES on the FP32 FMM operator to the
// relative tolerance inner_tol, all density columns in lockstep (a column already at the
// outer tolerance gets a zero correction).  The relative residual reported is the FP64-grade
// one, the largest over the columns.
static kfmm_status gmres_ir(bem_ctx *b, const bem_solve_opts &o, bem_stats *st)
{
    const int nc = b->ncol;
    const int64_t n = 3 * b->nt, N = n * nc;
    BK_CUDA(b->x.ensure(sizeof(double) * N));
    BK_CUDA(b->b.ensure(sizeof(double) * N));
    BK_CUDA(b->d.ensure(sizeof(double) * N));
    BK_CUDA(b->rhs_hi.ensure(sizeof(double) * N));
    BK_CUDA(b->w.ensure(sizeof(double) * N));
    double *x = b->x.as<double>(), *rhs = b->b.as<double>(), *d = b->d.as<double>(), *r = b->rhs_hi.as<double>();
    const int hi = o.refine == 2 ? BEM_DIRECT_FP64 : BEM_DIRECT_HI;  // the outer (FP64-grade) operator
    std::vector<double> bn;
    BK_TRY(rhs_norms(b, hi, rhs, bn));
    if (o.x0) BK_TRY(load_x0(b, o.x0, x));
    else BK_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * N, b->stream));
    std::vector<double> rn(nc), rel(nc, 1.0), x0_rel(nc, 1.0), itol(nc), irel(nc), rn1(nc);
    std::unique_ptr<bool[]> conv(new bool[nc]), iconv(new bool[nc]);
    int inner_total = 0, outer = 0;
    while (true) {
        // outer residual in FP64 with the FP64-grade operator
        if (o.x0 || outer > 0) {
            BK_TRY(bem_op_apply(b, 1, nullptr, nullptr, x, b->w.as<double>(), hi, nc));
            sub_kernel<<<kVecBlocks, kVecThreads, 0, b->stream>>>(r, rhs, b->w.as<double>(), N);
            BK_LAUNCH();
        } else {
            BK_CUDA(cudaMemcpyAsync(r, rhs, sizeof(double) * N, cudaMemcpyDeviceToDevice, b->stream));
        }
        BK_TRY(vnorm(b, r, nc, rn.data()));
        bool all = true;
        for (int c = 0; c < nc; ++c) {
            if (o.x0 && outer == 0) {
                x0_rel[c] = rn[c] / bn[c];
                if (rn[c] > bn[c]) {
                    // an initial guess worse than zero is dropped: this column starts from zero
                    BK_CUDA(cudaMemsetAsync(x + c * n, 0, sizeof(double) * n, b->stream));
                    BK_CUDA(cudaMemcpyAsync(r + c * n, rhs + c * n, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                                            b->stream));
                    rn[c] = bn[c];
                }
            }
            rel[c] = rn[c] / bn[c];
            conv[c] = rel[c] <= o.tol;
            all = all && conv[c];
        }
        if (all) break;
        if (outer >= o.max_outer || inner_total >= o.maxit) break;
        // corrections on the fast operator: A_fmm d = r to inner_tol relative to ||r||, or only
        // as far as the outer target needs (with a factor 5 of margin for the gap between the
        // FMM and the FP64-grade operator) when closer; converged columns get d = 0
        for (int c = 0; c < nc; ++c) {
            if (conv[c]) {
                BK_CUDA(cudaMemsetAsync(r + c * n, 0, sizeof(double) * n, b->stream));
                rn1[c] = 1.0;
                itol[c] = 1.0;
            } else {
                rn1[c] = rn[c];
                itol[c] = std::max(o.inner_tol, 0.2 * o.tol * bn[c] / rn[c]);
            }
        }
        int it = 0;
        BK_TRY(gmres_core(b, BEM_FMM, nc, r, d, true, rn1.data(), itol.data(), o.restart, o.maxit - inner_total, &it,
                          irel.data(), iconv.get()));
        inner_total += it;
        ++outer;
        add_kernel<<<kVecBlocks, kVecThreads, 0, b->stream>>>(x, d, N);
        BK_LAUNCH();
    }
    fill_stats(nc, rel.data(), conv.get(), x0_rel.data(), st);
    st->iters = inner_total;
    st->outer = outer;
    return KFMM_OK;
}

extern "C" {

void bem_default_solve_opts(bem_solve_opts *o)
{
    if (!o) return;
    o->tol = 1e-6;
    o->restart = 30;
    o->maxit = 1000;
    o->x0 = nullptr;
    o->refine = 0;
    o->inner_tol = 1e-3;
    o->max_outer = 30;
}

kfmm_status bem_create(bem_ctx **out, const kfmm_options *opt, int op, const double *verts, int64_t nv,
                       const int32_t *tris, int64_t nt)
{
    if (!out) return KFMM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!verts || !tris || nv < 3 || nt < 1 || (op != BEM_FMM && op != BEM_DIRECT_FP64 && op != BEM_DIRECT_HI) || 16 * nt > (1LL << 30))
        return KFMM_ERR_INVALID_ARG;
    bem_ctx *b = new (std::nothrow) bem_ctx();
    if (!b) return KFMM_ERR_OOM;
    kfmm_default_options(&b->opt);
    if (opt) b->opt = *opt;
    // leaf_cap 0 (or no options): the BEM's own caps.  Its sources are 16 quadrature points
    // per triangle, so the general-purpose cap of 64 leaves only 4 triangles per leaf; on
    // cantilevers of 52k and 400k triangles the surface matvec was fastest at 256 and 512
    // sources per leaf (1.35 against 3.0 ms; 6.2 against 15.7 ms).  With autotuning on (the
    // default) the boundary sums time 128 ... 1024 on the surface instead (bem_tune_leaf_cap).
    b->auto_cap = !opt || opt->leaf_cap == 0;
    if (b->auto_cap) b->opt.leaf_cap = 16 * nt <= (int64_t)(2 << 20) ? 256 : 512;
    b->op = op;
    b->nt = nt;
    b->nv = nv;
    kfmm_status s = kfmm_create(&b->surf, &b->opt);
    if (s != KFMM_OK) {
        delete b;
        return s;
    }
    // copy the mesh, check indices
    std::vector<int32_t> ht(3 * nt);
    bool host_tris = !is_device_ptr(tris);
    if (host_tris) std::memcpy(ht.data(), tris, sizeof(int32_t) * 3 * nt);
    else cudaMemcpy(ht.data(), tris, sizeof(int32_t) * 3 * nt, cudaMemcpyDeviceToHost);
    for (int64_t i = 0; i < 3 * nt; ++i)
        if (ht[i] < 0 || ht[i] >= nv) {
            kfmm_destroy(b->surf);
            delete b;
            return KFMM_ERR_INVALID_ARG;
        }
    const int64_t nq = 16 * nt;
    bool ok = b->verts.ensure(sizeof(double) * 3 * nv) == cudaSuccess && b->tris.ensure(sizeof(int) * 3 * nt) == cudaSuccess &&
              b->q32.ensure(sizeof(float) * 3 * nq) == cudaSuccess && b->qn32.ensure(sizeof(float) * 3 * nq) == cudaSuccess &&
              b->q64.ensure(sizeof(double) * 3 * nq) == cudaSuccess && b->qn64.ensure(sizeof(double) * 3 * nq) == cudaSuccess &&
              b->qw.ensure(sizeof(double) * nq) == cudaSuccess && b->cen32.ensure(sizeof(float) * 3 * nt) == cudaSuccess &&
              b->cen64.ensure(sizeof(double) * 3 * nt) == cudaSuccess && b->corrU.ensure(sizeof(double) * 9 * nt) == cudaSuccess &&
              b->corrT.ensure(sizeof(double) * 9 * nt) == cudaSuccess && b->mask.ensure(3 * nt) == cudaSuccess &&
              b->val.ensure(sizeof(double) * 3 * nt) == cudaSuccess && b->usol.ensure(sizeof(double) * 3 * nt) == cudaSuccess &&
              b->tsol.ensure(sizeof(double) * 3 * nt) == cudaSuccess;
    if (!ok) {
        kfmm_destroy(b->surf);
        delete b;
        return KFMM_ERR_OOM;
    }
    cudaMemcpy(b->verts.p, verts, sizeof(double) * 3 * nv, cudaMemcpyDefault);
    cudaMemcpy(b->tris.p, ht.data(), sizeof(int) * 3 * nt, cudaMemcpyHostToDevice);
    std::vector<double> hv(3 * nv);
    cudaMemcpy(hv.data(), b->verts.p, sizeof(double) * 3 * nv, cudaMemcpyDeviceToHost);
    for (double v : hv)
        if (!std::isfinite(v)) {
            kfmm_destroy(b->surf);
            delete b;
            return KFMM_ERR_INVALID_ARG;
        }
    // pairs of the compensated direct sum closer than 4 longest edges are summed in FP64.
    // The remaining FP32 pairs leave ~5e-7 of ||b|| on the residual of a cantilever solution
    // (51,840 triangles; the residual cancels by ||A| |x|| / ||b|| ~ 100), measured against
    // the FP64 direct sum: 7.8e-7 at 4 edges, 6.4e-7 at 8, 4.7e-7 at 16 -- the error comes
    // from rounding that repeats over many pairs (sources of one element share their
    // density, normal and nearly their difference to a far target), so a larger radius buys
    // little; 4 edges keep the FP64 pairs a few percent of the work.
    double emax2 = 0.0;
    for (int64_t k = 0; k < nt; ++k)
        for (int e = 0; e < 3; ++e) {
            const double *a = &hv[3 * (size_t)ht[3 * k + e]], *c = &hv[3 * (size_t)ht[3 * k + (e + 1) % 3]];
            const double dx = a[0] - c[0], dy = a[1] - c[1], dz = a[2] - c[2];
            emax2 = std::max(emax2, dx * dx + dy * dy + dz * dz);
        }
    b->near_radius = 4.0 * std::sqrt(emax2);
    *out = b;
    return KFMM_OK;
}

kfmm_status bem_destroy(bem_ctx *b)
{
    if (!b) return KFMM_ERR_INVALID_ARG;
    cudaStreamSynchronize(b->stream);
    if (b->surf) kfmm_destroy(b->surf);
    if (b->vol) kfmm_destroy(b->vol);
    delete b;
    return KFMM_OK;
}

kfmm_status bem_set_material(bem_ctx *b, double K, double G)
{
    if (!b) return KFMM_ERR_INVALID_ARG;
    kfmm_status s = kfmm_set_material(b->surf, K, G);
    if (s != KFMM_OK) return b->fail(s, "bem: material needs K > 0 and G > 0");
    if (b->vol) kfmm_set_material(b->vol, K, G);
    b->G = G;
    b->K = K;
    b->nu = (3.0 * K - 2.0 * G) / (2.0 * (3.0 * K + G));
    return KFMM_OK;
}

kfmm_status bem_set_stream(bem_ctx *b, void *stream)
{
    if (!b) return KFMM_ERR_INVALID_ARG;
    b->stream = (cudaStream_t)stream;
    kfmm_set_stream(b->surf, stream);
    if (b->vol) kfmm_set_stream(b->vol, stream);
    return KFMM_OK;
}

kfmm_status bem_set_quadrature(bem_ctx *b, int near_levels)
{
    if (!b || near_levels < 1 || near_levels > 5) return KFMM_ERR_INVALID_ARG;
    b->near_levels = near_levels;
    return KFMM_OK;
}

kfmm_status bem_set_periodic(bem_ctx *b, int on, const double *lo, double side)
{
    if (!b) return KFMM_ERR_INVALID_ARG;
    b->err.clear();
    if (on && b->op != BEM_FMM)
        return b->fail(KFMM_ERR_INVALID_ARG, "bem: periodic sums need the FMM operator (the direct sums are free-space)");
    kfmm_status s = kfmm_set_periodic(b->surf, on, lo, side);
    if (s != KFMM_OK) return b->fail(s, std::string("bem: ") + kfmm_last_error(b->surf));
    if (b->vol) kfmm_set_periodic(b->vol, on, lo, side);
    b->periodic = on != 0;
    if (on) {
        for (int c = 0; c < 3; ++c) b->cell_lo[c] = lo[c];
        b->cell_side = side;
    }
    b->surf_built = false;  // the tree is built again at the next application
    return KFMM_OK;
}

kfmm_status bem_set_macro_stress(bem_ctx *b, const double *stress6, int ncol)
{
    if (!b) return KFMM_ERR_INVALID_ARG;
    b->err.clear();
    if (!stress6) {
        b->macro_ncol = 0;
        return KFMM_OK;
    }
    if (ncol < 1 || ncol > 32) return b->fail(KFMM_ERR_INVALID_ARG, "bem: macro stress needs 1 <= ncol <= 32");
    for (int i = 0; i < 6 * ncol; ++i)
        if (!std::isfinite(stress6[i])) return b->fail(KFMM_ERR_INVALID_ARG, "bem: non-finite macro stress");
    BK_CUDA(b->macro.ensure(sizeof(double) * 6 * ncol));
    BK_CUDA(cudaMemcpy(b->macro.p, stress6, sizeof(double) * 6 * ncol, cudaMemcpyHostToDevice));
    b->macro_ncol = ncol;
    return KFMM_OK;
}

kfmm_status bem_set_bc(bem_ctx *b, const uint8_t *known_is_disp, const double *values, int ncol)
{
    if (!b || !known_is_disp || !values || ncol < 1 || ncol > 32) return KFMM_ERR_INVALID_ARG;
    if (first_foreign({known_is_disp, values}))
        return b->fail(KFMM_ERR_INVALID_ARG, "bem: an array is device memory of another GPU");
    const int64_t N = 3 * b->nt * ncol;
    BK_CUDA(b->val.ensure(sizeof(double) * N));
    const void *dv;
    BK_TRY(bem_stage(b, b->stage[0], values, sizeof(double) * N, &dv));
    BK_CUDA(cudaMemcpyAsync(b->mask.p, known_is_disp, 3 * b->nt, cudaMemcpyDefault, b->stream));
    transpose_cols_kernel<<<g1(N), 256, 0, b->stream>>>(b->nt, ncol, 1, (const double *)dv, b->val.as<double>());
    BK_LAUNCH();
    BK_CUDA(cudaStreamSynchronize(b->stream));
    b->ncol = ncol;
    b->have_bc = true;
    return KFMM_OK;
}

kfmm_status bem_apply(bem_ctx *b, const double *u, const double *t, double *out)
{
    if (!b || !out || (!u && !t)) return KFMM_ERR_INVALID_ARG;
    if (first_foreign({u, t, out})) return b->fail(KFMM_ERR_INVALID_ARG, "bem: an array is device memory of another GPU");
    const size_t bytes = sizeof(double) * 3 * b->nt;
    const void *du, *dt;
    BK_TRY(bem_stage(b, b->stage[0], u, bytes, &du));
    BK_TRY(bem_stage(b, b->stage[1], t, bytes, &dt));
    double *dout = out;
    const bool host_out = !is_device_ptr(out);
    if (host_out) {
        BK_CUDA(b->out64.ensure(bytes));
        dout = b->out64.as<double>();
    }
    BK_TRY(bem_op_apply(b, 0, (const double *)du, (const double *)dt, nullptr, dout));
    if (host_out) BK_CUDA(cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, b->stream));
    BK_CUDA(cudaStreamSynchronize(b->stream));
    return KFMM_OK;
}

// y = A x or (x == NULL) y = B y_known for every column, ABI layout [nt][3 ncol] in and out
static kfmm_status bem_apply_cols(bem_ctx *b, const double *x, double *y)
{
    const int nc = b->ncol;
    const int64_t N = 3 * b->nt * nc;
    BK_CUDA(b->w.ensure(sizeof(double) * N));
    BK_CUDA(b->r.ensure(sizeof(double) * N));
    if (x) {
        const void *dx;
        BK_TRY(bem_stage(b, b->stage[0], x, sizeof(double) * N, &dx));
        transpose_cols_kernel<<<g1(N), 256, 0, b->stream>>>(b->nt, nc, 1, (const double *)dx, b->r.as<double>());
        BK_LAUNCH();
        BK_TRY(bem_op_apply(b, 1, nullptr, nullptr, b->r.as<double>(), b->w.as<double>(), -1, nc));
    } else {
        BK_TRY(bem_op_apply(b, 2, nullptr, nullptr, b->val.as<double>(), b->w.as<double>(), -1, nc));
    }
    double *dy = y;
    const bool host_out = !is_device_ptr(y);
    if (host_out) {
        BK_CUDA(b->out64.ensure(sizeof(double) * N));
        dy = b->out64.as<double>();
    }
    transpose_cols_kernel<<<g1(N), 256, 0, b->stream>>>(b->nt, nc, 0, b->w.as<double>(), dy);
    BK_LAUNCH();
    if (host_out) BK_CUDA(cudaMemcpyAsync(y, dy, sizeof(double) * N, cudaMemcpyDeviceToHost, b->stream));
    BK_CUDA(cudaStreamSynchronize(b->stream));
    return KFMM_OK;
}

kfmm_status bem_matvec(bem_ctx *b, const double *x, double *y)
{
    if (!b || !x || !y) return KFMM_ERR_INVALID_ARG;
    if (!b->have_bc) return b->fail(KFMM_ERR_NOT_BUILT, "bem: boundary conditions not set");
    if (first_foreign({x, y})) return b->fail(KFMM_ERR_INVALID_ARG, "bem: an array is device memory of another GPU");
    return bem_apply_cols(b, x, y);
}

kfmm_status bem_rhs(bem_ctx *b, double *rhs)
{
    if (!b || !rhs) return KFMM_ERR_INVALID_ARG;
    if (!b->have_bc) return b->fail(KFMM_ERR_NOT_BUILT, "bem: boundary conditions not set");
    if (foreign_device_ptr(rhs)) return b->fail(KFMM_ERR_INVALID_ARG, "bem: an array is device memory of another GPU");
    return bem_apply_cols(b, nullptr, rhs);
}

kfmm_status bem_solve(bem_ctx *b, const bem_solve_opts *opts, double *u, double *t, bem_stats *st)
{
    if (!b) return KFMM_ERR_INVALID_ARG;
    if (!b->have_bc) return b->fail(KFMM_ERR_NOT_BUILT, "bem: boundary conditions not set");
    bem_solve_opts o;
    bem_default_solve_opts(&o);
    if (opts) o = *opts;
    if (!(o.tol > 0) || o.restart < 1 || o.restart > 200 || o.maxit < 1)
        return b->fail(KFMM_ERR_INVALID_ARG, "bem_solve: need tol > 0, 1 <= restart <= 200, maxit >= 1");
    if (o.refine < 0 || o.refine > 2 ||
        (o.refine && (b->op != BEM_FMM || !(o.inner_tol > 0 && o.inner_tol < 1) || o.max_outer < 1)))
        return b->fail(KFMM_ERR_INVALID_ARG,
                       "bem_solve: refinement needs an FMM context, 0 < inner_tol < 1 and max_outer >= 1");
    if (o.refine && b->periodic)
        return b->fail(KFMM_ERR_INVALID_ARG, "bem_solve: no refinement with periodic sums (its outer operator is "
                                             "a free-space direct sum)");
    if (first_foreign({u, t, o.x0})) return b->fail(KFMM_ERR_INVALID_ARG, "bem: an array is device memory of another GPU");
    const auto t0 = std::chrono::steady_clock::now();
    bem_stats s{};
    const int mv0 = b->matvecs, mh0 = b->matvecs_hi;
    if (o.refine) BK_TRY(gmres_ir(b, o, &s));
    else BK_TRY(gmres(b, o, &s));
    const int nc = b->ncol;
    const int64_t n = 3 * b->nt, N = n * nc;
    BK_CUDA(b->usol.ensure(sizeof(double) * N));
    BK_CUDA(b->tsol.ensure(sizeof(double) * N));
    split_kernel<<<g1(N), 256, 0, b->stream>>>(n, nc, b->x.as<double>(), b->mask.as<uint8_t>(), b->val.as<double>(),
                                                b->usol.as<double>(), b->tsol.as<double>());
    BK_LAUNCH();
    b->have_sol = true;
    b->sol_ncol = nc;
    for (int k = 0; k < 2; ++k) {
        double *dst = k == 0 ? u : t;
        if (!dst) continue;
        const double *src = k == 0 ? b->usol.as<double>() : b->tsol.as<double>();
        double *d = dst;
        const bool host = !is_device_ptr(dst);
        if (host) {
            BK_CUDA(b->out64.ensure(sizeof(double) * N));
            d = b->out64.as<double>();
        }
        transpose_cols_kernel<<<g1(N), 256, 0, b->stream>>>(b->nt, nc, 0, src, d);
        BK_LAUNCH();
        if (host) BK_CUDA(cudaMemcpyAsync(dst, d, sizeof(double) * N, cudaMemcpyDeviceToHost, b->stream));
        BK_CUDA(cudaStreamSynchronize(b->stream));
    }
    s.matvecs = b->matvecs - mv0;
    s.matvecs_hi = b->matvecs_hi - mh0;
    s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (st) *st = s;
    if (!s.converged) return b->fail(KFMM_ERR_NOT_CONVERGED, "bem_solve: iteration cap reached");
    return KFMM_OK;
}

kfmm_status bem_set_solution(bem_ctx *b, const double *u, const double *t, int ncol)
{
    if (!b || !u || !t || ncol < 1 || ncol > 32) return KFMM_ERR_INVALID_ARG;
    if (first_foreign({u, t})) return b->fail(KFMM_ERR_INVALID_ARG, "bem: an array is device memory of another GPU");
    const int64_t N = 3 * b->nt * ncol;
    BK_CUDA(b->usol.ensure(sizeof(double) * N));
    BK_CUDA(b->tsol.ensure(sizeof(double) * N));
    for (int k = 0; k < 2; ++k) {
        const void *d;
        BK_TRY(bem_stage(b, b->stage[k], k == 0 ? u : t, sizeof(double) * N, &d));
        transpose_cols_kernel<<<g1(N), 256, 0, b->stream>>>(b->nt, ncol, 1, (const double *)d,
                                                            k == 0 ? b->usol.as<double>() : b->tsol.as<double>());
        BK_LAUNCH();
    }
    BK_CUDA(cudaStreamSynchronize(b->stream));
    b->have_sol = true;
    b->sol_ncol = ncol;
    return KFMM_OK;
}

kfmm_status bem_interior(bem_ctx *b, const float *pts, int64_t n, float *disp, float *stress)
{
    if (!b || !pts || n < 1 || (!disp && !stress)) return KFMM_ERR_INVALID_ARG;
    if (!b->have_sol) return b->fail(KFMM_ERR_NOT_BUILT, "bem: no boundary solution (solve or set_solution first)");
    if (first_foreign({pts, disp, stress}))
        return b->fail(KFMM_ERR_INVALID_ARG, "bem: an array is device memory of another GPU");
    BK_TRY(bem_setup(b));
    const int64_t nt = b->nt, nq = 16 * nt;
    const int nc = b->sol_ncol;
    const void *dp;
    BK_TRY(bem_stage(b, b->stage[2], pts, sizeof(float) * 3 * n, &dp));
    if (b->op == BEM_FMM) {
        if (!b->vol) {
            // interior stresses are far-field-dominated sums of a single and a double layer
            // that cancel each other in part: the interior context runs at p >= 8 with the M2L
            // basis cut at 1e-7 (p = 6 leaves ~3e-3 on the double-layer stress, p = 8 ~7e-5)
            kfmm_options vo = b->opt;
            vo.p = std::max(vo.p, 8);
            // p = 8 makes every box's far field dearer, so larger leaves pay: the 4.2M-point
            // stress evaluation of a 400k-triangle cantilever took 360 ms at 256 sources per
            // leaf and 109 ms at 768
            if (b->auto_cap) vo.leaf_cap = BEM_INTERIOR_LEAF_CAP;
            vo.m2l_rtol = vo.m2l_rtol > 0.0 ? std::min(vo.m2l_rtol, 1e-7) : 0.0;
            kfmm_status s = kfmm_create(&b->vol, &vo);
            if (s != KFMM_OK) return b->fail(s, "bem: interior FMM context");
            kfmm_set_material(b->vol, b->K, b->G);
            kfmm_set_stream(b->vol, b->stream);
            if (b->periodic) kfmm_set_periodic(b->vol, 1, b->cell_lo, b->cell_side);
        }
        BK_CUDA(b->slq.ensure(sizeof(float) * 3 * nq * nc));
        BK_CUDA(b->dlq.ensure(sizeof(float) * 3 * nq * nc));
        interior_density_kernel<float><<<g1(nq * nc), 256, 0, b->stream>>>(nt, 0, nc, b->usol.as<double>(),
                                                                           b->tsol.as<double>(), b->qw.as<double>(),
                                                                           b->slq.as<float>(), b->dlq.as<float>());
        BK_LAUNCH();
        kfmm_status s = kfmm_build(b->vol, b->q32.as<float>(), b->qn32.as<float>(), nq, (const float *)dp, n);
        if (s != KFMM_OK) return b->fail(s, std::string("interior fmm: ") + kfmm_last_error(b->vol));
        if (disp) {
            s = kfmm_eval(b->vol, b->slq.as<float>(), b->dlq.as<float>(), nc, KFMM_DISP, disp);
            if (s != KFMM_OK) return b->fail(s, std::string("interior fmm: ") + kfmm_last_error(b->vol));
        }
        if (stress) {
            s = kfmm_eval(b->vol, b->slq.as<float>(), b->dlq.as<float>(), nc, KFMM_STRESS, stress);
            if (s != KFMM_OK) return b->fail(s, std::string("interior fmm: ") + kfmm_last_error(b->vol));
        }
    } else {
        BK_CUDA(b->slq.ensure(sizeof(double) * 3 * nq));
        BK_CUDA(b->dlq.ensure(sizeof(double) * 3 * nq));
        BK_CUDA(b->pts64.ensure(sizeof(double) * 3 * n));
        BK_CUDA(b->out64.ensure(sizeof(double) * 6 * n));
        f2d_kernel<<<g1(3 * n), 256, 0, b->stream>>>(3 * n, (const float *)dp, b->pts64.as<double>());
        BK_LAUNCH();
        DevBuf of[2];
        float *dd[2] = {disp, stress};
        bool host[2] = {false, false};
        for (int kind = 0; kind < 2; ++kind) {
            if (!dd[kind]) continue;
            host[kind] = !is_device_ptr(dd[kind]);
            if (host[kind]) {
                BK_CUDA(of[kind].ensure(sizeof(float) * (kind == 0 ? 3 : 6) * n * nc));
                dd[kind] = of[kind].as<float>();
            }
        }
        for (int c = 0; c < nc; ++c) {
            interior_density_kernel<double><<<g1(nq), 256, 0, b->stream>>>(nt, c, 1, b->usol.as<double>(),
                                                                           b->tsol.as<double>(), b->qw.as<double>(),
                                                                           b->slq.as<double>(), b->dlq.as<double>());
            BK_LAUNCH();
            for (int kind = 0; kind < 2; ++kind) {
                if (!dd[kind]) continue;
                const int no = kind == 0 ? 3 : 6;
                BK_FMM(kfmm_direct(b->surf, KFMM_FP64, b->pts64.p, n, b->q64.p, b->qn64.p, nq, b->slq.p, b->dlq.p,
                                   kind == 0 ? KFMM_DISP : KFMM_STRESS, b->out64.p));
                d2f_cols_kernel<<<g1(no * n), 256, 0, b->stream>>>(n, no, nc, c, b->out64.as<double>(), dd[kind]);
                BK_LAUNCH();
            }
        }
        for (int kind = 0; kind < 2; ++kind)
            if (host[kind])
                BK_CUDA(cudaMemcpyAsync(kind == 0 ? disp : stress, dd[kind], sizeof(float) * (kind == 0 ? 3 : 6) * n * nc,
                                        cudaMemcpyDeviceToHost, b->stream));
        BK_CUDA(cudaStreamSynchronize(b->stream));
    }
    BK_CUDA(cudaStreamSynchronize(b->stream));
    return KFMM_OK;
}

kfmm_status bem_topo_derivative(bem_ctx *b, const float *pts, int64_t n, float *td, float *energy, float *stress)
{
    if (!b || !pts || n < 1 || (!td && !energy && !stress)) return KFMM_ERR_INVALID_ARG;
    if (!b->have_sol) return b->fail(KFMM_ERR_NOT_BUILT, "bem: no boundary solution (solve or set_solution first)");
    if (first_foreign({pts, td, energy, stress}))
        return b->fail(KFMM_ERR_INVALID_ARG, "bem: an array is device memory of another GPU");
    const int nc = b->sol_ncol;
    DevBuf sbuf, tdb, enb;
    float *ds = stress;
    const bool host_s = stress && !is_device_ptr(stress);
    if (!stress || host_s) {
        BK_CUDA(sbuf.ensure(sizeof(float) * 6 * n * nc));
        ds = sbuf.as<float>();
    }
    BK_TRY(bem_interior(b, pts, n, nullptr, ds));
    if (b->macro_ncol) {
        if (b->macro_ncol != nc) return b->fail(KFMM_ERR_INVALID_ARG, "bem: macro stress and solution columns differ");
        add_macro_kernel<<<g1(6 * n * nc), 256, 0, b->stream>>>(6 * n * nc, 6 * nc, b->macro.as<double>(), ds);
        BK_LAUNCH();
    }
    float *dtd = td, *den = energy;
    const bool host_td = td && !is_device_ptr(td), host_en = energy && !is_device_ptr(energy);
    if (host_td) {
        BK_CUDA(tdb.ensure(sizeof(float) * n * nc));
        dtd = tdb.as<float>();
    }
    if (host_en) {
        BK_CUDA(enb.ensure(sizeof(float) * n * nc));
        den = enb.as<float>();
    }
    const double E = 2.0 * b->G * (1.0 + b->nu);
    topo_kernel<<<g1(n * nc), 256, 0, b->stream>>>(n, nc, ds, (float)E, (float)b->nu, dtd, den);
    BK_LAUNCH();
    if (host_td) BK_CUDA(cudaMemcpyAsync(td, dtd, sizeof(float) * n * nc, cudaMemcpyDeviceToHost, b->stream));
    if (host_en) BK_CUDA(cudaMemcpyAsync(energy, den, sizeof(float) * n * nc, cudaMemcpyDeviceToHost, b->stream));
    if (host_s) BK_CUDA(cudaMemcpyAsync(stress, ds, sizeof(float) * 6 * n * nc, cudaMemcpyDeviceToHost, b->stream));
    BK_CUDA(cudaStreamSynchronize(b->stream));
    return KFMM_OK;
}

const char *bem_last_error(const bem_ctx *b) { return b ? b->err.c_str() : "null context"; }

}  // extern "C"
