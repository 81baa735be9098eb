/*
 * kelvin_oracle.c -- plain FP64 CPU oracle for the Kelvin elasticity sums and the
 * piecewise-constant collocation BEM of arXiv 1612.04082 ("What Lies Beneath the
 * Surface: Topological-Shape Optimization With the Kernel-Independent FMM").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls this
 * file; only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code with the CUDA path: every formula is written out again here
 * from the paper, in FP64, without blocking, fusion or reordering beyond the
 * definitions, so that it can be checked against the paper by eye.
 *
 * Conventions used throughout (readings of the paper, listed in the design notes):
 *   d = x_target - y_source, r = |d|, rhat = d / r.  Every kernel is set to 0 at r = 0
 *   (the sum of Eq. fmm_summation skips coincident points).
 *   U  : Eq. disp_1, 3x3, out_i += U_ij s_j          (single layer, "SL")
 *   T  : Eq. disp_2, 3x3, normal n at the source,    (double layer, "DL")
 *        out_i += T_ij s_j.  With r_,i = (xi - x)_i / r, i.e. target minus source, the
 *        printed form is the textbook traction kernel; the BIE of Eq. BIE reads
 *        1/2 u + int T u = int U t.
 *   D  : Eq. stress_2, stress at the target of the SL field, D = C : grad U.  The
 *        printed constant 1/(2 pi) is read as the textbook 1/(8 pi) (D = C:grad U is
 *        what Eq. stress_1 needs; the finite-difference pin checks it).
 *   S  : Eq. stress_3, stress at the target of the DL field, S = C : grad T, with the
 *        factor G the printed form omits.
 *   Stress components are stored in the order xx, yy, zz, yz, xz, xy.
 *   DISP(sl, dl)   = sum_j U(d) sl_j + T(d, n_j) dl_j
 *   STRESS(sl, dl) = sum_j D(d) sl_j + S(d, n_j) dl_j  (= Hooke of grad DISP)
 *   Somigliana (Eq. stress_1) is then STRESS(sl = t w, dl = -u w) and the interior
 *   displacement is DISP(sl = t w, dl = -u w).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define KO_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------ */
/* Kernels                                                                         */
/* ------------------------------------------------------------------------------ */

/* Eq. disp_1: U_ij = [(3-4nu) delta_ij + r_,i r_,j] / (16 pi (1-nu) G r). */
void ko_kernel_U(const double *d, double G, double nu, double *U)
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 == 0.0) {
        memset(U, 0, 9 * sizeof(double));
        return;
    }
    double r = sqrt(r2);
    double c = 1.0 / (16.0 * KO_PI * (1.0 - nu) * G * r);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            U[3 * i + j] = c * ((i == j ? 3.0 - 4.0 * nu : 0.0) + d[i] * d[j] / r2);
}

/* Eq. disp_2: P_ij = 1/(8 pi (1-nu) r^2) { dr/dn [(1-2nu) delta_ij + 3 r_,i r_,j]
 *                                          - (1-2nu) (r_,i n_j - r_,j n_i) }
 * with r_,i = d_i / r and dr/dn = r_,k n_k (n = normal at the source). */
void ko_kernel_T(const double *d, const double *n, double nu, double *T)
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 == 0.0) {
        memset(T, 0, 9 * sizeof(double));
        return;
    }
    double r = sqrt(r2);
    double rh[3] = {d[0] / r, d[1] / r, d[2] / r};
    double drdn = rh[0] * n[0] + rh[1] * n[1] + rh[2] * n[2];
    double c = 1.0 / (8.0 * KO_PI * (1.0 - nu) * r2);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = c * (drdn * ((i == j ? 1.0 - 2.0 * nu : 0.0) + 3.0 * rh[i] * rh[j]) -
                                (1.0 - 2.0 * nu) * (rh[i] * n[j] - rh[j] * n[i]));
}

static const int KO_VI[6] = {0, 1, 2, 1, 0, 0};
static const int KO_VJ[6] = {0, 1, 2, 2, 2, 1};

/* Eq. stress_2 (textbook constant): stress ij at the target from a unit SL force k at
 * the source.  With r_,i = (x_src - x_trg)_i / r = -rhat_i:
 *   D_kij = 1/(8 pi (1-nu) r^2) [(1-2nu)(delta_ki r_,j + delta_kj r_,i - delta_ij r_,k)
 *                                + 3 r_,i r_,j r_,k]
 * Output D[6 k + s], s over (xx, yy, zz, yz, xz, xy). */
void ko_kernel_D(const double *d, double nu, double *D)
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 == 0.0) {
        memset(D, 0, 18 * sizeof(double));
        return;
    }
    double r = sqrt(r2);
    double g[3] = {-d[0] / r, -d[1] / r, -d[2] / r}; /* r_,i: source minus target */
    double c = 1.0 / (8.0 * KO_PI * (1.0 - nu) * r2);
    for (int k = 0; k < 3; ++k)
        for (int s = 0; s < 6; ++s) {
            int i = KO_VI[s], j = KO_VJ[s];
            double v = (1.0 - 2.0 * nu) * ((k == i ? g[j] : 0.0) + (k == j ? g[i] : 0.0) -
                                           (i == j ? g[k] : 0.0)) +
                       3.0 * g[i] * g[j] * g[k];
            D[6 * k + s] = c * v;
        }
}

/* Eq. stress_3 with the factor G: stress ij at the target from a unit DL density k
 * at the source (normal n).  With r_,i = (x_src - x_trg)_i / r and dr/dn = r_,m n_m:
 *   S_kij = G/(4 pi (1-nu) r^3) { 3 dr/dn [(1-2nu) delta_ij r_,k + nu (delta_ki r_,j
 *           + delta_kj r_,i) - 5 r_,i r_,j r_,k] + 3 nu (n_i r_,j r_,k + n_j r_,i r_,k)
 *           + (1-2nu)(3 n_k r_,i r_,j + n_j delta_ki + n_i delta_kj)
 *           - (1-4nu) n_k delta_ij }                                               */
void ko_kernel_S(const double *d, const double *n, double G, double nu, double *S)
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 == 0.0) {
        memset(S, 0, 18 * sizeof(double));
        return;
    }
    double r = sqrt(r2);
    double g[3] = {-d[0] / r, -d[1] / r, -d[2] / r};
    double drdn = g[0] * n[0] + g[1] * n[1] + g[2] * n[2];
    double c = G / (4.0 * KO_PI * (1.0 - nu) * r2 * r);
    for (int k = 0; k < 3; ++k)
        for (int s = 0; s < 6; ++s) {
            int i = KO_VI[s], j = KO_VJ[s];
            double dij = (i == j) ? 1.0 : 0.0, dki = (k == i) ? 1.0 : 0.0, dkj = (k == j) ? 1.0 : 0.0;
            double v = 3.0 * drdn *
                           ((1.0 - 2.0 * nu) * dij * g[k] + nu * (dki * g[j] + dkj * g[i]) -
                            5.0 * g[i] * g[j] * g[k]) +
                       3.0 * nu * (n[i] * g[j] * g[k] + n[j] * g[i] * g[k]) +
                       (1.0 - 2.0 * nu) * (3.0 * n[k] * g[i] * g[j] + n[j] * dki + n[i] * dkj) -
                       (1.0 - 4.0 * nu) * n[k] * dij;
            S[6 * k + s] = c * v;
        }
}

/* ------------------------------------------------------------------------------ */
/* Direct sums (Eq. fmm_summation written out: all pairs, r = 0 skipped)            */
/* ------------------------------------------------------------------------------ */

/* out[3 i + a] = sum_j U(x_i - y_j) sl_j + T(x_i - y_j, n_j) dl_j.  sl, dl may be NULL. */
void ko_direct_disp(const double *trg, int64_t ntrg, const double *src, const double *nrm,
                    const double *sl, const double *dl, int64_t nsrc, double G, double nu,
                    double *out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < ntrg; ++i) {
        double acc[3] = {0.0, 0.0, 0.0};
        double K[9];
        for (int64_t j = 0; j < nsrc; ++j) {
            double d[3] = {trg[3 * i] - src[3 * j], trg[3 * i + 1] - src[3 * j + 1],
                           trg[3 * i + 2] - src[3 * j + 2]};
            if (sl) {
                ko_kernel_U(d, G, nu, K);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) acc[a] += K[3 * a + b] * sl[3 * j + b];
            }
            if (dl) {
                ko_kernel_T(d, nrm + 3 * j, nu, K);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) acc[a] += K[3 * a + b] * dl[3 * j + b];
            }
        }
        out[3 * i] = acc[0];
        out[3 * i + 1] = acc[1];
        out[3 * i + 2] = acc[2];
    }
}

/* out[6 i + s] = sum_j D(x_i - y_j)_k,s sl_jk + S(x_i - y_j, n_j)_k,s dl_jk. */
void ko_direct_stress(const double *trg, int64_t ntrg, const double *src, const double *nrm,
                      const double *sl, const double *dl, int64_t nsrc, double G, double nu,
                      double *out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < ntrg; ++i) {
        double acc[6] = {0, 0, 0, 0, 0, 0};
        double K[18];
        for (int64_t j = 0; j < nsrc; ++j) {
            double d[3] = {trg[3 * i] - src[3 * j], trg[3 * i + 1] - src[3 * j + 1],
                           trg[3 * i + 2] - src[3 * j + 2]};
            if (sl) {
                ko_kernel_D(d, nu, K);
                for (int k = 0; k < 3; ++k)
                    for (int s = 0; s < 6; ++s) acc[s] += K[6 * k + s] * sl[3 * j + k];
            }
            if (dl) {
                ko_kernel_S(d, nrm + 3 * j, G, nu, K);
                for (int k = 0; k < 3; ++k)
                    for (int s = 0; s < 6; ++s) acc[s] += K[6 * k + s] * dl[3 * j + k];
            }
        }
        for (int s = 0; s < 6; ++s) out[6 * i + s] = acc[s];
    }
}

/* ------------------------------------------------------------------------------ */
/* Triangle geometry and the 16-point rule of the two-pass matvec                  */
/* ------------------------------------------------------------------------------ */

static void tri_geom(const double *p0, const double *p1, const double *p2, double *nrm,
                     double *area, double *cen)
{
    double e1[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
    double e2[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
    double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                   e1[0] * e2[1] - e1[1] * e2[0]};
    double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    *area = 0.5 * len;
    for (int a = 0; a < 3; ++a) {
        nrm[a] = (len > 0.0) ? c[a] / len : 0.0;
        cen[a] = (p0[a] + p1[a] + p2[a]) / 3.0;
    }
}

/* Per-triangle normal (right-hand rule on the vertex order), area and centroid. */
void ko_tri_geometry(const double *verts, const int32_t *tris, int64_t nt, double *nrm,
                     double *area, double *cen)
{
    for (int64_t k = 0; k < nt; ++k)
        tri_geom(verts + 3 * tris[3 * k], verts + 3 * tris[3 * k + 1], verts + 3 * tris[3 * k + 2],
                 nrm + 3 * k, area + k, cen + 3 * k);
}

/* The 16-point rule (Sec. "Matrix-vector products"): split the triangle into four by
 * its edge midpoints and use on each part the 4-node degree-3 Gauss rule: the centroid
 * with weight -27/48 and the points with barycentric coordinates (3/5, 1/5, 1/5) and
 * permutations with weight 25/48 each.  Weights w are multiplied by the part's area,
 * so that they sum to the triangle's area.  Points q[16 k + m], weights w[16 k + m]. */
void ko_tri_quadrature(const double *verts, const int32_t *tris, int64_t nt, double *q, double *w)
{
    static const double bary[4][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                                      {0.6, 0.2, 0.2},
                                      {0.2, 0.6, 0.2},
                                      {0.2, 0.2, 0.6}};
    static const double wt[4] = {-27.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0};
    for (int64_t k = 0; k < nt; ++k) {
        const double *A = verts + 3 * tris[3 * k];
        const double *B = verts + 3 * tris[3 * k + 1];
        const double *C = verts + 3 * tris[3 * k + 2];
        double mAB[3], mBC[3], mCA[3];
        for (int a = 0; a < 3; ++a) {
            mAB[a] = 0.5 * (A[a] + B[a]);
            mBC[a] = 0.5 * (B[a] + C[a]);
            mCA[a] = 0.5 * (C[a] + A[a]);
        }
        const double *sub[4][3] = {{A, mAB, mCA}, {mAB, B, mBC}, {mCA, mBC, C}, {mBC, mCA, mAB}};
        double nrm[3], area, cen[3];
        tri_geom(A, B, C, nrm, &area, cen);
        int m = 0;
        for (int s = 0; s < 4; ++s)
            for (int g = 0; g < 4; ++g, ++m) {
                for (int a = 0; a < 3; ++a)
                    q[3 * (16 * k + m) + a] = bary[g][0] * sub[s][0][a] + bary[g][1] * sub[s][1][a] +
                                              bary[g][2] * sub[s][2][a];
                w[16 * k + m] = wt[g] * 0.25 * area;
            }
    }
}

/* ------------------------------------------------------------------------------ */
/* Singular self-integrals at the centroid of a flat triangle                      */
/* ------------------------------------------------------------------------------ */

/* Polar coordinates around the centroid xi: x = xi + rho e(theta).  The triangle is the
 * union of the three sectors (xi, v_a, v_b); in a sector let u be the unit direction of
 * the foot of the perpendicular from xi onto the edge line (distance h), w the unit
 * edge direction from v_a to v_b, and phi the angle from u, so that e = cos(phi) u +
 * sin(phi) w and the edge is at R(phi) = h / cos(phi), phi in [phi_a, phi_b].
 *   int_tri U dA    = 1/(16 pi (1-nu) G) int [(3-4nu) I + e e^T] R dphi   (radial part
 *                     exact: U(rho e) rho = U(e));
 *   PV int_tri P dA = (1-2nu)/(8 pi (1-nu)) [E_i n_j - E_j n_i], E = int e ln R dphi
 *                     (in the plane dr/dn = 0; the 1/rho^2 radial part gives ln R - ln eps
 *                     and int e dtheta over the full circle vanishes).
 * The phi-integrals are elementary (F = asinh(tan phi) = ln(sec phi + tan phi)):
 *   int R          = h F
 *   int cos^2 R    = h sin,      int cos sin R = -h cos,    int sin^2 R = h (F - sin)
 *   int cos ln R   = ln h sin - (sin ln cos + F - sin)
 *   int sin ln R   = -ln h cos - (cos - cos ln cos)                                    */
static double ko_F(double p) { return asinh(tan(p)); }

void ko_self_integrals(const double *A, const double *B, const double *C, double G, double nu,
                       double *Uself, double *Tself)
{
    double nrm[3], area, xi[3];
    tri_geom(A, B, C, nrm, &area, xi);
    const double *V[3] = {A, B, C};
    double Iee[9] = {0}, Ie0 = 0.0, E[3] = {0, 0, 0};
    for (int e = 0; e < 3; ++e) {
        const double *va = V[e], *vb = V[(e + 1) % 3];
        double a[3], d[3];
        for (int c = 0; c < 3; ++c) {
            a[c] = va[c] - xi[c];
            d[c] = vb[c] - va[c];
        }
        double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double w[3] = {d[0] / L, d[1] / L, d[2] / L};
        double aw = a[0] * w[0] + a[1] * w[1] + a[2] * w[2];
        double foot[3] = {a[0] - aw * w[0], a[1] - aw * w[1], a[2] - aw * w[2]};
        double h = sqrt(foot[0] * foot[0] + foot[1] * foot[1] + foot[2] * foot[2]);
        double u[3] = {foot[0] / h, foot[1] / h, foot[2] / h};
        double pa = atan2(aw, h), pb = atan2(aw + L, h);
        double sa = sin(pa), sb = sin(pb), ca = cos(pa), cb = cos(pb);
        double dF = ko_F(pb) - ko_F(pa);
        double i_r = h * dF, i_cc = h * (sb - sa), i_cs = -h * (cb - ca), i_ss = h * (dF - (sb - sa));
        double lh = log(h);
        double i_clr = lh * (sb - sa) - ((sb * log(cb) + ko_F(pb) - sb) - (sa * log(ca) + ko_F(pa) - sa));
        double i_slr = -lh * (cb - ca) - ((cb - cb * log(cb)) - (ca - ca * log(ca)));
        Ie0 += i_r;
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j)
                Iee[3 * i + j] += i_cc * u[i] * u[j] + i_cs * (u[i] * w[j] + w[i] * u[j]) + i_ss * w[i] * w[j];
            E[i] += i_clr * u[i] + i_slr * w[i];
        }
    }
    double cu = 1.0 / (16.0 * KO_PI * (1.0 - nu) * G);
    double ct = (1.0 - 2.0 * nu) / (8.0 * KO_PI * (1.0 - nu));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Uself[3 * i + j] = cu * ((i == j ? (3.0 - 4.0 * nu) * Ie0 : 0.0) + Iee[3 * i + j]);
            Tself[3 * i + j] = ct * (E[i] * nrm[j] - E[j] * nrm[i]);
        }
}

/* ------------------------------------------------------------------------------ */
/* Dense collocation BEM: Eq. num, Eq. coef, Eq. num2                              */
/* ------------------------------------------------------------------------------ */

/* H = 1/2 I + P^Delta and Gm = U^Delta (Eq. num, Eq. coef), row 3l+m = collocation
 * point l (centroid of triangle l), component m; column 3k+n = element k, component n.
 * Off-diagonal blocks by the 16-point rule; diagonal blocks analytic.  Row-major
 * (3 nt) x (3 nt). */
/* int_T U and int_T T(., n) over the triangle (A, B, C) at the point x, by the 4-node degree-3
 * rule on each of the 4^levels sub-triangles of `levels` rounds of midpoint subdivision
 * (levels = 1 is the 16-point rule of Sec. "Matrix-vector products"; larger values are the
 * upsampled quadrature of triangles near the collocation point).  Adds into bu, bt. */
static void tri_block_rec(const double *A, const double *B, const double *C, const double *n, const double *x,
                          int levels, double G, double nu, double *bu, double *bt)
{
    if (levels == 0) {
        static const double bary[4][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {0.6, 0.2, 0.2}, {0.2, 0.6, 0.2}, {0.2, 0.2, 0.6}};
        static const double wt[4] = {-27.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0};
        double nn[3], area, cen[3], Ku[9], Kt[9];
        tri_geom(A, B, C, nn, &area, cen);
        for (int g = 0; g < 4; ++g) {
            double d[3];
            for (int a = 0; a < 3; ++a)
                d[a] = x[a] - (bary[g][0] * A[a] + bary[g][1] * B[a] + bary[g][2] * C[a]);
            ko_kernel_U(d, G, nu, Ku);
            ko_kernel_T(d, n, nu, Kt);
            for (int a = 0; a < 9; ++a) {
                bu[a] += Ku[a] * wt[g] * area;
                bt[a] += Kt[a] * wt[g] * area;
            }
        }
        return;
    }
    double mAB[3], mBC[3], mCA[3];
    for (int a = 0; a < 3; ++a) {
        mAB[a] = 0.5 * (A[a] + B[a]);
        mBC[a] = 0.5 * (B[a] + C[a]);
        mCA[a] = 0.5 * (C[a] + A[a]);
    }
    tri_block_rec(A, mAB, mCA, n, x, levels - 1, G, nu, bu, bt);
    tri_block_rec(mAB, B, mBC, n, x, levels - 1, G, nu, bu, bt);
    tri_block_rec(mCA, mBC, C, n, x, levels - 1, G, nu, bu, bt);
    tri_block_rec(mBC, mCA, mAB, n, x, levels - 1, G, nu, bu, bt);
}

void ko_tri_block(const double *A, const double *B, const double *C, const double *x, int levels, double G,
                  double nu, double *bu, double *bt)
{
    double n[3], area, cen[3];
    tri_geom(A, B, C, n, &area, cen);
    for (int a = 0; a < 9; ++a) bu[a] = bt[a] = 0.0;
    tri_block_rec(A, B, C, n, x, levels, G, nu, bu, bt);
}

static int share_vertex(const int32_t *ta, const int32_t *tb)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (ta[i] == tb[j]) return 1;
    return 0;
}

void ko_bem_assemble(const double *verts, const int32_t *tris, int64_t nt, double G, double nu,
                     double *H, double *Gm);

/* ko_bem_assemble with the blocks of triangles that share a vertex with the collocation
 * triangle integrated on 4^near_levels sub-triangles (near_levels >= 1; 1 gives
 * ko_bem_assemble's operator). */
void ko_bem_assemble_near(const double *verts, const int32_t *tris, int64_t nt, double G, double nu,
                          int near_levels, double *H, double *Gm)
{
    ko_bem_assemble(verts, tris, nt, G, nu, H, Gm);
    if (near_levels <= 1) return;
    int64_t n3 = 3 * nt;
    double *cen = (double *)malloc(sizeof(double) * 3 * nt);
    double *nrm = (double *)malloc(sizeof(double) * 3 * nt);
    double *area = (double *)malloc(sizeof(double) * nt);
    ko_tri_geometry(verts, tris, nt, nrm, area, cen);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t l = 0; l < nt; ++l) {
        for (int64_t k = 0; k < nt; ++k) {
            if (k == l || !share_vertex(tris + 3 * l, tris + 3 * k)) continue;
            double bu[9], bt[9];
            ko_tri_block(verts + 3 * tris[3 * k], verts + 3 * tris[3 * k + 1], verts + 3 * tris[3 * k + 2],
                         cen + 3 * l, near_levels, G, nu, bu, bt);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    H[(3 * l + a) * n3 + 3 * k + b] = bt[3 * a + b];
                    Gm[(3 * l + a) * n3 + 3 * k + b] = bu[3 * a + b];
                }
        }
    }
    free(cen);
    free(nrm);
    free(area);
}

void ko_bem_assemble(const double *verts, const int32_t *tris, int64_t nt, double G, double nu,
                     double *H, double *Gm)
{
    int64_t n3 = 3 * nt;
    double *q = (double *)malloc(sizeof(double) * 48 * nt);
    double *w = (double *)malloc(sizeof(double) * 16 * nt);
    double *nrm = (double *)malloc(sizeof(double) * 3 * nt);
    double *area = (double *)malloc(sizeof(double) * nt);
    double *cen = (double *)malloc(sizeof(double) * 3 * nt);
    ko_tri_quadrature(verts, tris, nt, q, w);
    ko_tri_geometry(verts, tris, nt, nrm, area, cen);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t l = 0; l < nt; ++l) {
        double Ku[9], Kt[9];
        for (int64_t k = 0; k < nt; ++k) {
            double bu[9] = {0}, bt[9] = {0};
            if (k == l) {
                ko_self_integrals(verts + 3 * tris[3 * k], verts + 3 * tris[3 * k + 1],
                                  verts + 3 * tris[3 * k + 2], G, nu, bu, bt);
            } else {
                for (int m = 0; m < 16; ++m) {
                    const double *y = q + 3 * (16 * k + m);
                    double d[3] = {cen[3 * l] - y[0], cen[3 * l + 1] - y[1], cen[3 * l + 2] - y[2]};
                    ko_kernel_U(d, G, nu, Ku);
                    ko_kernel_T(d, nrm + 3 * k, nu, Kt);
                    for (int a = 0; a < 9; ++a) {
                        bu[a] += Ku[a] * w[16 * k + m];
                        bt[a] += Kt[a] * w[16 * k + m];
                    }
                }
            }
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    H[(3 * l + a) * n3 + 3 * k + b] = bt[3 * a + b] + (k == l && a == b ? 0.5 : 0.0);
                    Gm[(3 * l + a) * n3 + 3 * k + b] = bu[3 * a + b];
                }
        }
    }
    free(q);
    free(w);
    free(nrm);
    free(area);
    free(cen);
}

/* Column rearrangement of Eq. num2.  For each (element k, component n):
 *   known_is_disp[3k+n] = 1: u known (= val), t unknown -> A column = -Gm column
 *   known_is_disp[3k+n] = 0: t known (= val), u unknown -> A column =  H column
 * and b = sum_known (Gm col * t_known) - (H col * u_known).  Row-major A. */
void ko_bem_system(const double *H, const double *Gm, int64_t n3, const uint8_t *known_is_disp,
                   const double *val, double *A, double *b)
{
#pragma omp parallel for
    for (int64_t r = 0; r < n3; ++r) {
        double acc = 0.0;
        for (int64_t c = 0; c < n3; ++c) {
            if (known_is_disp[c]) {
                A[r * n3 + c] = -Gm[r * n3 + c];
                acc -= H[r * n3 + c] * val[c];
            } else {
                A[r * n3 + c] = H[r * n3 + c];
                acc += Gm[r * n3 + c] * val[c];
            }
        }
        b[r] = acc;
    }
}

/* ------------------------------------------------------------------------------ */
/* Restarted GMRES (Saad & Schultz), dense matvec, FP64                             */
/* ------------------------------------------------------------------------------ */

static void dense_mv(const double *A, int64_t n, const double *x, double *y)
{
#pragma omp parallel for
    for (int64_t r = 0; r < n; ++r) {
        double s = 0.0;
        for (int64_t c = 0; c < n; ++c) s += A[r * n + c] * x[c];
        y[r] = s;
    }
}

static double vnorm(const double *x, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += x[i] * x[i];
    return sqrt(s);
}

/* GMRES(m) from x (x holds the initial guess on entry), stopping when
 * ||b - A x|| / ||b|| <= tol.  Arnoldi by classical Gram-Schmidt applied twice,
 * least-squares problem by Givens rotations.  Returns 0 on convergence, 1 otherwise;
 * *iters = total inner iterations, *relres = final true relative residual. */
int ko_gmres(const double *A, int64_t n, const double *b, double *x, double tol, int restart,
             int maxit, int *iters, double *relres)
{
    int m = restart;
    double *V = (double *)calloc((size_t)(m + 1) * n, sizeof(double));
    double *Hh = (double *)calloc((size_t)(m + 1) * m, sizeof(double));
    double *cs = (double *)calloc(m, sizeof(double)), *sn = (double *)calloc(m, sizeof(double));
    double *g = (double *)calloc(m + 1, sizeof(double)), *y = (double *)calloc(m, sizeof(double));
    double *r = (double *)malloc(sizeof(double) * n), *h = (double *)malloc(sizeof(double) * (m + 1));
    double bn = vnorm(b, n);
    if (bn == 0.0) bn = 1.0;
    int it = 0, conv = 0;
    double rel = 0.0;
    while (it < maxit) {
        dense_mv(A, n, x, r);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        double beta = vnorm(r, n);
        rel = beta / bn;
        if (rel <= tol) {
            conv = 1;
            break;
        }
        for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
        memset(g, 0, sizeof(double) * (m + 1));
        g[0] = beta;
        int j;
        for (j = 0; j < m && it < maxit; ++j, ++it) {
            double *w = V + (size_t)(j + 1) * n;
            dense_mv(A, n, V + (size_t)j * n, w);
            memset(h, 0, sizeof(double) * (m + 1));
            for (int pass = 0; pass < 2; ++pass) {
                double hc[256];
                for (int i = 0; i <= j; ++i) {
                    double s = 0.0;
                    for (int64_t t = 0; t < n; ++t) s += V[(size_t)i * n + t] * w[t];
                    hc[i] = s;
                }
                for (int i = 0; i <= j; ++i) {
                    for (int64_t t = 0; t < n; ++t) w[t] -= hc[i] * V[(size_t)i * n + t];
                    h[i] += hc[i];
                }
            }
            h[j + 1] = vnorm(w, n);
            if (h[j + 1] > 0.0)
                for (int64_t t = 0; t < n; ++t) w[t] /= h[j + 1];
            for (int i = 0; i < j; ++i) {
                double t0 = cs[i] * h[i] + sn[i] * h[i + 1];
                h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
                h[i] = t0;
            }
            double den = sqrt(h[j] * h[j] + h[j + 1] * h[j + 1]);
            cs[j] = (den > 0.0) ? h[j] / den : 1.0;
            sn[j] = (den > 0.0) ? h[j + 1] / den : 0.0;
            h[j] = den;
            h[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int i = 0; i <= j; ++i) Hh[i * m + j] = h[i];
            if (fabs(g[j + 1]) / bn <= tol) {
                ++j;
                ++it;
                break;
            }
        }
        /* back substitution and update */
        for (int i = j - 1; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k < j; ++k) s -= Hh[i * m + k] * y[k];
            y[i] = s / Hh[i * m + i];
        }
        for (int i = 0; i < j; ++i)
            for (int64_t t = 0; t < n; ++t) x[t] += y[i] * V[(size_t)i * n + t];
    }
    if (!conv) {
        dense_mv(A, n, x, r);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        rel = vnorm(r, n) / bn;
        conv = rel <= tol;
    }
    *iters = it;
    *relres = rel;
    free(V);
    free(Hh);
    free(cs);
    free(sn);
    free(g);
    free(y);
    free(r);
    free(h);
    return conv ? 0 : 1;
}

/* ------------------------------------------------------------------------------ */
/* Interior fields: Eq. stress_1, Eq. deriv, Eq. functional                        */
/* ------------------------------------------------------------------------------ */

/* Interior displacement (the BIE at an interior point, free term 1) and stress
 * (Eq. stress_1, Somigliana) from the piecewise-constant boundary solution, using
 * the same 16-point rule: sl = t_k w, dl = -u_k w.  disp [np,3] and/or sig [np,6]. */
void ko_bem_interior(const double *pts, int64_t np, const double *verts, const int32_t *tris,
                     int64_t nt, const double *u, const double *t, double G, double nu,
                     double *disp, double *sig)
{
    double *q = (double *)malloc(sizeof(double) * 48 * nt);
    double *w = (double *)malloc(sizeof(double) * 16 * nt);
    double *nrm = (double *)malloc(sizeof(double) * 3 * nt);
    double *area = (double *)malloc(sizeof(double) * nt);
    double *cen = (double *)malloc(sizeof(double) * 3 * nt);
    double *qn = (double *)malloc(sizeof(double) * 48 * nt);
    double *sl = (double *)malloc(sizeof(double) * 48 * nt);
    double *dl = (double *)malloc(sizeof(double) * 48 * nt);
    ko_tri_quadrature(verts, tris, nt, q, w);
    ko_tri_geometry(verts, tris, nt, nrm, area, cen);
    for (int64_t k = 0; k < nt; ++k)
        for (int m = 0; m < 16; ++m)
            for (int a = 0; a < 3; ++a) {
                int64_t j = 16 * k + m;
                qn[3 * j + a] = nrm[3 * k + a];
                sl[3 * j + a] = t[3 * k + a] * w[j];
                dl[3 * j + a] = -u[3 * k + a] * w[j];
            }
    if (disp) ko_direct_disp(pts, np, q, qn, sl, dl, 16 * nt, G, nu, disp);
    if (sig) ko_direct_stress(pts, np, q, qn, sl, dl, 16 * nt, G, nu, sig);
    free(q);
    free(w);
    free(nrm);
    free(area);
    free(cen);
    free(qn);
    free(sl);
    free(dl);
}

/* Eq. deriv: D^T = 3/(4E) (1-nu)/(7-5nu) [10 (1+nu) sigma:sigma - (1+5nu) (tr sigma)^2],
 * "tr sigma_ij(p)^2" read as the square of the trace.  sigma:sigma counts each
 * off-diagonal component twice.  Energy density (Eq. functional integrand)
 * w = 1/2 sigma:eps with eps = ((1+nu) sigma - nu tr(sigma) I) / E. */
void ko_topo_derivative(const double *sig, int64_t n, double G, double nu, double *td,
                        double *energy)
{
    double E = 2.0 * G * (1.0 + nu);
    for (int64_t i = 0; i < n; ++i) {
        const double *s = sig + 6 * i;
        double tr = s[0] + s[1] + s[2];
        double ss = s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + 2.0 * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]);
        if (td)
            td[i] = 3.0 / (4.0 * E) * (1.0 - nu) / (7.0 - 5.0 * nu) *
                    (10.0 * (1.0 + nu) * ss - (1.0 + 5.0 * nu) * tr * tr);
        if (energy) energy[i] = 0.5 * ((1.0 + nu) * ss - nu * tr * tr) / E;
    }
}

/* ------------------------------------------------------------------------------ */
/* Periodic sums (Sec. "Periodic cell of a metamaterial": the integrals over the   */
/* infinite periodic surface of a cell repeated in all three directions)           */
/* ------------------------------------------------------------------------------ */
/* The cell is a cube of side Lc repeated on the lattice Lc Z^3, V = Lc^3.  The periodic
 * single layer is defined by its Fourier series
 *     U_per(d) = (1/V) sum_{k != 0} Uhat(k) e^{i k.d},   k = (2 pi / Lc) m,  m in Z^3,
 *     Uhat_ij(k) = [delta_ij - c2 k_i k_j / k^2] / (G k^2),   c2 = 1 / (2 (1 - nu)),
 * the Fourier transform of Eq. disp_1.  Leaving out k = 0 makes the cell mean of every
 * field zero and, for sources with a net force F, adds the uniform body force -F/V that
 * balances it (without it the lattice sum has no limit).  The double layer is the traction
 * kernel of that field: with v^(i)(y) = U_per(y - x) e_i, the field at y of a unit force at
 * x, T_per,ij = sigma_jk[v^(i)](y) n_k(y), which at d = x - y reads
 *     T_per,ij = -[lambda n_j dU_mi/dd_m + G n_k (dU_ki/dd_j + dU_ji/dd_k)]
 * (the free-space kernel of Eq. disp_2 is the same expression of U; a test checks it).
 *
 * Evaluation by Ewald's split with screening parameter xi.  With
 *     U_ij = [delta_ij phi(r) + c2 d_i d_j psi(r)] / G,  phi = 1/(4 pi r) <-> 1/k^2,
 *     psi = -r/(8 pi) <-> 1/k^4,
 * the short-range parts are
 *     phi_R = erfc(xi r) / (4 pi r),
 *     psi_R = -[r erfc(xi r) - exp(-xi^2 r^2) / (xi sqrt(pi))] / (8 pi),
 * the long-range parts have the transforms g/k^2 and (1 + a) g/k^4, a = k^2/(4 xi^2),
 * g = exp(-a), and by Poisson's summation formula
 *     U_per(d) = sum_n U_R(d - n Lc) + (1/V) sum_{k != 0} Uhat_K(k) e^{i k.d} - delta_ij / (4 xi^2 G V),
 * the last term the transform of U_R at k = 0 (its integral), which the series leaves out.
 * A pair at distance 0 (a target on a source, image n = 0) contributes the regular part
 * lim_{d->0} [U_per(d) - U(d)], the periodic analogue of skipping r = 0. */

#define KO_SQRTPI 1.77245385090551602730

/* short-range kernel U_R and its gradient dU[(3i+j)*3+m] = dU_R,ij/dd_m at e != 0; at e = 0 the
 * regular part U_R - U = -U_smooth(0) (and a zero gradient) */
static void ewald_real(const double *e, double G, double nu, double xi, double *U, double *dU)
{
    const double c2 = 1.0 / (2.0 * (1.0 - nu));
    const double r2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    if (r2 == 0.0) {
        /* U_smooth(0): erf(xi r)/(4 pi r) -> xi/(2 pi^1.5); Hessian of (psi - psi_R) -> -xi/(4 pi^1.5) I */
        const double s = xi / (KO_PI * KO_SQRTPI) * (0.5 - 0.25 * c2) / G;
        for (int a = 0; a < 9; ++a) U[a] = (a % 4 == 0) ? -s : 0.0;
        if (dU) memset(dU, 0, 27 * sizeof(double));
        return;
    }
    const double r = sqrt(r2), rh[3] = {e[0] / r, e[1] / r, e[2] / r};
    const double ec = erfc(xi * r), ex = exp(-xi * xi * r2);
    const double phi = ec / (4.0 * KO_PI * r);
    const double dphi = -(ec / r + 2.0 * xi / KO_SQRTPI * ex) / (4.0 * KO_PI * r);
    const double p1 = -ec / (8.0 * KO_PI);                                /* psi_R'   */
    const double p2 = xi * ex / (4.0 * KO_PI * KO_SQRTPI);                /* psi_R''  */
    const double p3 = -xi * xi * xi * r * ex / (2.0 * KO_PI * KO_SQRTPI); /* psi_R''' */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const double dij = i == j ? 1.0 : 0.0;
            const double H = (p2 - p1 / r) * rh[i] * rh[j] + (p1 / r) * dij;
            U[3 * i + j] = (dij * phi + c2 * H) / G;
            if (!dU) continue;
            for (int m = 0; m < 3; ++m) {
                const double dim = i == m ? 1.0 : 0.0, djm = j == m ? 1.0 : 0.0;
                const double H3 = (p3 - 3.0 * p2 / r + 3.0 * p1 / r2) * rh[i] * rh[j] * rh[m] +
                                  (p2 / r - p1 / r2) * (dij * rh[m] + dim * rh[j] + djm * rh[i]);
                dU[(3 * i + j) * 3 + m] = (dij * dphi * rh[m] + c2 * H3) / G;
            }
        }
}

/* screened transform Uhat_K(k) (without the 1/V) */
static void ewald_recip(const double *k, double G, double nu, double xi, double *Uk)
{
    const double c2 = 1.0 / (2.0 * (1.0 - nu));
    const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    const double a = k2 / (4.0 * xi * xi), g = exp(-a);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Uk[3 * i + j] = ((i == j ? g / k2 : 0.0) - c2 * k[i] * k[j] * (1.0 + a) * g / (k2 * k2)) / G;
}

/* cut-offs: erfc(xi rc) and exp(-kc^2 / (4 xi^2)) below 1e-16 */
static double ewald_xi(double Lc, double xi) { return xi > 0.0 ? xi : 4.5 / Lc; }
static double ewald_rc(double xi) { return 6.2 / xi; }
static double ewald_kc(double xi) { return 12.4 * xi; }

/* d reduced to the image nearest the origin (the sum over the lattice does not change) */
static void min_image(double *d, double Lc)
{
    for (int c = 0; c < 3; ++c) d[c] -= Lc * floor(d[c] / Lc + 0.5);
}

/* U_per(d) and its gradient dU[(3i+j)*3+m] (the regular part at d = 0 mod Lc) */
void ko_periodic_U(const double *d_in, double G, double nu, double Lc, double xi, double *U, double *dU)
{
    xi = ewald_xi(Lc, xi);
    const double V = Lc * Lc * Lc, rc = ewald_rc(xi), kc = ewald_kc(xi);
    double d[3] = {d_in[0], d_in[1], d_in[2]};
    min_image(d, Lc);
    memset(U, 0, 9 * sizeof(double));
    memset(dU, 0, 27 * sizeof(double));
    const int nr = (int)ceil(rc / Lc + 0.5), nk = (int)ceil(kc * Lc / (2.0 * KO_PI));
    double Ut[9], dUt[27];
    for (int a = -nr; a <= nr; ++a)
        for (int b = -nr; b <= nr; ++b)
            for (int c = -nr; c <= nr; ++c) {
                const double e[3] = {d[0] - a * Lc, d[1] - b * Lc, d[2] - c * Lc};
                if (e[0] * e[0] + e[1] * e[1] + e[2] * e[2] >= rc * rc) continue;
                ewald_real(e, G, nu, xi, Ut, dUt);
                for (int q = 0; q < 9; ++q) U[q] += Ut[q];
                for (int q = 0; q < 27; ++q) dU[q] += dUt[q];
            }
    for (int a = -nk; a <= nk; ++a)
        for (int b = -nk; b <= nk; ++b)
            for (int c = -nk; c <= nk; ++c) {
                if (a == 0 && b == 0 && c == 0) continue;
                const double k[3] = {2.0 * KO_PI * a / Lc, 2.0 * KO_PI * b / Lc, 2.0 * KO_PI * c / Lc};
                if (k[0] * k[0] + k[1] * k[1] + k[2] * k[2] > kc * kc) continue;
                ewald_recip(k, G, nu, xi, Ut);
                const double th = k[0] * d[0] + k[1] * d[1] + k[2] * d[2], cs = cos(th), sn = sin(th);
                for (int q = 0; q < 9; ++q) {
                    U[q] += Ut[q] * cs / V;
                    for (int m = 0; m < 3; ++m) dU[q * 3 + m] -= k[m] * Ut[q] * sn / V;
                }
            }
    const double c0 = 1.0 / (4.0 * xi * xi * G * V);
    U[0] -= c0;
    U[4] -= c0;
    U[8] -= c0;
}

/* out[3 i + a] = sum_j U_per(x_i - y_j) sl_j + T_per(x_i - y_j, n_j) dl_j; sl, dl may be NULL.
 * The real-space part is summed pair by pair over the images within the cut-off; the
 * reciprocal part in its structure-factor form,
 *   (1/V) sum_k sum_j Re[(Uhat_K sl_j - i w_j) e^{i k.(x - y_j)}]
 *     = (1/V) sum_k [cos(k.x) (C1 - S2) + sin(k.x) (S1 + C2)],
 * with w_j = lambda (n.dl) Uhat_K k + G [(k.dl) Uhat_K n + (k.n) Uhat_K dl] the transform of
 * T_per dl_j and C1, S1 (C2, S2) the sums of Uhat_K sl_j (w_j) times cos, sin(k.y_j). */
void ko_periodic_disp(const double *trg, int64_t ntrg, const double *src, const double *nrm,
                      const double *sl, const double *dl, int64_t nsrc, double G, double nu, double Lc,
                      double xi, double *out)
{
    xi = ewald_xi(Lc, xi);
    const double V = Lc * Lc * Lc, rc = ewald_rc(xi), kc = ewald_kc(xi);
    const double lam = 2.0 * G * nu / (1.0 - 2.0 * nu);
    const int nr = (int)ceil(rc / Lc + 0.5), nk = (int)ceil(kc * Lc / (2.0 * KO_PI));
    /* real space */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < ntrg; ++i) {
        double acc[3] = {0.0, 0.0, 0.0}, Ut[9], dUt[27];
        for (int64_t j = 0; j < nsrc; ++j) {
            double d[3] = {trg[3 * i] - src[3 * j], trg[3 * i + 1] - src[3 * j + 1], trg[3 * i + 2] - src[3 * j + 2]};
            min_image(d, Lc);
            for (int a = -nr; a <= nr; ++a)
                for (int b = -nr; b <= nr; ++b)
                    for (int c = -nr; c <= nr; ++c) {
                        const double e[3] = {d[0] - a * Lc, d[1] - b * Lc, d[2] - c * Lc};
                        if (e[0] * e[0] + e[1] * e[1] + e[2] * e[2] >= rc * rc) continue;
                        ewald_real(e, G, nu, xi, Ut, dl ? dUt : NULL);
                        if (sl)
                            for (int p = 0; p < 3; ++p)
                                for (int q = 0; q < 3; ++q) acc[p] += Ut[3 * p + q] * sl[3 * j + q];
                        if (dl) {
                            const double *n = nrm + 3 * j;
                            for (int p = 0; p < 3; ++p)
                                for (int q = 0; q < 3; ++q) {
                                    double div = 0.0, sym = 0.0;
                                    for (int m = 0; m < 3; ++m) {
                                        div += dUt[(3 * m + p) * 3 + m];
                                        sym += n[m] * (dUt[(3 * m + p) * 3 + q] + dUt[(3 * q + p) * 3 + m]);
                                    }
                                    acc[p] -= (lam * n[q] * div + G * sym) * dl[3 * j + q];
                                }
                        }
                    }
        }
        out[3 * i] = acc[0];
        out[3 * i + 1] = acc[1];
        out[3 * i + 2] = acc[2];
    }
    /* reciprocal space: the wave vectors within the cut-off, their structure factors
     * (C1, S1, C2, S2 per vector), then the sum over the vectors at every target */
    int nkv = 0;
    double *kv = (double *)malloc(sizeof(double) * 3 * (size_t)(2 * nk + 1) * (2 * nk + 1) * (2 * nk + 1));
    for (int a = -nk; a <= nk; ++a)
        for (int b = -nk; b <= nk; ++b)
            for (int c = -nk; c <= nk; ++c) {
                const double k[3] = {2.0 * KO_PI * a / Lc, 2.0 * KO_PI * b / Lc, 2.0 * KO_PI * c / Lc};
                const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                if ((a == 0 && b == 0 && c == 0) || k2 > kc * kc) continue;
                memcpy(kv + 3 * nkv++, k, sizeof(k));
            }
    double *sf = (double *)calloc((size_t)nkv * 12, sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
    for (int q = 0; q < nkv; ++q) {
        const double *k = kv + 3 * q;
        double Uk[9];
        ewald_recip(k, G, nu, xi, Uk);
        double *C1 = sf + 12 * (size_t)q, *S1 = C1 + 3, *C2 = C1 + 6, *S2 = C1 + 9;
        for (int64_t j = 0; j < nsrc; ++j) {
            const double th = k[0] * src[3 * j] + k[1] * src[3 * j + 1] + k[2] * src[3 * j + 2];
            const double cs = cos(th), sn = sin(th);
            for (int p = 0; p < 3; ++p) {
                if (sl) {
                    const double v = Uk[3 * p] * sl[3 * j] + Uk[3 * p + 1] * sl[3 * j + 1] + Uk[3 * p + 2] * sl[3 * j + 2];
                    C1[p] += v * cs;
                    S1[p] += v * sn;
                }
                if (dl) {
                    const double *n = nrm + 3 * j, *u = dl + 3 * j;
                    const double ndl = n[0] * u[0] + n[1] * u[1] + n[2] * u[2];
                    const double kdl = k[0] * u[0] + k[1] * u[1] + k[2] * u[2];
                    const double kn = k[0] * n[0] + k[1] * n[1] + k[2] * n[2];
                    double w = 0.0;
                    for (int r = 0; r < 3; ++r) w += Uk[3 * p + r] * (lam * ndl * k[r] + G * (kdl * n[r] + kn * u[r]));
                    C2[p] += w * cs;
                    S2[p] += w * sn;
                }
            }
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ntrg; ++i)
        for (int q = 0; q < nkv; ++q) {
            const double *k = kv + 3 * q, *C1 = sf + 12 * (size_t)q, *S1 = C1 + 3, *C2 = C1 + 6, *S2 = C1 + 9;
            const double th = k[0] * trg[3 * i] + k[1] * trg[3 * i + 1] + k[2] * trg[3 * i + 2];
            const double cs = cos(th), sn = sin(th);
            for (int p = 0; p < 3; ++p) out[3 * i + p] += (cs * (C1[p] - S2[p]) + sn * (S1[p] + C2[p])) / V;
        }
    free(sf);
    free(kv);
    /* the mean of U_R, left out with k = 0 */
    if (sl) {
        double F[3] = {0, 0, 0};
        for (int64_t j = 0; j < nsrc; ++j)
            for (int p = 0; p < 3; ++p) F[p] += sl[3 * j + p];
        const double c0 = 1.0 / (4.0 * xi * xi * G * V);
        for (int64_t i = 0; i < ntrg; ++i)
            for (int p = 0; p < 3; ++p) out[3 * i + p] -= c0 * F[p];
    }
}
