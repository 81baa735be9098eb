// periodic.cpp -- FP64 host precompute of the far-lattice operator of the periodic KIFMM
// (Sec. "Periodic cell of a metamaterial": the sums run over an infinite periodic surface, and
// the FMM tree is made periodic at every level).
//
// In a periodic tree the interaction lists wrap around the cell, so that every level sees the
// images of the cell's boxes; what no list reaches are the cell images n with |n|_inf >= 2 as
// seen from the root (the root's 26 neighbours are its near field).  Their field at the root's
// downward check surface is one fixed linear map of the root's upward equivalent density.  For
// the unit cell (root half-width 1/2, G = 1), with x_a = y_a = (r_inner / 2) s_a the points of
// both surfaces:
//     T[3a+i][3b+j] = sum_{|n|_inf >= 2} U_ij(x_a - y_b - n).
// The lattice sum is taken in the sense of the Fourier series of U without the k = 0 term (zero
// cell mean of the field; a net force balanced by a uniform body force), split by Ewald:
//     sum_{|n|>=2} U(d - n) = sum_{|n|>=2} U_R(d - n) - sum_{|n|<=1} U_L(d - n)
//                             + sum_{k != 0} Uhat_L(k) e^{i k.d} - I / (4 xi^2)
// with U = U_R + U_L, the short- and long-range parts of U_ij = delta_ij phi + c2 d_i d_j psi,
// c2 = 1 / (2 (1 - nu)), phi = 1/(4 pi r), psi = -r / (8 pi):
//     phi_L = erf(xi r) / (4 pi r),                     Uhat: g / k^2,
//     psi_L = -[r erf(xi r) + exp(-xi^2 r^2) / (xi sqrt(pi))] / (8 pi),   Uhat: (1 + a) g / k^4,
// a = k^2 / (4 xi^2), g = exp(-a), k = 2 pi m; the last term is the k = 0 limit of Uhat_R.
// T depends on d = x_a - y_b only, and d takes the (2p - 1)^3 values of the surface lattice's
// differences: the sum is made once per difference.
//
// With a net force F in the cell, the balancing body force -F/V acts inside the root too, and
// there the far field is no Navier solution: G lap u + (lambda + G) grad div u = F/V.  Equivalent
// densities hold Navier solutions only, so the particular solution P(x_a) F,
// P(x) = x x^T / (4 lambda + 6 G) (about the cell centre, V = 1), is taken out of T row by row
// (it depends on the check point alone, and sum_b phi_b = F) and added exactly at the targets
// by the evaluation.
//
// The operator on the singular-basis densities: the root (half-width h, cell side 2h) has
// phi_up = V_u alpha and beta = G h S_d^-1 U_d^T chk with chk = T phi_up / (G 2h), so
//     beta_root += R alpha_root,   R = 1/2 S_d^-1 U_d^T T V_u,
// independent of the cell size and of G.
#include <cmath>
#include <vector>

#include "precompute.h"

namespace kfmm {
namespace host {

namespace {

const double kPi = 3.14159265358979323846;
const double kSqrtPi = 1.77245385090551602730;

// 3x3 block of the long-range part U_L at e (G = 1)
void long_range(const double *e, double xi, double c2, double *out)
{
    const double r2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    if (r2 < 1e-24) {  // limits at r = 0: phi_L -> xi / (2 pi^1.5), Hess psi_L -> -xi / (4 pi^1.5) I
        const double v = xi / (kPi * kSqrtPi) * (0.5 - 0.25 * c2);
        for (int q = 0; q < 9; ++q) out[q] = (q % 4 == 0) ? v : 0.0;
        return;
    }
    const double r = std::sqrt(r2), ef = std::erf(xi * r), ex = std::exp(-xi * xi * r2);
    const double phi = ef / (4.0 * kPi * r);
    const double d1 = -ef / (8.0 * kPi);                   // psi_L'
    const double d2 = -xi * ex / (4.0 * kPi * kSqrtPi);    // psi_L''
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const double dij = i == j ? 1.0 : 0.0;
            out[3 * i + j] = dij * phi + c2 * ((d2 - d1 / r) * e[i] * e[j] / r2 + (d1 / r) * dij);
        }
}

// 3x3 block of the short-range part U_R = U - U_L at e != 0 (G = 1)
void short_range(const double *e, double xi, double c2, double *out)
{
    const double r2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    const double r = std::sqrt(r2), ec = std::erfc(xi * r), ex = std::exp(-xi * xi * r2);
    const double phi = ec / (4.0 * kPi * r);
    const double d1 = -ec / (8.0 * kPi);                  // psi_R'
    const double d2 = xi * ex / (4.0 * kPi * kSqrtPi);    // psi_R''
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const double dij = i == j ? 1.0 : 0.0;
            out[3 * i + j] = dij * phi + c2 * ((d2 - d1 / r) * e[i] * e[j] / r2 + (d1 / r) * dij);
        }
}

// sum over the images |n|_inf >= 2 of U(d - n), unit cell, G = 1
void far_lattice(const double *d, double nu, double *out)
{
    const double xi = 2.5, c2 = 1.0 / (2.0 * (1.0 - nu));
    const double rc = 6.1 / xi;            // erfc(xi rc) < 1e-17
    const double kc = 2.0 * xi * 6.1;      // exp(-kc^2 / (4 xi^2)) < 1e-16
    for (int q = 0; q < 9; ++q) out[q] = 0.0;
    double blk[9];
    const int nr = (int)std::ceil(rc + 1.1), nk = (int)std::ceil(kc / (2.0 * kPi));
    for (int a = -nr; a <= nr; ++a)
        for (int b = -nr; b <= nr; ++b)
            for (int c = -nr; c <= nr; ++c) {
                const double e[3] = {d[0] - a, d[1] - b, d[2] - c};
                const bool near = std::abs(a) <= 1 && std::abs(b) <= 1 && std::abs(c) <= 1;
                if (near) {
                    long_range(e, xi, c2, blk);
                    for (int q = 0; q < 9; ++q) out[q] -= blk[q];
                } else if (e[0] * e[0] + e[1] * e[1] + e[2] * e[2] < rc * rc) {
                    short_range(e, xi, c2, blk);
                    for (int q = 0; q < 9; ++q) out[q] += blk[q];
                }
            }
    for (int a = -nk; a <= nk; ++a)
        for (int b = -nk; b <= nk; ++b)
            for (int c = -nk; c <= nk; ++c) {
                if (a == 0 && b == 0 && c == 0) continue;
                const double k[3] = {2.0 * kPi * a, 2.0 * kPi * b, 2.0 * kPi * c};
                const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                if (k2 > kc * kc) continue;
                const double al = k2 / (4.0 * xi * xi), g = std::exp(-al);
                const double cs = std::cos(k[0] * d[0] + k[1] * d[1] + k[2] * d[2]);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        out[3 * i + j] += cs * ((i == j ? g / k2 : 0.0) - c2 * k[i] * k[j] * (1.0 + al) * g / (k2 * k2));
            }
    const double c0 = 1.0 / (4.0 * xi * xi);
    out[0] -= c0;
    out[4] -= c0;
    out[8] -= c0;
}

}  // namespace

bool compute_lattice(const OpsParams &prm, const OpsHost &H, std::vector<double> &R)
{
    const int p = prm.p, n = H.n_surf, m = 3 * n, ku = H.ku, kd = H.kd;
    if (p < 2 || n <= 0) return false;
    // the far sum at every difference of two surface points: d = (r_inner / 2) (2 / (p - 1)) q,
    // q in [-(p-1), p-1]^3
    const int w = 2 * p - 1;
    const double step = 0.5 * prm.r_inner * 2.0 / (p - 1);
    std::vector<double> tab((size_t)w * w * w * 9);
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < w * w * w; ++t) {
        const int qx = t / (w * w) - (p - 1), qy = (t / w) % w - (p - 1), qz = t % w - (p - 1);
        const double d[3] = {qx * step, qy * step, qz * step};
        far_lattice(d, prm.nu, &tab[(size_t)t * 9]);
    }
    // lattice index of each surface point (its coordinates are -1 + 2 i / (p - 1))
    std::vector<int> li(3 * (size_t)n);
    for (int a = 0; a < 3 * n; ++a) li[a] = (int)std::lround((H.surf[a] + 1.0) * (p - 1) / 2.0);
    const double lam = 2.0 * prm.nu / (1.0 - 2.0 * prm.nu);  // G = 1
    std::vector<double> T((size_t)m * m);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            const int qx = li[3 * a] - li[3 * b] + (p - 1), qy = li[3 * a + 1] - li[3 * b + 1] + (p - 1),
                      qz = li[3 * a + 2] - li[3 * b + 2] + (p - 1);
            const double *blk = &tab[((size_t)(qx * w + qy) * w + qz) * 9];
            // less P(x_a), the particular part of the balancing body force (added at the targets
            // instead): what remains is a Navier solution in the root
            const double xa[3] = {0.5 * prm.r_inner * H.surf[3 * a], 0.5 * prm.r_inner * H.surf[3 * a + 1],
                                  0.5 * prm.r_inner * H.surf[3 * a + 2]};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    T[(size_t)(3 * a + i) * m + 3 * b + j] = blk[3 * i + j] - xa[i] * xa[j] / (4.0 * lam + 6.0);
        }
    // R = 1/2 s2a_d T V_u: first TV = T V_u (m x ku), then R = 1/2 s2a_d TV (kd x ku)
    std::vector<double> TV((size_t)m * ku, 0.0);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i)
        for (int k = 0; k < m; ++k) {
            const double t = T[(size_t)i * m + k];
            const double *v = &H.vu[(size_t)k * ku];
            double *o = &TV[(size_t)i * ku];
            for (int j = 0; j < ku; ++j) o[j] += t * v[j];
        }
    R.assign((size_t)kd * ku, 0.0);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < kd; ++i)
        for (int k = 0; k < m; ++k) {
            const double s = 0.5 * H.s2a_d[(size_t)i * m + k];
            const double *v = &TV[(size_t)k * ku];
            double *o = &R[(size_t)i * ku];
            for (int j = 0; j < ku; ++j) o[j] += s * v[j];
        }
    return true;
}

}  // namespace host
}  // namespace kfmm
