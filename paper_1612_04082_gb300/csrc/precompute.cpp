// precompute.cpp -- FP64 host precompute of the kernel-independent FMM operators
// (Sec. "Kernel-independent fast multipole method": far fields are densities phi_i on
// samples x_i of an equivalent surface, sum_i phi_i K(x_i, y); the M2M, L2L and M2L
// operators are matrices computed automatically from the kernel).
//
// Surfaces are the boundary of a p x p x p lattice on [-1,1]^3 (6(p-1)^2 + 2 points),
// scaled by r_inner (upward equivalent, downward check) or r_outer (upward check, downward
// equivalent) box half-widths.  Every matrix is built for half-width 1 and G = 1; the
// Kelvin kernel U is homogeneous of degree -1 and proportional to 1/G, so the
// pseudo-inverses scale by G h and the translations (M2M, L2L, M2L) do not scale at all.
//
// The M2L matrices K_v for the 316 directions v in [-3,3]^3 \ [-1,1]^3 are compressed with
// one shared basis: the inner surfaces are the same point set, so K_{-v} = K_v^T and the
// left and right singular vectors of [K_v]_v coincide; with U_r the leading eigenvectors of
// sum_v K_v K_v^T, K_v ~ U_r C_v U_r^T, C_v = U_r^T K_v U_r.
//
// Linear algebra written here: a parallel cyclic Jacobi eigensolver and OpenMP loops for
// the products.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "precompute.h"

namespace kfmm {
namespace host {

static const double kPi = 3.14159265358979323846;

std::vector<double> lattice_surface(int p)
{
    std::vector<double> pts;
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j)
            for (int k = 0; k < p; ++k) {
                if (i == 0 || j == 0 || k == 0 || i == p - 1 || j == p - 1 || k == p - 1) {
                    pts.push_back(-1.0 + 2.0 * i / (p - 1));
                    pts.push_back(-1.0 + 2.0 * j / (p - 1));
                    pts.push_back(-1.0 + 2.0 * k / (p - 1));
                }
            }
    return pts;
}

// U_ij(d) with G = 1 (Eq. disp_1).
static inline void kelvin_U(const double *d, double nu, double *U)
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 == 0.0) {
        for (int a = 0; a < 9; ++a) U[a] = 0.0;
        return;
    }
    double r = std::sqrt(r2);
    double c = 1.0 / (16.0 * kPi * (1.0 - nu) * r);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) U[3 * i + j] = c * ((i == j ? 3.0 - 4.0 * nu : 0.0) + d[i] * d[j] / r2);
}

// K[3a+i][3b+j] = U_ij(x_a - y_b); x = ct + rt * surf, y = cs + rs * surf.
static void kernel_matrix(const std::vector<double> &surf, double nu, const double *ct, double rt,
                          const double *cs, double rs, double *K)
{
    const int n = (int)surf.size() / 3, m = 3 * n;
#pragma omp parallel for schedule(static)
    for (int a = 0; a < n; ++a) {
        double x[3], U[9];
        for (int c = 0; c < 3; ++c) x[c] = ct[c] + rt * surf[3 * a + c];
        for (int b = 0; b < n; ++b) {
            double d[3];
            for (int c = 0; c < 3; ++c) d[c] = x[c] - (cs[c] + rs * surf[3 * b + c]);
            kelvin_U(d, nu, U);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) K[(size_t)(3 * a + i) * m + 3 * b + j] = U[3 * i + j];
        }
    }
}

// C = A (m x k) * B (k x n), row-major.
static void gemm(int m, int n, int k, const double *A, const double *B, double *C)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i) {
        double *c = C + (size_t)i * n;
        for (int j = 0; j < n; ++j) c[j] = 0.0;
        for (int l = 0; l < k; ++l) {
            const double a = A[(size_t)i * k + l];
            const double *b = B + (size_t)l * n;
            for (int j = 0; j < n; ++j) c[j] += a * b[j];
        }
    }
}

// C = A^T (A: k x m) * B (k x n).
static void gemm_tn(int m, int n, int k, const double *A, const double *B, double *C)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i) {
        double *c = C + (size_t)i * n;
        for (int j = 0; j < n; ++j) c[j] = 0.0;
        for (int l = 0; l < k; ++l) {
            const double a = A[(size_t)l * m + i];
            const double *b = B + (size_t)l * n;
            for (int j = 0; j < n; ++j) c[j] += a * b[j];
        }
    }
}

// Symmetric eigendecomposition A = Z diag(w) Z^T (eigenvalues descending) by the cyclic
// Jacobi method.  Each step applies n/2 plane rotations on disjoint index pairs, chosen by a
// round-robin schedule so that every pair (p, q) is visited once per sweep; a rotation in
// the (p, q) plane with tan(phi) = t, t^2 + 2 theta t - 1 = 0, theta = (A_qq - A_pp) / (2 A_pq)
// (the smaller root) zeroes A_pq.  Disjoint rotations commute, so a step's rotations are
// computed from the same A and applied in parallel.  A pair is skipped once
// |A_pq| <= eps sqrt(|A_pp A_qq|), which gives the small eigenvalues high relative accuracy;
// the iteration stops after a sweep without rotations.  A (n x n, row-major) is overwritten
// by Z (columns are eigenvectors).
static bool sym_eig(int n, double *A, double *w)
{
    const int np = n + (n & 1);  // an odd n gets a dummy index that never rotates
    std::vector<double> Zt((size_t)n * n, 0.0);  // rows are eigenvectors
    for (int i = 0; i < n; ++i) Zt[(size_t)i * n + i] = 1.0;
    std::vector<int> ring(np);
    for (int i = 0; i < np; ++i) ring[i] = i;
    std::vector<int> pp(np / 2), qq(np / 2);
    std::vector<double> cs(np / 2), sn(np / 2);
    const double eps = 2.2e-16;
    bool converged = false;
    for (int sweep = 0; sweep < 40 && !converged; ++sweep) {
        long rotations = 0;
        for (int step = 0; step < np - 1; ++step) {
            // pairs of this step: ring[k] with ring[np-1-k]
            for (int k = 0; k < np / 2; ++k) {
                int p = ring[k], q = ring[np - 1 - k];
                if (p > q) std::swap(p, q);
                pp[k] = p;
                qq[k] = q;
                cs[k] = 1.0;
                sn[k] = 0.0;
                if (q >= n) continue;
                const double apq = A[(size_t)p * n + q];
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                if (std::fabs(apq) <= eps * std::sqrt(std::fabs(app * aqq)) || apq == 0.0) continue;
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                cs[k] = 1.0 / std::sqrt(t * t + 1.0);
                sn[k] = t * cs[k];
                ++rotations;
            }
            // A <- A J (columns p, q), then A <- J^T A (rows p, q), Zt <- J^T Zt
#pragma omp parallel for schedule(static)
            for (int k = 0; k < np / 2; ++k) {
                if (sn[k] == 0.0) continue;
                const int p = pp[k], q = qq[k];
                const double c = cs[k], s = sn[k];
                for (int i = 0; i < n; ++i) {
                    const double x = A[(size_t)i * n + p], y = A[(size_t)i * n + q];
                    A[(size_t)i * n + p] = c * x - s * y;
                    A[(size_t)i * n + q] = s * x + c * y;
                }
            }
#pragma omp parallel for schedule(static)
            for (int k = 0; k < np / 2; ++k) {
                if (sn[k] == 0.0) continue;
                const int p = pp[k], q = qq[k];
                const double c = cs[k], s = sn[k];
                double *rp = A + (size_t)p * n, *rq = A + (size_t)q * n;
                for (int j = 0; j < n; ++j) {
                    const double x = rp[j], y = rq[j];
                    rp[j] = c * x - s * y;
                    rq[j] = s * x + c * y;
                }
                rp[q] = rq[p] = 0.0;
                double *zp = Zt.data() + (size_t)p * n, *zq = Zt.data() + (size_t)q * n;
                for (int j = 0; j < n; ++j) {
                    const double x = zp[j], y = zq[j];
                    zp[j] = c * x - s * y;
                    zq[j] = s * x + c * y;
                }
            }
            // rotate the ring, keeping ring[0] fixed
            const int last = ring[np - 1];
            for (int k = np - 1; k > 1; --k) ring[k] = ring[k - 1];
            ring[1] = last;
        }
        converged = rotations == 0;
    }
    if (!converged) return false;
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(),
              [&](int a, int b) { return A[(size_t)a * n + a] > A[(size_t)b * n + b]; });
    std::vector<double> diag(n);
    for (int i = 0; i < n; ++i) diag[i] = A[(size_t)i * n + i];
    for (int j = 0; j < n; ++j) {
        w[j] = diag[ord[j]];
        for (int i = 0; i < n; ++i) A[(size_t)i * n + j] = Zt[(size_t)ord[j] * n + i];
    }
    return true;
}

// Truncated SVD K = U S V^T through the eigendecomposition of K^T K = V S^2 V^T, keeping
// s_i > rtol s_1; U = K V S^-1.  U (m x k), s (k), V (m x k), row-major.
static bool svd_trunc(int m, const double *K, double rtol, std::vector<double> &U, std::vector<double> &s,
                      std::vector<double> &V, int *rank_out)
{
    std::vector<double> KtK((size_t)m * m), w(m);
    gemm_tn(m, m, m, K, K, KtK.data());
    if (!sym_eig(m, KtK.data(), w.data())) return false;
    const double s1 = std::sqrt(std::max(w[0], 0.0));
    int r = 0;
    while (r < m && w[r] > 0.0 && std::sqrt(w[r]) > rtol * s1) ++r;
    s.resize(r);
    V.assign((size_t)m * r, 0.0);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < r; ++j) V[(size_t)i * r + j] = KtK[(size_t)i * m + j];
    for (int j = 0; j < r; ++j) s[j] = std::sqrt(w[j]);
    U.assign((size_t)m * r, 0.0);
    gemm(m, r, m, K, V.data(), U.data());
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < r; ++j) U[(size_t)i * r + j] /= s[j];
    *rank_out = r;
    return true;
}

// S^-1 U^T (k x m) from U (m x k) and s (k)
static std::vector<double> sinv_ut(int m, int k, const std::vector<double> &U, const std::vector<double> &s)
{
    std::vector<double> out((size_t)k * m);
    for (int i = 0; i < k; ++i)
        for (int a = 0; a < m; ++a) out[(size_t)i * m + a] = U[(size_t)a * k + i] / s[i];
    return out;
}

int m2l_directions(int *dirs /* [316][3] or NULL */)
{
    int n = 0;
    for (int dx = -3; dx <= 3; ++dx)
        for (int dy = -3; dy <= 3; ++dy)
            for (int dz = -3; dz <= 3; ++dz) {
                if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) < 2) continue;
                if (dirs) {
                    dirs[3 * n] = dx;
                    dirs[3 * n + 1] = dy;
                    dirs[3 * n + 2] = dz;
                }
                ++n;
            }
    return n;
}

bool compute_operators(const OpsParams &prm, OpsHost *out)
{
    const int p = prm.p;
    out->surf = lattice_surface(p);
    const int ns = (int)out->surf.size() / 3, m = 3 * ns;
    out->n_surf = ns;
    const double zero[3] = {0, 0, 0};
    const double ri = prm.r_inner, ro = prm.r_outer, nu = prm.nu;
    std::vector<double> K((size_t)m * m), tmp, tmp2;

    // singular bases of the check-to-equivalent maps at h = G = 1
    std::vector<double> Uu, su, Vu, Ud, sd, Vd;
    kernel_matrix(out->surf, nu, zero, ro, zero, ri, K.data());  // upward check <- upward equivalent
    if (!svd_trunc(m, K.data(), prm.pinv_rtol, Uu, su, Vu, &out->ku)) return false;
    kernel_matrix(out->surf, nu, zero, ri, zero, ro, K.data());  // downward check <- downward equivalent
    if (!svd_trunc(m, K.data(), prm.pinv_rtol, Ud, sd, Vd, &out->kd)) return false;
    const int ku = out->ku, kd = out->kd;
    out->sv_u = su;
    out->sv_d = sd;
    out->s2a_u = sinv_ut(m, ku, Uu, su);
    out->s2a_d = sinv_ut(m, kd, Ud, sd);
    out->vu = Vu;
    out->vd = Vd;

    // M2M in alpha space: parent half-width 2, child 1 at c_o:
    //   alpha_p = (G 2h) S^-1 U^T K(parent check <- child equiv) / (G h) V alpha_c
    // L2L in beta space: beta_c = S^-1 U^T K(child check <- parent equiv) V beta_p
    out->mb.assign((size_t)8 * ku * ku, 0.0);
    out->lb.assign((size_t)8 * kd * kd, 0.0);
    for (int o = 0; o < 8; ++o) {
        const double co[3] = {(o & 4) ? 1.0 : -1.0, (o & 2) ? 1.0 : -1.0, (o & 1) ? 1.0 : -1.0};
        kernel_matrix(out->surf, nu, zero, 2.0 * ro, co, ri, K.data());
        tmp.assign((size_t)m * ku, 0.0);
        gemm(m, ku, m, K.data(), Vu.data(), tmp.data());
        gemm(ku, ku, m, out->s2a_u.data(), tmp.data(), out->mb.data() + (size_t)o * ku * ku);
        for (size_t a = 0; a < (size_t)ku * ku; ++a) out->mb[(size_t)o * ku * ku + a] *= 2.0;
        kernel_matrix(out->surf, nu, co, ri, zero, 2.0 * ro, K.data());
        tmp.assign((size_t)m * kd, 0.0);
        gemm(m, kd, m, K.data(), Vd.data(), tmp.data());
        gemm(kd, kd, m, out->s2a_d.data(), tmp.data(), out->lb.data() + (size_t)o * kd * kd);
    }

    // M2L: K_v = K(target downward check at 0 <- source upward equivalent at 2v), h = 1
    int dirs[316 * 3];
    const int nd = m2l_directions(dirs);
    std::vector<double> Kall((size_t)nd * m * m);
    for (int v = 0; v < nd; ++v) {
        const double cs[3] = {2.0 * dirs[3 * v], 2.0 * dirs[3 * v + 1], 2.0 * dirs[3 * v + 2]};
        kernel_matrix(out->surf, nu, zero, ri, cs, ri, Kall.data() + (size_t)v * m * m);
    }
    // Gram = sum_v K_v K_v^T (symmetric; lower triangle then mirrored)
    std::vector<double> Gram((size_t)m * m, 0.0);
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < m; ++i)
        for (int v = 0; v < nd; ++v) {
            const double *Kv = Kall.data() + (size_t)v * m * m;
            const double *ri_ = Kv + (size_t)i * m;
            for (int j = 0; j <= i; ++j) {
                const double *rj = Kv + (size_t)j * m;
                double acc = 0.0;
                for (int k = 0; k < m; ++k) acc += ri_[k] * rj[k];
                Gram[(size_t)i * m + j] += acc;
            }
        }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < i; ++j) Gram[(size_t)j * m + i] = Gram[(size_t)i * m + j];
    std::vector<double> lam(m);
    if (!sym_eig(m, Gram.data(), lam.data())) return false;
    const double s1 = std::sqrt(std::max(lam[0], 0.0));
    int r = 0;
    if (prm.m2l_rtol <= 0.0) {
        r = m;
    } else {
        while (r < m && lam[r] > 0.0 && std::sqrt(lam[r]) > prm.m2l_rtol * s1) ++r;
    }
    r = std::min(m, (r + 15) / 16 * 16);  // padding to 16 costs the same, so keep those columns
    if (prm.m2l_rank_max > 0 && r > prm.m2l_rank_max) r = prm.m2l_rank_max;
    r = std::max(r, 1);
    out->rank = r;
    out->m2l_sv.resize(m);
    for (int i = 0; i < m; ++i) out->m2l_sv[i] = std::sqrt(std::max(lam[i], 0.0));
    std::vector<double> Ur((size_t)m * r);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < r; ++j) Ur[(size_t)i * r + j] = Gram[(size_t)i * m + j];
    out->m2l_c.assign((size_t)nd * r * r, 0.0);
    {
        std::vector<double> KU((size_t)m * r);
        for (int v = 0; v < nd; ++v) {
            gemm(m, r, m, Kall.data() + (size_t)v * m * m, Ur.data(), KU.data());
            gemm_tn(r, r, m, Ur.data(), KU.data(), out->m2l_c.data() + (size_t)v * r * r);
        }
    }
    out->cb.assign((size_t)r * ku, 0.0);  // U_r^T V_u
    gemm_tn(r, ku, m, Ur.data(), Vu.data(), out->cb.data());
    out->wb.assign((size_t)kd * r, 0.0);  // S_d^-1 U_d^T U_r
    gemm(kd, r, m, out->s2a_d.data(), Ur.data(), out->wb.data());
    return true;
}

}  // namespace host
}  // namespace kfmm
