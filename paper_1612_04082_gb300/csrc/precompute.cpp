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

// Truncated pseudo-inverse through the eigendecomposition of K^T K = V diag(s^2) V^T:
// pinv(K) = sum_{s_i > rtol s_1} v_i v_i^T K^T / s_i^2.
static bool pinv(int m, const double *K, double rtol, double *P, int *rank_out)
{
    std::vector<double> KtK((size_t)m * m), w(m);
    gemm_tn(m, m, m, K, K, KtK.data());
    if (!sym_eig(m, KtK.data(), w.data())) return false;
    const double s1 = std::sqrt(std::max(w[0], 0.0));
    int r = 0;
    while (r < m && w[r] > 0.0 && std::sqrt(w[r]) > rtol * s1) ++r;
    // B = V_r diag(1/s^2) V_r^T  (m x m), then P = B K^T
    std::vector<double> Vs((size_t)m * r);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < r; ++j) Vs[(size_t)i * r + j] = KtK[(size_t)i * m + j] / w[j];
    std::vector<double> B((size_t)m * m);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i)
        for (int k = 0; k < m; ++k) {
            double s = 0.0;
            for (int j = 0; j < r; ++j) s += Vs[(size_t)i * r + j] * KtK[(size_t)k * m + j];
            B[(size_t)i * m + k] = s;
        }
    // P = B K^T: P[i][a] = sum_k B[i][k] K[a][k]
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i)
        for (int a = 0; a < m; ++a) {
            double s = 0.0;
            for (int k = 0; k < m; ++k) s += B[(size_t)i * m + k] * K[(size_t)a * m + k];
            P[(size_t)i * m + a] = s;
        }
    *rank_out = r;
    return true;
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

    // check-to-equivalent pseudo-inverses at h = 1
    std::vector<double> K((size_t)m * m);
    out->pinv_uc.assign((size_t)m * m, 0.0);
    out->pinv_dc.assign((size_t)m * m, 0.0);
    kernel_matrix(out->surf, nu, zero, ro, zero, ri, K.data());  // upward check <- upward equivalent
    if (!pinv(m, K.data(), prm.pinv_rtol, out->pinv_uc.data(), &out->rank_uc)) return false;
    kernel_matrix(out->surf, nu, zero, ri, zero, ro, K.data());  // downward check <- downward equivalent
    if (!pinv(m, K.data(), prm.pinv_rtol, out->pinv_dc.data(), &out->rank_dc)) return false;

    // M2M_o = pinv_uc(parent, half-width 2) K(parent check <- child equivalent)
    //       = 2 pinv_uc K;  L2L_o = pinv_dc(child) K(child check <- parent equivalent)
    out->m2m.assign((size_t)8 * m * m, 0.0);
    out->l2l.assign((size_t)8 * m * m, 0.0);
    std::vector<double> tmp((size_t)m * m);
    for (int o = 0; o < 8; ++o) {
        const double co[3] = {(o & 4) ? 1.0 : -1.0, (o & 2) ? 1.0 : -1.0, (o & 1) ? 1.0 : -1.0};
        kernel_matrix(out->surf, nu, zero, 2.0 * ro, co, ri, K.data());
        gemm(m, m, m, out->pinv_uc.data(), K.data(), tmp.data());
        for (size_t a = 0; a < tmp.size(); ++a) out->m2m[(size_t)o * m * m + a] = 2.0 * tmp[a];
        kernel_matrix(out->surf, nu, co, ri, zero, 2.0 * ro, K.data());
        gemm(m, m, m, out->pinv_dc.data(), K.data(), out->l2l.data() + (size_t)o * m * m);
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
                double s = 0.0;
                for (int k = 0; k < m; ++k) s += ri_[k] * rj[k];
                Gram[(size_t)i * m + j] += s;
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
    if (prm.m2l_rank_max > 0 && r > prm.m2l_rank_max) r = prm.m2l_rank_max;
    r = std::max(r, 1);
    out->rank = r;
    out->m2l_sv.resize(m);
    for (int i = 0; i < m; ++i) out->m2l_sv[i] = std::sqrt(std::max(lam[i], 0.0));
    // Ur: m x r (first r columns of Gram's eigenvectors)
    std::vector<double> Ur((size_t)m * r);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < r; ++j) Ur[(size_t)i * r + j] = Gram[(size_t)i * m + j];
    out->m2l_vt.assign((size_t)r * m, 0.0);  // Ur^T
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < r; ++j) out->m2l_vt[(size_t)j * m + i] = Ur[(size_t)i * r + j];
    out->m2l_c.assign((size_t)nd * r * r, 0.0);
    {
        std::vector<double> KU((size_t)m * r);
        for (int v = 0; v < nd; ++v) {
            gemm(m, r, m, Kall.data() + (size_t)v * m * m, Ur.data(), KU.data());
            gemm_tn(r, r, m, Ur.data(), KU.data(), out->m2l_c.data() + (size_t)v * r * r);
        }
    }
    out->m2l_w.assign((size_t)m * r, 0.0);  // pinv_dc Ur
    gemm(m, r, m, out->pinv_dc.data(), Ur.data(), out->m2l_w.data());
    return true;
}

}  // namespace host
}  // namespace kfmm
