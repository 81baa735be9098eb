// precompute.h -- FP64 host precompute of the equivalent-surface operators (no CUDA).
//
// Equivalent densities are carried in the singular bases of the check-to-equivalent maps:
// with K_uc = U_u S_u V_u^T (upward check <- upward equivalent, truncated at pinv_rtol) the
// upward density of a box is phi_up = V_u alpha, alpha = G h S_u^-1 U_u^T chk_up, and
// likewise phi_dn = V_d beta for the downward pass.  Every translation acts on alpha / beta,
// so the 1/s amplification of the pseudo-inverse only ever multiplies rounding errors that
// lie along the matching singular direction, whose field the kernel damps by s again.
#pragma once

#include <vector>

namespace kfmm {
namespace host {

struct OpsParams {
    int p;
    double nu, r_inner, r_outer, pinv_rtol, m2l_rtol;
    int m2l_rank_max;
};

struct OpsHost {
    int n_surf = 0;  // lattice surface points; m = 3 n_surf
    int ku = 0;      // rank kept of K_uc (upward)
    int kd = 0;      // rank kept of K_dc (downward)
    int rank = 0;    // shared M2L basis rank r
    std::vector<double> surf;    // [n_surf][3] in [-1,1]^3
    std::vector<double> s2a_u;   // [ku][m]:  S_u^-1 U_u^T         (upward check -> alpha, x G h)
    std::vector<double> mb;      // [8][ku][ku]: 2 S_u^-1 U_u^T K_o V_u (child alpha -> parent alpha)
    std::vector<double> vu;      // [m][ku]:  V_u                  (alpha -> phi_up)
    std::vector<double> cb;      // [rank][ku]: U_r^T V_u          (alpha -> psi, the M2L input)
    std::vector<double> m2l_c;   // [316][rank][rank]: U_r^T K_v U_r
    std::vector<double> wb;      // [kd][rank]: S_d^-1 U_d^T U_r   (M2L output c -> beta)
    std::vector<double> s2a_d;   // [kd][m]:  S_d^-1 U_d^T         (downward check -> beta, x G h)
    std::vector<double> lb;      // [8][kd][kd]: S_d^-1 U_d^T K'_o V_d (parent beta -> child beta)
    std::vector<double> vd;      // [m][kd]:  V_d                  (beta -> phi_dn)
    std::vector<double> sv_u, sv_d, m2l_sv;  // singular values (for inspection)
};

std::vector<double> lattice_surface(int p);
int m2l_directions(int *dirs);
bool compute_operators(const OpsParams &prm, OpsHost *out);
// periodic.cpp: R [kd][ku], the far-lattice operator of a periodic tree's root (root alpha ->
// root beta) for the operators H computed with prm
bool compute_lattice(const OpsParams &prm, const OpsHost &H, std::vector<double> &R);

}  // namespace host
}  // namespace kfmm
