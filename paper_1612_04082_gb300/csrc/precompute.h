// precompute.h -- FP64 host precompute of the equivalent-surface operators (no CUDA).
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
    int n_surf = 0, rank = 0, rank_uc = 0, rank_dc = 0;
    std::vector<double> surf;     // [n_surf][3] in [-1,1]^3
    std::vector<double> pinv_uc;  // [3n][3n]
    std::vector<double> pinv_dc;  // [3n][3n]
    std::vector<double> m2m;      // [8][3n][3n]
    std::vector<double> l2l;      // [8][3n][3n]
    std::vector<double> m2l_vt;   // [rank][3n]
    std::vector<double> m2l_c;    // [316][rank][rank]
    std::vector<double> m2l_w;    // [3n][rank]
    std::vector<double> m2l_sv;   // [3n] singular values of the stacked M2L matrices
};

std::vector<double> lattice_surface(int p);
int m2l_directions(int *dirs);
bool compute_operators(const OpsParams &prm, OpsHost *out);

}  // namespace host
}  // namespace kfmm
