// voxel.cpp -- host side of the optimisation procedure of Sec. "Parallel optimization
// procedure": the boundary of the material voxels as flat triangles (every face between a
// material voxel and a void voxel or the outside gives 4 triangles fanned to the face centre,
// Sec. "Performance and scalability"), the hard-kill update by thresholding the topological
// derivative, D_C = D_min + C (D_max - D_min), and the post-processing that drops isolated
// voxels and material not connected to the supports.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/kifmm_elastic.h"

namespace {

struct Surface {
    std::vector<double> verts;
    std::vector<int32_t> tris;
    std::vector<int64_t> cell;
    std::vector<int8_t> dir;
};

// face directions -x, +x, -y, +y, -z, +z as (axis, sign)
constexpr int kAxis[6] = {0, 0, 1, 1, 2, 2};
constexpr int kSign[6] = {-1, 1, -1, 1, -1, 1};

// periodic: the array is one cell of a periodic voxel pattern, a voxel's neighbour across a
// face of the array is the voxel on the opposite side, and no face lies on the array's boundary
// unless the wrapped neighbour is void (the surface then crosses the cell's faces)
void build_surface(const uint8_t *m, int nx, int ny, int nz, double h, const double *o, bool periodic, Surface &S)
{
    const int64_t cx = nx + 1, cy = ny + 1, cz = nz + 1;
    std::vector<int64_t> corner_id((size_t)(cx * cy * cz), -1);
    std::vector<int32_t> corners;  // lattice coordinates, 3 per corner, in first-use order
    std::vector<int64_t> centers;  // 4x the face centre in lattice units, 3 per face
    std::vector<int64_t> tri_ref;  // per triangle: -1 - face index, corner a, corner b
    const int n[3] = {nx, ny, nz};
    auto filled = [&](int i, int j, int k) {
        if (periodic) {
            i = (i + nx) % nx;
            j = (j + ny) % ny;
            k = (k + nz) % nz;
        } else if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) {
            return false;
        }
        return m[((int64_t)i * ny + j) * nz + k] != 0;
    };
    auto corner = [&](const int c[3]) {
        const int64_t key = ((int64_t)c[0] * cy + c[1]) * cz + c[2];
        int64_t &id = corner_id[(size_t)key];
        if (id < 0) {
            id = (int64_t)corners.size() / 3;
            corners.insert(corners.end(), {c[0], c[1], c[2]});
        }
        return id;
    };
    (void)n;
    for (int fd = 0; fd < 6; ++fd) {
        const int ax = kAxis[fd], sgn = kSign[fd];
        int a1 = -1, a2 = -1;
        for (int a = 0; a < 3; ++a)
            if (a != ax) (a1 < 0 ? a1 : a2) = a;
        // (e_a1, e_a2, e_ax) right-handed when a2 follows a1 cyclically; the normal must
        // point along sgn * e_ax
        const bool cyc = (a2 - a1 + 3) % 3 == 1;
        const bool flip = (sgn > 0) != cyc;
        for (int i = 0; i < nx; ++i)
            for (int j = 0; j < ny; ++j)
                for (int k = 0; k < nz; ++k) {
                    if (!filled(i, j, k)) continue;
                    int nb[3] = {i, j, k};
                    nb[ax] += sgn;
                    if (filled(nb[0], nb[1], nb[2])) continue;
                    int base[3] = {i, j, k};
                    if (sgn > 0) base[ax] += 1;
                    static const int uv[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
                    int64_t q[4];
                    int64_t csum[3] = {0, 0, 0};
                    for (int t = 0; t < 4; ++t) {
                        int c[3] = {base[0], base[1], base[2]};
                        c[a1] += uv[t][0];
                        c[a2] += uv[t][1];
                        q[t] = corner(c);
                        for (int a = 0; a < 3; ++a) csum[a] += c[a];
                    }
                    if (flip) std::swap(q[0], q[3]), std::swap(q[1], q[2]);
                    const int64_t f = (int64_t)centers.size() / 3;
                    centers.insert(centers.end(), {csum[0], csum[1], csum[2]});
                    const int64_t lin = ((int64_t)i * ny + j) * nz + k;
                    for (int t = 0; t < 4; ++t) {
                        tri_ref.insert(tri_ref.end(), {-1 - f, q[t], q[(t + 1) % 4]});
                        S.cell.push_back(lin);
                        S.dir.push_back((int8_t)fd);
                    }
                }
    }
    const int64_t nc = (int64_t)corners.size() / 3, nf = (int64_t)centers.size() / 3;
    S.verts.resize((size_t)(3 * (nc + nf)));
    for (int64_t c = 0; c < nc; ++c)
        for (int a = 0; a < 3; ++a) S.verts[(size_t)(3 * c + a)] = corners[(size_t)(3 * c + a)] * h + o[a];
    for (int64_t f = 0; f < nf; ++f)
        for (int a = 0; a < 3; ++a)
            S.verts[(size_t)(3 * (nc + f) + a)] = 0.25 * (double)centers[(size_t)(3 * f + a)] * h + o[a];
    S.tris.resize(tri_ref.size());
    for (size_t t = 0; t < tri_ref.size(); ++t) {
        const int64_t v = tri_ref[t];
        S.tris[t] = (int32_t)(v < 0 ? nc + (-1 - v) : v);
    }
}

bool dims_ok(int nx, int ny, int nz)
{
    return nx > 0 && ny > 0 && nz > 0 && (int64_t)nx * ny * nz <= (int64_t)1 << 31;
}

}  // namespace

extern "C" {

static kfmm_status voxel_surface(const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, double h,
                                 const double *origin, bool periodic, double *verts, int64_t *nv, int32_t *tris,
                                 int64_t *nt, int64_t *face_cell, int8_t *face_dir)
{
    if (!mask || !nv || !nt || !dims_ok(nx, ny, nz) || !(h > 0)) return KFMM_ERR_INVALID_ARG;
    const double zero[3] = {0, 0, 0};
    Surface S;
    build_surface(mask, nx, ny, nz, h, origin ? origin : zero, periodic, S);
    const int64_t n_v = (int64_t)S.verts.size() / 3, n_t = (int64_t)S.tris.size() / 3;
    if (n_t > INT32_MAX || n_v > INT32_MAX) return KFMM_ERR_INVALID_ARG;
    const bool fill = verts || tris || face_cell || face_dir;
    if (fill && (*nv < n_v || *nt < n_t)) {
        *nv = n_v;
        *nt = n_t;
        return KFMM_ERR_INVALID_ARG;
    }
    *nv = n_v;
    *nt = n_t;
    if (verts) std::memcpy(verts, S.verts.data(), sizeof(double) * S.verts.size());
    if (tris) std::memcpy(tris, S.tris.data(), sizeof(int32_t) * S.tris.size());
    if (face_cell) std::memcpy(face_cell, S.cell.data(), sizeof(int64_t) * S.cell.size());
    if (face_dir) std::memcpy(face_dir, S.dir.data(), S.dir.size());
    return KFMM_OK;
}

kfmm_status kfmm_voxel_surface(const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, double h,
                               const double *origin, double *verts, int64_t *nv, int32_t *tris, int64_t *nt,
                               int64_t *face_cell, int8_t *face_dir)
{
    return voxel_surface(mask, nx, ny, nz, h, origin, false, verts, nv, tris, nt, face_cell, face_dir);
}

kfmm_status kfmm_voxel_surface_periodic(const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, double h,
                                        const double *origin, double *verts, int64_t *nv, int32_t *tris,
                                        int64_t *nt, int64_t *face_cell, int8_t *face_dir)
{
    return voxel_surface(mask, nx, ny, nz, h, origin, true, verts, nv, tris, nt, face_cell, face_dir);
}

kfmm_status kfmm_voxel_threshold(uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, const float *td,
                                 const uint8_t *frozen, double C, int64_t *removed)
{
    if (!mask || !td || !dims_ok(nx, ny, nz) || !(C >= 0 && C <= 1)) return KFMM_ERR_INVALID_ARG;
    const int64_t n = (int64_t)nx * ny * nz;
    float lo = 0, hi = 0;
    bool any = false;
    for (int64_t c = 0; c < n; ++c) {
        if (!mask[c]) continue;
        if (!any) lo = hi = td[c], any = true;
        lo = std::min(lo, td[c]);
        hi = std::max(hi, td[c]);
    }
    int64_t cnt = 0;
    if (any) {
        const double thr = (double)lo + C * ((double)hi - (double)lo);
        for (int64_t c = 0; c < n; ++c)
            if (mask[c] && !(frozen && frozen[c]) && (double)td[c] < thr) {
                mask[c] = 0;
                ++cnt;
            }
    }
    if (removed) *removed = cnt;
    return KFMM_OK;
}

kfmm_status kfmm_voxel_clean(uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, const uint8_t *support,
                             const uint8_t *keep, int64_t *removed)
{
    if (!mask || !dims_ok(nx, ny, nz)) return KFMM_ERR_INVALID_ARG;
    const int64_t n = (int64_t)nx * ny * nz;
    auto lin = [&](int i, int j, int k) { return ((int64_t)i * ny + j) * nz + k; };
    const int di[6] = {-1, 1, 0, 0, 0, 0}, dj[6] = {0, 0, -1, 1, 0, 0}, dk[6] = {0, 0, 0, 0, -1, 1};
    int64_t cnt = 0;
    // material voxels without a material face neighbour
    std::vector<int64_t> iso;
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k) {
                const int64_t c = lin(i, j, k);
                if (!mask[c] || (support && support[c]) || (keep && keep[c])) continue;
                bool nb = false;
                for (int d = 0; d < 6 && !nb; ++d) {
                    const int a = i + di[d], b = j + dj[d], e = k + dk[d];
                    if (a >= 0 && b >= 0 && e >= 0 && a < nx && b < ny && e < nz && mask[lin(a, b, e)]) nb = true;
                }
                if (!nb) iso.push_back(c);
            }
    for (int64_t c : iso) mask[c] = 0;
    cnt += (int64_t)iso.size();
    // material not face-connected to a support voxel
    if (support) {
        std::vector<uint8_t> seen((size_t)n, 0);
        std::vector<int64_t> stack;
        for (int64_t c = 0; c < n; ++c)
            if (support[c] && mask[c]) {
                seen[(size_t)c] = 1;
                stack.push_back(c);
            }
        while (!stack.empty()) {
            const int64_t c = stack.back();
            stack.pop_back();
            const int i = (int)(c / ((int64_t)ny * nz)), j = (int)((c / nz) % ny), k = (int)(c % nz);
            for (int d = 0; d < 6; ++d) {
                const int a = i + di[d], b = j + dj[d], e = k + dk[d];
                if (a < 0 || b < 0 || e < 0 || a >= nx || b >= ny || e >= nz) continue;
                const int64_t q = lin(a, b, e);
                if (mask[q] && !seen[(size_t)q]) {
                    seen[(size_t)q] = 1;
                    stack.push_back(q);
                }
            }
        }
        for (int64_t c = 0; c < n; ++c)
            if (mask[c] && !seen[(size_t)c] && !(keep && keep[c])) {
                mask[c] = 0;
                ++cnt;
            }
    }
    if (removed) *removed = cnt;
    return KFMM_OK;
}

}  // extern "C"
