// shard.cpp -- the partition of the FMM over several GPUs (Sec. "Numerical solution": the
// evaluation is parallelised by giving each process a part of the octree; the data a
// process needs from the others is its locally essential tree).  Host code on a tree given
// as host arrays (kfmm_tree_view; kfmm_export_tree and kfmm_export_list give them for a
// built tree).
//
// Plan: the leaves, in Morton order, are cut into n_ranks contiguous ranges of about equal
// cost.  A leaf belongs to the rank of its range; a box belongs to a rank when all the leaves
// below it do, and is shared otherwise (only boxes on the paths between the ranges' ends and
// the roots are shared: the coarse levels).
//
// Locally essential tree of rank r, for its target leaves L and their ancestors (the boxes
// whose downward densities it forms):
//   sources      -- leaves of U(l), l in L, and of X(B), B in L or an ancestor, that rank r
//                   does not own: their points and densities are received (all-to-all);
//   upward       -- boxes of V(B), B in L or an ancestor, and of W(l), l in L, owned by
//                   another rank: their upward equivalent densities are received;
//   shared       -- boxes in those lists, or ancestors of rank r's leaves, that are shared:
//                   their upward densities are sums of every rank's part (all-reduce).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/kifmm_elastic.h"

namespace {

// Morton key of a box at the finest level, led by its root's index (independent point sets)
uint64_t box_key(const kfmm_tree_view *t, int b, int max_level, const std::vector<int> &root)
{
    const int lev = t->level[b];
    const int sh = max_level - lev;
    uint64_t k = 0;
    const uint64_t xyz[3] = {(uint64_t)t->anchor[3 * b] << sh, (uint64_t)t->anchor[3 * b + 1] << sh,
                             (uint64_t)t->anchor[3 * b + 2] << sh};
    for (int bit = max_level - 1; bit >= 0; --bit)
        for (int c = 0; c < 3; ++c) k = (k << 1) | ((xyz[c] >> bit) & 1u);
    return ((uint64_t)root[b] << (3 * max_level)) | k;
}

bool valid_view(const kfmm_tree_view *t)
{
    return t && t->n_boxes > 0 && t->level && t->anchor && t->parent && t->box_src && t->box_trg && t->u_off &&
           t->u_idx && t->v_off && t->v_idx && t->w_off && t->w_idx && t->x_off && t->x_idx;
}

}  // namespace

extern "C" {

kfmm_status kfmm_shard_plan(const kfmm_tree_view *t, int32_t n_ranks, const double *box_cost, int32_t *box_owner,
                            int32_t *leaf_order, double *rank_cost)
{
    if (!valid_view(t) || n_ranks < 1 || !box_owner) return KFMM_ERR_INVALID_ARG;
    const int nb = t->n_boxes;
    std::vector<char> has_child(nb, 0);
    std::vector<int> root(nb, -1);
    int max_level = 0, n_roots = 0;
    for (int b = 0; b < nb; ++b) {
        const int p = t->parent[b];
        if (p < -1 || p >= nb || t->level[b] < 0 || t->level[b] > 21) return KFMM_ERR_INVALID_ARG;
        if (p >= 0) has_child[p] = 1;
        max_level = std::max(max_level, (int)t->level[b]);
    }
    // roots: walk up (boxes are listed coarse to fine, so a parent precedes its children)
    for (int b = 0; b < nb; ++b) {
        const int p = t->parent[b];
        if (p < 0) root[b] = n_roots++;
        else if (p < b) root[b] = root[p];
        else return KFMM_ERR_INVALID_ARG;
    }
    if (max_level > 21 || (n_roots > 1 && 3 * max_level + 32 - __builtin_clz((unsigned)n_roots) > 64))
        return KFMM_ERR_INVALID_ARG;
    std::vector<int> leaves;
    for (int b = 0; b < nb; ++b)
        if (!has_child[b]) leaves.push_back(b);
    std::vector<uint64_t> key(nb, 0);
    for (int b : leaves) key[b] = box_key(t, b, max_level, root);
    std::sort(leaves.begin(), leaves.end(), [&](int a, int b) { return key[a] < key[b]; });
    // cost of a leaf: its pairs with the sources of its U list, plus its own sources and
    // targets (upward and local work), plus one
    std::vector<double> cost(leaves.size());
    for (size_t i = 0; i < leaves.size(); ++i) {
        const int b = leaves[i];
        if (box_cost) {
            cost[i] = std::max(0.0, box_cost[b]);
            continue;
        }
        const double nt = t->box_trg[2 * b + 1] - t->box_trg[2 * b];
        const double ns = t->box_src[2 * b + 1] - t->box_src[2 * b];
        double near = 0.0;
        for (int e = t->u_off[b]; e < t->u_off[b + 1]; ++e) {
            const int s = t->u_idx[e];
            near += t->box_src[2 * s + 1] - t->box_src[2 * s];
        }
        cost[i] = nt * near + ns + nt + 1.0;
    }
    const double total = std::accumulate(cost.begin(), cost.end(), 0.0);
    for (int b = 0; b < nb; ++b) box_owner[b] = -2;  // not yet assigned
    if (rank_cost)
        for (int r = 0; r < n_ranks; ++r) rank_cost[r] = 0.0;
    // leaf i goes to the rank whose share of the total holds the middle of its cost
    double run = 0.0;
    for (size_t i = 0; i < leaves.size(); ++i) {
        const double mid = run + 0.5 * cost[i];
        int r = total > 0.0 ? (int)(mid / total * n_ranks) : (int)(i * n_ranks / leaves.size());
        r = std::min(std::max(r, 0), n_ranks - 1);
        box_owner[leaves[i]] = r;
        if (rank_cost) rank_cost[r] += cost[i];
        run += cost[i];
        if (leaf_order) leaf_order[i] = leaves[i];
    }
    // a box belongs to a rank when all its leaves do (children are listed after parents)
    for (int b = nb - 1; b >= 0; --b) {
        const int p = t->parent[b];
        if (p < 0) continue;
        const int o = box_owner[b];
        if (box_owner[p] == -2) box_owner[p] = o;
        else if (box_owner[p] != o) box_owner[p] = -1;
    }
    for (int b = 0; b < nb; ++b)
        if (box_owner[b] == -2) box_owner[b] = -1;  // cannot happen for a tree of leaves
    return KFMM_OK;
}

kfmm_status kfmm_shard_let(const kfmm_tree_view *t, const int32_t *box_owner, int32_t rank, int32_t *src_boxes,
                           int64_t *n_src, int32_t *up_boxes, int64_t *n_up, int32_t *shared_boxes,
                           int64_t *n_shared)
{
    if (!valid_view(t) || !box_owner || rank < 0 || !n_src || !n_up || !n_shared) return KFMM_ERR_INVALID_ARG;
    const int nb = t->n_boxes;
    std::vector<char> has_child(nb, 0), target_side(nb, 0), need_src(nb, 0), need_up(nb, 0), need_shared(nb, 0);
    for (int b = 0; b < nb; ++b) {
        const int p = t->parent[b];
        if (p < -1 || p >= nb) return KFMM_ERR_INVALID_ARG;
        if (p >= 0) has_child[p] = 1;
    }
    // rank r's leaves and all their ancestors
    for (int b = 0; b < nb; ++b)
        if (!has_child[b] && box_owner[b] == rank)
            for (int a = b; a >= 0 && !target_side[a]; a = t->parent[a]) target_side[a] = 1;
    auto add_src = [&](int s) {
        if (box_owner[s] != rank) need_src[s] = 1;
    };
    auto add_up = [&](int s) {
        if (box_owner[s] == -1) need_shared[s] = 1;
        else if (box_owner[s] != rank) need_up[s] = 1;
    };
    for (int b = 0; b < nb; ++b) {
        if (!target_side[b]) continue;
        const bool leaf = !has_child[b];
        if (leaf) {
            for (int e = t->u_off[b]; e < t->u_off[b + 1]; ++e) add_src(t->u_idx[e]);
            for (int e = t->w_off[b]; e < t->w_off[b + 1]; ++e) add_up(t->w_idx[e]);
        }
        for (int e = t->x_off[b]; e < t->x_off[b + 1]; ++e) add_src(t->x_idx[e]);
        for (int e = t->v_off[b]; e < t->v_off[b + 1]; ++e) add_up(t->v_idx[e]);
        // the upward pass of a shared ancestor combines every rank's part of it
        if (box_owner[b] == -1) need_shared[b] = 1;
    }
    const int64_t cap_s = *n_src, cap_u = *n_up, cap_h = *n_shared;
    int64_t ks = 0, ku = 0, kh = 0;
    for (int b = 0; b < nb; ++b) {
        if (need_src[b]) {
            if (src_boxes && ks < cap_s) src_boxes[ks] = b;
            ++ks;
        }
        if (need_up[b]) {
            if (up_boxes && ku < cap_u) up_boxes[ku] = b;
            ++ku;
        }
        if (need_shared[b]) {
            if (shared_boxes && kh < cap_h) shared_boxes[kh] = b;
            ++kh;
        }
    }
    *n_src = ks;
    *n_up = ku;
    *n_shared = kh;
    if ((src_boxes && ks > cap_s) || (up_boxes && ku > cap_u) || (shared_boxes && kh > cap_h))
        return KFMM_ERR_INVALID_ARG;
    return KFMM_OK;
}

}  // extern "C"
