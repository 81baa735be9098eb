// common.cuh -- internal types of the kifmm_elastic library: the context, device buffers,
// error handling.  Not part of the public ABI (include/kifmm_elastic.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include "../../include/kifmm_elastic.h"

namespace kfmm {

// ------------------------------------------------------------------------------------
// Errors: every internal routine returns kfmm_status; the first failure records a message
// in the context and is passed straight up to the ABI.
// ------------------------------------------------------------------------------------
struct Error {
    kfmm_status code;
    std::string msg;
};

#define KF_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            return ctx->fail(KFMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                                  \
    } while (0)

#define KF_LAUNCH()                                                                        \
    do {                                                                                   \
        ++ctx->n_launch;                                                                   \
        cudaError_t e_ = cudaGetLastError();                                               \
        if (e_ != cudaSuccess)                                                             \
            return ctx->fail(KFMM_ERR_CUDA, std::string("kernel launch at ") + __FILE__ + ":" + \
                                                std::to_string(__LINE__) + ": " +          \
                                                cudaGetErrorString(e_));                   \
    } while (0)

#define KF_TRY(expr)                                                                       \
    do {                                                                                   \
        kfmm_status s_ = (expr);                                                           \
        if (s_ != KFMM_OK) return s_;                                                      \
    } while (0)

// Grow-only device buffer.  Contents are not preserved across growth.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes) {
        o.p = nullptr;
        o.bytes = 0;
    }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            bytes = o.bytes;
            o.p = nullptr;
            o.bytes = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t nbytes) {
        if (nbytes <= bytes) return cudaSuccess;
        release();
        size_t nb = nbytes < 256 ? 256 : nbytes;
        cudaError_t e = cudaMalloc(&p, nb);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = nb;
        return cudaSuccess;
    }
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// Equivalent-surface operators for one (p, nu, radii, tolerances); FP32 copies on device.
struct Operators {
    bool ready = false;
    int p = 0, n_surf = 0, rank = 0;  // rank of the shared M2L basis
    double nu = -1, r_inner = 0, r_outer = 0, pinv_rtol = 0, m2l_rtol = 0;
    int m2l_rank_max = 0;
    int ku = 0, kd = 0;  // ranks kept of the upward / downward check-to-equivalent maps
    // FP32, rows padded to multiples of 16 (see precompute.h for the definitions)
    DevBuf surf;      // float [n_surf][4]: unit lattice surface points in [-1,1]^3
    DevBuf s2a_u;     // [ku][3n]   upward check -> alpha (x G h)
    DevBuf mb;        // [8][ku][ku] child alpha -> parent alpha
    DevBuf vu;        // [3n][ku]   alpha -> upward equivalent density
    DevBuf cb;        // [r][ku]    alpha -> psi (M2L input)
    DevBuf m2l_c;     // [316][r][r] translation in the shared basis
    DevBuf wb;        // [kd][r]    M2L output -> beta
    DevBuf s2a_d;     // [kd][3n]   downward check -> beta (x G h)
    DevBuf lb;        // [8][kd][kd] parent beta -> child beta
    DevBuf vd;        // [3n][kd]   beta -> downward equivalent density
    // M2L translations as BF16 split-pair operand images for the tensor cores:
    // [316][ceil(r/128)][hi, lo][128 x rp] in the UMMA core-matrix layout (see tc_gemm.cuh)
    DevBuf m2l_tc;
    int m2l_tc_mtiles = 0;
    bool m2l_pairs_rows = false;  // tensor-core M2L with the pairs as rows (tc_m2l_kernel)
    // box operators for the K-streamed tensor-core product: [n_mat][n_mtile][n_kc][2][128 x 64]
    struct TcOp {
        DevBuf img;
        int n_mat = 0, M = 0, K = 0, n_mtile = 0, n_kc = 0;
        bool on = false;  // product runs on the tensor cores
    };
    bool box_tc = false;  // any box operator on the tensor cores
    // far-lattice operator of a periodic tree's root, root alpha -> root beta (periodic.cpp)
    DevBuf lat;           // float [kd][kup]
    bool lat_ready = false;
    TcOp tc_s2a_u, tc_mb, tc_cb, tc_vu, tc_wb, tc_s2a_d, tc_lb, tc_vd;
};

// points on the surface of a p x p x p lattice (equivalent and check surfaces)
constexpr int surface_points(int p) { return 6 * (p - 1) * (p - 1) + 2; }

// Entries of the colleague table and the interaction lists: the box index in the low 26 bits
// and, in a periodic tree, the image of the box that the entry means (the box moved by s cells,
// s in {-1, 0, 1}^3) in bits 26-30 as (9 (sx + 1) + 3 (sy + 1) + (sz + 1)) ^ 13.  The unmoved
// image has code 0, so every entry of a free-space tree is the box index itself; entries stay
// non-negative (-1 marks a missing colleague).
constexpr int kEntBits = 26;
constexpr int kEntMask = (1 << kEntBits) - 1;
__host__ __device__ inline int ent_box(int e) { return e & kEntMask; }
__host__ __device__ inline int ent_image(int e) { return ((e >> kEntBits) & 31) ^ 13; }  // 0..26
__host__ __device__ inline int ent_make(int box, int image) { return box | ((image ^ 13) << kEntBits); }
__host__ __device__ inline void ent_shift(int e, int &sx, int &sy, int &sz)
{
    const int c = ent_image(e);
    sx = c / 9 - 1;
    sy = (c / 3) % 3 - 1;
    sz = c % 3 - 1;
}

// Octree and interaction lists (device arrays unless noted).
struct Tree {
    bool built = false;
    int64_t nsrc = 0, ntrg = 0;
    int max_depth = 0;
    double root_lo[3] = {0, 0, 0};  // lower corner of the root cube (of the first set)
    double root_w = 1;              // root cube side
    int n_sets = 1;                 // independent point sets, one root box each (level 0)
    std::vector<double> set_roots;  // host: 8 per set: lower corner x, y, z, side, 1 / side
    DevBuf set_root_dev;            // the same on the device
    int n_boxes = 0, n_leaves = 0, n_levels = 0;
    std::vector<int> level_off;  // host: first box of each level, size n_levels + 1
    bool has_nrm = false;

    // points, sorted by Morton key
    DevBuf src_xyz;   // float4 [nsrc]: x, y, z, 0
    DevBuf src_nrm;   // float4 [nsrc]
    DevBuf trg_xyz;   // float4 [ntrg]
    DevBuf src_perm;  // int [nsrc]: sorted position -> input index
    DevBuf trg_perm;  // int [ntrg]
    DevBuf src_key, trg_key;  // uint64 [n]

    // boxes (level-major, Morton order within a level)
    DevBuf box_key;     // uint64
    DevBuf box_level;   // int
    DevBuf box_anchor;  // int4: ix, iy, iz, level
    DevBuf box_parent;  // int
    DevBuf box_child;   // int [8] per box, -1 if absent
    DevBuf box_src;     // int2 [begin, end) into sorted sources
    DevBuf box_trg;     // int2
    DevBuf box_leaf;    // int: 1 if leaf
    DevBuf colleague;   // int [27] per box, -1 if absent (index 13 = itself)

    // interaction lists, CSR by target box
    DevBuf u_off, u_idx;  // U: leaves adjacent to a leaf (incl. itself)
    DevBuf w_off, w_idx;  // W: for leaf B, descendants of colleagues, not adjacent, parent adjacent
    DevBuf x_off, x_idx;  // X: dual of W
    DevBuf xd_off, xd_idx;  // per box (entries at leaves only): the X-list leaves of the leaf and
                            // of its ancestors with at most x_direct_max targets, whose sources
                            // the leaf evaluation sums directly at the leaf's targets
    int64_t n_xd = 0;
    DevBuf v_off, v_idx;  // V: children of the parent's colleagues, not adjacent
    // V pairs grouped by direction (for the M2L product)
    DevBuf vp_src, vp_trg;  // int [n_v]
    std::vector<int> vdir_off;  // host: 317 offsets into the grouped V pairs
    DevBuf leaves;              // int [n_leaves]: leaf box indices
    DevBuf xboxes;              // int: boxes with a non-empty X list
    int n_xboxes = 0;
    DevBuf wboxes;              // int: boxes that appear in some W list
    int n_wboxes = 0;
    // octant groups per level for M2M / L2L: children at level l with octant o
    DevBuf oct_child;           // int: grouped child indices
    std::vector<int> oct_off;   // host: [(n_levels) * 8 + 1] offsets (level-major, then octant)
    int64_t n_u = 0, n_v = 0, n_w = 0, n_x = 0;
    int64_t p2p_pairs = 0, l2p_pairs = 0, p2l_pairs = 0;
    bool counts_valid = false;  // the three counts above are made on request
    // a W-list box with at most this many sources is evaluated directly at the targets (exact
    // and cheaper than its n_surf equivalent points); larger ones through their densities
    int w_direct_max = 0;
    int x_direct_max = 0;  // a box with an X list and at most this many targets skips P2L
    int split_grid = 0;  // blocks of the cooperative split launch (all resident)
    // periodic tree: the root is the cell, colleagues and lists wrap around it (list entries
    // carry the image of their box), and the cell's far images act through the lattice operator
    bool periodic = false;
    float cell = 0.f;  // cell side (the shift of an image by one cell)
};

// Per-evaluation work arrays.
struct Work {
    DevBuf src_rec;   // packed, pre-scaled source records in sorted order
    DevBuf up_chk;    // float [n_boxes][3n]   upward check potentials (leaves)
    DevBuf alpha;     // float [n_boxes][ku]   upward densities in the singular basis
    DevBuf psi;       // float [n_boxes][rank] M2L inputs
    DevBuf psi2;      // bf16 [n_boxes][2][rank] their split pairs (tensor-core M2L)
    DevBuf cdn;       // float [n_boxes][rank] M2L outputs
    DevBuf dn_chk;    // float [n_boxes][3n]   downward check potentials (X-list boxes)
    DevBuf beta;      // float [n_boxes][kd]   downward densities in the singular basis
    DevBuf up_phi;    // float [n_boxes][3n]   upward equivalent densities (W-list boxes)
    DevBuf dn_phi;    // float [n_boxes][3n]   downward equivalent densities (leaves)
    DevBuf scan_tmp[4];  // per-level partial sums of the device scan
    DevBuf tree_tmp[16]; // tree-build temporaries (sort ping-pong, histograms, child ranges...)
    DevBuf stage_in[4];  // staging of host inputs
    DevBuf stage_out;
    DevBuf tmp;
    DevBuf hi_rec;       // source records of the compensated direct sum (direct_hi.cu)
    DevBuf hi_part;      // its per-block coordinate bounds
    DevBuf td_stress;    // stresses behind a KFMM_TD evaluation
    DevBuf net_force;    // double [ncol][3]: net single-layer force of a periodic sum
    // box-vector buffers whose padding lanes are known to be zero: their allocations and the
    // density-column layout they were zeroed for
    void *zero_ptr[8] = {};
    int zero_ld[8] = {};
    int zero_ncol = 0, zero_nb = 0;
};

// Pinned host memory for tables built on the host and copied to the device in stream order,
// without a synchronisation per copy.  Space is handed out in order and given back by reset(),
// which is called only right after a synchronisation of the context stream (all copies done).
struct Staging {
    struct Chunk {
        void *p = nullptr;
        size_t bytes = 0;
    };
    std::vector<Chunk> chunks;
    size_t cur = 0, used = 0;
    Staging() = default;
    Staging(const Staging &) = delete;
    Staging &operator=(const Staging &) = delete;
    void *take(size_t n) {
        n = (n + 15) & ~(size_t)15;
        while (cur < chunks.size() && used + n > chunks[cur].bytes) {
            ++cur;
            used = 0;
        }
        if (cur == chunks.size()) {
            Chunk c;
            c.bytes = n > ((size_t)4 << 20) ? n : ((size_t)4 << 20);
            if (cudaMallocHost(&c.p, c.bytes) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            chunks.push_back(c);
            used = 0;
        }
        void *r = (char *)chunks[cur].p + used;
        used += n;
        return r;
    }
    void reset() {
        cur = 0;
        used = 0;
    }
    ~Staging() {
        for (Chunk &c : chunks) cudaFreeHost(c.p);
    }
};

// Tile tables of the grouped gather-GEMM, built once per tree.
struct GemmPlan {
    DevBuf tiles;  // int4 {matrix index, first column, end column, density column}
    int n_tiles = 0;      // device tiles: host tiles x ncol
    int ncol = 1;         // density columns the device tiles and items were made for
    std::vector<int4> host_tiles;  // one density column: {matrix, first, end, 0}
    // tensor-core work items {column * n_mat + matrix, row tile, first column, end column}, by
    // row-tile count
    DevBuf tc_items[9];
    int n_tc_items[9] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
};

struct FmmPlans {
    bool valid = false;
    GemmPlan all, leaves, xboxes, wboxes, m2l;
    std::vector<GemmPlan> oct_lvl;  // per level: children grouped by octant (M2M, L2L)
    DevBuf geom;                    // float4 per box: centre x, y, z and half-width
    DevBuf m2l_items;               // int4 {column * 316 + direction, row tile, c0, c1} (tensor-core M2L)
    int n_m2l_items = 0;
    std::vector<int4> m2l_host;     // one density column
    int m2l_ncol = 1;
    DevBuf err;                     // int: set by kernels whose bounded waits gave up
    // leaf-evaluation work items, int4 {leaf box, first target, first segment, end segment}:
    // one list over all segments, or (eval_split) a near list (P2P: U leaves and direct W
    // boxes) followed by a far list (L2P and M2P), launched separately
    DevBuf eval_items;
    DevBuf eval_cnt;                // int per leaf and list: items, then their offsets
    int n_eval_items = 0, n_eval_far = 0;
    bool eval_split = false;
    // item totals of a new tree, copied asynchronously to pinned memory (event ev_items)
    bool items_pending = false;
    int *items_host = nullptr;
    cudaEvent_t ev_items = nullptr;
};

// Per-phase CUDA-event timing (off unless enabled).
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    struct Pending {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    double ms[KFMM_N_PHASES] = {0};
    int64_t count[KFMM_N_PHASES] = {0};
    cudaEvent_t take() {
        if (pool.empty()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    ~Profiler() {
        for (auto &p : pending) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

}  // namespace kfmm

namespace kfmm {
// A captured evaluation (CUDA graph) and the arguments it was captured with.
struct EvalGraph {
    const void *sl = nullptr, *dl = nullptr;
    void *out = nullptr;
    int ncol = -1, kind = -1;
    int seen = 0;          // evaluations with these arguments since the last reset
    bool valid = false;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    int64_t launches = 0;  // kernels in the graph
    void reset();
};
}  // namespace kfmm

struct kfmm_ctx {
    kfmm_options opt;
    kfmm::EvalGraph graph;
    // launch shapes tuned on the first evaluation (kept across builds)
    struct Tune {
        bool eval_done = false, m2l_done = false;
        float eval_cost = 1024.f;  // cap of a leaf-evaluation work item, warp pair-steps
        int m2l_chunk = 1024;      // columns per M2L work item
    } tune;
    cudaStream_t stream = nullptr;
    kfmm::Staging staging;  // pinned host side of the in-order table uploads
    // second stream of the overlapped evaluation and its fork/join events (made on first use)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_p2l = nullptr, ev_near = nullptr, ev_plans = nullptr;
    double G = 1.0, nu = 0.3;
    // periodic cell (kfmm_set_periodic): lower corner and side; applies to the next build
    bool periodic = false;
    double cell_lo[3] = {0, 0, 0}, cell_side = 1.0;
    std::string err;
    kfmm::Operators ops;
    kfmm::Tree tree;
    kfmm::Work work;
    kfmm::FmmPlans plans;
    kfmm::Profiler prof;
    int cur_phase = -1;
    cudaEvent_t cur_ev = nullptr;
    int64_t n_launch = 0;  // kernels launched by this context since creation
    int n_sms = 152;       // multiprocessors of opt.device (queried at create; sizes grids)
    // Close the open phase (if any) and open phase `ph` (ph < 0: only close).
    void phase(int ph) {
        if (!prof.on) return;
        if (cur_phase >= 0) {
            cudaEvent_t e = prof.take();
            cudaEventRecord(e, stream);
            prof.pending.push_back({cur_phase, cur_ev, e});
            cur_ev = nullptr;
        }
        if (ph >= 0) {
            cur_ev = prof.take();
            cudaEventRecord(cur_ev, stream);
        }
        cur_phase = ph;
    }

    kfmm_status fail(kfmm_status code, const std::string &msg) {
        if (err.empty() || code != KFMM_OK) err = msg;
        return code;
    }
};

namespace kfmm {
// tree.cu
kfmm_status build_tree(kfmm_ctx *ctx, const float *src_xyz, const float *src_nrm, int64_t nsrc,
                       const float *trg_xyz, int64_t ntrg);
// independent point sets (offsets [n_sets + 1] on the host, points concatenated on the device)
kfmm_status build_forest(kfmm_ctx *ctx, int n_sets, const int64_t *src_off, const float *src_xyz,
                         const float *src_nrm, const int64_t *trg_off, const float *trg_xyz);
kfmm_status tree_work_counts(kfmm_ctx *ctx);  // interaction counts for the statistics
// precompute.cpp (host, FP64) + upload
kfmm_status ensure_operators(kfmm_ctx *ctx);
// fmm.cu
kfmm_status fmm_eval(kfmm_ctx *ctx, const float *sl, const float *dl, int ncol, int kind, float *out);
// D^T and energy density per target and column from stresses [n][6 ncol] -> out [n][2 ncol]
kfmm_status fmm_td(kfmm_ctx *ctx, const float *stress, int64_t n, int ncol, float *out);
kfmm_status selftest_bounded_wait(kfmm_ctx *ctx, long long polls);
// direct.cu
kfmm_status direct_sum(kfmm_ctx *ctx, int precision, const void *trg, int64_t ntrg, const void *src,
                       const void *nrm, int64_t nsrc, const void *sl, const void *dl, int kind, void *out);
// direct_hi.cu: FP64-grade displacement sum at FP32 rate (FP64 arrays, device pointers)
kfmm_status direct_hi_sum(kfmm_ctx *ctx, const double *trg, int64_t ntrg, const double *src, const double *nrm,
                          int64_t nsrc, const double *sl, const double *dl, double near_radius, double *out);
// peak.cu: measured FP32 FMA throughput (TFLOP/s) and the kernel's time
kfmm_status measure_fp32_peak(kfmm_ctx *ctx, double *tflops, double *ms);
// api.cu helpers
// Device (or managed) memory, as opposed to host memory.
bool is_device_ptr(const void *p);
// Device memory that belongs to a GPU other than the current one: the entry points reject it
// (a kernel here would read another GPU's memory without peer access).
bool foreign_device_ptr(const void *p);
// The first non-null pointer of `ptrs` that foreign_device_ptr() flags, or nullptr.
const void *first_foreign(std::initializer_list<const void *> ptrs);
}  // namespace kfmm
