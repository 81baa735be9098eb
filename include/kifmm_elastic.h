/*
 * kifmm_elastic.h -- C ABI of the GB300 (sm_103a) kernel-independent FMM for the 3D Kelvin
 * elasticity boundary-integral operators, and of the collocation BEM built on it.
 *
 * Method: arXiv 1612.04082, "What Lies Beneath the Surface: Topological-Shape Optimization
 * With the Kernel-Independent Fast Multipole Method".
 *
 * General conventions (every entry point):
 *  - Return value: KFMM_OK (0) or a negative kfmm_status.  No exception crosses the ABI.
 *    On error kfmm_last_error(ctx) holds a one-line message.  Outputs are unspecified
 *    after an error unless the entry point says otherwise.
 *  - Array arguments are plain pointers that may point to device memory of the context's GPU
 *    or to host memory (pageable or pinned); the library inspects each pointer and stages
 *    host arrays through its own device buffers.  Device memory of another GPU is rejected
 *    with KFMM_ERR_INVALID_ARG.  The caller owns every array passed in; each must stay valid
 *    for the duration of the call.  The library owns only its internal buffers (tree,
 *    operators, workspaces), released by the matching *_destroy.
 *  - Layouts are row-major arrays of structures: points [n][3] (x, y, z); 3-vector densities
 *    [n][3 * ncol] (column c occupies entries 3c .. 3c+2 of each row); displacements
 *    [n][3 * ncol]; stresses [n][6 * ncol] in the order xx, yy, zz, yz, xz, xy.
 *  - Work is enqueued on the context's CUDA stream (kfmm_set_stream; default: the legacy
 *    default stream).  Entry points that return data to host pointers, or that need a count
 *    on the host (tree build, GMRES convergence tests), synchronise that stream.
 *  - Kernels follow the paper's Eq. disp_1 (U, single layer, "SL"), Eq. disp_2 (P, double
 *    layer, "DL"; normal at the source, pointing out of the material), Eq. stress_2 (D) and
 *    Eq. stress_3 (S, with the factor G).  With d = x_target - y_source every kernel is 0
 *    at d = 0 (coincident points are skipped, as in the direct sum of Eq. fmm_summation).
 *      DISP   (3 outputs): out_i = sum_j U(d) sl_j + P(d, n_j) dl_j
 *      STRESS (6 outputs): out_i = sum_j D(d) sl_j + S(d, n_j) dl_j   (Hooke of grad DISP)
 *    so the interior displacement of the BIE is DISP(sl = t w, dl = -u w) and Eq. stress_1
 *    (Somigliana) is STRESS(sl = t w, dl = -u w) for quadrature weights w.
 */
#ifndef KIFMM_ELASTIC_H
#define KIFMM_ELASTIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum kfmm_status {
    KFMM_OK = 0,
    KFMM_ERR_INVALID_ARG = -1,    /* bad size, NULL where an array is required, NaN input   */
    KFMM_ERR_OOM = -2,            /* device or host allocation failed                        */
    KFMM_ERR_CUDA = -3,           /* a CUDA runtime call or kernel launch failed             */
    KFMM_ERR_NOT_CONVERGED = -4,  /* iterative solve stopped at its iteration cap            */
    KFMM_ERR_DEVICE_TIMEOUT = -5, /* a bounded device-side wait gave up                      */
    KFMM_ERR_NOT_BUILT = -6,      /* kfmm_eval before kfmm_build, or BEM use before set-up   */
    KFMM_ERR_INTERNAL = -7        /* an internal consistency check failed                    */
} kfmm_status;

typedef enum kfmm_kind {
    KFMM_DISP = 0,   /* 3 outputs per target and column: SL (Eq. disp_1) + DL (Eq. disp_2) */
    KFMM_STRESS = 1, /* 6 outputs per target and column: Eq. stress_2 + Eq. stress_3        */
    KFMM_TD = 2      /* 2 outputs per target and column from that stress sigma: the
                        topological derivative of the compliance, Eq. deriv,
                        D^T = 3 (1-nu) / (4 E (7-5nu)) [10 (1+nu) sigma:sigma - (1+5nu) (tr sigma)^2],
                        and the energy density 1/2 sigma:eps (integrand of Eq. functional);
                        with sl = t w, dl = -u w (Eq. stress_1) these are the fields of the
                        optimisation loop.  kfmm_eval only.                                  */
} kfmm_kind;

typedef enum kfmm_precision {
    KFMM_FP32 = 0,  /* FP32 arithmetic and FP32 arrays                                       */
    KFMM_FP64 = 1   /* FP64 arithmetic and FP64 arrays (direct sums only)                   */
} kfmm_precision;

/* Options of the kernel-independent FMM (Sec. "Kernel-independent fast multipole method":
 * far fields are represented by densities on equivalent surfaces, matched on check
 * surfaces; the translation operators are matrices built from the kernel alone). */
typedef struct kfmm_options {
    int p;              /* points per edge of the cube lattice whose surface carries the
                           equivalent densities: 6 (p - 1)^2 + 2 points (152 at p = 6)     */
    int leaf_cap;       /* a box is split while it holds more than leaf_cap sources or
                           targets (64)                                                     */
    int max_depth;      /* deepest octree level, <= 20 (20)                                 */
    double r_inner;     /* radius of the inner surfaces (upward equivalent, downward check),
                           in box half-widths (1.05)                                         */
    double r_outer;     /* radius of the outer surfaces (upward check, downward equivalent)
                           (2.95)                                                            */
    double pinv_rtol;   /* relative singular-value cutoff of the check-to-equivalent maps,
                           factored in FP64 (1e-7)                                           */
    double m2l_rtol;    /* relative singular-value cutoff of the shared M2L basis (3e-5);
                           the rank is rounded up to a multiple of 16; 0 keeps full rank    */
    int m2l_rank_max;   /* upper bound on the M2L rank (0 = no bound)                       */
    int m2l_tensor_cores; /* bit field of the products run on the tcgen05 tensor cores with
                           FP32 accumulation; clear bits use FP32 SIMT:
                           1 = M2L translations, BF16 split pairs (rank <= 288; up to
                           rank 208 the translation pairs are the rows of the products and
                           the whole translation stays in shared memory);
                           2 = check-to-equivalent factors, 4 = M2M and L2L,
                           8 = equivalent-density and M2L basis changes, all three with
                           three-term BF16 splits (FP32-grade);
                           16 = with 1: M2L by row tiles of the translation at every rank
                           (the kernel used above rank 208) (15)                              */
    int device;         /* CUDA device ordinal (0)                                          */
    int graphs;         /* 1: an evaluation repeated with the same arguments (e.g. the matvecs
                           of a GMRES solve) is captured once into a CUDA graph and replayed;
                           not while profiling (1)                                          */
    int autotune;       /* 1: the context's first evaluation times candidate launch shapes on
                           its tree (columns per M2L work item; cost cap of the leaf-
                           evaluation work items) and keeps the fastest for later builds (1)  */
    int streams;        /* 1: the parts of an evaluation that need no multipole data (P2L and
                           the leaf-to-leaf P2P) run on a second stream, concurrently with the
                           upward pass and M2L; not while profiling (1)                      */
    int eval_item_cost; /* cap of one leaf-evaluation work item, in warp pair-steps; > 0 fixes
                           it (and leaves it out of the tuning), 0 takes 1024 or the tuned
                           value (0)                                                         */
} kfmm_options;

/* Tree and work counts of the last kfmm_build (for tests and roofline accounting). */
typedef struct kfmm_stats {
    int64_t n_src, n_trg;
    int32_t n_boxes, n_leaves, n_levels, m2l_rank, n_surf;
    int64_t n_u_pairs;      /* (target leaf, source leaf) pairs of the U lists               */
    int64_t n_v_pairs;      /* (target box, source box) pairs of the V lists                 */
    int64_t n_w_pairs, n_x_pairs;
    int64_t p2p_interactions;  /* sum over target leaves of n_trg * (U-list sources + sources
                                  of the W-list boxes evaluated directly + sources of the
                                  X lists summed directly: those of the leaf and of its
                                  ancestors with at most n_surf / 2 targets)                  */
    int64_t s2m_interactions;  /* n_src * n_surf                                             */
    int64_t l2p_interactions;  /* n_trg * n_surf * (1 + W-list boxes evaluated through their
                                  upward densities)                                          */
    int64_t p2l_interactions;  /* sum over the X pairs of boxes with more than n_surf / 2
                                  targets of n_src(leaf) * n_surf                             */
    int64_t kernel_launches;   /* CUDA kernels this context has launched since kfmm_create   */
    int32_t up_rank, down_rank;  /* kept singular values of the upward / downward check-to-
                                    equivalent maps (0 before the first evaluation)          */
    int32_t n_xboxes, n_wboxes;  /* boxes whose X list goes through their downward check
                                    surface (more than n_surf / 2 targets); W-list boxes with
                                    their own upward density evaluated at targets            */
    int32_t m2l_chunk;           /* columns per M2L work item in use (tuned or default)     */
    float eval_item_cost;        /* cost cap of the leaf-evaluation items in use            */
    float fp32_box_ratio;        /* half-width of a box at the deepest level over the FP32
                                    spacing of the largest coordinate of its root cube (the
                                    smallest over the point sets).  Positions are FP32, so the
                                    check and equivalent surfaces of the deepest boxes sit up
                                    to 1 / ratio of a half-width off: measured 4e-4 relative
                                    error at a ratio of ~17, 1.3e-5 at 1e6 points on a 2x1x1
                                    box (ratio 16384).  Below ~100 shift the points towards
                                    the origin or expect the FMM error to grow.                */
} kfmm_stats;

typedef struct kfmm_ctx kfmm_ctx;

/* Fill *opt with the defaults listed above. */
void kfmm_default_options(kfmm_options *opt);

/* Create a context on opt->device (opt may be NULL for defaults).  Material defaults to
 * G = 1, nu = 0.3.  The FP64 operator precompute runs at the first build for a material. */
kfmm_status kfmm_create(kfmm_ctx **out, const kfmm_options *opt);
kfmm_status kfmm_destroy(kfmm_ctx *ctx);

/* Bulk modulus K and shear modulus G of Eq. elast; nu = (3K - 2G) / (2 (3K + G)).
 * Requires K > 0, G > 0 (so -1 < nu < 1/2). */
kfmm_status kfmm_set_material(kfmm_ctx *ctx, double K, double G);

/* Periodic sums over a cubic cell (Sec. "Periodic cell of a metamaterial": the integrals run
 * over the infinite periodic surface, and the FMM tree is periodic at every level).  With
 * on != 0 the next kfmm_build uses the cube [lo, lo + side]^3 as its root, every point must
 * lie in it (to 1e-6 of side), the interaction lists wrap around the cell and every list
 * entry names the image of its box that it means; the cell's images beyond the root's 26
 * neighbours act on the root's downward density through a lattice operator made once per
 * operator set (FP64 host precompute, Ewald's split).  kfmm_eval then returns
 *   sum over n in Z^3 of sum_j K(x_i - y_j - n side) den_j
 * in the sense of the Fourier series without its k = 0 term: the field has zero mean over the
 * cell, and a net force of the single layer is balanced by a uniform body force.  A target
 * on a source skips that source only (its other images count).  The displacement sum is
 * defined up to a constant vector per column (a rigid translation of the periodic field), and
 * the FMM fixes that constant otherwise than by the zero mean: its lattice operator acts on
 * the root's equivalent density, which reproduces the cell's field outside the root but not
 * its cell mean.  Stresses (and TD) carry no constant.  Not with kfmm_build_sets (one cell
 * per tree).  on = 0 returns to free space; either way the tree must be built again.
 * lo: 3 doubles (may be NULL with on = 0); side > 0. */
kfmm_status kfmm_set_periodic(kfmm_ctx *ctx, int on, const double *lo, double side);

/* Enqueue all later work of this context on `stream` (a cudaStream_t; NULL = default). */
kfmm_status kfmm_set_stream(kfmm_ctx *ctx, void *stream);

/* Octree build for the sum of Eq. fmm_summation (Sec. "Kernel-independent fast multipole
 * method", first step): Morton keys in the bounding cube, radix sort, split while a box
 * holds more than leaf_cap points, U/V/W/X interaction lists.  src_xyz [nsrc][3],
 * src_nrm [nsrc][3] (may be NULL when no double-layer density will be passed),
 * trg_xyz [ntrg][3], FP32.  nsrc, ntrg >= 1 and all coordinates finite.  The tree and the
 * sorted copies of the points are kept until the next build or destroy. */
kfmm_status kfmm_build(kfmm_ctx *ctx, const float *src_xyz, const float *src_nrm, int64_t nsrc,
                       const float *trg_xyz, int64_t ntrg);

/* One build over n_sets independent point sets (a batch of surfaces of uneven size): set k
 * owns sources src_off[k] .. src_off[k+1] - 1 and targets trg_off[k] .. trg_off[k+1] - 1 of
 * the concatenated arrays (offsets: n_sets + 1 host int64 values from 0, every set at least
 * one source and one target; 1 <= n_sets <= 65535).  Each set gets its own root cube (one level-0 box); no list
 * crosses sets, so kfmm_eval computes Eq. fmm_summation within every set, all sets in the
 * same launches.  The set index leads every Morton key, so the depth is capped at
 * (64 - ceil(log2 n_sets)) / 3 levels.  kfmm_build is the case n_sets = 1. */
kfmm_status kfmm_build_sets(kfmm_ctx *ctx, int32_t n_sets, const int64_t *src_off, const float *src_xyz,
                            const float *src_nrm, const int64_t *trg_off, const float *trg_xyz);

/* One FMM evaluation of Eq. fmm_summation on the built tree: sl_den, dl_den [nsrc][3*ncol]
 * (either may be NULL, not both), out [ntrg][3*ncol] (DISP), [ntrg][6*ncol] (STRESS) or
 * [ntrg][2*ncol] (TD: D^T then energy density per column), FP32, overwritten.  ncol in
 * 1..32. */
kfmm_status kfmm_eval(kfmm_ctx *ctx, const float *sl_den, const float *dl_den, int ncol, int kind,
                      float *out);

/* The same sum by all-pairs direct summation (no tree), in FP32 or FP64 (`precision`):
 * arrays are float or double accordingly.  out is overwritten.  Used for small problems,
 * the dense-equivalent BEM and as the GPU reference of the near field. */
kfmm_status kfmm_direct(kfmm_ctx *ctx, int precision, const void *trg_xyz, int64_t ntrg,
                        const void *src_xyz, const void *src_nrm, int64_t nsrc, const void *sl_den,
                        const void *dl_den, int kind, void *out);

/* The displacement sum of kfmm_direct (DISP kind) to FP64-grade accuracy at FP32 arithmetic
 * rate, for the outer residual of mixed-precision GMRES (the system of Eq. num2, solved by
 * GMRES as in Sec. "Numerical solution").  Such a residual b - A x cancels: its terms exceed
 * the result by a factor ||A| |x|| / ||b|| of ~100 on a clamped cantilever, so a relative
 * residual of 1e-6 needs the operator to ~1e-9 of its terms, beyond FP32 and too slow in
 * FP64 on this GPU (1/64 of the FP32 rate).  Arithmetic: points split into FP32 hi + lo
 * parts so that every difference x - y is exact to FP32 rounding of the difference itself;
 * the sum carried as four partial sums free of material constants, which are applied in
 * FP64 per target; FP32 partial sums folded into FP64 every 128 sources; 1/r refined by one
 * Newton-Raphson step; pairs closer than near_radius (the largest terms) evaluated wholly in
 * FP64.  What is left is the random rounding of the far pairs' FP32 kernel evaluation.
 *  - All arrays FP64: trg_xyz [ntrg][3], src_xyz [nsrc][3], src_nrm [nsrc][3] (required with
 *    dl_den), sl_den, dl_den [nsrc][3] (either may be NULL, not both), out [ntrg][3]
 *    (overwritten); host or device memory as for every entry point.
 *  - near_radius >= 0 (same length unit as the points): pairs with |x - y| < near_radius use
 *    FP64 throughout.  The remaining pairs' FP32 rounding (~4e-7 of each term, of either
 *    sign) adds up to ~1e-8 of the sum on smooth densities over a surface (measured), where
 *    plain FP32 summation is off by ~1e-6; the BEM layer passes four times its longest
 *    element edge.
 *    Coincident points (r = 0) are skipped, as in every sum here.
 *  - The context's material (kfmm_set_material) applies; no tree is needed.  Work is enqueued
 *    on the context stream; the call synchronises only when it staged host arrays. */
kfmm_status kfmm_direct_hi(kfmm_ctx *ctx, const double *trg_xyz, int64_t ntrg, const double *src_xyz,
                           const double *src_nrm, int64_t nsrc, const double *sl_den, const double *dl_den,
                           double near_radius, double *out);

/* The same all-pairs sum as kfmm_direct, for callers that cannot allocate device memory:
 * a process whose device memory is already handed to a caching allocator (a new
 * cudaMalloc would fail), or code that must not call cudaMalloc / cudaFree while it runs
 * because those calls synchronise the device.  The paper has no counterpart of this entry
 * point; it is a deployment variant.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.  The sum is
 *    split over source slices whose partial results go to one fixed 16 MiB scratch array
 *    in device memory, reserved on every GPU that loads the library until process exit.
 *  - Every array (trg_xyz, src_xyz, src_nrm, sl_den, dl_den, out) must be device memory of
 *    the context's GPU; host pointers and other GPUs' memory are rejected with
 *    KFMM_ERR_INVALID_ARG (staging them would allocate).
 *  - Limit: ntrg * (3 for DISP, 6 for STRESS) * (4 for FP32, 8 for FP64) bytes must not
 *    exceed 16 MiB (e.g. 699,050 FP32 or 349,525 FP64 displacement targets); larger
 *    sizes are rejected with KFMM_ERR_INVALID_ARG.  nsrc is not limited.
 *  - The first call on a device looks up the scratch array's device address (once per
 *    device, with that device current); make that first call before any stream capture.
 *    The cached address is not valid across cudaDeviceReset (the module is loaded again).
 *  - All calls share the scratch array, which keeps the last call's contents; each call
 *    writes every entry it reads.  Calls that overlap on the GPU (other streams, other host
 *    threads) race on it: the caller must serialise them.
 *  - Work is enqueued on the context stream; the call does not synchronise. */
kfmm_status kfmm_direct_noalloc(kfmm_ctx *ctx, int precision, const void *trg_xyz, int64_t ntrg,
                                const void *src_xyz, const void *src_nrm, int64_t nsrc,
                                const void *sl_den, const void *dl_den, int kind, void *out);

kfmm_status kfmm_get_stats(const kfmm_ctx *ctx, kfmm_stats *st);

/* Copies of the built tree for inspection (host arrays sized from kfmm_get_stats):
 * box_level [n_boxes], box_anchor [n_boxes][3] (integer box coordinates at its level),
 * box_parent [n_boxes], box_src [n_boxes][2] and box_trg [n_boxes][2] (ranges into the
 * sorted point order), src_perm [nsrc] and trg_perm [ntrg] (sorted position -> input index).
 * Any pointer may be NULL. */
kfmm_status kfmm_export_tree(const kfmm_ctx *ctx, int32_t *box_level, int32_t *box_anchor,
                             int32_t *box_parent, int32_t *box_src, int32_t *box_trg,
                             int32_t *src_perm, int32_t *trg_perm);

/* Interaction lists as CSR over boxes: which = 'U', 'V', 'W' or 'X'; offsets [n_boxes+1],
 * items [n_pairs] (source box indices).  Either pointer may be NULL; *n_pairs receives the
 * total.  U and W lists are defined for leaves only (empty rows elsewhere).  In a periodic
 * tree (kfmm_set_periodic) an item names an image of a box: the box index in bits 0-25 and,
 * in bits 26-30, c ^ 13 with c = 9 (sx + 1) + 3 (sy + 1) + (sz + 1) for the image moved by
 * (sx, sy, sz) in {-1, 0, 1}^3 cells (0 for the unmoved box, so free-space items are plain
 * box indices). */
kfmm_status kfmm_export_list(const kfmm_ctx *ctx, char which, int32_t *offsets, int32_t *items,
                             int64_t *n_pairs);

/* ------------------------------------------------------------------------------------
 * Partition over several GPUs (Sec. "Numerical solution": the evaluation is parallelised by
 * giving each process a part of the octree).  Host code on a tree given as host arrays --
 * the arrays of kfmm_export_tree and kfmm_export_list for a built free-space tree; boxes are
 * listed coarse to fine (a parent before its children).  No GPU is needed.
 * ------------------------------------------------------------------------------------ */
typedef struct kfmm_tree_view {
    int32_t n_boxes;
    const int32_t *level;    /* [n_boxes] octree level (0 = a root)                          */
    const int32_t *anchor;   /* [n_boxes][3] integer box coordinates at its level            */
    const int32_t *parent;   /* [n_boxes], -1 at a root                                      */
    const int32_t *box_src;  /* [n_boxes][2] source range [begin, end) in the sorted order   */
    const int32_t *box_trg;  /* [n_boxes][2] target range                                    */
    const int32_t *u_off, *u_idx, *v_off, *v_idx, *w_off, *w_idx, *x_off, *x_idx;  /* lists,
                                CSR by target box (the U, V, W, X lists of the build)       */
} kfmm_tree_view;

/* Cost-weighted partition: the leaves in Morton order (led by their root for independent
 * point sets) are cut into n_ranks contiguous ranges of about equal cost; box_cost [n_boxes]
 * gives each leaf's cost (NULL: targets x U-list sources + sources + targets + 1).  Outputs:
 * box_owner [n_boxes] = the rank of a leaf, the rank of a box whose leaves all belong to one
 * rank, -1 for a box shared by several ranks (the coarse levels); leaf_order [n_leaves] (may
 * be NULL) = the leaves in Morton order; rank_cost [n_ranks] (may be NULL) = each rank's
 * total cost. */
kfmm_status kfmm_shard_plan(const kfmm_tree_view *t, int32_t n_ranks, const double *box_cost, int32_t *box_owner,
                            int32_t *leaf_order, double *rank_cost);

/* Locally essential tree of `rank` under the partition box_owner: for its leaves and their
 * ancestors (the boxes whose downward densities it forms), the boxes whose data come from
 * elsewhere, each list in increasing box order:
 *   src_boxes    -- leaves of U (its leaves) and X lists owned by another rank: their points
 *                   and densities are received;
 *   up_boxes     -- boxes of V lists and W (its leaves) owned by another rank: their upward
 *                   equivalent densities are received;
 *   shared_boxes -- shared boxes (owner -1) in those lists or among its ancestors: their
 *                   upward densities are the sum of every rank's part (all-reduce).
 * On entry *n_src, *n_up, *n_shared are the capacities of the arrays (arrays may be NULL to
 * count only); on return the counts (KFMM_ERR_INVALID_ARG if an array was too small). */
kfmm_status kfmm_shard_let(const kfmm_tree_view *t, const int32_t *box_owner, int32_t rank, int32_t *src_boxes,
                           int64_t *n_src, int32_t *up_boxes, int64_t *n_up, int32_t *shared_boxes,
                           int64_t *n_shared);

/* Phases timed when profiling is on (CUDA events on the context stream around each phase). */
typedef enum kfmm_phase {
    KFMM_PH_TREE = 0,     /* kfmm_build: bounding cube, Morton keys, sort, sorted points   */
    KFMM_PH_PACK = 1,     /* source records (sorted, pre-scaled densities)                 */
    KFMM_PH_S2M = 2,      /* sources -> upward check surfaces of the leaves                 */
    KFMM_PH_UP_PINV = 3,  /* upward check -> upward equivalent densities (leaves)          */
    KFMM_PH_M2M = 4,      /* child -> parent upward densities, bottom-up                   */
    KFMM_PH_M2L = 5,      /* V-list translation (M2L) in the shared basis                  */
    KFMM_PH_P2L = 6,      /* X-list sources -> downward check surfaces                      */
    KFMM_PH_DOWN = 7,     /* downward densities and L2L, top-down                          */
    KFMM_PH_EVAL = 8,     /* leaf evaluation: L2P + M2P (W list) + P2P (U list)             */
    KFMM_PH_M2L_BASIS = 9, /* upward densities into the shared M2L basis (compression)       */
    KFMM_PH_TREE_SPLIT = 10, /* kfmm_build: boxes level by level, leaves, colleagues         */
    KFMM_PH_TREE_LISTS = 11, /* kfmm_build: U, V, W, X lists, V directions, box groups       */
    KFMM_PH_PLANS = 12,   /* first evaluation on a new tree: the host part of its work plans  */
    KFMM_N_PHASES = 13
} kfmm_phase;

/* Turn per-phase timing on or off (off by default).  Timing adds two event records per
 * phase and changes no result. */
kfmm_status kfmm_set_profiling(kfmm_ctx *ctx, int enable);

/* Milliseconds and call counts per phase accumulated since the last reset (arrays of
 * KFMM_N_PHASES; either may be NULL).  Synchronises the context stream.  reset != 0 clears
 * the accumulators after reading. */
kfmm_status kfmm_get_phase_times(kfmm_ctx *ctx, double *ms, int64_t *counts, int reset);

const char *kfmm_status_str(kfmm_status s);
const char *kfmm_last_error(const kfmm_ctx *ctx);

/* Measured FP32 FMA throughput of the context's GPU, the peak the pair-evaluation kernels
 * (Eq. fmm_summation's near field and the check-surface sums) are bounded by: 8 CTAs of
 * 256 threads per multiprocessor, each thread 8 independent chains of dependent FMAs
 * (2 flop each); the fastest of 5 timed launches after one warm-up, timed with CUDA events
 * on the context stream.  *tflops receives TFLOP/s, *ms (may be NULL) the launch time,
 * *n_sms (may be NULL) the multiprocessor count.  Synchronises the context stream. */
kfmm_status kfmm_measure_fp32_peak(kfmm_ctx *ctx, double *tflops, double *ms, int32_t *n_sms);

/* Failure-detection check of the bounded device waits: one thread waits on a shared-memory
 * mbarrier that nothing arrives on, polling at most `polls` times (1..2^24) with the wait
 * the tensor-core kernels use, then records the time-out in the context's device error
 * word, which the host reads back as those kernels' errors are read.  Returns
 * KFMM_ERR_DEVICE_TIMEOUT, as designed (KFMM_OK would mean the wait completed); nothing
 * faults or hangs and the context stays usable. */
kfmm_status kfmm_selftest_bounded_wait(kfmm_ctx *ctx, int64_t polls);

/* ====================================================================================== */
/* Collocation BEM on the FMM (Eq. BIE; Eq. num, coef, num2; Sec. "Matrix-vector products") */
/* ====================================================================================== */
/* Piecewise-constant u and t on flat triangles, collocation at the centroids.  Off-diagonal
 * blocks use the 16-point rule (4 midpoint sub-triangles x the 4-node degree-3 rule:
 * centroid weight -27/48, (3/5,1/5,1/5) weights 25/48); the matvec is the paper's two-pass
 * scheme: one fast summation over all quadrature sources (weights = element value x area x
 * rule weight, targets = centroids), then a local pass per element that removes its own
 * quadrature terms and adds the analytic singular integrals.  Diagonal blocks: int U over
 * the flat triangle in closed form (polar coordinates about the centroid) and the principal
 * value of int P, whose only in-plane term is (1-2nu)/(8 pi (1-nu)) (r_,i n_j - r_,j n_i)/r^2.
 *
 * The boundary operator is M(u, t) = 1/2 u + P^D u - U^D t at the collocation points (Eq. num);
 * for mixed conditions (Eq. num2) the unknowns x are, per element and component, t where
 * the displacement is prescribed and u where the traction is prescribed: A x = M(x_u, x_t),
 * B y = -M(y_u, y_t).  Arrays of the BEM layer are FP64 [nt][3] unless stated. */
typedef struct bem_ctx bem_ctx;

typedef enum bem_operator {
    BEM_FMM = 0,         /* FP32 KIFMM summation (SL + DL) + FP64 local pass               */
    BEM_DIRECT_FP64 = 1, /* FP64 all-pairs summation on the GPU + FP64 local pass (O(N^2)) */
    BEM_DIRECT_HI = 2    /* compensated all-pairs summation (kfmm_direct_hi: FP64-grade at
                            FP32 rate, O(N^2)) + FP64 local pass                           */
} bem_operator;

typedef struct bem_solve_opts {
    double tol;        /* stop at ||b - A x|| / ||b|| <= tol (1e-6)                           */
    int restart;       /* GMRES restart length (30; <= 200)                                  */
    int maxit;         /* cap on inner GMRES iterations in total (1000)                      */
    const double *x0;  /* initial guess of the unknowns [nt][3], or NULL for zero; a guess
                          whose residual exceeds ||b|| is dropped for zero                    */
    int refine;        /* 0: GMRES on the context's operator.  1 or 2 (FMM contexts): mixed-
                          precision iterative refinement -- right-hand side, outer residuals
                          and updates in FP64 with an FP64-grade all-pairs operator (1: the
                          compensated sum of kfmm_direct_hi; 2: the FP64 direct sum), each
                          correction by GMRES on the FP32 FMM operator (0)                    */
    double inner_tol;  /* relative tolerance of each refinement correction, loosened to what
                          the outer tolerance still needs near the end (1e-3)                 */
    int max_outer;     /* cap on refinement steps (30)                                       */
} bem_solve_opts;

typedef struct bem_stats {
    int iters;        /* inner GMRES iterations                                             */
    int matvecs;      /* FMM operator applications (including residual checks)              */
    int converged;    /* 1 if the tolerance was met                                          */
    double relres;    /* final true relative residual ||b - A x|| / ||b|| (with refinement:
                         against the FP64-grade direct operator)                             */
    double seconds;   /* wall time of bem_solve                                              */
    int outer;        /* refinement steps (1 without refinement)                            */
    int matvecs_hi;   /* FP64-grade direct operator applications (refinement)               */
    double x0_relres; /* ||b - A x0|| / ||b|| of the initial guess (1 for zero; a value > 1
                         means the guess was dropped for zero)                               */
} bem_stats;

void bem_default_solve_opts(bem_solve_opts *o);

/* Triangulated boundary: verts [nv][3] FP64, tris [nt][3] int32 (vertex order gives the
 * normal by the right-hand rule; it must point out of the material).  `op` is a
 * bem_operator.  opt as for kfmm_create (NULL = defaults), except that leaf_cap = 0 (and
 * opt = NULL) lets the BEM pick its leaf caps: for the boundary sums, with autotune on, the
 * fastest of 128, 256, 512 and 1024 quadrature sources per leaf, timed on the surface at the
 * first operator application (without autotune: 256 up to 2^21 sources, 512 above); 1024
 * for the interior evaluations of bem_interior / bem_topo_derivative.  Rejects zero-area
 * triangles. */
kfmm_status bem_create(bem_ctx **out, const kfmm_options *opt, int op, const double *verts, int64_t nv,
                       const int32_t *tris, int64_t nt);
kfmm_status bem_destroy(bem_ctx *b);
kfmm_status bem_set_material(bem_ctx *b, double K, double G);
kfmm_status bem_set_stream(bem_ctx *b, void *stream);

/* Quadrature of the triangles next to a collocation point (Sec. "Matrix-vector products":
 * the sums over triangles neighbouring the one that holds the collocation point become
 * inaccurate on fine meshes, which an upsampled quadrature fixes).  near_levels = 1: every
 * off-diagonal block uses the 16-point rule (4 midpoint sub-triangles x the 4-node rule;
 * the default).  near_levels = s in 2..5: the blocks of triangles sharing a vertex with the
 * collocation triangle use the 4-node rule on 4^s sub-triangles (64, 256, 1024, 4096
 * points); the summation keeps the 16-point sources and the local pass adds, per
 * (triangle, neighbour) pair, the FP64 difference of the two rules.  Takes effect at the
 * next operator application. */
kfmm_status bem_set_quadrature(bem_ctx *b, int near_levels);

/* Periodic boundary sums (Sec. "Periodic cell of a metamaterial"): the surface is the part in
 * one cell [lo, lo + side]^3 of an infinite periodic surface, and every sum of the operator
 * runs over the whole lattice (kfmm_set_periodic on the BEM's FMM contexts; the solution of
 * the periodic traction problem is fixed up to a rigid translation).  Every vertex must lie in
 * the cell.  A surface may cross the cell's faces (kfmm_voxel_surface_periodic gives such
 * surfaces their own vertices on both faces); the upsampled rule of bem_set_quadrature then
 * finds a collocation triangle's neighbours within the cell only, those across a face keep
 * the 16-point rule.  Needs the FMM operator (BEM_FMM) and a solve without refinement (the
 * refinement's outer operator is a free-space direct sum).  on = 0 returns to free space.
 * Takes effect at the next operator application. */
kfmm_status bem_set_periodic(bem_ctx *b, int on, const double *lo, double side);

/* A uniform stress per load case, stress6 [ncol][6] (xx, yy, zz, yz, xz, xy; NULL clears),
 * added to the stresses of bem_topo_derivative before the TD and the energy density: the
 * homogeneous part sigma^h of a periodic cell's total stress, whose fluctuation the BEM
 * solves (Sec. "Periodic cell of a metamaterial": the TD of the total stress).  ncol must
 * match the boundary solution's columns when the TD is taken; bem_interior is unaffected. */
kfmm_status bem_set_macro_stress(bem_ctx *b, const double *stress6, int ncol);

/* Boundary conditions of Eq. elast for ncol load cases (1..32) sharing one mask:
 * known_is_disp [nt][3] (uint8: 1 = u_i prescribed, 0 = t_i prescribed), values [nt][3*ncol]
 * (the prescribed u or t of load case c in entries 3c .. 3c+2 of each row).  The load cases
 * are solved together: every GMRES step sums all columns in one FMM evaluation (the six
 * unit-strain cases of a periodic-cell homogenisation are 6 columns, Sec. "Periodic cell of
 * a metamaterial"). */
kfmm_status bem_set_bc(bem_ctx *b, const uint8_t *known_is_disp, const double *values, int ncol);

/* out = M(u, t) = 1/2 u + P^D u - U^D t at the centroids (either input may be NULL = 0); one
 * column, [nt][3]. */
kfmm_status bem_apply(bem_ctx *b, const double *u, const double *t, double *out);
/* y = A x and rhs = B y of Eq. num2 for the boundary conditions set last: x, y, rhs
 * [nt][3*ncol]. */
kfmm_status bem_matvec(bem_ctx *b, const double *x, double *y);
kfmm_status bem_rhs(bem_ctx *b, double *rhs);

/* Restarted GMRES (Saad & Schultz) on A x = B y, FP64 vectors and Arnoldi (classical
 * Gram-Schmidt applied twice) on the device, all ncol load cases in lockstep: each Arnoldi
 * step applies the operator to every column at once; each column has its own Krylov basis
 * and stops extending it once it meets the tolerance.  On return u, t [nt][3*ncol] (either
 * may be NULL) hold the boundary solution, which is also kept for bem_interior.  The stats
 * report the largest relative residual over the columns and the lockstep iteration count.
 * opts->x0, when given, is [nt][3*ncol].  Returns KFMM_ERR_NOT_CONVERGED (with the last
 * iterate stored and returned) at the iteration cap. */
kfmm_status bem_solve(bem_ctx *b, const bem_solve_opts *o, double *u, double *t, bem_stats *st);

/* Store a boundary solution of ncol columns (u, t [nt][3*ncol]) without solving, e.g. from an
 * earlier solve. */
kfmm_status bem_set_solution(bem_ctx *b, const double *u, const double *t, int ncol);

/* Interior fields from the stored boundary solution (Sec. "Computing topological
 * derivatives"): displacement [n][3*ncol] by the BIE at interior points and stress
 * [n][6*ncol] by Eq. stress_1 (Somigliana), summed over the same quadrature sources, all
 * stored columns in one evaluation; either output may be NULL.  pts [n][3] FP32; outputs
 * FP32.  FMM contexts evaluate these sums with their own interior FMM at p = max(p, 8) and
 * M2L cutoff min(m2l_rtol, 1e-7): the stress sums are far-field dominated and their single-
 * and double-layer parts partly cancel. */
kfmm_status bem_interior(bem_ctx *b, const float *pts, int64_t n, float *disp, float *stress);

/* Topological derivative of the compliance (Eq. deriv) and the energy density
 * 1/2 sigma:eps (integrand of Eq. functional) at interior points, td and energy [n][ncol];
 * stress [n][6*ncol] is also returned when non-NULL.  FP32. */
kfmm_status bem_topo_derivative(bem_ctx *b, const float *pts, int64_t n, float *td, float *energy,
                                float *stress);

const char *bem_last_error(const bem_ctx *b);

/* ------------------------------------------------------------------------------------
 * Optimisation driver, host side (Sec. "Parallel optimization procedure"): voxel array
 * M(i,j,k) uint8 [nx][ny][nz] (1 = material), linear index (i*ny + j)*nz + k; host memory.
 * ------------------------------------------------------------------------------------ */

/* Boundary of the material voxels: every face between a material voxel and a void voxel or
 * the outside becomes 4 flat triangles fanned to the face centre (Sec. "Performance and
 * scalability": 24 N^2 triangles for an N^3 cube), vertex order giving the normal out of
 * the material.  Corner vertices are shared, then one centre vertex per face.  Outputs:
 * verts [nv][3] = lattice point * h + origin (origin may be NULL), tris [nt][3],
 * face_cell [nt] (linear index of the owning voxel), face_dir [nt] (0..5 = -x,+x,-y,+y,
 * -z,+z).  With all four output pointers NULL only *nv and *nt are set; otherwise *nv and
 * *nt give the capacities on entry (too small -> KFMM_ERR_INVALID_ARG with the needed
 * sizes). */
kfmm_status kfmm_voxel_surface(const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, double h,
                               const double *origin, double *verts, int64_t *nv, int32_t *tris,
                               int64_t *nt, int64_t *face_cell, int8_t *face_dir);

/* The same for one cell of a periodic voxel pattern (Sec. "Periodic cell of a metamaterial";
 * the cell is origin + [0, n h] per axis): a voxel's neighbour across a face of the array is
 * the voxel on the opposite side, so faces lie only between material and void, and a void
 * that meets a face of the cell continues across it (its triangles on both sides, with their
 * own vertices on the cell's faces).  Arguments as kfmm_voxel_surface. */
kfmm_status kfmm_voxel_surface_periodic(const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, double h,
                                        const double *origin, double *verts, int64_t *nv, int32_t *tris,
                                        int64_t *nt, int64_t *face_cell, int8_t *face_dir);

/* Hard-kill update by thresholding the topological derivative td [nx*ny*nz] over the
 * material voxels: D_C = D_min + C (D_max - D_min); material voxels with td < D_C that are
 * not frozen (frozen may be NULL) become void.  0 <= C <= 1.  *removed (may be NULL)
 * receives the count. */
kfmm_status kfmm_voxel_threshold(uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, const float *td,
                                 const uint8_t *frozen, double C, int64_t *removed);

/* Post-processing: material voxels with no material face neighbour become void, then, when
 * support is non-NULL, so does material not face-connected to a support voxel.  Support
 * voxels and keep voxels (may be NULL; e.g. the loaded ones) are never removed.  *removed
 * (may be NULL) receives the count. */
kfmm_status kfmm_voxel_clean(uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, const uint8_t *support,
                             const uint8_t *keep, int64_t *removed);

/* ------------------------------------------------------------------------------------
 * Learned warm start of the optimisation loop's GMRES solves (not in the paper, which
 * restarts every solve from zero): a multilayer perceptron from per-element features to
 * the initial guess of the element's unknowns, trained on the GPU on the (features,
 * converged unknowns) pairs of earlier iterations.  Widths n_in -> n_hidden (ReLU) x
 * (n_layers - 1) -> n_out; FP32 master weights, forward with their BF16 roundings; inputs
 * and targets standardised per column with statistics of the last training set (identity
 * before any training); loss = mean squared error; Adam (beta 0.9, 0.999).  Parameters are
 * one flat FP32 array: for each layer W [out][in] row-major, then b [out].  Arrays may be
 * host or device memory.
 * ------------------------------------------------------------------------------------ */
typedef struct kfmm_mlp kfmm_mlp;

typedef struct mlp_train_opts {
    int epochs;      /* passes over the training rows, shuffled each pass (200)        */
    int batch;       /* rows per Adam step; the last partial batch is dropped (4096)   */
    double lr;       /* Adam step size (1e-3)                                          */
    uint64_t seed;   /* shuffling seed (1612)                                           */
} mlp_train_opts;

typedef struct mlp_train_stats {
    double final_loss;  /* mean standardised squared error over the last epoch          */
    int64_t steps;      /* Adam steps taken                                             */
} mlp_train_stats;

void mlp_default_train_opts(mlp_train_opts *o);
/* He-uniform initial weights from `seed`, zero biases. */
kfmm_status mlp_create(kfmm_mlp **out, int n_in, int n_hidden, int n_layers, int n_out, uint64_t seed);
kfmm_status mlp_destroy(kfmm_mlp *m);
kfmm_status mlp_set_stream(kfmm_mlp *m, void *stream);
int64_t mlp_num_params(const kfmm_mlp *m);
/* on != 0 (default): forward and gradients use the BF16 roundings of the weights; 0: FP32. */
kfmm_status mlp_set_bf16(kfmm_mlp *m, int on);
kfmm_status mlp_get_params(const kfmm_mlp *m, float *params);
kfmm_status mlp_set_params(kfmm_mlp *m, const float *params);
kfmm_status mlp_get_normalizers(const kfmm_mlp *m, float *x_mu, float *x_sd, float *y_mu, float *y_sd);
/* Y [n][n_out] = network(X [n][n_in]) in the original (de-standardised) units. */
kfmm_status mlp_forward(kfmm_mlp *m, const float *X, int64_t n, float *Y);
/* Loss and its gradient with respect to the parameters on n <= 2^20 rows (current
 * standardisation), for gradient checks. */
kfmm_status mlp_loss_grad(kfmm_mlp *m, const float *X, const float *Y, int64_t n, double *loss, float *grad);
/* Standardisation from (X, Y), then `epochs` of shuffled mini-batch Adam. */
kfmm_status mlp_train(kfmm_mlp *m, const float *X, const float *Y, int64_t n, const mlp_train_opts *o,
                      mlp_train_stats *st);
const char *mlp_last_error(const kfmm_mlp *m);

#ifdef __cplusplus
}
#endif

#endif /* KIFMM_ELASTIC_H */
