// fmm.cu -- the evaluation pass of the kernel-independent FMM (Sec. "Kernel-independent fast
// multipole method"): upward pass (S2M, M2M), M2L on the V lists, P2L on the X lists,
// downward pass (L2L), and the leaf evaluation (L2P + M2P on the W lists + P2P on the U
// lists, the "direct summation" of the near zone).
//
// Densities on equivalent surfaces are 3-vectors of the single-layer kernel U; sources may
// carry single- and double-layer densities (Eq. fmm_summation with the normal at the source).
// The dense operators (pseudo-inverses, M2M, L2L, compressed M2L) are applied by one
// grouped gather-GEMM kernel: each column of a group is a box vector gathered by index, each
// group has its own matrix.
#include <algorithm>
#include <climits>
#include <cmath>
#include <deque>
#include <mutex>

#include "common.cuh"
#include "kelvin.cuh"
#include "precompute.h"
#include "tc_gemm.cuh"
#include "util.cuh"

namespace kfmm {

static inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// largest padded M2L rank whose operand tiles fit the shared memory of one CTA
static inline bool tc_rank_ok(int rp) { return tc::smem_bytes(rp) <= 227 * 1024; }

// raise a kernel's dynamic shared-memory limit to at least `bytes` (the limit belongs to the
// function, shared by every context of the process)
template <class K> static cudaError_t raise_smem_limit(K *kernel, int bytes)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    if (a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// round-to-nearest-even FP32 -> BF16 (finite inputs)
static inline uint16_t host_bf16(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
static inline float host_bf16_to_f32(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// tensor-core image of nmat row-major [M][K] FP64 matrices, three BF16 terms per entry
// (hi = bf16(a), mid = bf16(a - hi), lo = bf16(a - hi - mid)): [mat][mtile][kc][term][128 x KC]
static kfmm_status upload_tc_op(kfmm_ctx *ctx, Operators::TcOp &op, const double *A, int nmat, int M, int K)
{
    op.n_mat = nmat;
    op.M = M;
    op.K = K;
    op.n_mtile = (M + tc::BM - 1) / tc::BM;
    op.n_kc = (K + tc::KC - 1) / tc::KC;
    const size_t term = tc::A_TERM / 2;  // uint16 per term of a chunk
    std::vector<uint16_t> img((size_t)nmat * op.n_mtile * op.n_kc * tc::NTERM * term, 0);
    for (int g = 0; g < nmat; ++g)
        for (int mt = 0; mt < op.n_mtile; ++mt)
            for (int kc = 0; kc < op.n_kc; ++kc) {
                uint16_t *t0 = img.data() + (((size_t)g * op.n_mtile + mt) * op.n_kc + kc) * tc::NTERM * term;
                for (int i = 0; i < tc::BM; ++i) {
                    const int row = mt * tc::BM + i;
                    if (row >= M) break;
                    for (int kk = 0; kk < tc::KC; ++kk) {
                        const int k = kc * tc::KC + kk;
                        if (k >= K) break;
                        double rem = A[((size_t)g * M + row) * K + k];
                        const uint32_t off = tc::core_offset(i, kk, tc::BM) / 2;
                        for (int t = 0; t < tc::NTERM; ++t) {
                            const uint16_t h = host_bf16((float)rem);
                            t0[t * term + off] = h;
                            rem -= (double)host_bf16_to_f32(h);
                        }
                    }
                }
            }
    KF_CUDA(op.img.ensure(sizeof(uint16_t) * img.size()));
    KF_CUDA(cudaMemcpy(op.img.p, img.data(), sizeof(uint16_t) * img.size(), cudaMemcpyHostToDevice));
    op.on = true;
    return KFMM_OK;
}

// ------------------------------------------------------------------------------------
// Operators: FP64 host precompute (cached per parameter set) and FP32 upload
// ------------------------------------------------------------------------------------
namespace {
struct CacheEntry {
    host::OpsParams prm;
    host::OpsHost ops;
    std::vector<double> lat;  // far-lattice operator of a periodic root (made on first use)
};
std::mutex g_cache_mu;
std::deque<CacheEntry> g_cache;  // entries keep their addresses as the cache grows

bool same_params(const host::OpsParams &a, const host::OpsParams &b)
{
    return a.p == b.p && a.nu == b.nu && a.r_inner == b.r_inner && a.r_outer == b.r_outer &&
           a.pinv_rtol == b.pinv_rtol && a.m2l_rtol == b.m2l_rtol && a.m2l_rank_max == b.m2l_rank_max;
}

// Copy a [rows][cols] FP64 matrix into a zero-padded [rows][ld] FP32 device matrix.
kfmm_status upload_padded(kfmm_ctx *ctx, DevBuf &dst, const double *src, int nmat, int rows, int cols, int ld,
                          int rows_pad)
{
    std::vector<float> h((size_t)nmat * rows_pad * ld, 0.0f);
    for (int m = 0; m < nmat; ++m)
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c)
                h[((size_t)m * rows_pad + r) * ld + c] = (float)src[((size_t)m * rows + r) * cols + c];
    KF_CUDA(dst.ensure(sizeof(float) * h.size()));
    KF_CUDA(cudaMemcpy(dst.p, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice));
    return KFMM_OK;
}
}  // namespace

// The far-lattice operator of a periodic tree's root for the context's operators (host FP64,
// made once per operator set and kept with it in the cache), uploaded as FP32 [kd][kup].
static kfmm_status ensure_lattice(kfmm_ctx *ctx, const host::OpsParams &prm)
{
    Operators &O = ctx->ops;
    std::vector<double> R;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        CacheEntry *E = nullptr;
        for (auto &e : g_cache)
            if (same_params(e.prm, prm)) E = &e;
        if (!E) return ctx->fail(KFMM_ERR_INTERNAL, "lattice operator: operators not in the cache");
        if (E->lat.empty() && !host::compute_lattice(prm, E->ops, E->lat))
            return ctx->fail(KFMM_ERR_INTERNAL, "lattice operator precompute failed");
        R = E->lat;
    }
    KF_TRY(upload_padded(ctx, O.lat, R.data(), 1, O.kd, O.ku, round_up(O.ku, 16), O.kd));
    O.lat_ready = true;
    return KFMM_OK;
}

kfmm_status ensure_operators(kfmm_ctx *ctx)
{
    Operators &O = ctx->ops;
    host::OpsParams prm{ctx->opt.p, ctx->nu, ctx->opt.r_inner, ctx->opt.r_outer, ctx->opt.pinv_rtol,
                        ctx->opt.m2l_rtol, ctx->opt.m2l_rank_max};
    if (O.ready && O.p == prm.p && O.nu == prm.nu && O.r_inner == prm.r_inner && O.r_outer == prm.r_outer &&
        O.pinv_rtol == prm.pinv_rtol && O.m2l_rtol == prm.m2l_rtol && O.m2l_rank_max == prm.m2l_rank_max)
        return ctx->periodic && !O.lat_ready ? ensure_lattice(ctx, prm) : KFMM_OK;
    const host::OpsHost *H = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        for (auto &e : g_cache)
            if (same_params(e.prm, prm)) H = &e.ops;
        if (!H) {
            CacheEntry e;
            e.prm = prm;
            if (!host::compute_operators(prm, &e.ops))
                return ctx->fail(KFMM_ERR_INTERNAL, "operator precompute: eigensolver did not converge");
            g_cache.push_back(std::move(e));
            H = &g_cache.back().ops;
        }
    }
    const int n = H->n_surf, m = 3 * n, ld = round_up(m, 16), r = H->rank, rp = round_up(r, 16);
    (void)rp;
    {
        std::vector<float> s((size_t)n * 4, 0.f);
        for (int a = 0; a < n; ++a)
            for (int c = 0; c < 3; ++c) s[4 * a + c] = (float)H->surf[3 * a + c];
        KF_CUDA(O.surf.ensure(sizeof(float) * s.size()));
        KF_CUDA(cudaMemcpy(O.surf.p, s.data(), sizeof(float) * s.size(), cudaMemcpyHostToDevice));
    }
    const int ku = H->ku, kd = H->kd, kup = round_up(ku, 16), kdp = round_up(kd, 16);
    KF_TRY(upload_padded(ctx, O.s2a_u, H->s2a_u.data(), 1, ku, m, ld, ku));
    KF_TRY(upload_padded(ctx, O.mb, H->mb.data(), 8, ku, ku, kup, ku));
    KF_TRY(upload_padded(ctx, O.vu, H->vu.data(), 1, m, ku, kup, m));
    KF_TRY(upload_padded(ctx, O.cb, H->cb.data(), 1, r, ku, kup, r));
    KF_TRY(upload_padded(ctx, O.m2l_c, H->m2l_c.data(), 316, r, r, rp, r));
    KF_TRY(upload_padded(ctx, O.wb, H->wb.data(), 1, kd, r, rp, kd));
    KF_TRY(upload_padded(ctx, O.s2a_d, H->s2a_d.data(), 1, kd, m, ld, kd));
    KF_TRY(upload_padded(ctx, O.lb, H->lb.data(), 8, kd, kd, kdp, kd));
    KF_TRY(upload_padded(ctx, O.vd, H->vd.data(), 1, m, kd, kdp, m));
    O.ku = ku;
    O.kd = kd;
    // tensor-core images of the M2L translations: rows in tiles of 128, split pairs
    O.m2l_tc_mtiles = 0;
    O.m2l_pairs_rows = false;
    if ((ctx->opt.m2l_tensor_cores & 1) && !(ctx->opt.m2l_tensor_cores & 16) && tc::mt_rank_ok(rp)) {
        // pairs as rows: each translation as one B operand image [hi | lo], row i = output index
        const size_t half = (size_t)rp * rp;  // uint16 per half
        std::vector<uint16_t> img((size_t)316 * 2 * half, 0);
        for (int d = 0; d < 316; ++d) {
            uint16_t *hi = img.data() + (size_t)d * 2 * half, *lo = hi + half;
            for (int i = 0; i < r; ++i)
                for (int k = 0; k < r; ++k) {
                    const float v = (float)H->m2l_c[((size_t)d * r + i) * r + k];
                    const uint16_t h = host_bf16(v);
                    const uint16_t l = host_bf16(v - host_bf16_to_f32(h));
                    const uint32_t off = tc::core_offset(i, k, rp) / 2;
                    hi[off] = h;
                    lo[off] = l;
                }
        }
        KF_CUDA(O.m2l_tc.ensure(sizeof(uint16_t) * img.size()));
        KF_CUDA(cudaMemcpy(O.m2l_tc.p, img.data(), sizeof(uint16_t) * img.size(), cudaMemcpyHostToDevice));
        O.m2l_tc_mtiles = 1;
        O.m2l_pairs_rows = true;
    } else if ((ctx->opt.m2l_tensor_cores & 1) && tc_rank_ok(rp)) {
        const int nmt = (r + tc::BM - 1) / tc::BM;
        const size_t half = tc::half_bytes(tc::BM, rp) / 2;  // uint16 per half
        std::vector<uint16_t> img((size_t)316 * nmt * 2 * half, 0);
        for (int d = 0; d < 316; ++d)
            for (int mt = 0; mt < nmt; ++mt) {
                uint16_t *hi = img.data() + ((size_t)d * nmt + mt) * 2 * half, *lo = hi + half;
                for (int i = 0; i < tc::BM; ++i) {
                    const int row = mt * tc::BM + i;
                    if (row >= r) continue;
                    for (int k = 0; k < r; ++k) {
                        const float v = (float)H->m2l_c[((size_t)d * r + row) * r + k];
                        const uint16_t h = host_bf16(v);
                        const uint16_t l = host_bf16(v - host_bf16_to_f32(h));
                        const uint32_t off = tc::core_offset(i, k, tc::BM) / 2;
                        hi[off] = h;
                        lo[off] = l;
                    }
                }
            }
        KF_CUDA(O.m2l_tc.ensure(sizeof(uint16_t) * img.size()));
        KF_CUDA(cudaMemcpy(O.m2l_tc.p, img.data(), sizeof(uint16_t) * img.size(), cudaMemcpyHostToDevice));
        O.m2l_tc_mtiles = nmt;
    }
    // tensor-core images of the box operators (K streamed in chunks, any size)
    // bit 1: check-to-equivalent factors, bit 2: M2M and L2L, bit 3: basis changes
    const int tcb = ctx->opt.m2l_tensor_cores;
    O.box_tc = false;
    for (Operators::TcOp *op : {&O.tc_s2a_u, &O.tc_mb, &O.tc_cb, &O.tc_vu, &O.tc_wb, &O.tc_s2a_d, &O.tc_lb, &O.tc_vd})
        op->on = false;
    if (tcb & 2) {
        KF_TRY(upload_tc_op(ctx, O.tc_s2a_u, H->s2a_u.data(), 1, ku, m));
        KF_TRY(upload_tc_op(ctx, O.tc_s2a_d, H->s2a_d.data(), 1, kd, m));
    }
    if (tcb & 4) {
        KF_TRY(upload_tc_op(ctx, O.tc_mb, H->mb.data(), 8, ku, ku));
        KF_TRY(upload_tc_op(ctx, O.tc_lb, H->lb.data(), 8, kd, kd));
    }
    if (tcb & 8) {
        KF_TRY(upload_tc_op(ctx, O.tc_cb, H->cb.data(), 1, r, ku));
        KF_TRY(upload_tc_op(ctx, O.tc_wb, H->wb.data(), 1, kd, r));
        KF_TRY(upload_tc_op(ctx, O.tc_vu, H->vu.data(), 1, m, ku));
        KF_TRY(upload_tc_op(ctx, O.tc_vd, H->vd.data(), 1, m, kd));
    }
    O.box_tc = (tcb & 14) != 0;
    // dynamic shared memory of the tensor-core kernels (set here, outside any graph capture;
    // raised, never lowered: another context of this process may use a larger rank)
    KF_CUDA(raise_smem_limit(tc::tc_box_gemm_kernel, (int)tc::box_smem_bytes()));
    if (O.m2l_pairs_rows) KF_CUDA(raise_smem_limit(tc::tc_m2l_kernel, (int)tc::mt_smem_bytes(rp)));
    else if (O.m2l_tc_mtiles > 0) KF_CUDA(raise_smem_limit(tc::tc_gather_gemm_kernel, (int)tc::smem_bytes(rp)));
    O.p = prm.p;
    O.nu = prm.nu;
    O.r_inner = prm.r_inner;
    O.r_outer = prm.r_outer;
    O.pinv_rtol = prm.pinv_rtol;
    O.m2l_rtol = prm.m2l_rtol;
    O.m2l_rank_max = prm.m2l_rank_max;
    O.n_surf = n;
    O.rank = r;
    O.ready = true;
    O.lat_ready = false;
    ctx->plans.valid = false;  // box-vector layouts depend on the rank
    return ctx->periodic ? ensure_lattice(ctx, prm) : KFMM_OK;
}

namespace {

// ------------------------------------------------------------------------------------
// source records: 4 x float4 = {y, nu'}, {t}, {u}, {n} in sorted order.  Displacement
// records carry u pre-multiplied by 1 - 2 nu and nu' = n . u (acc_sl_dl_s); stress records
// carry u scaled by c_S / c_D and nu' = (1 - 2 nu) n . u.
// ------------------------------------------------------------------------------------
struct SrcRec {
    float4 y, t, u, n;
};

// records of all ncol density columns: rec[col * ns + i]
__global__ void pack_sources_kernel(int64_t ns, const float4 *__restrict__ xyz, const float4 *__restrict__ nrm,
                                    const int *__restrict__ perm, const float *__restrict__ sl,
                                    const float *__restrict__ dl, int ld, int ncol, float st, float su,
                                    float nscale, SrcRec *__restrict__ rec)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ns * ncol; e += stride) {
        const int64_t i = e % ns;
        const int col = (int)(e / ns);
        const int j = perm[i];
        SrcRec r;
        float4 p = xyz[i];
        float3 t = make_float3(0.f, 0.f, 0.f), u = make_float3(0.f, 0.f, 0.f);
        float4 nn = make_float4(0.f, 0.f, 0.f, 0.f);
        if (sl) {
            const float *s = sl + (int64_t)j * ld + 3 * col;
            t = make_float3(st * s[0], st * s[1], st * s[2]);
        }
        if (dl) {
            const float *s = dl + (int64_t)j * ld + 3 * col;
            u = make_float3(su * s[0], su * s[1], su * s[2]);
            nn = nrm[i];
        }
        const float nup = nscale * (nn.x * u.x + nn.y * u.y + nn.z * u.z);
        r.y = make_float4(p.x, p.y, p.z, nup);
        r.t = make_float4(t.x, t.y, t.z, 0.f);
        r.u = make_float4(u.x, u.y, u.z, 0.f);
        r.n = make_float4(nn.x, nn.y, nn.z, 0.f);
        rec[e] = r;
    }
}

// centre and half-width of every box, in the root cube of its point set (the set index leads
// the box key; roots: 8 doubles per set, lower corner x, y, z, side, ...)
__global__ void box_geom_kernel(int nb, const int4 *__restrict__ anchor, const uint64_t *__restrict__ key,
                                const double *__restrict__ roots, float4 *__restrict__ geom)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int4 a = anchor[b];
    const double *r = roots + 8 * (key[b] >> (3 * a.w));
    const double s = r[3] / (double)(1 << a.w);
    geom[b] = make_float4((float)(r[0] + (a.x + 0.5) * s), (float)(r[1] + (a.y + 0.5) * s),
                          (float)(r[2] + (a.z + 0.5) * s), (float)(0.5 * s));
}

// ------------------------------------------------------------------------------------
// check-surface potentials from sources (S2M on leaves, P2L on X lists)
// One CTA per box, one thread per check point; sources staged through shared memory.
// ------------------------------------------------------------------------------------
constexpr int kChkThreads = 80;  // 2 check points per thread up to p = 6 (152), 4 up to p = 8 (296)
static_assert(surface_points(8) <= 4 * kChkThreads, "check points of the largest order per CTA");
constexpr int kChkStage = 256;

template <bool SL, bool DL>
__device__ __forceinline__ void chk_pair(float x, float y, float z, const SrcRec &q, float a34, float c3, float &ox,
                                         float &oy, float &oz)
{
    const float dx = x - q.y.x, dy = y - q.y.y, dz = z - q.y.z;
    if (SL && DL)
        acc_sl_dl_s<float>(dx, dy, dz, q.t.x, q.t.y, q.t.z, q.u.x, q.u.y, q.u.z, q.n.x, q.n.y, q.n.z, q.y.w, a34, c3,
                           ox, oy, oz);
    else if (SL)
        acc_sl<float>(dx, dy, dz, q.t.x, q.t.y, q.t.z, a34, ox, oy, oz);
    else
        acc_dl_s<float>(dx, dy, dz, q.u.x, q.u.y, q.u.z, q.n.x, q.n.y, q.n.z, q.y.w, c3, ox, oy, oz);
}

// NPT check points per thread: tid, tid + kChkThreads, ... (n_surf <= NPT kChkThreads); each
// staged source record serves NPT independent pairs.  An X-list entry of a periodic tree that
// names a moved image of its box stages the box's sources moved by whole cells (cell side).
template <bool SL, bool DL, int NPT>
__global__ void __launch_bounds__(kChkThreads)
check_potential_kernel(const int *__restrict__ boxes, int nbox, int use_xlist, const int *__restrict__ xo,
                       const int *__restrict__ xi, const int2 *__restrict__ bsrc, const float4 *__restrict__ geom,
                       const float4 *__restrict__ surf, int n_surf, float radius, const SrcRec *__restrict__ rec,
                       float a34, float c3, float *__restrict__ out, int ldo, int64_t rec_col, int64_t out_col,
                       float cell)
{
    __shared__ SrcRec sh[kChkStage];
    rec += blockIdx.y * rec_col;  // density column blockIdx.y
    out += blockIdx.y * out_col;
    const int b = boxes ? boxes[blockIdx.x] : blockIdx.x;
    const float4 g = geom[b];
    const int tid = threadIdx.x;
    float x[NPT], y[NPT], z[NPT], o[NPT][3];
    bool has[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int c = tid + j * kChkThreads;
        has[j] = c < n_surf;
        x[j] = y[j] = z[j] = 0.f;
        o[j][0] = o[j][1] = o[j][2] = 0.f;
        if (has[j]) {
            const float4 sp = surf[c];
            x[j] = g.x + radius * g.w * sp.x;
            y[j] = g.y + radius * g.w * sp.y;
            z[j] = g.z + radius * g.w * sp.z;
        }
    }
    const int nlist = use_xlist ? xo[b + 1] - xo[b] : 1;
    for (int li = 0; li < nlist; ++li) {
        const int ent = use_xlist ? xi[xo[b] + li] : b;
        const int2 r = bsrc[ent_box(ent)];
        int sx, sy, sz;
        ent_shift(ent, sx, sy, sz);
        const float ox = sx * cell, oy = sy * cell, oz = sz * cell;
        for (int base = r.x; base < r.y; base += kChkStage) {
            const int cnt = min(kChkStage, r.y - base);
            __syncthreads();
            for (int k = tid; k < cnt; k += kChkThreads) {
                SrcRec q = rec[base + k];
                q.y.x += ox;
                q.y.y += oy;
                q.y.z += oz;
                sh[k] = q;
            }
            __syncthreads();
            if (has[0]) {
                for (int k = 0; k < cnt; ++k) {
                    const SrcRec q = sh[k];
#pragma unroll
                    for (int j = 0; j < NPT; ++j) chk_pair<SL, DL>(x[j], y[j], z[j], q, a34, c3, o[j][0], o[j][1], o[j][2]);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NPT; ++j)
        if (has[j]) {
            float *q = out + (int64_t)b * ldo + 3 * (tid + j * kChkThreads);
            q[0] = o[j][0];
            q[1] = o[j][1];
            q[2] = o[j][2];
        }
}

// ------------------------------------------------------------------------------------
// grouped gather-GEMM: for each tile (group g, columns c0..c1):
//   y_j = alpha_j * A_g (M x K) * X[src_j]   ->  Y[dst_j] (= | += | atomic +=)
// FP32 SIMT, 64 x 64 output tile per CTA, K in steps of 16, 4 x 4 per thread.
// ------------------------------------------------------------------------------------
struct GemmArgs {
    const float *A;
    int64_t a_stride;
    int M, K, lda;
    const int4 *tiles;  // {matrix index, c0, c1, 0}
    const int *src_idx;
    const int *dst_idx;
    const int *parent;
    int src_par, dst_par;
    const float *X;
    int ldx;
    float *Y;
    int ldy;
    const float4 *geom;  // alpha_j = alpha * geom[dst].w when non-null
    float alpha;
    int mode;  // 0 store, 1 add, 2 atomic add
    int64_t x_col_rows, y_col_rows;  // rows of one density column (tile.w) in X and Y
};

constexpr int GBM = 64, GBN = 64, GBK = 16;

// TAG only separates the launches by name in profiles: 0 = box operators, 1 = M2L.
template <int TAG>
__global__ void __launch_bounds__(256) gemm_gather_kernel(GemmArgs g)
{
    __shared__ float As[GBK][GBM + 4];
    __shared__ float Bs[GBK][GBN + 4];
    __shared__ int s_src[GBN], s_dst[GBN];
    const int4 tile = g.tiles[blockIdx.x];
    const int m0 = blockIdx.y * GBM;
    const int tid = threadIdx.x;
    const int ncols = tile.z - tile.y;
    if (tid < GBN) {
        int j = tile.y + tid;
        int s = -1, d = -1;
        if (tid < ncols) {
            s = g.src_idx ? g.src_idx[j] : j;
            d = g.dst_idx ? g.dst_idx[j] : j;
            if (g.src_par) s = g.parent[s];
            if (g.dst_par) d = g.parent[d];
        }
        s_src[tid] = s;
        s_dst[tid] = d;
    }
    __syncthreads();
    const float *A = g.A + (int64_t)tile.x * g.a_stride;
    const float *Xc = g.X + (int64_t)tile.w * g.x_col_rows * g.ldx;
    float *Yc = g.Y + (int64_t)tile.w * g.y_col_rows * g.ldy;
    const int tx = tid & 15, ty = tid >> 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    // load mapping
    const int am = tid >> 2, ak = (tid & 3) * 4;       // A: row am, cols ak..ak+3
    const int bn = tid & 63, bk = (tid >> 6) * 4;      // B: column bn, rows bk..bk+3
    const int bsrc = s_src[bn];
    for (int k0 = 0; k0 < g.K; k0 += GBK) {
        float4 av = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m0 + am < g.M) av = *reinterpret_cast<const float4 *>(A + (int64_t)(m0 + am) * g.lda + k0 + ak);
        As[ak + 0][am] = av.x;
        As[ak + 1][am] = av.y;
        As[ak + 2][am] = av.z;
        As[ak + 3][am] = av.w;
        float4 bv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (bsrc >= 0) bv = *reinterpret_cast<const float4 *>(Xc + (int64_t)bsrc * g.ldx + k0 + bk);
        Bs[bk + 0][bn] = bv.x;
        Bs[bk + 1][bn] = bv.y;
        Bs[bk + 2][bn] = bv.z;
        Bs[bk + 3][bn] = bv.w;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    const int mrow = m0 + ty * 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = tx * 4 + j;
        const int d = s_dst[c];
        if (d < 0) continue;
        const float al = g.geom ? g.alpha * g.geom[d].w : g.alpha;
        float *y = Yc + (int64_t)d * g.ldy + mrow;
        if (mrow + 3 < g.M) {
            float4 v = make_float4(al * acc[0][j], al * acc[1][j], al * acc[2][j], al * acc[3][j]);
            if (g.mode == 0) {
                *reinterpret_cast<float4 *>(y) = v;
            } else if (g.mode == 1) {
                float4 o = *reinterpret_cast<float4 *>(y);
                *reinterpret_cast<float4 *>(y) = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
            } else {
                atomicAdd(reinterpret_cast<float4 *>(y), v);
            }
        } else {
            for (int i = 0; i < 4; ++i) {
                if (mrow + i >= g.M) break;
                const float v = al * acc[i][j];
                if (g.mode == 0) y[i] = v;
                else if (g.mode == 1) y[i] += v;
                else atomicAdd(y + i, v);
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// leaf evaluation: L2P (downward equivalent density of the leaf), M2P (upward equivalent
// densities of the W list), P2P (sources of the U list).
//
// Work items (one warp each, one warp per CTA): a chunk of at most 64 targets of a leaf and a
// range of its source segments -- segment 0 the leaf's own downward density (L2P), then the
// W-list boxes (M2P through the upward density, or directly from the sources of a box with
// at most w_direct_max of them), then the U-list leaves (P2P).  Heavy leaves (long W and U
// lists) are cut into several items of bounded cost whose results are added atomically into
// the zeroed output, so no warp runs far longer than the others.  A chunk of nt targets
// gives each lane T = 1, 2 or 4 of them (ti, ti + L, ...; L = ceil(nt / T)) and splits the 32
// lanes into nsl = 32 / L source slices, lane = slice * L + ti; the slices are summed by
// shuffles at the end (eval_layout picks T), so small and ragged leaves keep their lanes
// busy and large ones read each staged source once per four pairs.
// Sources are staged per warp in batches of 32 records through shared memory, the next
// batch prefetched into registers while the current one is evaluated.  Coincident points
// share a Morton key and so a leaf: only the leaf's own sources take the r = 0 test.
// ------------------------------------------------------------------------------------
constexpr int kEvalWarps = 1;  // one warp per CTA: the block scheduler balances the leaves
constexpr int kEvalThreads = 32 * kEvalWarps;
constexpr unsigned kFull = 0xffffffffu;

template <int KIND, bool SL, bool DL, bool CHK>
__device__ __forceinline__ void p2p_pair(float x, float y, float z, const SrcRec &q, float a34, float b12, float c3,
                                         float nu, float *o)
{
    const float dx = x - q.y.x, dy = y - q.y.y, dz = z - q.y.z;
    if (KIND == KFMM_DISP) {
        // displacement records carry the double-layer density pre-multiplied by 1 - 2 nu
        if (SL && DL)
            acc_sl_dl_s<float, CHK>(dx, dy, dz, q.t.x, q.t.y, q.t.z, q.u.x, q.u.y, q.u.z, q.n.x, q.n.y, q.n.z,
                                    q.y.w, a34, c3, o[0], o[1], o[2]);
        else if (SL)
            acc_sl<float, CHK>(dx, dy, dz, q.t.x, q.t.y, q.t.z, a34, o[0], o[1], o[2]);
        else
            acc_dl_s<float, CHK>(dx, dy, dz, q.u.x, q.u.y, q.u.z, q.n.x, q.n.y, q.n.z, q.y.w, c3, o[0], o[1], o[2]);
    } else {
        if (SL) acc_D<float, CHK>(dx, dy, dz, q.t.x, q.t.y, q.t.z, b12, o);
        if (DL) acc_S<float, CHK>(dx, dy, dz, q.u.x, q.u.y, q.u.z, q.n.x, q.n.y, q.n.z, nu, b12, o);
    }
}

// equivalent source (position p, density f): single layer only, never coincident
template <int KIND>
__device__ __forceinline__ void equiv_pair(float x, float y, float z, const float4 &p, const float4 &f, float a34,
                                           float b12, float *o)
{
    const float dx = x - p.x, dy = y - p.y, dz = z - p.z;
    if (KIND == KFMM_DISP) acc_sl<float, false>(dx, dy, dz, f.x, f.y, f.z, a34, o[0], o[1], o[2]);
    else acc_D<float, false>(dx, dy, dz, f.x, f.y, f.z, b12, o);
}

struct EvalArgs {
    const int4 *items;
    int n_items;
    int w_direct_max;
    const int2 *btrg, *bsrc;
    const float4 *geom;
    const int *uo, *ui, *wo, *wi;
    const int *xdo, *xdi;  // X-list leaves summed directly at the leaf's targets
    const float4 *trg;
    const int *trg_perm;
    const SrcRec *rec;
    const float4 *surf;
    int n_surf;
    float r_in, r_out;
    const float *dn_phi, *up_phi;
    int ld_phi;
    float phi_scale;  // c_sl for DISP, 1 for STRESS (D carries c_D at the end)
    float a34, b12, nu;
    float c3;         // 3 / (1 - 2 nu): displacement records carry (1 - 2 nu) u
    float out_scale;  // 1 for DISP, c_D for STRESS
    float *out;
    int ldo;
    int64_t rec_col, phi_col;  // strides of one density column (blockIdx.y) in rec and the phis
    int part;                  // 0: all segments; 1: P2P only (U leaves, direct W boxes);
                               // 2: L2P and M2P only
    float cell;                // periodic tree: cell side (list entries may name moved images)
};

// the offset of a moved image from its entry bits (e >> kEntBits, 0 for the unmoved box)
__device__ __forceinline__ void image_offset(int bits, float cell, float &ox, float &oy, float &oz)
{
    const int c = bits ^ 13;
    ox = (float)(c / 9 - 1) * cell;
    oy = (float)((c / 3) % 3 - 1) * cell;
    oz = (float)(c % 3 - 1) * cell;
}

// one source record, only the fields the kernel family reads
template <bool SL, bool DL>
__device__ __forceinline__ SrcRec load_rec(const SrcRec *__restrict__ rec, int64_t i)
{
    SrcRec r;
    r.y = __ldg(&rec[i].y);
    if (SL) r.t = __ldg(&rec[i].t);
    if (DL) {
        r.u = __ldg(&rec[i].u);
        r.n = __ldg(&rec[i].n);
    }
    return r;
}

template <bool SL, bool DL>
__device__ __forceinline__ void store_rec(SrcRec *sh, const SrcRec &r)
{
    sh->y = r.y;
    if (SL) sh->t = r.t;
    if (DL) {
        sh->u = r.u;
        sh->n = r.n;
    }
}

// Lane layout of a chunk of nt <= 64 targets: T targets per lane (1, 2 or 4), L = ceil(nt / T)
// lanes per source slice, nsl = 32 / L slices taking every nsl-th source.  A warp step then
// evaluates nt * nsl useful pairs at the cost of T pair evaluations per lane: the layout with
// the most pairs per step wins, on a tie the larger T (fewer shared-memory loads per pair,
// more independent work per lane).  Returns T.
__host__ __device__ inline int eval_layout(int nt, int &L, int &nsl)
{
    int best_t = 0;
    float best = -1.f;
    for (int t = 1; t <= 4; t *= 2) {
        const int l = (nt + t - 1) / t;
        if (l > 32) continue;
        const float score = (float)(32 / l) / (float)t;
        if (score >= best) {
            best = score;
            best_t = t;
            L = l;
            nsl = 32 / l;
        }
    }
    return best_t;
}

// staged records k = kbeg, kbeg + nsl, ... < cnt against this lane's NT targets; with one or
// two targets two sources per step (independent pairs), with four one
template <int KIND, bool SL, bool DL, bool CHK, int NO, int NT>
__device__ __forceinline__ void eval_batch(const SrcRec *sh, int kbeg, int cnt, int nsl, const float (&x)[4],
                                           const float (&y)[4], const float (&z)[4], const EvalArgs &e,
                                           float (&o)[4][NO])
{
    int k = kbeg;
    if constexpr (NT == 4) {
        for (; k < cnt; k += nsl) {
            const SrcRec q = sh[k];
#pragma unroll
            for (int t = 0; t < 4; ++t) p2p_pair<KIND, SL, DL, CHK>(x[t], y[t], z[t], q, e.a34, e.b12, e.c3, e.nu, o[t]);
        }
    } else {
        for (; k + nsl < cnt; k += 2 * nsl) {
            const SrcRec qa = sh[k], qb = sh[k + nsl];
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                p2p_pair<KIND, SL, DL, CHK>(x[t], y[t], z[t], qa, e.a34, e.b12, e.c3, e.nu, o[t]);
                p2p_pair<KIND, SL, DL, CHK>(x[t], y[t], z[t], qb, e.a34, e.b12, e.c3, e.nu, o[t]);
            }
        }
        if (k < cnt) {
            const SrcRec q = sh[k];
#pragma unroll
            for (int t = 0; t < NT; ++t)
                p2p_pair<KIND, SL, DL, CHK>(x[t], y[t], z[t], q, e.a34, e.b12, e.c3, e.nu, o[t]);
        }
    }
}

// the same for the layout's T (warp-uniform)
template <int KIND, bool SL, bool DL, bool CHK, int NO>
__device__ __forceinline__ void eval_batch_t(int T, const SrcRec *sh, int kbeg, int cnt, int nsl, const float (&x)[4],
                                             const float (&y)[4], const float (&z)[4], const EvalArgs &e,
                                             float (&o)[4][NO])
{
    if (T == 4) eval_batch<KIND, SL, DL, CHK, NO, 4>(sh, kbeg, cnt, nsl, x, y, z, e, o);
    else if (T == 2) eval_batch<KIND, SL, DL, CHK, NO, 2>(sh, kbeg, cnt, nsl, x, y, z, e, o);
    else eval_batch<KIND, SL, DL, CHK, NO, 1>(sh, kbeg, cnt, nsl, x, y, z, e, o);
}

// staged equivalent sources k = kbeg, kbeg + nsl, ... < n against this lane's NT targets
template <int KIND, int NO, int NT>
__device__ __forceinline__ void equiv_batch(const float4 *eqp, const float4 *eqf, int kbeg, int n, int nsl,
                                            const float (&x)[4], const float (&y)[4], const float (&z)[4],
                                            const EvalArgs &e, float (&o)[4][NO])
{
    int k = kbeg;
    for (; k + nsl < n; k += 2 * nsl) {  // two independent pairs per target and step
        const float4 pa = eqp[k], fa = eqf[k], pb = eqp[k + nsl], fb = eqf[k + nsl];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            equiv_pair<KIND>(x[t], y[t], z[t], pa, fa, e.a34, e.b12, o[t]);
            equiv_pair<KIND>(x[t], y[t], z[t], pb, fb, e.a34, e.b12, o[t]);
        }
    }
    if (k < n) {
        const float4 pp = eqp[k], f = eqf[k];
#pragma unroll
        for (int t = 0; t < NT; ++t) equiv_pair<KIND>(x[t], y[t], z[t], pp, f, e.a34, e.b12, o[t]);
    }
}

// PART: 0 all segments, 1 the near list (P2P only), 2 the far list (L2P and M2P only); a
// compile-time part leaves the other part's code, and its registers, out of the kernel.
template <int KIND, bool SL, bool DL, int PART>
__global__ void __launch_bounds__(kEvalThreads) eval_leaf_kernel(EvalArgs e)
{
    constexpr int NO = KIND == KFMM_DISP ? 3 : 6;
    __shared__ SrcRec stage[kEvalWarps][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    SrcRec *sh = stage[wid];
    if ((int)blockIdx.x * kEvalWarps + wid >= e.n_items) return;  // the whole warp
    const int4 it = e.items[blockIdx.x * kEvalWarps + wid];
    const int dcol = blockIdx.y;  // density column
    const SrcRec *rec = e.rec + dcol * e.rec_col;
    const float *dn_phi = e.dn_phi + dcol * e.phi_col, *up_phi = e.up_phi + dcol * e.phi_col;
    const int b = it.x, c0 = it.y, s0 = it.z, s1 = it.w;
    const int2 tr = e.btrg[b];
    const int uo0 = e.uo[b], nU = e.uo[b + 1] - uo0;
    const int wo0 = e.wo[b], nW = e.wo[b + 1] - wo0;
    const int xdo0 = e.xdo[b];

    const int nt = min(64, tr.y - c0);
    int L, nsl;
    const int T = eval_layout(nt, L, nsl);             // targets per lane (warp-uniform)
    const int ti = lane % L, si = lane / L;            // first target, source slice
    const bool act = si < nsl;
    float x[4], y[4], z[4];
    bool tact[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        tact[t] = act && t < T && ti + t * L < nt;  // targets ti, ti + L, ...
        x[t] = y[t] = z[t] = 0.f;
        if (tact[t]) {
            const float4 p = e.trg[c0 + ti + t * L];
            x[t] = p.x;
            y[t] = p.y;
            z[t] = p.z;
        }
    }
    float o[4][NO];
#pragma unroll
    for (int t = 0; t < 4; ++t)
        for (int a = 0; a < NO; ++a) o[t][a] = 0.f;
    const int kbeg = act ? si : 32;  // inactive lanes skip every evaluation loop

    // ---- L2P (segment 0) and M2P (W boxes above the direct threshold): the equivalent
    //      sources of one box are staged whole in shared memory (all their loads in flight
    //      at once), then evaluated two per step
    extern __shared__ float4 eq_smem[];  // per warp: n_surf positions, then n_surf densities
    float4 *eqp = eq_smem + (size_t)wid * 2 * e.n_surf, *eqf = eqp + e.n_surf;
    const int n_eq = e.n_surf;
    for (int j = s0; PART != 1 && j < s1 && j <= nW; ++j) {
        const int ent = j == 0 ? b : e.wi[wo0 + j - 1];
        const int src_box = ent_box(ent);
        if (j > 0) {
            const int2 r = e.bsrc[src_box];
            if (r.y - r.x <= e.w_direct_max) continue;  // evaluated directly below
        }
        float4 g = e.geom[src_box];
        if (ent >> kEntBits) {  // a moved image (periodic tree)
            float ox, oy, oz;
            image_offset(ent >> kEntBits, e.cell, ox, oy, oz);
            g.x += ox;
            g.y += oy;
            g.z += oz;
        }
        const float rad = (j == 0 ? e.r_out : e.r_in) * g.w;
        const float *__restrict__ phi = (j == 0 ? dn_phi : up_phi) + (int64_t)src_box * e.ld_phi;
        __syncwarp();
        for (int k = lane; k < n_eq; k += 32) {
            const float4 sp = __ldg(&e.surf[k]);
            const float f0 = __ldg(&phi[3 * k]), f1 = __ldg(&phi[3 * k + 1]), f2 = __ldg(&phi[3 * k + 2]);
            eqp[k] = make_float4(g.x + rad * sp.x, g.y + rad * sp.y, g.z + rad * sp.z, 0.f);
            eqf[k] = make_float4(e.phi_scale * f0, e.phi_scale * f1, e.phi_scale * f2, 0.f);
        }
        __syncwarp();
        const int kb = act ? si : n_eq;
        if (T == 4) equiv_batch<KIND, NO, 4>(eqp, eqf, kb, n_eq, nsl, x, y, z, e, o);
        else if (T == 2) equiv_batch<KIND, NO, 2>(eqp, eqf, kb, n_eq, nsl, x, y, z, e, o);
        else equiv_batch<KIND, NO, 1>(eqp, eqf, kb, n_eq, nsl, x, y, z, e, o);
    }

    // ---- P2P with the direct W boxes, the U-list leaves other than the leaf itself and the
    //      X-list leaves summed directly: up to 32 source ranges at a time, batches of 32
    //      records filled across ranges
    bool has_self = false;
    for (int j0 = max(s0, 1); PART != 2 && j0 < s1; j0 += 32) {
        const int nr = min(32, s1 - j0);
        int beg = 0, cnt = 0;
        bool self = false;
        int mbits = 0;  // a moved image of a box (periodic tree): summed after the others
        if (lane < nr) {
            const int j = j0 + lane;
            const int ent = j <= nW ? e.wi[wo0 + j - 1]
                                    : (j <= nW + nU ? e.ui[uo0 + j - 1 - nW] : e.xdi[xdo0 + j - 1 - nW - nU]);
            const int2 r = e.bsrc[ent_box(ent)];
            if (j <= nW) {
                if (r.y - r.x <= e.w_direct_max) {
                    beg = r.x;
                    cnt = r.y - r.x;
                }
            } else if (j <= nW + nU && ent == b) {
                self = true;
            } else {
                beg = r.x;
                cnt = r.y - r.x;
            }
            if (ent >> kEntBits) {
                mbits = ent >> kEntBits;
                cnt = 0;  // not in the batches below
            }
        }
        has_self |= __ballot_sync(kFull, self) != 0u;
        int incl = cnt;  // inclusive prefix over the lanes
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += v;
        }
        const int excl = incl - cnt;
        const int total = __shfl_sync(kFull, incl, 31);
        // source index of flat position f: the last range whose exclusive prefix is <= f
        auto locate = [&](int f) -> int {
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int mid = lo + step;
                const int v = __shfl_sync(kFull, excl, mid < 32 ? mid : 31);
                if (mid < nr && v <= f) lo = mid;
            }
            const int bb = __shfl_sync(kFull, beg, lo);
            const int ee = __shfl_sync(kFull, excl, lo);
            return bb + (f - ee);
        };
        SrcRec nxt;
        {
            const int src = locate(lane);
            if (lane < total) nxt = load_rec<SL, DL>(rec, src);
        }
        for (int base = 0; base < total; base += 32) {
            const int cnt2 = min(32, total - base);
            __syncwarp();
            if (lane < cnt2) store_rec<SL, DL>(sh + lane, nxt);
            __syncwarp();
            if (base + 32 < total) {
                const int src = locate(base + 32 + lane);
                if (base + 32 + lane < total) nxt = load_rec<SL, DL>(rec, src);
            }
            eval_batch_t<KIND, SL, DL, false, NO>(T, sh, kbeg, cnt2, nsl, x, y, z, e, o);
        }
        // moved images of boxes (a periodic tree near the cell's faces): one range at a time,
        // its sources staged moved by whole cells
        for (unsigned mv = __ballot_sync(kFull, mbits != 0); mv; mv &= mv - 1) {
            const int l = __ffs(mv) - 1;
            const int bits = __shfl_sync(kFull, mbits, l);
            const int j = j0 + l;  // the segment, read again by the whole warp
            const int ent = j <= nW ? e.wi[wo0 + j - 1]
                                    : (j <= nW + nU ? e.ui[uo0 + j - 1 - nW] : e.xdi[xdo0 + j - 1 - nW - nU]);
            const int2 rr = e.bsrc[ent_box(ent)];
            if (j <= nW && rr.y - rr.x > e.w_direct_max) continue;  // through its density
            float ox, oy, oz;
            image_offset(bits, e.cell, ox, oy, oz);
            for (int base = rr.x; base < rr.y; base += 32) {
                const int c2 = min(32, rr.y - base);
                __syncwarp();
                if (lane < c2) {
                    SrcRec q = load_rec<SL, DL>(rec, base + lane);
                    q.y.x += ox;
                    q.y.y += oy;
                    q.y.z += oz;
                    store_rec<SL, DL>(sh + lane, q);
                }
                __syncwarp();
                eval_batch_t<KIND, SL, DL, false, NO>(T, sh, kbeg, c2, nsl, x, y, z, e, o);
            }
        }
    }

    // ---- P2P with the leaf's own sources (the only ones that may coincide with a target)
    if (has_self) {
        const int2 r = e.bsrc[b];
        SrcRec nxt;
        if (r.x + lane < r.y) nxt = load_rec<SL, DL>(rec, r.x + lane);
        for (int base = r.x; base < r.y; base += 32) {
            const int cnt = min(32, r.y - base);
            __syncwarp();
            if (lane < cnt) store_rec<SL, DL>(sh + lane, nxt);
            __syncwarp();
            if (base + 32 + lane < r.y) nxt = load_rec<SL, DL>(rec, base + 32 + lane);
            eval_batch_t<KIND, SL, DL, true, NO>(T, sh, kbeg, cnt, nsl, x, y, z, e, o);
        }
    }

    // ---- sum the source slices into slice 0 (shuffling the unmodified partial sums) and add
    //      into the zeroed output in input order
    float tot[4][NO];
#pragma unroll
    for (int t = 0; t < 4; ++t)
        for (int a = 0; a < NO; ++a) tot[t][a] = o[t][a];
    for (int s = 1; s < nsl; ++s) {
        const int src = lane + s * L;
        const int sl = src < 32 ? src : 31;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (t >= T) break;  // warp-uniform
#pragma unroll
            for (int a = 0; a < NO; ++a) {
                const float v = __shfl_sync(kFull, o[t][a], sl);
                if (src < 32) tot[t][a] += v;
            }
        }
    }
    if (si == 0) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (!tact[t]) continue;
            float *q = e.out + (int64_t)e.trg_perm[c0 + ti + t * L] * e.ldo + NO * dcol;
#pragma unroll
            for (int a = 0; a < NO; ++a) atomicAdd(q + a, e.out_scale * tot[t][a]);
        }
    }
}

// zero the NO outputs of column col of every target (the evaluation adds into them)
__global__ void zero_out_kernel(int64_t n, float *__restrict__ out, int ldo, int c0, int no)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * no; i += stride)
        out[(i / no) * ldo + c0 + i % no] = 0.f;
}

// Work items of the leaf evaluation: one warp per leaf.  For each target chunk the lanes cost
// the source segments (L2P, W boxes, U leaves) 32 at a time; a warp prefix sum of the costs
// (warp pair-steps) cuts a new item wherever floor(prefix / item_cost) changes, so no item
// exceeds the cap by more than one segment.  An item is written once, when the next start
// (its end) is known.  item_cost is 1024 by default and tuned per context when autotuning is
// on.
// For a split evaluation (part 1: P2P, part 2: L2P and M2P) the segments of the other part
// cost nothing, so they never start an item.
template <bool EMIT>
__global__ void eval_items_kernel(int n_leaves, const int *__restrict__ leaves, const int2 *__restrict__ btrg,
                                  const int2 *__restrict__ bsrc, const int *__restrict__ uo,
                                  const int *__restrict__ ui, const int *__restrict__ wo,
                                  const int *__restrict__ wi, const int *__restrict__ xdo,
                                  const int *__restrict__ xdi, int w_direct_max, int n_surf, float item_cost,
                                  int split, const int *__restrict__ off, int *__restrict__ cnt,
                                  int4 *__restrict__ items)
{
    const int lane = threadIdx.x & 31;
    const int li = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (li >= n_leaves) return;  // the whole warp
    const int b = leaves[li];
    const int2 tr = btrg[b];
    const int w0 = wo[b], nW = wo[b + 1] - w0, u0 = uo[b], nU = uo[b + 1] - u0;
    const int x0 = xdo[b], nX = xdo[b + 1] - x0;
    const int nseg = 1 + nW + nU + nX;
    // one list (part 0), or the near (1) and far (2) lists with counts and offsets at
    // [list][leaf]
    for (int k = 0; k < (split ? 2 : 1); ++k) {
        const int part = split ? k + 1 : 0;
        const int pos = EMIT ? off[(size_t)k * n_leaves + li] : 0;
        int n = 0;
        for (int c0 = tr.x; c0 < tr.y; c0 += 64) {
            const int nt = min(64, tr.y - c0);
            int L, nsl;
            const int T = eval_layout(nt, L, nsl);
            const float w = (float)T / (float)nsl;  // pair evaluations per lane and source
            float base = 0.f;
            int q_last = -1;
            int pend_idx = -1, pend_sg = 0;  // last item started so far: its end is not known yet
            for (int sb = 0; sb < nseg; sb += 32) {
                const int sg = sb + lane;
                float c = 0.f;
                if (sg < nseg) {
                    bool far = true;  // an equivalent surface (L2P, M2P) rather than sources
                    if (sg == 0) {
                        c = 0.5f * (float)n_surf;
                    } else if (sg <= nW) {
                        const int2 r = bsrc[ent_box(wi[w0 + sg - 1])];
                        far = r.y - r.x > w_direct_max;
                        c = far ? 0.5f * (float)n_surf : (float)(r.y - r.x);
                    } else {
                        const int2 r = bsrc[ent_box(sg <= nW + nU ? ui[u0 + sg - 1 - nW] : xdi[x0 + sg - 1 - nW - nU])];
                        c = (float)(r.y - r.x);
                        far = false;
                    }
                    c *= (part == 1 && far) || (part == 2 && !far) ? 0.f : w;  // segments of the other part
                }
                float incl = c;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const float v = __shfl_up_sync(0xffffffffu, incl, d);
                    if (lane >= d) incl += v;
                }
                const int q = sg < nseg ? (int)floorf((base + incl - c) / item_cost) : INT_MAX;
                int qp = __shfl_up_sync(0xffffffffu, q, 1);
                if (lane == 0) qp = q_last;
                const bool start = sg < nseg && (sg == 0 || q != qp);
                const unsigned mask = __ballot_sync(0xffffffffu, start);
                // every item is written once, when its end (the next start) is known: the
                // pending item of the previous batch ends at this batch's first start; an item
                // with a later start in this batch ends there; the last one stays pending
                if (mask) {
                    if (EMIT && pend_idx >= 0 && lane == 0)
                        items[pos + pend_idx] = make_int4(b, c0, pend_sg, sb + __ffs(mask) - 1);
                    const unsigned later = mask & ~((2u << lane) - 1u);
                    if (EMIT && start && later)
                        items[pos + n + __popc(mask & ((1u << lane) - 1u))] =
                            make_int4(b, c0, sg, sb + __ffs(later) - 1);
                    pend_idx = n + __popc(mask) - 1;
                    pend_sg = sb + 31 - __clz(mask);
                }
                n += __popc(mask);
                base += __shfl_sync(0xffffffffu, incl, 31);
                q_last = __shfl_sync(0xffffffffu, q, 31);
            }
            if (EMIT && pend_idx >= 0 && lane == 0) items[pos + pend_idx] = make_int4(b, c0, pend_sg, nseg);
        }
        if (!EMIT && lane == 0) cnt[(size_t)k * n_leaves + li] = n;
    }
}

template <int KIND>
void launch_eval(const EvalArgs &e, int n_items, int ncol, bool sl, bool dl, cudaStream_t st)
{
    if (n_items <= 0) return;
    const dim3 grid((unsigned)((n_items + kEvalWarps - 1) / kEvalWarps), (unsigned)ncol);
    // staged equivalent sources of the L2P / M2P segments (none in the P2P-only part)
    const size_t smem = e.part == 1 ? 0 : sizeof(float4) * 2 * (size_t)e.n_surf * kEvalWarps;
    if (e.part == 1) {
        if (sl && dl) eval_leaf_kernel<KIND, true, true, 1><<<grid, kEvalThreads, smem, st>>>(e);
        else if (sl) eval_leaf_kernel<KIND, true, false, 1><<<grid, kEvalThreads, smem, st>>>(e);
        else eval_leaf_kernel<KIND, false, true, 1><<<grid, kEvalThreads, smem, st>>>(e);
    } else if (e.part == 2) {
        if (sl && dl) eval_leaf_kernel<KIND, true, true, 2><<<grid, kEvalThreads, smem, st>>>(e);
        else if (sl) eval_leaf_kernel<KIND, true, false, 2><<<grid, kEvalThreads, smem, st>>>(e);
        else eval_leaf_kernel<KIND, false, true, 2><<<grid, kEvalThreads, smem, st>>>(e);
    } else {
        if (sl && dl) eval_leaf_kernel<KIND, true, true, 0><<<grid, kEvalThreads, smem, st>>>(e);
        else if (sl) eval_leaf_kernel<KIND, true, false, 0><<<grid, kEvalThreads, smem, st>>>(e);
        else eval_leaf_kernel<KIND, false, true, 0><<<grid, kEvalThreads, smem, st>>>(e);
    }
}

}  // namespace

// ------------------------------------------------------------------------------------
// GEMM plans: tile tables built once per tree
// ------------------------------------------------------------------------------------
static kfmm_status make_plan(kfmm_ctx *ctx, GemmPlan &pl, const std::vector<int> &group_mat,
                             const std::vector<int> &group_begin, const std::vector<int> &group_end)
{
    std::vector<int4> t;
    for (size_t gi = 0; gi < group_mat.size(); ++gi)
        for (int c = group_begin[gi]; c < group_end[gi]; c += GBN)
            t.push_back(make_int4(group_mat[gi], c, std::min(c + GBN, group_end[gi]), 0));
    pl.n_tiles = (int)t.size();
    if (pl.n_tiles) {
        KF_CUDA(pl.tiles.ensure(sizeof(int4) * t.size()));
        KF_TRY(upload_async(ctx, pl.tiles.p, t.data(), sizeof(int4) * t.size()));
    }
    pl.host_tiles = t;
    pl.ncol = 1;
    for (int k = 0; k < 9; ++k) pl.n_tc_items[k] = -1;
    return KFMM_OK;
}

// Device tiles for ncol density columns (tile.w = column); drops the tensor-core items.
static kfmm_status plan_ncol(kfmm_ctx *ctx, GemmPlan &pl, int ncol)
{
    if (pl.ncol == ncol) return KFMM_OK;
    std::vector<int4> t;
    t.reserve(pl.host_tiles.size() * ncol);
    for (int c = 0; c < ncol; ++c)
        for (const int4 &h : pl.host_tiles) t.push_back(make_int4(h.x, h.y, h.z, c));
    pl.n_tiles = (int)t.size();
    if (pl.n_tiles) {
        KF_CUDA(pl.tiles.ensure(sizeof(int4) * t.size()));
        KF_TRY(upload_async(ctx, pl.tiles.p, t.data(), sizeof(int4) * t.size()));
    }
    for (int k = 0; k < 9; ++k) pl.n_tc_items[k] = -1;
    pl.ncol = ncol;
    return KFMM_OK;
}

// ------------------------------------------------------------------------------------
// box operators on the tensor cores (K-streamed kernel of tc_gemm.cuh)
// ------------------------------------------------------------------------------------
static_assert(GBN == tc::BN, "tensor-core box items are the 64-column tiles of the GEMM plans");

static kfmm_status run_tc_box(kfmm_ctx *ctx, GemmPlan &pl, const Operators::TcOp &op, const int *src,
                              const int *dst, int src_par, int dst_par, const float *X, int ldx, float *Y, int ldy,
                              const float4 *geom, float alpha, int mode, int ncol, int64_t col_rows)
{
    KF_TRY(plan_ncol(ctx, pl, ncol));
    if (pl.n_tiles == 0) return KFMM_OK;
    // work items for this row-tile count (built once per plan)
    const int nm = op.n_mtile;
    if (nm < 1 || nm > 8) return ctx->fail(KFMM_ERR_INTERNAL, "tensor-core box product: too many row tiles");
    if (ldx % 8 != 0) return ctx->fail(KFMM_ERR_INTERNAL, "tensor-core box product: source rows not padded to 8");
    if (pl.n_tc_items[nm] < 0) {
        std::vector<int4> items;
        for (int c = 0; c < pl.ncol; ++c)
            for (const int4 &t : pl.host_tiles)
                for (int mt = 0; mt < nm; ++mt) items.push_back(make_int4(c * op.n_mat + t.x, mt, t.y, t.z));
        pl.n_tc_items[nm] = (int)items.size();
        KF_CUDA(pl.tc_items[nm].ensure(sizeof(int4) * std::max<size_t>(1, items.size())));
        KF_TRY(upload_async(ctx, pl.tc_items[nm].p, items.data(), sizeof(int4) * items.size()));
    }
    tc::TcBoxArgs a;
    a.A = op.img.as<uint16_t>();
    a.n_mat = op.n_mat;
    a.x_col_rows = col_rows;
    a.y_col_rows = col_rows;
    a.n_mtile = nm;
    a.n_kc = op.n_kc;
    a.M = op.M;
    a.items = pl.tc_items[nm].as<int4>();
    a.src_idx = src;
    a.dst_idx = dst;
    a.parent = ctx->tree.box_parent.as<int>();
    a.src_par = src_par;
    a.dst_par = dst_par;
    a.X = X;
    a.ldx = ldx;
    a.Y = Y;
    a.ldy = ldy;
    a.geom = geom;
    a.alpha = alpha;
    a.mode = mode;
    a.err = ctx->plans.err.as<int>();
    const uint32_t smem = tc::box_smem_bytes();
    tc::tc_box_gemm_kernel<<<pl.n_tc_items[nm], tc::BOX_THREADS, smem, ctx->stream>>>(a);
    KF_LAUNCH();
    return KFMM_OK;
}

// M2L work items of one density column: per direction and row tile, chunks of `chunk`
// columns that share one load of the translation's operand tile (the device copy for the
// current number of density columns is made at the next evaluation)
static void make_m2l_host(kfmm_ctx *ctx, FmmPlans &P, int chunk)
{
    const Tree &T = ctx->tree;
    const int nmt = ctx->ops.m2l_tc_mtiles;
    P.m2l_host.clear();
    for (int d = 0; d < 316 && nmt > 0; ++d)
        for (int c = T.vdir_off[d]; c < T.vdir_off[d + 1]; c += chunk)
            for (int mt = 0; mt < nmt; ++mt)
                P.m2l_host.push_back(make_int4(d, mt, c, std::min(c + chunk, T.vdir_off[d + 1])));
    P.m2l_ncol = 0;
}

// work items of the leaf evaluation for a cost cap
// the leaf-item kernels: per-leaf counts ([list][leaf]) or the items at their offsets
static void eval_items_launch(kfmm_ctx *ctx, FmmPlans &P, float cost, bool emit)
{
    const Tree &T = ctx->tree;
    const int nl = T.n_leaves;
    int *cnt = P.eval_cnt.as<int>();
    const dim3 grid(grid_for((int64_t)nl * 32, 128, 1 << 30));
    if (emit)
        eval_items_kernel<true><<<grid, 128, 0, ctx->stream>>>(
            nl, T.leaves.as<int>(), T.box_trg.as<int2>(), T.box_src.as<int2>(), T.u_off.as<int>(), T.u_idx.as<int>(),
            T.w_off.as<int>(), T.w_idx.as<int>(), T.xd_off.as<int>(), T.xd_idx.as<int>(), T.w_direct_max,
            surface_points(ctx->opt.p), cost, P.eval_split, cnt, nullptr, P.eval_items.as<int4>());
    else
        eval_items_kernel<false><<<grid, 128, 0, ctx->stream>>>(
            nl, T.leaves.as<int>(), T.box_trg.as<int2>(), T.box_src.as<int2>(), T.u_off.as<int>(), T.u_idx.as<int>(),
            T.w_off.as<int>(), T.w_idx.as<int>(), T.xd_off.as<int>(), T.xd_idx.as<int>(), T.w_direct_max,
            surface_points(ctx->opt.p), cost, P.eval_split, nullptr, cnt, nullptr);
}

// counts of all lists side by side ([part][leaf]) and one scan: with a split the far items
// follow the near ones in the same buffer; the totals are at [nl] and [2 nl]
static kfmm_status eval_items_count(kfmm_ctx *ctx, FmmPlans &P, float cost)
{
    const int nl = ctx->tree.n_leaves, nparts = P.eval_split ? 2 : 1;
    KF_CUDA(P.eval_cnt.ensure(sizeof(int) * (size_t)(nparts * nl + 1)));
    int *cnt = P.eval_cnt.as<int>();
    eval_items_launch(ctx, P, cost, false);
    KF_LAUNCH();
    KF_TRY(scan_exclusive(ctx, cnt, cnt, nparts * nl, cnt + (size_t)nparts * nl));
    return KFMM_OK;
}

static kfmm_status eval_items_emit(kfmm_ctx *ctx, FmmPlans &P, float cost, int n_near, int n_far)
{
    P.n_eval_items = n_near;
    P.n_eval_far = n_far;
    KF_CUDA(P.eval_items.ensure(sizeof(int4) * (size_t)std::max(1, n_near + n_far)));
    eval_items_launch(ctx, P, cost, true);
    KF_LAUNCH();
    return KFMM_OK;
}

// all of it, synchronously (the launch-shape tuning)
static kfmm_status make_eval_items(kfmm_ctx *ctx, FmmPlans &P, float cost)
{
    const Tree &T = ctx->tree;
    const cudaStream_t st = ctx->stream;
    P.n_eval_items = P.n_eval_far = 0;
    P.eval_split = ctx->opt.streams != 0;
    if (!T.n_leaves) return KFMM_OK;
    const int nl = T.n_leaves;
    KF_TRY(eval_items_count(ctx, P, cost));
    const int *cnt = P.eval_cnt.as<int>();
    int h[2] = {0, 0};
    KF_CUDA(cudaMemcpyAsync(&h[0], cnt + nl, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (P.eval_split) KF_CUDA(cudaMemcpyAsync(&h[1], cnt + 2 * (size_t)nl, sizeof(int), cudaMemcpyDeviceToHost, st));
    KF_TRY(sync_stream(ctx));
    return eval_items_emit(ctx, P, cost, h[0], P.eval_split ? h[1] - h[0] : 0);
}

// Plans of a new tree, in two parts so that the host work overlaps the first kernels of the
// evaluation.  plans_begin enqueues the device part: box geometry, the leaf-item counts with
// their scan, and an asynchronous copy of the list totals to pinned memory (event ev_items);
// it also makes the leaves' tile table, which the first box product needs.
static kfmm_status plans_begin(kfmm_ctx *ctx, FmmPlans &P)
{
    Tree &T = ctx->tree;
    const cudaStream_t st = ctx->stream;
    KF_CUDA(P.err.ensure(sizeof(int)));
    KF_CUDA(cudaMemsetAsync(P.err.p, 0, sizeof(int), st));
    KF_CUDA(P.geom.ensure(sizeof(float4) * T.n_boxes));
    box_geom_kernel<<<grid_for(T.n_boxes, 256, 1 << 30), 256, 0, st>>>(
        T.n_boxes, T.box_anchor.as<int4>(), T.box_key.as<uint64_t>(), T.set_root_dev.as<double>(),
        P.geom.as<float4>());
    KF_LAUNCH();
    KF_TRY(make_plan(ctx, P.leaves, {0}, {0}, {T.n_leaves}));  // for the first box product
    P.n_eval_items = P.n_eval_far = 0;
    P.eval_split = ctx->opt.streams != 0;
    P.items_pending = false;
    if (!T.n_leaves) return KFMM_OK;
    KF_TRY(eval_items_count(ctx, P, ctx->tune.eval_cost));
    P.items_host = static_cast<int *>(ctx->staging.take(2 * sizeof(int)));
    if (!P.items_host) return ctx->fail(KFMM_ERR_OOM, "pinned staging for the item totals");
    const int nl = T.n_leaves, nparts = P.eval_split ? 2 : 1;
    const int *cnt = P.eval_cnt.as<int>();
    P.items_host[1] = 0;
    KF_CUDA(cudaMemcpyAsync(P.items_host, cnt + nl, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (nparts == 2)
        KF_CUDA(cudaMemcpyAsync(P.items_host + 1, cnt + 2 * (size_t)nl, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (!P.ev_items) KF_CUDA(cudaEventCreateWithFlags(&P.ev_items, cudaEventDisableTiming));
    KF_CUDA(cudaEventRecord(P.ev_items, st));
    P.items_pending = true;
    return KFMM_OK;
}

// plans_end: the host part (tile tables of the box products, M2L work items), then the leaf
// items once their totals have arrived.
static kfmm_status plans_end(kfmm_ctx *ctx, FmmPlans &P)
{
    Tree &T = ctx->tree;
    KF_TRY(make_plan(ctx, P.all, {0}, {0}, {T.n_boxes}));
    KF_TRY(make_plan(ctx, P.xboxes, {0}, {0}, {T.n_xboxes}));
    KF_TRY(make_plan(ctx, P.wboxes, {0}, {0}, {T.n_wboxes}));
    {
        std::vector<int> gm(316), gb(316), ge(316);
        for (int d = 0; d < 316; ++d) {
            gm[d] = d;
            gb[d] = T.vdir_off[d];
            ge[d] = T.vdir_off[d + 1];
        }
        KF_TRY(make_plan(ctx, P.m2l, gm, gb, ge));
        make_m2l_host(ctx, P, ctx->tune.m2l_chunk);
    }
    P.oct_lvl.clear();
    P.oct_lvl.resize(T.n_levels);
    for (int l = 1; l < T.n_levels; ++l) {
        std::vector<int> gm(8), gb(8), ge(8);
        for (int o = 0; o < 8; ++o) {
            gm[o] = o;
            gb[o] = T.oct_off[8 * l + o];
            ge[o] = T.oct_off[8 * l + o + 1];
        }
        KF_TRY(make_plan(ctx, P.oct_lvl[l], gm, gb, ge));
    }
    if (P.items_pending) {
        KF_CUDA(cudaEventSynchronize(P.ev_items));
        P.items_pending = false;
        const int h0 = P.items_host[0], h1 = P.items_host[1];
        KF_TRY(eval_items_emit(ctx, P, ctx->tune.eval_cost, h0, P.eval_split ? h1 - h0 : 0));
    }
    return KFMM_OK;
}

static kfmm_status run_gemm(kfmm_ctx *ctx, GemmPlan &pl, const float *A, int64_t a_stride, int M, int K,
                            int lda, const int *src, const int *dst, int src_par, int dst_par, const float *X,
                            int ldx, float *Y, int ldy, const float4 *geom, float alpha, int mode, int ncol,
                            int64_t col_rows, int tag = 0)
{
    KF_TRY(plan_ncol(ctx, pl, ncol));
    if (pl.n_tiles == 0) return KFMM_OK;
    GemmArgs g;
    g.A = A;
    g.a_stride = a_stride;
    g.M = M;
    g.K = K;
    g.lda = lda;
    g.tiles = pl.tiles.as<int4>();
    g.src_idx = src;
    g.dst_idx = dst;
    g.parent = ctx->tree.box_parent.as<int>();
    g.src_par = src_par;
    g.dst_par = dst_par;
    g.X = X;
    g.ldx = ldx;
    g.Y = Y;
    g.ldy = ldy;
    g.geom = geom;
    g.alpha = alpha;
    g.mode = mode;
    g.x_col_rows = col_rows;
    g.y_col_rows = col_rows;
    dim3 grid(pl.n_tiles, (M + GBM - 1) / GBM);
    if (tag == 1) gemm_gather_kernel<1><<<grid, 256, 0, ctx->stream>>>(g);
    else gemm_gather_kernel<0><<<grid, 256, 0, ctx->stream>>>(g);
    KF_LAUNCH();
    return KFMM_OK;
}

// Device time of the work `f` enqueues on the context stream (synchronises).
template <class F> static kfmm_status time_launch(kfmm_ctx *ctx, F f, float *ms)
{
    cudaEvent_t a, b;
    KF_CUDA(cudaEventCreate(&a));
    KF_CUDA(cudaEventCreate(&b));
    KF_CUDA(cudaEventRecord(a, ctx->stream));
    f();
    KF_LAUNCH();
    KF_CUDA(cudaEventRecord(b, ctx->stream));
    KF_CUDA(cudaEventSynchronize(b));
    KF_CUDA(cudaEventElapsedTime(ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return KFMM_OK;
}

// All work of one evaluation, enqueued on ctx->stream.  The first call after a build also
// makes the plans and lazily built tables (it may allocate and synchronise); later calls with
// the same arguments only enqueue, which is what a CUDA graph captures.
// The far images of a periodic cell (|n|_inf >= 2 from the root) into the root's downward
// density, beta_root += R alpha_root for every density column (the root is box 0): one CTA per
// column, one output row per thread; the root's alpha is read by all threads at once.
__global__ void __launch_bounds__(256) lattice_kernel(const float *__restrict__ R, int kd, int ku, int ldr,
                                                      const float *__restrict__ alpha, int64_t a_col,
                                                      float *__restrict__ beta, int64_t b_col)
{
    const float *a = alpha + blockIdx.x * a_col;
    float *b = beta + blockIdx.x * b_col;
    for (int i = threadIdx.x; i < kd; i += blockDim.x) {
        const float *r = R + (size_t)i * ldr;
        float s = 0.f;
        for (int j = 0; j < ku; ++j) s = fmaf(r[j], __ldg(&a[j]), s);
        b[i] += s;
    }
}

// A periodic sum whose single layer has a net force F carries the balancing uniform body force
// -F/V in every cell.  Inside the cell that force makes the far field a non-Navier field, which
// equivalent densities cannot hold; its particular part P(x - c) F, with
// P(d) = d d^T / ((4 lambda + 6 G) V) about the cell centre c, is left out of the lattice
// operator and added here at the targets.  First the net force per density column (FP64):
__global__ void net_force_kernel(int64_t ns, const float *__restrict__ sl, int ldd, double *__restrict__ F)
{
    const int col = blockIdx.y;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
        const float *q = sl + i * ldd + 3 * col;
        a0 += q[0];
        a1 += q[1];
        a2 += q[2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_down_sync(kFull, a0, o);
        a1 += __shfl_down_sync(kFull, a1, o);
        a2 += __shfl_down_sync(kFull, a2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&F[3 * col], a0);
        atomicAdd(&F[3 * col + 1], a1);
        atomicAdd(&F[3 * col + 2], a2);
    }
}

// then u += P(x - c) F at every target (DISP), or its Hooke stress (STRESS, Voigt order)
__global__ void net_force_field_kernel(int64_t nt, const float4 *__restrict__ trg, const int *__restrict__ perm,
                                       const double *__restrict__ F, double cx, double cy, double cz, double coef,
                                       double lam, double G, int stress, float *__restrict__ out, int ldo)
{
    const int col = blockIdx.y;
    const double f[3] = {F[3 * col], F[3 * col + 1], F[3 * col + 2]};
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nt; k += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = trg[k];
        const double d[3] = {p.x - cx, p.y - cy, p.z - cz};
        const double df = d[0] * f[0] + d[1] * f[1] + d[2] * f[2];
        float *o = out + (int64_t)perm[k] * ldo;
        if (!stress) {
            for (int a = 0; a < 3; ++a) o[3 * col + a] += (float)(coef * d[a] * df);
        } else {
            // grad u = coef (df I + d f^T): eps = coef (df I + sym(d f^T)), tr eps = 4 coef df
            const double dg = lam * 4.0 * coef * df + 2.0 * G * coef * df;
            o[6 * col + 0] += (float)(dg + 2.0 * G * coef * d[0] * f[0]);
            o[6 * col + 1] += (float)(dg + 2.0 * G * coef * d[1] * f[1]);
            o[6 * col + 2] += (float)(dg + 2.0 * G * coef * d[2] * f[2]);
            o[6 * col + 3] += (float)(G * coef * (d[1] * f[2] + d[2] * f[1]));
            o[6 * col + 4] += (float)(G * coef * (d[0] * f[2] + d[2] * f[0]));
            o[6 * col + 5] += (float)(G * coef * (d[0] * f[1] + d[1] * f[0]));
        }
    }
}

static kfmm_status fmm_enqueue(kfmm_ctx *ctx, const float *sl, const float *dl, int ncol, int kind, float *out)
{
    Tree &T = ctx->tree;
    Operators &O = ctx->ops;
    Work &W = ctx->work;
    const cudaStream_t st = ctx->stream;
    KF_TRY(ensure_operators(ctx));
    FmmPlans &P = ctx->plans;
    const int n = O.n_surf, m = 3 * n, ld = round_up(m, 16), r = O.rank, rp = round_up(r, 16);
    const int ku = O.ku, kd = O.kd, kup = round_up(ku, 16), kdp = round_up(kd, 16);
    const int nb = T.n_boxes;
    const int64_t ns = T.nsrc;
    // a new tree: its plans are made during this evaluation, the host part overlapping S2M and
    // P2L (plans_begin / plans_end)
    const bool new_tree = !P.valid;
    if (new_tree) KF_TRY(plans_begin(ctx, P));
    {
        // box vectors of all density columns ([column][box][ld]).  The GEMM K loops read their
        // padding lanes, which no kernel writes: a buffer is zeroed in full when it is
        // allocated, and again only when the layout moves the lanes (another row length or
        // column count, or more than one column over another number of boxes).
        DevBuf *bufs[8] = {&W.up_chk, &W.alpha, &W.psi, &W.cdn, &W.dn_chk, &W.beta, &W.up_phi, &W.dn_phi};
        const int lds[8] = {ld, kup, rp, rp, ld, kdp, ld, ld};
        const bool moved = W.zero_ncol != ncol || (ncol > 1 && W.zero_nb != nb);
        for (int k = 0; k < 8; ++k) {
            KF_CUDA(bufs[k]->ensure(sizeof(float) * (size_t)nb * lds[k] * ncol));
            if (moved || W.zero_ptr[k] != bufs[k]->p || W.zero_ld[k] != lds[k]) {
                KF_CUDA(cudaMemsetAsync(bufs[k]->p, 0, bufs[k]->bytes, st));
                W.zero_ptr[k] = bufs[k]->p;
                W.zero_ld[k] = lds[k];
            }
        }
        W.zero_ncol = ncol;
        W.zero_nb = nb;
        if (O.m2l_tc_mtiles > 0) KF_CUDA(W.psi2.ensure(sizeof(uint16_t) * 2 * (size_t)nb * rp * ncol));
    }
    // translation work items of all density columns: x = column * 316 + direction
    auto upload_m2l_items = [&]() -> kfmm_status {
        std::vector<int4> items;
        items.reserve(P.m2l_host.size() * ncol);
        for (int c = 0; c < ncol; ++c)
            for (const int4 &t : P.m2l_host) items.push_back(make_int4(c * 316 + t.x, t.y, t.z, t.w));
        P.n_m2l_items = (int)items.size();
        if (P.n_m2l_items) {
            KF_CUDA(P.m2l_items.ensure(sizeof(int4) * items.size()));
            KF_TRY(upload_async(ctx, P.m2l_items.p, items.data(), sizeof(int4) * items.size()));
        }
        P.m2l_ncol = ncol;
        return KFMM_OK;
    };
    KF_CUDA(W.src_rec.ensure(sizeof(SrcRec) * ns * ncol));
    if (kind == KFMM_STRESS) KF_CUDA(W.tmp.ensure(sizeof(SrcRec) * ns * ncol));
    // one box-operator product over all density columns: tensor cores (three-term split) or
    // FP32 SIMT
    auto box_gemm = [&](GemmPlan &pl, const Operators::TcOp &top, const float *A, int64_t a_stride,
                        int M, int K, int lda, const int *src, const int *dst, int src_par, int dst_par,
                        const float *X, int ldx, float *Y, int ldy, const float4 *gm, float alpha,
                        int mode) -> kfmm_status {
        if (top.on)
            return run_tc_box(ctx, pl, top, src, dst, src_par, dst_par, X, ldx, Y, ldy, gm, alpha, mode, ncol, nb);
        return run_gemm(ctx, pl, A, a_stride, M, K, lda, src, dst, src_par, dst_par, X, ldx, Y, ldy, gm, alpha, mode,
                        ncol, nb);
    };
    const auto kc = make_kelvin<float>(ctx->G, ctx->nu);
    const float4 *geom = P.geom.as<float4>();
    const int ldd = 3 * ncol;
    // every phase below treats the ncol density columns in one launch (grid.y or work items)
    // ---- pack sources (displacement scaling) for the upward pass and P2L
    ctx->phase(KFMM_PH_PACK);
    pack_sources_kernel<<<grid_for(ns * ncol, 256), 256, 0, st>>>(ns, T.src_xyz.as<float4>(), T.src_nrm.as<float4>(),
                                                                   T.src_perm.as<int>(), sl, dl, ldd, ncol, kc.c_sl,
                                                                   kc.c_dl * kc.b12, 1.f, W.src_rec.as<SrcRec>());
    KF_LAUNCH();
    auto check_pot = [&](const int *boxes, int nbx, int use_x, float radius, float *outp, cudaStream_t s) {
        const dim3 grid((unsigned)nbx, (unsigned)ncol);
        const int64_t rc = ns, oc = (int64_t)nb * ld;
        auto go = [&](auto kern) {
            kern<<<grid, kChkThreads, 0, s>>>(boxes, nbx, use_x, T.x_off.as<int>(), T.x_idx.as<int>(),
                                              T.box_src.as<int2>(), geom, O.surf.as<float4>(), n, radius,
                                              W.src_rec.as<SrcRec>(), kc.a34, 3.f / kc.b12, outp, ld, rc, oc,
                                              T.cell);
        };
        const bool two = n <= 2 * kChkThreads;  // check points per thread: 2, else 4
        if (sl && dl) two ? go(check_potential_kernel<true, true, 2>) : go(check_potential_kernel<true, true, 4>);
        else if (sl) two ? go(check_potential_kernel<true, false, 2>) : go(check_potential_kernel<true, false, 4>);
        else two ? go(check_potential_kernel<false, true, 2>) : go(check_potential_kernel<false, true, 4>);
    };
    // arguments of the leaf evaluation (the stress kind re-packs its sources below)
    EvalArgs e;
    e.items = P.eval_items.as<int4>();
    e.n_items = P.n_eval_items;
    e.w_direct_max = T.w_direct_max;
    e.btrg = T.box_trg.as<int2>();
    e.bsrc = T.box_src.as<int2>();
    e.geom = geom;
    e.uo = T.u_off.as<int>();
    e.ui = T.u_idx.as<int>();
    e.wo = T.w_off.as<int>();
    e.wi = T.w_idx.as<int>();
    e.xdo = T.xd_off.as<int>();
    e.xdi = T.xd_idx.as<int>();
    e.trg = T.trg_xyz.as<float4>();
    e.trg_perm = T.trg_perm.as<int>();
    e.rec = W.src_rec.as<SrcRec>();
    e.surf = O.surf.as<float4>();
    e.n_surf = n;
    e.r_in = (float)O.r_inner;
    e.r_out = (float)O.r_outer;
    e.dn_phi = W.dn_phi.as<float>();
    e.up_phi = W.up_phi.as<float>();
    e.ld_phi = ld;
    e.cell = T.cell;
    e.phi_scale = kind == KFMM_DISP ? kc.c_sl : 1.f;
    e.a34 = kc.a34;
    e.b12 = kc.b12;
    e.nu = kc.nu;
    e.c3 = 3.f / kc.b12;
    e.out_scale = kind == KFMM_DISP ? 1.f : kc.c_D;
    e.out = out;
    e.ldo = (kind == KFMM_DISP ? 3 : 6) * ncol;
    e.rec_col = ns;
    e.phi_col = (int64_t)nb * ld;
    e.part = 0;
    // the leaf evaluation: all segments (part 0) or the near (1) or far (2) list of a split
    auto eval_part = [&](int part, cudaStream_t s) {
        EvalArgs a = e;
        a.part = P.eval_split ? part : 0;
        a.items = P.eval_items.as<int4>() + (part == 2 ? P.n_eval_items : 0);
        a.n_items = part == 2 ? P.n_eval_far : P.n_eval_items;
        if (kind == KFMM_DISP) launch_eval<KFMM_DISP>(a, a.n_items, ncol, sl != nullptr, dl != nullptr, s);
        else launch_eval<KFMM_STRESS>(a, a.n_items, ncol, sl != nullptr, dl != nullptr, s);
    };
    // The near field (P2L into the downward check surfaces; the leaf-to-leaf P2P into the
    // zeroed output) needs no multipole data.  With streams on it runs on the side stream,
    // concurrently with the upward pass and M2L, and joins the context stream before the
    // downward pass (P2L) and before the far part of the leaf evaluation (P2P).  Profiling
    // serialises it on the one stream so that each phase keeps its own events.
    const bool overlap = ctx->opt.streams != 0 && !ctx->prof.on && P.eval_split;
    if (overlap && !ctx->side) return ctx->fail(KFMM_ERR_INTERNAL, "side stream missing");
    const cudaStream_t s2 = overlap ? ctx->side : st;
    if (overlap) {
        KF_CUDA(cudaEventRecord(ctx->ev_fork, st));
        KF_CUDA(cudaStreamWaitEvent(s2, ctx->ev_fork, 0));
    }
    // ---- P2L: X-list sources -> downward check surface
    ctx->phase(KFMM_PH_P2L);
    if (T.n_xboxes) {
        check_pot(T.xboxes.as<int>(), T.n_xboxes, 1, (float)O.r_inner, W.dn_chk.as<float>(), s2);
        KF_LAUNCH();
    }
    if (overlap) KF_CUDA(cudaEventRecord(ctx->ev_p2l, s2));
    // ---- S2M: sources -> upward check surface of each leaf
    ctx->phase(KFMM_PH_S2M);
    KF_CUDA(cudaMemsetAsync(W.alpha.p, 0, sizeof(float) * (size_t)nb * kup * ncol, st));
    if (T.n_leaves) {
        check_pot(T.leaves.as<int>(), T.n_leaves, 0, (float)O.r_outer, W.up_chk.as<float>(), st);
        KF_LAUNCH();
    }
    // upward densities of the leaves in the singular basis: alpha = G h S^-1 U^T chk
    ctx->phase(KFMM_PH_UP_PINV);
    KF_TRY(box_gemm(P.leaves, O.tc_s2a_u, O.s2a_u.as<float>(), 0, ku, ld, ld, T.leaves.as<int>(),
                    T.leaves.as<int>(), 0, 0, W.up_chk.as<float>(), ld, W.alpha.as<float>(), kup, geom,
                    (float)ctx->G, 0));
    if (new_tree) {
        // host part of the plans while the GPU runs S2M, P2L and the first box product; then
        // the leaf items
        ctx->phase(KFMM_PH_PLANS);
        KF_TRY(plans_end(ctx, P));
        P.valid = true;
        if (ctx->opt.autotune && !ctx->tune.eval_done && T.n_leaves) {
            // cost cap of the leaf-evaluation items: time each candidate on this tree (the
            // values of the equivalent densities do not change the work; the output is zeroed
            // below, after these launches)
            float best = 1e30f, best_cost = ctx->tune.eval_cost;
            for (float cost : {256.f, 512.f, 1024.f, 2048.f, 4096.f}) {
                KF_TRY(make_eval_items(ctx, P, cost));
                float ms = 0.f;
                KF_TRY(time_launch(ctx, [&]() {
                    eval_part(1, st);
                    if (P.eval_split) eval_part(2, st);
                }, &ms));
                if (ms < best) best = ms, best_cost = cost;
            }
            ctx->tune.eval_cost = best_cost;
            ctx->tune.eval_done = true;
            KF_TRY(make_eval_items(ctx, P, best_cost));
        }
        if (overlap) {  // the side stream's leaf pass needs the items (and the tuning finished)
            KF_CUDA(cudaEventRecord(ctx->ev_plans, st));
            KF_CUDA(cudaStreamWaitEvent(s2, ctx->ev_plans, 0));
        }
    }
    if (O.m2l_tc_mtiles > 0 && P.m2l_ncol != ncol) KF_TRY(upload_m2l_items());
    // ---- leaf evaluation, near part
    ctx->phase(KFMM_PH_EVAL);
    if (kind == KFMM_STRESS) {
        // re-pack with stress scaling: t unscaled, u scaled by c_S / c_D
        pack_sources_kernel<<<grid_for(ns * ncol, 256), 256, 0, s2>>>(
            ns, T.src_xyz.as<float4>(), T.src_nrm.as<float4>(), T.src_perm.as<int>(), sl, dl, ldd, ncol, 1.f,
            kc.c_S / kc.c_D, kc.b12, W.tmp.as<SrcRec>());
        KF_LAUNCH();
        e.rec = W.tmp.as<SrcRec>();
    }
    zero_out_kernel<<<grid_for(T.ntrg * e.ldo, 256), 256, 0, s2>>>(T.ntrg, out, e.ldo, 0, e.ldo);
    KF_LAUNCH();
    if (P.eval_split && P.n_eval_items) {
        eval_part(1, s2);
        KF_LAUNCH();
    }
    if (overlap) KF_CUDA(cudaEventRecord(ctx->ev_near, s2));
    // ---- M2M, bottom-up (children of level l into their parents)
    ctx->phase(KFMM_PH_M2M);
    for (int l = T.n_levels - 1; l >= 1; --l)
        KF_TRY(box_gemm(P.oct_lvl[l], O.tc_mb, O.mb.as<float>(), (int64_t)ku * kup, ku, kup, kup, T.oct_child.as<int>(),
                        T.oct_child.as<int>(), 0, 1, W.alpha.as<float>(), kup, W.alpha.as<float>(), kup, nullptr,
                        1.f, 2));
    // ---- M2L on the V lists in the shared basis: psi = U_r^T V_u alpha, c += C_v psi
    ctx->phase(KFMM_PH_M2L_BASIS);
    KF_TRY(box_gemm(P.all, O.tc_cb, O.cb.as<float>(), 0, r, kup, kup, nullptr, nullptr, 0, 0,
                    W.alpha.as<float>(), kup, W.psi.as<float>(), rp, nullptr, 1.f, 0));
    KF_CUDA(cudaMemsetAsync(W.cdn.p, 0, sizeof(float) * (size_t)nb * rp * ncol, st));
    if (O.m2l_tc_mtiles > 0) {
        if (P.n_m2l_items) {
            const int64_t nchunk = (int64_t)nb * ncol * (rp / 8);
            tc::split_pairs_kernel<<<(unsigned)((nchunk + 255) / 256), 256, 0, st>>>(
                W.psi.as<float>(), (int64_t)nb * ncol, rp, W.psi2.as<uint16_t>(), O.m2l_pairs_rows ? 1 : 0);
            KF_LAUNCH();
            ctx->phase(KFMM_PH_M2L);
            const bool rows = O.m2l_pairs_rows;
            const uint32_t smem = rows ? tc::mt_smem_bytes(rp) : tc::smem_bytes(rp);
            tc::TcArgs ta{O.m2l_tc.as<uint16_t>(), 316, nb, O.m2l_tc_mtiles, r, rp, P.m2l_items.as<int4>(),
                          T.vp_src.as<int>(), T.vp_trg.as<int>(), W.psi2.as<uint16_t>(), W.cdn.as<float>(), rp,
                          P.err.as<int>()};
            tc::TcM2lArgs tm{O.m2l_tc.as<uint16_t>(), 316, nb, rp, P.m2l_items.as<int4>(), T.vp_src.as<int>(),
                             T.vp_trg.as<int>(), W.psi2.as<uint16_t>(), W.cdn.as<float>(), P.err.as<int>()};
            auto launch = [&]() {
                if (rows) tc::tc_m2l_kernel<<<P.n_m2l_items, tc::MT_THREADS, smem, st>>>(tm);
                else tc::tc_gather_gemm_kernel<<<P.n_m2l_items, tc::M2L_THREADS, smem, st>>>(ta);
            };
            if (ctx->opt.autotune && !ctx->tune.m2l_done) {
                // columns (pairs) per work item: time each candidate on this tree, keep the fastest
                float best = 1e30f;
                int best_chunk = ctx->tune.m2l_chunk;
                const int rows_chunks[4] = {512, 1024, 2048, 4096}, tile_chunks[4] = {256, 512, 1024, 2048};
                for (int ci = 0; ci < 4; ++ci) {
                    const int chunk = rows ? rows_chunks[ci] : tile_chunks[ci];
                    make_m2l_host(ctx, P, chunk);
                    KF_TRY(upload_m2l_items());
                    ta.items = tm.items = P.m2l_items.as<int4>();
                    KF_CUDA(cudaMemsetAsync(W.cdn.p, 0, sizeof(float) * (size_t)nb * rp * ncol, st));
                    float ms = 0.f;
                    KF_TRY(time_launch(ctx, launch, &ms));
                    if (ms < best) best = ms, best_chunk = chunk;
                }
                ctx->tune.m2l_chunk = best_chunk;
                ctx->tune.m2l_done = true;
                make_m2l_host(ctx, P, best_chunk);
                KF_TRY(upload_m2l_items());
                ta.items = tm.items = P.m2l_items.as<int4>();
                KF_CUDA(cudaMemsetAsync(W.cdn.p, 0, sizeof(float) * (size_t)nb * rp * ncol, st));
            }
            launch();
            KF_LAUNCH();
        }
    } else {
        ctx->phase(KFMM_PH_M2L);
        KF_TRY(run_gemm(ctx, P.m2l, O.m2l_c.as<float>(), (int64_t)r * rp, r, rp, rp, T.vp_src.as<int>(),
                        T.vp_trg.as<int>(), 0, 0, W.psi.as<float>(), rp, W.cdn.as<float>(), rp, nullptr, 1.f, 2, ncol,
                        nb, 1));
    }
    // ---- downward densities in the singular basis: beta = S^-1 U^T (U_r c + G h chk_P2L),
    //      then L2L top-down, then the equivalent densities needed by the leaf pass
    ctx->phase(KFMM_PH_DOWN);
    KF_TRY(box_gemm(P.all, O.tc_wb, O.wb.as<float>(), 0, kd, rp, rp, nullptr, nullptr, 0, 0,
                    W.cdn.as<float>(), rp, W.beta.as<float>(), kdp, nullptr, 1.f, 0));
    if (T.periodic) {
        // the cell's images beyond the root's neighbours (no list reaches them)
        if (!O.lat_ready) return ctx->fail(KFMM_ERR_INTERNAL, "periodic tree without its lattice operator");
        lattice_kernel<<<(unsigned)ncol, 256, 0, st>>>(O.lat.as<float>(), kd, ku, kup, W.alpha.as<float>(),
                                                       (int64_t)nb * kup, W.beta.as<float>(), (int64_t)nb * kdp);
        KF_LAUNCH();
    }
    if (overlap) KF_CUDA(cudaStreamWaitEvent(st, ctx->ev_p2l, 0));
    KF_TRY(box_gemm(P.xboxes, O.tc_s2a_d, O.s2a_d.as<float>(), 0, kd,
                    ld, ld, T.xboxes.as<int>(), T.xboxes.as<int>(), 0, 0, W.dn_chk.as<float>(), ld,
                    W.beta.as<float>(), kdp, geom, (float)ctx->G, 1));
    // L2L into level l from level l - 1: free space from level 3 (the first far fields are at
    // level 2), a periodic tree from level 1 (the root has the lattice's)
    for (int l = T.periodic ? 1 : 3; l < T.n_levels; ++l)
        KF_TRY(box_gemm(P.oct_lvl[l], O.tc_lb, O.lb.as<float>(),
                        (int64_t)kd * kdp, kd, kdp, kdp, T.oct_child.as<int>(), T.oct_child.as<int>(), 1, 0,
                        W.beta.as<float>(), kdp, W.beta.as<float>(), kdp, nullptr, 1.f, 1));
    KF_TRY(box_gemm(P.leaves, O.tc_vd, O.vd.as<float>(), 0, m, kdp, kdp, T.leaves.as<int>(),
                    T.leaves.as<int>(), 0, 0, W.beta.as<float>(), kdp, W.dn_phi.as<float>(), ld, nullptr, 1.f, 0));
    KF_TRY(box_gemm(P.wboxes, O.tc_vu, O.vu.as<float>(), 0, m, kup,
                    kup, T.wboxes.as<int>(), T.wboxes.as<int>(), 0, 0, W.alpha.as<float>(), kup,
                    W.up_phi.as<float>(), ld, nullptr, 1.f, 0));
    // ---- leaf evaluation, far part (all of it when the lists are not split); joins the
    //      side stream first
    ctx->phase(KFMM_PH_EVAL);
    if (overlap) KF_CUDA(cudaStreamWaitEvent(st, ctx->ev_near, 0));
    if (P.eval_split ? P.n_eval_far > 0 : P.n_eval_items > 0) {
        eval_part(P.eval_split ? 2 : 0, st);
        KF_LAUNCH();
    }
    if (T.periodic && sl) {
        // the particular part of the balancing body force of a net single-layer force
        KF_CUDA(W.net_force.ensure(sizeof(double) * 3 * ncol));
        KF_CUDA(cudaMemsetAsync(W.net_force.p, 0, sizeof(double) * 3 * ncol, st));
        net_force_kernel<<<dim3((unsigned)(2 * ctx->n_sms), (unsigned)ncol), 256, 0, st>>>(ns, sl, ldd,
                                                                                       W.net_force.as<double>());
        KF_LAUNCH();
        const double side = ctx->cell_side, Gd = ctx->G, lam = 2.0 * Gd * ctx->nu / (1.0 - 2.0 * ctx->nu);
        net_force_field_kernel<<<dim3((unsigned)(2 * ctx->n_sms), (unsigned)ncol), 256, 0, st>>>(
            T.ntrg, T.trg_xyz.as<float4>(), T.trg_perm.as<int>(), W.net_force.as<double>(),
            ctx->cell_lo[0] + 0.5 * side, ctx->cell_lo[1] + 0.5 * side, ctx->cell_lo[2] + 0.5 * side,
            1.0 / ((4.0 * lam + 6.0 * Gd) * side * side * side), lam, Gd, kind == KFMM_STRESS ? 1 : 0, out, e.ldo);
        KF_LAUNCH();
    }
    ctx->phase(-1);
    return KFMM_OK;
}

// One thread waits on an mbarrier that nothing arrives on (bounded) and records the time-out.
// Topological derivative of the compliance (Eq. deriv) and the energy density 1/2 sigma:eps
// (integrand of Eq. functional) from stresses [n][6 ncol] (xx, yy, zz, yz, xz, xy per
// column): out [n][2 ncol] = (D^T, w) per column.
__global__ void td_from_stress_kernel(int64_t n, int ncol, const float *__restrict__ s6, float E, float nu,
                                      float *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * ncol) return;
    const int64_t i = e / ncol;
    const int c = (int)(e % ncol);
    const float *s = s6 + i * 6 * ncol + 6 * c;
    const float tr = s[0] + s[1] + s[2];
    const float ss = s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + 2.f * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]);
    out[i * 2 * ncol + 2 * c] =
        0.75f / E * (1.f - nu) / (7.f - 5.f * nu) * (10.f * (1.f + nu) * ss - (1.f + 5.f * nu) * tr * tr);
    out[i * 2 * ncol + 2 * c + 1] = 0.5f * ((1.f + nu) * ss - nu * tr * tr) / E;
}

kfmm_status fmm_td(kfmm_ctx *ctx, const float *stress, int64_t n, int ncol, float *out)
{
    const double E = 2.0 * ctx->G * (1.0 + ctx->nu);
    const int64_t ne = n * ncol;
    td_from_stress_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, ctx->stream>>>(n, ncol, stress, (float)E,
                                                                                  (float)ctx->nu, out);
    KF_LAUNCH();
    return KFMM_OK;
}

__global__ void bounded_wait_probe_kernel(long long polls, int *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!tc::mbar_wait_n(&bar, 0u, polls)) atomicExch(err, 1);
}

kfmm_status selftest_bounded_wait(kfmm_ctx *ctx, long long polls)
{
    if (polls < 1 || polls > (1LL << 24)) return ctx->fail(KFMM_ERR_INVALID_ARG, "polls must be in 1..2^24");
    const cudaStream_t st = ctx->stream;
    DevBuf &err = ctx->plans.err;
    KF_CUDA(err.ensure(sizeof(int)));
    KF_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    bounded_wait_probe_kernel<<<1, 32, 0, st>>>(polls, err.as<int>());
    KF_LAUNCH();
    int herr = 0;
    KF_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    KF_TRY(sync_stream(ctx));
    if (!herr) return KFMM_OK;
    KF_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    return ctx->fail(KFMM_ERR_DEVICE_TIMEOUT, "bounded wait probe: the wait gave up, as designed");
}

void EvalGraph::reset()
{
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    valid = false;
    seen = 0;
    sl = dl = nullptr;
    out = nullptr;
    ncol = kind = -1;
    launches = 0;
}

// One evaluation.  Repeated evaluations with the same arguments (the matvecs of a GMRES
// solve) are captured once into a CUDA graph on a private stream and then replayed on the
// context stream: one launch instead of a few hundred.
kfmm_status fmm_eval(kfmm_ctx *ctx, const float *sl, const float *dl, int ncol, int kind, float *out)
{
    EvalGraph &G = ctx->graph;
    const cudaStream_t st = ctx->stream;
    const bool use_graph = ctx->opt.graphs != 0 && !ctx->prof.on;
    const bool same = G.sl == sl && G.dl == dl && G.out == out && G.ncol == ncol && G.kind == kind;
    if (!same || !use_graph) {
        G.reset();
        G.sl = sl;
        G.dl = dl;
        G.out = out;
        G.ncol = ncol;
        G.kind = kind;
    }
    if (use_graph && same && G.valid) {
        KF_CUDA(cudaGraphLaunch(G.exec, st));
        ctx->n_launch += G.launches;
    } else if (use_graph && same && G.seen >= 1) {
        if (!G.cap_stream) KF_CUDA(cudaStreamCreateWithFlags(&G.cap_stream, cudaStreamNonBlocking));
        // the capture stream starts after the work already queued on the context stream
        cudaEvent_t ev;
        KF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        KF_CUDA(cudaEventRecord(ev, st));
        KF_CUDA(cudaStreamWaitEvent(G.cap_stream, ev, 0));
        KF_CUDA(cudaStreamSynchronize(G.cap_stream));
        cudaEventDestroy(ev);
        const int64_t l0 = ctx->n_launch;
        ctx->stream = G.cap_stream;
        cudaGraph_t graph = nullptr;
        KF_CUDA(cudaStreamBeginCapture(G.cap_stream, cudaStreamCaptureModeThreadLocal));
        const kfmm_status s = fmm_enqueue(ctx, sl, dl, ncol, kind, out);
        const cudaError_t ce = cudaStreamEndCapture(G.cap_stream, &graph);
        ctx->stream = st;
        if (s != KFMM_OK) {
            if (graph) cudaGraphDestroy(graph);
            G.reset();
            return s;
        }
        if (ce != cudaSuccess) return ctx->fail(KFMM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        const cudaError_t ie = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            G.exec = nullptr;
            return ctx->fail(KFMM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
        }
        G.valid = true;
        G.launches = ctx->n_launch - l0;
        KF_CUDA(cudaGraphLaunch(G.exec, st));
    } else {
        KF_TRY(fmm_enqueue(ctx, sl, dl, ncol, kind, out));
        ++G.seen;
    }
    Operators &O = ctx->ops;
    if (O.m2l_tc_mtiles > 0 || O.box_tc) {
        // the tensor-core kernels bound their barrier waits and report a time-out here
        int herr = 0;
        KF_CUDA(cudaMemcpyAsync(&herr, ctx->plans.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        KF_TRY(sync_stream(ctx));
        if (herr) {
            KF_CUDA(cudaMemsetAsync(ctx->plans.err.p, 0, sizeof(int), st));
            return ctx->fail(KFMM_ERR_DEVICE_TIMEOUT, "tensor-core product: a bounded barrier wait gave up");
        }
    }
    return KFMM_OK;
}

}  // namespace kfmm
