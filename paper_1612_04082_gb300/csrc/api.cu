// api.cu -- the extern "C" entry points declared in include/kifmm_elastic.h.
// Argument checks, host-pointer staging and dispatch; the work happens in tree.cu, fmm.cu
// and direct.cu.
#include <algorithm>
#include <cmath>
#include <new>

#include "common.cuh"

namespace kfmm {

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool foreign_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return false;
    return a.type == cudaMemoryTypeDevice && a.device != cur;
}

const void *first_foreign(std::initializer_list<const void *> ptrs)
{
    for (const void *p : ptrs)
        if (foreign_device_ptr(p)) return p;
    return nullptr;
}

// Device copy of a possibly-host array (returned pointer is p itself for device memory).
static kfmm_status to_device(kfmm_ctx *ctx, DevBuf &buf, const void *p, size_t bytes, const void **out)
{
    if (foreign_device_ptr(p))
        return ctx->fail(KFMM_ERR_INVALID_ARG, "an array is device memory of another GPU than the context's");
    if (!p || is_device_ptr(p)) {
        *out = p;
        return KFMM_OK;
    }
    KF_CUDA(buf.ensure(bytes));
    KF_CUDA(cudaMemcpyAsync(buf.p, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *out = buf.p;
    return KFMM_OK;
}

}  // namespace kfmm

using namespace kfmm;

extern "C" {

void kfmm_default_options(kfmm_options *opt)
{
    if (!opt) return;
    opt->p = 6;
    opt->leaf_cap = 64;
    opt->max_depth = 20;
    opt->r_inner = 1.05;
    opt->r_outer = 2.95;
    opt->pinv_rtol = 1e-7;
    opt->m2l_rtol = 3e-5;
    opt->m2l_rank_max = 0;
    opt->m2l_tensor_cores = 15;
    opt->device = 0;
    opt->graphs = 1;
    opt->autotune = 1;
    opt->streams = 1;
    opt->eval_item_cost = 0;
}

kfmm_status kfmm_create(kfmm_ctx **out, const kfmm_options *opt)
{
    if (!out) return KFMM_ERR_INVALID_ARG;
    *out = nullptr;
    kfmm_options o;
    kfmm_default_options(&o);
    if (opt) o = *opt;
    if (o.p < 2 || o.p > 8 || o.leaf_cap < 1 || o.max_depth < 1 || o.max_depth > 20 || !(o.r_inner > 1.0) ||
        !(o.r_outer > o.r_inner) || !(o.r_outer < 3.0) || !(o.pinv_rtol > 0.0) || o.m2l_rtol < 0.0 ||
        o.m2l_rank_max < 0 || o.eval_item_cost < 0)
        return KFMM_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device < 0 || o.device >= ndev) {
        cudaGetLastError();
        return KFMM_ERR_CUDA;
    }
    if (cudaSetDevice(o.device) != cudaSuccess) return KFMM_ERR_CUDA;
    kfmm_ctx *c = new (std::nothrow) kfmm_ctx();
    if (!c) return KFMM_ERR_OOM;
    c->opt = o;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o.device) == cudaSuccess && sms > 0)
        c->n_sms = sms;
    cudaGetLastError();
    if (o.eval_item_cost > 0) {
        c->tune.eval_cost = (float)o.eval_item_cost;
        c->tune.eval_done = true;  // fixed by the caller
    }
    if (o.streams) {
        // second stream and fork/join events of the overlapped evaluation (made here, outside
        // any graph capture)
        bool ok = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) == cudaSuccess;
        for (cudaEvent_t *ev : {&c->ev_fork, &c->ev_p2l, &c->ev_near, &c->ev_plans})
            ok = ok && cudaEventCreateWithFlags(ev, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            kfmm_destroy(c);
            return KFMM_ERR_CUDA;
        }
    }
    *out = c;
    return KFMM_OK;
}

kfmm_status kfmm_destroy(kfmm_ctx *ctx)
{
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    cudaSetDevice(ctx->opt.device);
    cudaStreamSynchronize(ctx->stream);
    ctx->graph.reset();
    if (ctx->graph.cap_stream) cudaStreamDestroy(ctx->graph.cap_stream);
    if (ctx->side) {
        cudaStreamSynchronize(ctx->side);
        cudaStreamDestroy(ctx->side);
    }
    for (cudaEvent_t e : {ctx->ev_fork, ctx->ev_p2l, ctx->ev_near, ctx->ev_plans, ctx->plans.ev_items})
        if (e) cudaEventDestroy(e);
    delete ctx;
    return KFMM_OK;
}

kfmm_status kfmm_set_material(kfmm_ctx *ctx, double K, double G)
{
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    if (!(K > 0.0) || !(G > 0.0) || !std::isfinite(K) || !std::isfinite(G))
        return ctx->fail(KFMM_ERR_INVALID_ARG, "material: need K > 0 and G > 0");
    ctx->G = G;
    ctx->nu = (3.0 * K - 2.0 * G) / (2.0 * (3.0 * K + G));
    ctx->graph.reset();  // the constants are arguments of the captured kernels
    return KFMM_OK;
}

kfmm_status kfmm_set_periodic(kfmm_ctx *ctx, int on, const double *lo, double side)
{
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (on) {
        if (!lo || !(side > 0.0) || !std::isfinite(side) || !std::isfinite(lo[0]) || !std::isfinite(lo[1]) ||
            !std::isfinite(lo[2]))
            return ctx->fail(KFMM_ERR_INVALID_ARG, "periodic: need a finite lower corner and side > 0");
        for (int c = 0; c < 3; ++c) ctx->cell_lo[c] = lo[c];
        ctx->cell_side = side;
    }
    ctx->periodic = on != 0;
    ctx->tree.built = false;  // the root and the lists change: build again
    ctx->plans.valid = false;
    ctx->graph.reset();
    return KFMM_OK;
}

kfmm_status kfmm_set_stream(kfmm_ctx *ctx, void *stream)
{
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    if (ctx->stream != (cudaStream_t)stream) {
        // work (and table uploads) queued on the old stream complete first
        KF_CUDA(cudaStreamSynchronize(ctx->stream));
        ctx->staging.reset();
    }
    ctx->stream = (cudaStream_t)stream;
    return KFMM_OK;
}

kfmm_status kfmm_build(kfmm_ctx *ctx, const float *src_xyz, const float *src_nrm, int64_t nsrc, const float *trg_xyz,
                       int64_t ntrg)
{
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    const int64_t so[2] = {0, nsrc}, to[2] = {0, ntrg};
    return kfmm_build_sets(ctx, 1, so, src_xyz, src_nrm, to, trg_xyz);
}

kfmm_status kfmm_build_sets(kfmm_ctx *ctx, int32_t n_sets, const int64_t *src_off, const float *src_xyz,
                            const float *src_nrm, const int64_t *trg_off, const float *trg_xyz)
{
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (n_sets < 1 || n_sets > 65535 || !src_off || !trg_off || !src_xyz || !trg_xyz)
        return ctx->fail(KFMM_ERR_INVALID_ARG, "build: need 1 <= n_sets <= 65535, offsets and point arrays");
    if (src_off[0] != 0 || trg_off[0] != 0)
        return ctx->fail(KFMM_ERR_INVALID_ARG, "build: set offsets must start at 0");
    for (int k = 0; k < n_sets; ++k)
        if (src_off[k + 1] <= src_off[k] || trg_off[k + 1] <= trg_off[k])
            return ctx->fail(KFMM_ERR_INVALID_ARG, "build: every set needs at least one source and one target");
    const int64_t nsrc = src_off[n_sets], ntrg = trg_off[n_sets];
    if (cudaSetDevice(ctx->opt.device) != cudaSuccess) return ctx->fail(KFMM_ERR_CUDA, "cudaSetDevice");
    DevBuf a, b, c;
    const void *ds, *dn, *dt;
    KF_TRY(to_device(ctx, a, src_xyz, sizeof(float) * 3 * nsrc, &ds));
    KF_TRY(to_device(ctx, b, src_nrm, sizeof(float) * 3 * nsrc, &dn));
    bool same = trg_xyz == src_xyz;
    for (int k = 0; k <= n_sets && same; ++k) same = src_off[k] == trg_off[k];
    if (same) dt = ds;  // targets are the sources: one copy, one sort
    else KF_TRY(to_device(ctx, c, trg_xyz, sizeof(float) * 3 * ntrg, &dt));
    ctx->plans.valid = false;
    ctx->graph.reset();
    ctx->phase(KFMM_PH_TREE);
    kfmm_status s = build_forest(ctx, n_sets, src_off, (const float *)ds, (const float *)dn, trg_off,
                                 (const float *)dt);
    ctx->phase(-1);
    cudaStreamSynchronize(ctx->stream);
    return s;
}

kfmm_status kfmm_eval(kfmm_ctx *ctx, const float *sl_den, const float *dl_den, int ncol, int kind, float *out)
{
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->tree.built) return ctx->fail(KFMM_ERR_NOT_BUILT, "eval before build");
    if ((!sl_den && !dl_den) || !out || ncol < 1 || ncol > 32 ||
        (kind != KFMM_DISP && kind != KFMM_STRESS && kind != KFMM_TD))
        return ctx->fail(KFMM_ERR_INVALID_ARG, "eval: need a density, an output, 1 <= ncol <= 32, a valid kind");
    if (dl_den && !ctx->tree.has_nrm)
        return ctx->fail(KFMM_ERR_INVALID_ARG, "eval: double-layer density but the tree was built without normals");
    if (cudaSetDevice(ctx->opt.device) != cudaSuccess) return ctx->fail(KFMM_ERR_CUDA, "cudaSetDevice");
    const int64_t ns = ctx->tree.nsrc, nt = ctx->tree.ntrg;
    const int nout = (kind == KFMM_DISP ? 3 : (kind == KFMM_STRESS ? 6 : 2)) * ncol;
    const void *dsl, *ddl;
    KF_TRY(to_device(ctx, ctx->work.stage_in[0], sl_den, sizeof(float) * 3 * ncol * ns, &dsl));
    KF_TRY(to_device(ctx, ctx->work.stage_in[1], dl_den, sizeof(float) * 3 * ncol * ns, &ddl));
    if (foreign_device_ptr(out))
        return ctx->fail(KFMM_ERR_INVALID_ARG, "eval: out is device memory of another GPU than the context's");
    float *dout = out;
    const bool host_out = !is_device_ptr(out);
    if (host_out) {
        KF_CUDA(ctx->work.stage_out.ensure(sizeof(float) * nout * nt));
        dout = ctx->work.stage_out.as<float>();
    }
    if (kind == KFMM_TD) {
        // the stress sum (Eq. stress_1's kernels), then Eq. deriv and the energy density
        KF_CUDA(ctx->work.td_stress.ensure(sizeof(float) * 6 * ncol * nt));
        KF_TRY(fmm_eval(ctx, (const float *)dsl, (const float *)ddl, ncol, KFMM_STRESS, ctx->work.td_stress.as<float>()));
        KF_TRY(fmm_td(ctx, ctx->work.td_stress.as<float>(), nt, ncol, dout));
    } else {
        KF_TRY(fmm_eval(ctx, (const float *)dsl, (const float *)ddl, ncol, kind, dout));
    }
    if (host_out) {
        KF_CUDA(cudaMemcpyAsync(out, dout, sizeof(float) * nout * nt, cudaMemcpyDeviceToHost, ctx->stream));
        KF_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return KFMM_OK;
}

kfmm_status kfmm_direct(kfmm_ctx *ctx, int precision, const void *trg_xyz, int64_t ntrg, const void *src_xyz,
                        const void *src_nrm, int64_t nsrc, const void *sl_den, const void *dl_den, int kind, void *out)
{
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!trg_xyz || !src_xyz || ntrg < 1 || nsrc < 1 || (!sl_den && !dl_den) || !out ||
        (precision != KFMM_FP32 && precision != KFMM_FP64) || (kind != KFMM_DISP && kind != KFMM_STRESS) ||
        (dl_den && !src_nrm))
        return ctx->fail(KFMM_ERR_INVALID_ARG, "direct: bad arguments");
    if (cudaSetDevice(ctx->opt.device) != cudaSuccess) return ctx->fail(KFMM_ERR_CUDA, "cudaSetDevice");
    if (first_foreign({trg_xyz, src_xyz, src_nrm, sl_den, dl_den, out}))
        return ctx->fail(KFMM_ERR_INVALID_ARG, "direct: an array is device memory of another GPU than the context's");
    return direct_sum(ctx, precision, trg_xyz, ntrg, src_xyz, src_nrm, nsrc, sl_den, dl_den, kind, out);
}

kfmm_status kfmm_direct_hi(kfmm_ctx *ctx, const double *trg_xyz, int64_t ntrg, const double *src_xyz,
                           const double *src_nrm, int64_t nsrc, const double *sl_den, const double *dl_den,
                           double near_radius, double *out)
{
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!trg_xyz || !src_xyz || ntrg < 1 || nsrc < 1 || (!sl_den && !dl_den) || !out || (dl_den && !src_nrm) ||
        !(near_radius >= 0.0) || !std::isfinite(near_radius))
        return ctx->fail(KFMM_ERR_INVALID_ARG, "direct_hi: bad arguments");
    if (cudaSetDevice(ctx->opt.device) != cudaSuccess) return ctx->fail(KFMM_ERR_CUDA, "cudaSetDevice");
    if (first_foreign({trg_xyz, src_xyz, src_nrm, sl_den, dl_den, out}))
        return ctx->fail(KFMM_ERR_INVALID_ARG, "direct_hi: an array is device memory of another GPU than the context's");
    DevBuf a, b, c, d, e, o;
    const void *dt, *ds, *dn, *dsl, *ddl;
    KF_TRY(to_device(ctx, a, trg_xyz, sizeof(double) * 3 * ntrg, &dt));
    KF_TRY(to_device(ctx, b, src_xyz, sizeof(double) * 3 * nsrc, &ds));
    KF_TRY(to_device(ctx, c, src_nrm, sizeof(double) * 3 * nsrc, &dn));
    KF_TRY(to_device(ctx, d, sl_den, sizeof(double) * 3 * nsrc, &dsl));
    KF_TRY(to_device(ctx, e, dl_den, sizeof(double) * 3 * nsrc, &ddl));
    double *dout = out;
    const bool host_out = !is_device_ptr(out);
    if (host_out) {
        KF_CUDA(o.ensure(sizeof(double) * 3 * ntrg));
        dout = o.as<double>();
    }
    KF_TRY(direct_hi_sum(ctx, (const double *)dt, ntrg, (const double *)ds, (const double *)dn, nsrc,
                         (const double *)dsl, (const double *)ddl, near_radius, dout));
    if (host_out) KF_CUDA(cudaMemcpyAsync(out, dout, sizeof(double) * 3 * ntrg, cudaMemcpyDeviceToHost, ctx->stream));
    // staged inputs are freed at return; make sure the stream no longer uses them
    if (host_out || a.p || b.p || c.p || d.p || e.p) KF_CUDA(cudaStreamSynchronize(ctx->stream));
    return KFMM_OK;
}

kfmm_status kfmm_get_stats(const kfmm_ctx *ctx, kfmm_stats *st)
{
    if (!ctx || !st) return KFMM_ERR_INVALID_ARG;
    const Tree &T = ctx->tree;
    std::memset(st, 0, sizeof(*st));
    st->kernel_launches = ctx->n_launch;
    if (!T.built) return KFMM_ERR_NOT_BUILT;
    // the interaction counts are made on first request after a build (synchronises)
    const kfmm_status cs = tree_work_counts(const_cast<kfmm_ctx *>(ctx));
    if (cs != KFMM_OK) return cs;
    st->kernel_launches = ctx->n_launch;
    st->n_src = T.nsrc;
    st->n_trg = T.ntrg;
    st->n_boxes = T.n_boxes;
    st->n_leaves = T.n_leaves;
    st->n_levels = T.n_levels;
    st->m2l_rank = ctx->ops.ready ? ctx->ops.rank : 0;
    const int p = ctx->opt.p;
    st->n_surf = 6 * (p - 1) * (p - 1) + 2;
    st->n_u_pairs = T.n_u;
    st->n_v_pairs = T.n_v;
    st->n_w_pairs = T.n_w;
    st->n_x_pairs = T.n_x;
    st->p2p_interactions = T.p2p_pairs;
    st->s2m_interactions = T.nsrc * st->n_surf;
    st->l2p_interactions = T.l2p_pairs * st->n_surf;
    st->p2l_interactions = T.p2l_pairs * st->n_surf;
    st->kernel_launches = ctx->n_launch;
    st->up_rank = ctx->ops.ready ? ctx->ops.ku : 0;
    st->down_rank = ctx->ops.ready ? ctx->ops.kd : 0;
    st->n_xboxes = T.n_xboxes;
    st->n_wboxes = T.n_wboxes;
    st->m2l_chunk = ctx->tune.m2l_chunk;
    st->eval_item_cost = ctx->tune.eval_cost;
    // resolution of the FP32 positions at the deepest level: half-width of a box there over
    // the FP32 spacing of the largest coordinate of its root cube, the smallest over the sets
    double ratio = 0.0;
    for (int k = 0; k < T.n_sets && 8 * (size_t)k + 3 < T.set_roots.size(); ++k) {
        const double *r = &T.set_roots[8 * (size_t)k];  // lower corner x, y, z, side
        double cmax = 0.0;
        for (int c = 0; c < 3; ++c) cmax = std::max(cmax, std::max(std::fabs(r[c]), std::fabs(r[c] + r[3])));
        const double half = 0.5 * r[3] / std::ldexp(1.0, std::max(0, T.n_levels - 1));
        const double spacing = cmax > 0.0 ? std::ldexp(1.0, (int)std::floor(std::log2(cmax)) - 23) : 1e-45;
        const double q = half / spacing;
        ratio = k == 0 ? q : std::min(ratio, q);
    }
    st->fp32_box_ratio = (float)ratio;
    return KFMM_OK;
}

kfmm_status kfmm_export_tree(const kfmm_ctx *cctx, int32_t *box_level, int32_t *box_anchor, int32_t *box_parent,
                             int32_t *box_src, int32_t *box_trg, int32_t *src_perm, int32_t *trg_perm)
{
    kfmm_ctx *ctx = const_cast<kfmm_ctx *>(cctx);
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    const Tree &T = ctx->tree;
    if (!T.built) return KFMM_ERR_NOT_BUILT;
    const int nb = T.n_boxes;
    if (box_level || box_anchor) {
        std::vector<int4> a(nb);
        KF_CUDA(cudaMemcpy(a.data(), T.box_anchor.p, sizeof(int4) * nb, cudaMemcpyDeviceToHost));
        for (int b = 0; b < nb; ++b) {
            if (box_level) box_level[b] = a[b].w;
            if (box_anchor) {
                box_anchor[3 * b] = a[b].x;
                box_anchor[3 * b + 1] = a[b].y;
                box_anchor[3 * b + 2] = a[b].z;
            }
        }
    }
    if (box_parent) KF_CUDA(cudaMemcpy(box_parent, T.box_parent.p, sizeof(int) * nb, cudaMemcpyDeviceToHost));
    if (box_src) KF_CUDA(cudaMemcpy(box_src, T.box_src.p, sizeof(int2) * nb, cudaMemcpyDeviceToHost));
    if (box_trg) KF_CUDA(cudaMemcpy(box_trg, T.box_trg.p, sizeof(int2) * nb, cudaMemcpyDeviceToHost));
    if (src_perm) KF_CUDA(cudaMemcpy(src_perm, T.src_perm.p, sizeof(int) * T.nsrc, cudaMemcpyDeviceToHost));
    if (trg_perm) KF_CUDA(cudaMemcpy(trg_perm, T.trg_perm.p, sizeof(int) * T.ntrg, cudaMemcpyDeviceToHost));
    return KFMM_OK;
}

kfmm_status kfmm_export_list(const kfmm_ctx *cctx, char which, int32_t *offsets, int32_t *items, int64_t *n_pairs)
{
    kfmm_ctx *ctx = const_cast<kfmm_ctx *>(cctx);
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    const Tree &T = ctx->tree;
    if (!T.built) return KFMM_ERR_NOT_BUILT;
    const DevBuf *o = nullptr, *it = nullptr;
    int64_t n = 0;
    switch (which) {
    case 'U': o = &T.u_off; it = &T.u_idx; n = T.n_u; break;
    case 'V': o = &T.v_off; it = &T.v_idx; n = T.n_v; break;
    case 'W': o = &T.w_off; it = &T.w_idx; n = T.n_w; break;
    case 'X': o = &T.x_off; it = &T.x_idx; n = T.n_x; break;
    default: return ctx->fail(KFMM_ERR_INVALID_ARG, "export_list: which must be U, V, W or X");
    }
    if (n_pairs) *n_pairs = n;
    if (offsets) KF_CUDA(cudaMemcpy(offsets, o->p, sizeof(int) * (T.n_boxes + 1), cudaMemcpyDeviceToHost));
    if (items && n) KF_CUDA(cudaMemcpy(items, it->p, sizeof(int) * n, cudaMemcpyDeviceToHost));
    return KFMM_OK;
}

kfmm_status kfmm_set_profiling(kfmm_ctx *ctx, int enable)
{
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    ctx->prof.on = enable != 0;
    return KFMM_OK;
}

kfmm_status kfmm_get_phase_times(kfmm_ctx *ctx, double *ms, int64_t *counts, int reset)
{
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    KF_CUDA(cudaStreamSynchronize(ctx->stream));
    Profiler &P = ctx->prof;
    for (auto &q : P.pending) {
        float t = 0.f;
        KF_CUDA(cudaEventElapsedTime(&t, q.a, q.b));
        P.ms[q.phase] += t;
        P.count[q.phase] += 1;
        P.pool.push_back(q.a);
        P.pool.push_back(q.b);
    }
    P.pending.clear();
    for (int k = 0; k < KFMM_N_PHASES; ++k) {
        if (ms) ms[k] = P.ms[k];
        if (counts) counts[k] = P.count[k];
        if (reset) {
            P.ms[k] = 0.0;
            P.count[k] = 0;
        }
    }
    return KFMM_OK;
}

kfmm_status kfmm_selftest_bounded_wait(kfmm_ctx *ctx, int64_t polls)
{
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (cudaSetDevice(ctx->opt.device) != cudaSuccess) return ctx->fail(KFMM_ERR_CUDA, "cudaSetDevice");
    return selftest_bounded_wait(ctx, (long long)polls);
}

kfmm_status kfmm_measure_fp32_peak(kfmm_ctx *ctx, double *tflops, double *ms, int32_t *n_sms)
{
    if (!ctx || !tflops) return KFMM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (cudaSetDevice(ctx->opt.device) != cudaSuccess) return ctx->fail(KFMM_ERR_CUDA, "cudaSetDevice");
    if (n_sms) *n_sms = ctx->n_sms;
    return measure_fp32_peak(ctx, tflops, ms);
}

const char *kfmm_status_str(kfmm_status s)
{
    switch (s) {
    case KFMM_OK: return "ok";
    case KFMM_ERR_INVALID_ARG: return "invalid argument";
    case KFMM_ERR_OOM: return "out of memory";
    case KFMM_ERR_CUDA: return "CUDA error";
    case KFMM_ERR_NOT_CONVERGED: return "not converged";
    case KFMM_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    case KFMM_ERR_NOT_BUILT: return "not built";
    case KFMM_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

const char *kfmm_last_error(const kfmm_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

}  // extern "C"
