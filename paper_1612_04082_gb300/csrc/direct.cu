// direct.cu -- all-pairs summation of Eq. fmm_summation on the GPU (no tree), FP32 or FP64.
// One thread per target; sources are staged through shared memory in tiles, pre-scaled
// once per tile so the inner loop carries no constant factors.  When the targets alone give
// too few CTAs to fill the GPU, the sources are split over a second grid dimension and the
// partial sums are added atomically into the zeroed output.
#include <algorithm>

#include "common.cuh"
#include "kelvin.cuh"

namespace kfmm {

namespace {

constexpr int kDirThreads = 256;

template <typename R> struct SrcTile {
    R y[3][kDirThreads];
    R t[3][kDirThreads];
    R u[3][kDirThreads];
    R n[3][kDirThreads];
    R nup[kDirThreads];
};

template <typename R, int KIND, bool SL, bool DL>
__global__ void __launch_bounds__(kDirThreads)
direct_kernel(const R *__restrict__ trg, int64_t ntrg, const R *__restrict__ src,
              const R *__restrict__ nrm, const R *__restrict__ sl, const R *__restrict__ dl,
              int64_t nsrc, int64_t chunk, KelvinConst<R> kc, R *__restrict__ out)
{
    __shared__ SrcTile<R> tile;
    const int64_t s_begin = (int64_t)blockIdx.y * chunk;
    const int64_t s_end = s_begin + chunk < nsrc ? s_begin + chunk : nsrc;
    const bool split = gridDim.y > 1;
    const int64_t i = (int64_t)blockIdx.x * kDirThreads + threadIdx.x;
    const bool active = i < ntrg;
    R x = 0, y = 0, z = 0;
    if (active) {
        x = trg[3 * i];
        y = trg[3 * i + 1];
        z = trg[3 * i + 2];
    }
    R o[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t base = s_begin; base < s_end; base += kDirThreads) {
        const int64_t j = base + threadIdx.x;
        __syncthreads();
        if (j < s_end) {
            for (int a = 0; a < 3; ++a) tile.y[a][threadIdx.x] = src[3 * j + a];
            R tv[3] = {0, 0, 0}, uv[3] = {0, 0, 0}, nv[3] = {0, 0, 0};
            if (SL)
                for (int a = 0; a < 3; ++a) tv[a] = sl[3 * j + a];
            if (DL)
                for (int a = 0; a < 3; ++a) {
                    uv[a] = dl[3 * j + a];
                    nv[a] = nrm[3 * j + a];
                }
            if (KIND == KFMM_DISP) {
                for (int a = 0; a < 3; ++a) {
                    tv[a] *= kc.c_sl;
                    uv[a] *= kc.c_dl;
                }
            }
            for (int a = 0; a < 3; ++a) {
                tile.t[a][threadIdx.x] = tv[a];
                tile.u[a][threadIdx.x] = uv[a];
                tile.n[a][threadIdx.x] = nv[a];
            }
            tile.nup[threadIdx.x] = kc.b12 * (nv[0] * uv[0] + nv[1] * uv[1] + nv[2] * uv[2]);
        } else {
            // a far-away zero-density source contributes exactly 0
            for (int a = 0; a < 3; ++a) {
                tile.y[a][threadIdx.x] = R(1e30);
                tile.t[a][threadIdx.x] = 0;
                tile.u[a][threadIdx.x] = 0;
                tile.n[a][threadIdx.x] = 0;
            }
            tile.nup[threadIdx.x] = 0;
        }
        __syncthreads();
        const int cnt = (int)((s_end - base) < kDirThreads ? (s_end - base) : kDirThreads);
        for (int s = 0; s < cnt; ++s) {
            R dx = x - tile.y[0][s], dy = y - tile.y[1][s], dz = z - tile.y[2][s];
            if (KIND == KFMM_DISP) {
                if (SL && DL)
                    acc_sl_dl<R>(dx, dy, dz, tile.t[0][s], tile.t[1][s], tile.t[2][s], tile.u[0][s],
                                 tile.u[1][s], tile.u[2][s], tile.n[0][s], tile.n[1][s], tile.n[2][s],
                                 tile.nup[s], kc.a34, kc.b12, o[0], o[1], o[2]);
                else if (SL)
                    acc_sl<R>(dx, dy, dz, tile.t[0][s], tile.t[1][s], tile.t[2][s], kc.a34, o[0], o[1],
                              o[2]);
                else
                    acc_dl<R>(dx, dy, dz, tile.u[0][s], tile.u[1][s], tile.u[2][s], tile.n[0][s],
                              tile.n[1][s], tile.n[2][s], tile.nup[s], kc.b12, o[0], o[1], o[2]);
            } else {
                if (SL) acc_D<R>(dx, dy, dz, tile.t[0][s], tile.t[1][s], tile.t[2][s], kc.b12, o);
                if (DL) {
                    R s6[6] = {0, 0, 0, 0, 0, 0};
                    acc_S<R>(dx, dy, dz, tile.u[0][s], tile.u[1][s], tile.u[2][s], tile.n[0][s],
                             tile.n[1][s], tile.n[2][s], kc.nu, kc.b12, s6);
                    // S carries c_S, D carries c_D; keep D's scale in o and fold S's ratio here
                    const R ratio = kc.c_S / kc.c_D;
                    for (int a = 0; a < 6; ++a) o[a] += ratio * s6[a];
                }
            }
        }
    }
    if (!active) return;
    constexpr int NO = KIND == KFMM_DISP ? 3 : 6;
    const R sc = KIND == KFMM_DISP ? R(1) : kc.c_D;
    for (int a = 0; a < NO; ++a) {
        if (split) atomicAdd(out + NO * i + a, sc * o[a]);
        else out[NO * i + a] = sc * o[a];
    }
}

template <typename R, int KIND>
void launch_direct(const R *trg, int64_t ntrg, const R *src, const R *nrm, const R *sl, const R *dl,
                   int64_t nsrc, KelvinConst<R> kc, R *out, cudaStream_t st, int n_sms)
{
    // source chunks: enough CTAs for ~4 per SM, at least 1024 sources per chunk
    const int64_t tb = (ntrg + kDirThreads - 1) / kDirThreads;
    int64_t ns = (4 * (int64_t)n_sms + tb - 1) / tb;
    ns = std::min<int64_t>(ns, (nsrc + 1023) / 1024);
    ns = std::max<int64_t>(ns, 1);
    ns = std::min<int64_t>(ns, 65535);
    int64_t chunk = (nsrc + ns - 1) / ns;
    chunk = (chunk + kDirThreads - 1) / kDirThreads * kDirThreads;
    ns = std::max<int64_t>(1, (nsrc + chunk - 1) / chunk);
    if (ns > 1) cudaMemsetAsync(out, 0, sizeof(R) * (KIND == KFMM_DISP ? 3 : 6) * ntrg, st);
    dim3 grid((unsigned)tb, (unsigned)ns);
    if (sl && dl)
        direct_kernel<R, KIND, true, true><<<grid, kDirThreads, 0, st>>>(trg, ntrg, src, nrm, sl, dl,
                                                                         nsrc, chunk, kc, out);
    else if (sl)
        direct_kernel<R, KIND, true, false><<<grid, kDirThreads, 0, st>>>(trg, ntrg, src, nrm, sl, dl,
                                                                          nsrc, chunk, kc, out);
    else
        direct_kernel<R, KIND, false, true><<<grid, kDirThreads, 0, st>>>(trg, ntrg, src, nrm, sl, dl,
                                                                          nsrc, chunk, kc, out);
}

}  // namespace

// Stage a possibly-host array on the device; returns the device pointer to use.
static kfmm_status stage(kfmm_ctx *ctx, DevBuf &buf, const void *p, size_t bytes, const void **dp)
{
    if (p == nullptr || is_device_ptr(p)) {
        *dp = p;
        return KFMM_OK;
    }
    KF_CUDA(buf.ensure(bytes));
    KF_CUDA(cudaMemcpyAsync(buf.p, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *dp = buf.p;
    return KFMM_OK;
}

kfmm_status direct_sum(kfmm_ctx *ctx, int precision, const void *trg, int64_t ntrg, const void *src,
                       const void *nrm, int64_t nsrc, const void *sl, const void *dl, int kind,
                       void *out)
{
    const size_t es = precision == KFMM_FP64 ? 8 : 4;
    DevBuf tb, sb, nb, lb, db, ob;
    const void *dtrg, *dsrc, *dnrm, *dsl, *ddl;
    KF_TRY(stage(ctx, tb, trg, es * 3 * ntrg, &dtrg));
    KF_TRY(stage(ctx, sb, src, es * 3 * nsrc, &dsrc));
    KF_TRY(stage(ctx, nb, nrm, es * 3 * nsrc, &dnrm));
    KF_TRY(stage(ctx, lb, sl, es * 3 * nsrc, &dsl));
    KF_TRY(stage(ctx, db, dl, es * 3 * nsrc, &ddl));
    const int nout = kind == KFMM_DISP ? 3 : 6;
    void *dout = out;
    const bool host_out = !is_device_ptr(out);
    if (host_out) {
        KF_CUDA(ob.ensure(es * nout * ntrg));
        dout = ob.p;
    }
    if (precision == KFMM_FP64) {
        auto kc = make_kelvin<double>(ctx->G, ctx->nu);
        if (kind == KFMM_DISP)
            launch_direct<double, KFMM_DISP>((const double *)dtrg, ntrg, (const double *)dsrc,
                                             (const double *)dnrm, (const double *)dsl,
                                             (const double *)ddl, nsrc, kc, (double *)dout, ctx->stream, ctx->n_sms);
        else
            launch_direct<double, KFMM_STRESS>((const double *)dtrg, ntrg, (const double *)dsrc,
                                               (const double *)dnrm, (const double *)dsl,
                                               (const double *)ddl, nsrc, kc, (double *)dout,
                                               ctx->stream, ctx->n_sms);
    } else {
        auto kc = make_kelvin<float>(ctx->G, ctx->nu);
        if (kind == KFMM_DISP)
            launch_direct<float, KFMM_DISP>((const float *)dtrg, ntrg, (const float *)dsrc,
                                            (const float *)dnrm, (const float *)dsl, (const float *)ddl,
                                            nsrc, kc, (float *)dout, ctx->stream, ctx->n_sms);
        else
            launch_direct<float, KFMM_STRESS>((const float *)dtrg, ntrg, (const float *)dsrc,
                                              (const float *)dnrm, (const float *)dsl, (const float *)ddl,
                                              nsrc, kc, (float *)dout, ctx->stream, ctx->n_sms);
    }
    KF_LAUNCH();
    if (host_out) {
        KF_CUDA(cudaMemcpyAsync(out, dout, es * nout * ntrg, cudaMemcpyDeviceToHost, ctx->stream));
    }
    // temporaries are freed at return; make sure the stream no longer uses them
    KF_CUDA(cudaStreamSynchronize(ctx->stream));
    return KFMM_OK;
}

}  // namespace kfmm
