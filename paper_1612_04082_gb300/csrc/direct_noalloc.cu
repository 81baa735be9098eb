// direct_noalloc.cu -- a variant of the all-pairs direct sum that allocates nothing.
//
// Some callers cannot call cudaMalloc: a process whose device memory is already handed out
// to a caching allocator (a fresh cudaMalloc fails with out-of-memory even though the
// allocator has room), or code that must not call cudaMalloc / cudaFree once it runs,
// because those calls synchronise the device and stall the caller's other streams.  This
// entry point serves them: the caller passes device inputs and outputs, and the only extra
// memory is a fixed scratch array below, reserved when the library is loaded.
//
// The sum is split over source slices so that few targets still fill the GPU: each CTA
// sums one slice of sources for a tile of targets into the scratch array, and a second
// kernel adds the slices into the output.  Every scratch entry a call reads is first written
// by the same call, so nothing needs clearing between calls.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kelvin.cuh"

namespace kfmm {

// Scratch of the source-split direct sum: 16 MiB, held by every GPU that loads the library
// until the process exits.  Calls share it; calls that overlap on the GPU (different
// streams, or different host threads) race on it and must be serialised by the caller.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kNaThreads = 256;
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device;
// in host code the array's name is only a host-side stand-in).  The cache is keyed by the
// device ordinal only: it is not valid across cudaDeviceReset, after which the module is
// loaded again and the array may sit elsewhere.
kfmm_status scratch_address(kfmm_ctx *ctx, void **out)
{
    int dev = 0;
    KF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return ctx->fail(KFMM_ERR_INVALID_ARG, "direct_noalloc: device ordinal");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        KF_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return KFMM_OK;
}

template <typename R> struct NaTile {
    R y[3][kNaThreads];
    R t[3][kNaThreads];
    R u[3][kNaThreads];
    R n[3][kNaThreads];
    R nup[kNaThreads];
};

// partial[(slice * ntrg + i) * NO + a]: the sum over sources of slice `blockIdx.y` for target i.
template <typename R, int KIND, bool SL, bool DL>
__global__ void __launch_bounds__(kNaThreads)
direct_slice_kernel(const R *__restrict__ trg, int64_t ntrg, const R *__restrict__ src, const R *__restrict__ nrm,
                    const R *__restrict__ sl, const R *__restrict__ dl, int64_t nsrc, int64_t slice_len,
                    KelvinConst<R> kc, R *__restrict__ partial)
{
    constexpr int NO = KIND == KFMM_DISP ? 3 : 6;
    __shared__ NaTile<R> tile;
    const int64_t i = (int64_t)blockIdx.x * kNaThreads + threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.y * slice_len;
    const int64_t s1 = min(nsrc, s0 + slice_len);
    const bool active = i < ntrg;
    R x = 0, y = 0, z = 0;
    if (active) {
        x = trg[3 * i];
        y = trg[3 * i + 1];
        z = trg[3 * i + 2];
    }
    R o[6] = {0, 0, 0, 0, 0, 0};
    const R ratio = kc.c_S / kc.c_D;  // S carries c_S, the sum is scaled by c_D at the end
    for (int64_t base = s0; base < s1; base += kNaThreads) {
        const int64_t j = base + threadIdx.x;
        __syncthreads();
        if (j < s1) {
            R tv[3] = {0, 0, 0}, uv[3] = {0, 0, 0}, nv[3] = {0, 0, 0};
            for (int a = 0; a < 3; ++a) tile.y[a][threadIdx.x] = src[3 * j + a];
            if (SL)
                for (int a = 0; a < 3; ++a) tv[a] = sl[3 * j + a];
            if (DL)
                for (int a = 0; a < 3; ++a) {
                    uv[a] = dl[3 * j + a];
                    nv[a] = nrm[3 * j + a];
                }
            if (KIND == KFMM_DISP)
                for (int a = 0; a < 3; ++a) {
                    tv[a] *= kc.c_sl;
                    uv[a] *= kc.c_dl;
                }
            for (int a = 0; a < 3; ++a) {
                tile.t[a][threadIdx.x] = tv[a];
                tile.u[a][threadIdx.x] = uv[a];
                tile.n[a][threadIdx.x] = nv[a];
            }
            tile.nup[threadIdx.x] = kc.b12 * (nv[0] * uv[0] + nv[1] * uv[1] + nv[2] * uv[2]);
        }
        __syncthreads();
        const int cnt = (int)((s1 - base) < kNaThreads ? (s1 - base) : kNaThreads);
        for (int s = 0; s < cnt; ++s) {
            const R dx = x - tile.y[0][s], dy = y - tile.y[1][s], dz = z - tile.y[2][s];
            if (KIND == KFMM_DISP) {
                if (SL && DL)
                    acc_sl_dl<R>(dx, dy, dz, tile.t[0][s], tile.t[1][s], tile.t[2][s], tile.u[0][s], tile.u[1][s],
                                 tile.u[2][s], tile.n[0][s], tile.n[1][s], tile.n[2][s], tile.nup[s], kc.a34, kc.b12,
                                 o[0], o[1], o[2]);
                else if (SL)
                    acc_sl<R>(dx, dy, dz, tile.t[0][s], tile.t[1][s], tile.t[2][s], kc.a34, o[0], o[1], o[2]);
                else
                    acc_dl<R>(dx, dy, dz, tile.u[0][s], tile.u[1][s], tile.u[2][s], tile.n[0][s], tile.n[1][s],
                              tile.n[2][s], tile.nup[s], kc.b12, o[0], o[1], o[2]);
            } else {
                if (SL) acc_D<R>(dx, dy, dz, tile.t[0][s], tile.t[1][s], tile.t[2][s], kc.b12, o);
                if (DL) {
                    R s6[6] = {0, 0, 0, 0, 0, 0};
                    acc_S<R>(dx, dy, dz, tile.u[0][s], tile.u[1][s], tile.u[2][s], tile.n[0][s], tile.n[1][s],
                             tile.n[2][s], kc.nu, kc.b12, s6);
                    for (int a = 0; a < 6; ++a) o[a] += ratio * s6[a];
                }
            }
        }
    }
    if (!active) return;
    R *p = partial + ((int64_t)blockIdx.y * ntrg + i) * NO;
    for (int a = 0; a < NO; ++a) p[a] = o[a];
}

// out[i * NO + a] = scale * sum over slices of partial
template <typename R>
__global__ void sum_slices_kernel(const R *__restrict__ partial, int nslice, int64_t ntrg, int no, R scale,
                                  R *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ntrg * no) return;
    R s = 0;
    for (int k = 0; k < nslice; ++k) s += partial[(int64_t)k * ntrg * no + e];
    out[e] = scale * s;
}

template <typename R, int KIND>
kfmm_status run_noalloc(kfmm_ctx *ctx, const R *trg, int64_t ntrg, const R *src, const R *nrm, const R *sl,
                        const R *dl, int64_t nsrc, R *out)
{
    constexpr int NO = KIND == KFMM_DISP ? 3 : 6;
    const size_t per_slice = sizeof(R) * NO * (size_t)ntrg;
    if (per_slice > kNoAllocScratchBytes)
        return ctx->fail(KFMM_ERR_INVALID_ARG,
                         "direct_noalloc: ntrg * outputs * element size exceeds the 16 MiB scratch array");
    void *scr = nullptr;
    KF_TRY(scratch_address(ctx, &scr));
    // source slices: enough CTAs to fill the GPU, bounded by the scratch and by one tile each
    const int64_t tiles = (ntrg + kNaThreads - 1) / kNaThreads;
    int64_t nslice = (4 * (int64_t)ctx->n_sms + tiles - 1) / tiles;
    nslice = std::min<int64_t>(nslice, (nsrc + kNaThreads - 1) / kNaThreads);
    nslice = std::min<int64_t>(nslice, (int64_t)(kNoAllocScratchBytes / per_slice));
    nslice = std::max<int64_t>(1, std::min<int64_t>(nslice, 65535));
    const int64_t slice_len = (nsrc + nslice - 1) / nslice;
    const auto kc = make_kelvin<R>(ctx->G, ctx->nu);
    dim3 grid((unsigned)tiles, (unsigned)nslice);
    R *partial = reinterpret_cast<R *>(scr);
    if (sl && dl)
        direct_slice_kernel<R, KIND, true, true><<<grid, kNaThreads, 0, ctx->stream>>>(trg, ntrg, src, nrm, sl, dl, nsrc,
                                                                                       slice_len, kc, partial);
    else if (sl)
        direct_slice_kernel<R, KIND, true, false><<<grid, kNaThreads, 0, ctx->stream>>>(trg, ntrg, src, nrm, sl, dl,
                                                                                        nsrc, slice_len, kc, partial);
    else
        direct_slice_kernel<R, KIND, false, true><<<grid, kNaThreads, 0, ctx->stream>>>(trg, ntrg, src, nrm, sl, dl,
                                                                                        nsrc, slice_len, kc, partial);
    KF_LAUNCH();
    const R scale = KIND == KFMM_DISP ? R(1) : kc.c_D;
    const int64_t ne = ntrg * NO;
    sum_slices_kernel<R><<<(unsigned)((ne + 255) / 256), 256, 0, ctx->stream>>>(partial, (int)nslice, ntrg, NO, scale,
                                                                                 out);
    KF_LAUNCH();
    return KFMM_OK;
}

}  // namespace
}  // namespace kfmm

using namespace kfmm;

extern "C" kfmm_status kfmm_direct_noalloc(kfmm_ctx *ctx, int precision, const void *trg_xyz, int64_t ntrg,
                                           const void *src_xyz, const void *src_nrm, int64_t nsrc, const void *sl_den,
                                           const void *dl_den, int kind, void *out)
{
    if (!ctx) return KFMM_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!trg_xyz || !src_xyz || ntrg < 1 || nsrc < 1 || (!sl_den && !dl_den) || !out ||
        (precision != KFMM_FP32 && precision != KFMM_FP64) || (kind != KFMM_DISP && kind != KFMM_STRESS) ||
        (dl_den && !src_nrm))
        return ctx->fail(KFMM_ERR_INVALID_ARG, "direct_noalloc: bad arguments");
    const void *ptrs[6] = {trg_xyz, src_xyz, src_nrm, sl_den, dl_den, out};
    if (cudaSetDevice(ctx->opt.device) != cudaSuccess) return ctx->fail(KFMM_ERR_CUDA, "cudaSetDevice");
    // every array must be device memory of the context's GPU (checked with it current)
    for (const void *p : ptrs)
        if (p && (!is_device_ptr(p) || foreign_device_ptr(p)))
            return ctx->fail(KFMM_ERR_INVALID_ARG,
                             "direct_noalloc: every array must be device memory of the context's GPU");
    if (precision == KFMM_FP64) {
        if (kind == KFMM_DISP)
            return run_noalloc<double, KFMM_DISP>(ctx, (const double *)trg_xyz, ntrg, (const double *)src_xyz,
                                                  (const double *)src_nrm, (const double *)sl_den,
                                                  (const double *)dl_den, nsrc, (double *)out);
        return run_noalloc<double, KFMM_STRESS>(ctx, (const double *)trg_xyz, ntrg, (const double *)src_xyz,
                                                (const double *)src_nrm, (const double *)sl_den, (const double *)dl_den,
                                                nsrc, (double *)out);
    }
    if (kind == KFMM_DISP)
        return run_noalloc<float, KFMM_DISP>(ctx, (const float *)trg_xyz, ntrg, (const float *)src_xyz,
                                             (const float *)src_nrm, (const float *)sl_den, (const float *)dl_den, nsrc,
                                             (float *)out);
    return run_noalloc<float, KFMM_STRESS>(ctx, (const float *)trg_xyz, ntrg, (const float *)src_xyz,
                                           (const float *)src_nrm, (const float *)sl_den, (const float *)dl_den, nsrc,
                                           (float *)out);
}
