// peak.cu -- FP32 FMA throughput of the GPU the context runs on, measured: the denominator of
// the roofline fraction of the pair-evaluation kernels (P2P, S2M, P2L, L2P, M2P), whose
// bound is the FP32 FMA pipe.
//
// Every thread runs 8 independent chains of dependent FMAs (a <- a * b + c), enough
// independent work per warp to cover the FMA latency with a few resident warps per
// scheduler; the grid is 8 CTAs of 256 threads per multiprocessor.  One FMA counts 2 flop.
// The result is kept live through a conditional store that never happens for these inputs,
// so the compiler keeps every FMA.
#include <algorithm>

#include "common.cuh"

namespace kfmm {

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;

__global__ void __launch_bounds__(kPeakThreads) fma_chain_kernel(int iters, float b, float c, float *sink)
{
    float a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) a[k] = (float)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kPeakChains; ++k) a[k] = __fmaf_rn(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += a[k];
    if (s == -1.2345e-30f) sink[blockIdx.x] = s;  // never true for b < 1, c > 0 (keeps the chains)
}

}  // namespace

kfmm_status measure_fp32_peak(kfmm_ctx *ctx, double *tflops, double *ms_out)
{
    const int blocks = 8 * ctx->n_sms;
    const int iters = 4096;  // 16 x 8 x 4096 FMAs per thread
    DevBuf sink;
    KF_CUDA(sink.ensure(sizeof(float) * blocks));
    cudaEvent_t e0, e1;
    KF_CUDA(cudaEventCreate(&e0));
    KF_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 6; ++rep) {  // the first launch warms up; the fastest counts
        cudaEventRecord(e0, ctx->stream);
        fma_chain_kernel<<<blocks, kPeakThreads, 0, ctx->stream>>>(iters, 0.999f, 1e-3f, sink.as<float>());
        cudaEventRecord(e1, ctx->stream);
        ++ctx->n_launch;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return ctx->fail(KFMM_ERR_CUDA, std::string("fp32 peak: ") + cudaGetErrorString(e));
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0) best = std::min(best, t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    KF_CUDA(cudaGetLastError());
    const double flop = 2.0 * 16.0 * kPeakChains * (double)iters * kPeakThreads * (double)blocks;
    if (tflops) *tflops = flop / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
    return KFMM_OK;
}

}  // namespace kfmm
