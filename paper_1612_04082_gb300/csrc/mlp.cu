// mlp.cu -- the learned warm start of the GMRES solves: a multilayer perceptron mapping the
// per-element features of an optimisation iteration to the initial guess of its unknowns,
// trained on the GPU on (features, converged unknowns) pairs of earlier iterations.  The paper
// has no learned component (it reuses nothing between iterations); this is the layer the
// optimisation loop adds on top of the method, with plain GMRES from zero as its fallback.
//
// Network: d_0 inputs -> (hidden, ReLU) x (L - 1) -> d_L outputs.  Inputs and targets are
// standardised per column with statistics of the training set.  Master weights are FP32; the
// forward pass uses their BF16 roundings (straight-through: the gradient of the rounded
// weights updates the masters).  Loss: mean squared error over rows and outputs.  Adam.
//
// Kernels: one tiled FP32 GEMM (64 x 64 tiles, K steps of 16, 4 x 4 outputs per thread) with
// arbitrary strides and fused epilogues (bias, ReLU, ReLU mask of the layer input, split-K
// atomic accumulation), plus small elementwise kernels.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "../../include/kifmm_elastic.h"
#include "common.cuh"

using kfmm::DevBuf;
using kfmm::is_device_ptr;

struct kfmm_mlp {
    int L = 0;                  // weight layers
    std::vector<int> d;         // widths d_0 .. d_L
    std::vector<int64_t> w_off, b_off;
    int64_t n_params = 0;
    int bf16 = 1;
    cudaStream_t stream = nullptr;
    std::string err;
    DevBuf master, rounded, grad, m1, m2;  // parameters, rounded copy, gradient, Adam moments
    DevBuf x_mu, x_sd, y_mu, y_sd;         // standardisation
    DevBuf acts;                            // activations H_0 .. H_L for a batch
    DevBuf dacts;                           // gradients of the activations (two buffers)
    DevBuf xs, ys, batch_x, batch_y, idx, loss, tmpx, tmpy, stats;
    int64_t adam_t = 0;
    int64_t cap_rows = 0;
    kfmm_status fail(kfmm_status c, const std::string &m) {
        err = m;
        return c;
    }
};

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

// epilogues
enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_RELU = 2, EPI_RELU_MASK = 3, EPI_ATOMIC = 4 };

// C[i][j] (=|+=) sum_k A(i, k) B(k, j), A(i, k) = A[i sa0 + k sa1], B(k, j) = B[k sb0 + j sb1];
// blockIdx.z splits K into chunks of kchunk (EPI_ATOMIC only).
template <int EPI>
__global__ void __launch_bounds__(256) mlp_gemm_kernel(int M, int N, int K, const float *__restrict__ A, int64_t sa0,
                                                       int64_t sa1, const float *__restrict__ B, int64_t sb0,
                                                       int64_t sb1, float *__restrict__ C, int64_t ldc,
                                                       const float *__restrict__ bias, const float *__restrict__ mask,
                                                       int64_t ldm, int kchunk)
{
    __shared__ float As[TK][TM + 1];
    __shared__ float Bs[TK][TN + 1];
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int k_begin = blockIdx.z * kchunk, k_end = min(K, k_begin + kchunk);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    float acc[4][4] = {};
    for (int k0 = k_begin; k0 < k_end; k0 += TK) {
        for (int e = tid; e < TM * TK; e += 256) {
            const int mm = e / TK, kk = e % TK;
            const int i = m0 + mm, k = k0 + kk;
            As[kk][mm] = (i < M && k < k_end) ? A[(int64_t)i * sa0 + (int64_t)k * sa1] : 0.f;
        }
        for (int e = tid; e < TN * TK; e += 256) {
            const int nn = e % TN, kk = e / TN;
            const int j = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (j < N && k < k_end) ? B[(int64_t)k * sb0 + (int64_t)j * sb1] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx * 4 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = m0 + ty * 4 + r;
        if (i >= M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = n0 + tx * 4 + c;
            if (j >= N) continue;
            float v = acc[r][c];
            float *dst = C + (int64_t)i * ldc + j;
            if (EPI == EPI_BIAS || EPI == EPI_BIAS_RELU) v += bias[j];
            if (EPI == EPI_BIAS_RELU) v = fmaxf(v, 0.f);
            if (EPI == EPI_RELU_MASK) v = mask[(int64_t)i * ldm + j] > 0.f ? v : 0.f;
            if (EPI == EPI_ATOMIC) atomicAdd(dst, v);
            else *dst = v;
        }
    }
}

template <int EPI>
void gemm(cudaStream_t st, int M, int N, int K, const float *A, int64_t sa0, int64_t sa1, const float *B, int64_t sb0,
          int64_t sb1, float *C, int64_t ldc, const float *bias = nullptr, const float *mask = nullptr,
          int64_t ldm = 0)
{
    int splits = 1, kchunk = K;
    if (EPI == EPI_ATOMIC) {
        // enough CTAs for the GPU: split the (long) reduction dimension
        const int tiles = ((M + TM - 1) / TM) * ((N + TN - 1) / TN);
        splits = std::max(1, std::min((K + 255) / 256, (4 * 152 + tiles - 1) / tiles));
        kchunk = ((K + splits - 1) / splits + TK - 1) / TK * TK;
        splits = (K + kchunk - 1) / kchunk;
    }
    dim3 grid((unsigned)((N + TN - 1) / TN), (unsigned)((M + TM - 1) / TM), (unsigned)std::max(1, splits));
    mlp_gemm_kernel<EPI><<<grid, 256, 0, st>>>(M, N, K, A, sa0, sa1, B, sb0, sb1, C, ldc, bias, mask, ldm,
                                               std::max(1, kchunk));
}

// column sums (db = sum over rows of dY)
__global__ void colsum_kernel(int64_t n, int d, const float *__restrict__ X, float *__restrict__ out)
{
    const int j = blockIdx.x;
    float s = 0.f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += X[i * d + j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < blockDim.x / 32 ? w[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(&out[j], s);
    }
}

// column mean and standard deviation (FP64 accumulation), sd floored at 1e-6 (1 if constant)
__global__ void colstats_kernel(int64_t n, int d, const float *__restrict__ X, float *__restrict__ mu,
                                float *__restrict__ sd)
{
    const int j = blockIdx.x;
    double s = 0.0, s2 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = X[i * d + j];
        s += v;
        s2 += v * v;
    }
    __shared__ double a[256], b[256];
    a[threadIdx.x] = s;
    b[threadIdx.x] = s2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            a[threadIdx.x] += a[threadIdx.x + o];
            b[threadIdx.x] += b[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = a[0] / (double)n, var = fmax(b[0] / (double)n - m * m, 0.0);
        mu[j] = (float)m;
        const double s_ = sqrt(var);
        sd[j] = (float)(s_ > 1e-6 * (fabs(m) + 1.0) ? s_ : 1.0);
    }
}

// out = (X - mu) / sd (dir 0) or X * sd + mu (dir 1), rows gathered by idx when non-null
__global__ void affine_kernel(int64_t n, int d, const float *__restrict__ X, const int64_t *__restrict__ idx,
                              const float *__restrict__ mu, const float *__restrict__ sd, int dir,
                              float *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * d) return;
    const int64_t i = e / d;
    const int j = (int)(e % d);
    const float v = X[(idx ? idx[i] : i) * d + j];
    out[e] = dir == 0 ? (v - mu[j]) / sd[j] : v * sd[j] + mu[j];
}

// dY = 2 (Yhat - Y) / (n d), loss += sum (Yhat - Y)^2 / (n d)
__global__ void mse_kernel(int64_t n, int d, const float *__restrict__ Yh, const float *__restrict__ Y,
                           float *__restrict__ dY, double *__restrict__ loss)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    const double inv = 1.0 / ((double)n * d);
    if (e < n * d) {
        const float r = Yh[e] - Y[e];
        dY[e] = (float)(2.0 * inv) * r;
        l = (double)r * r * inv;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
}

// Adam step on the masters, then the BF16-rounded (or plain) forward copy
__global__ void adam_kernel(int64_t n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                            int bf16, float *__restrict__ wr)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wr[i] = bf16 ? __bfloat162float(__float2bfloat16_rn(wi)) : wi;
}

__global__ void round_kernel(int64_t n, const float *__restrict__ w, int bf16, float *__restrict__ wr)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wr[i] = bf16 ? __bfloat162float(__float2bfloat16_rn(w[i])) : w[i];
}

unsigned g1(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

#define MK_CUDA(call)                                                                             \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return m->fail(KFMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
#define MK_LAUNCH()                                                                               \
    do {                                                                                          \
        cudaError_t e_ = cudaGetLastError();                                                      \
        if (e_ != cudaSuccess) return m->fail(KFMM_ERR_CUDA, std::string("mlp kernel: ") + cudaGetErrorString(e_)); \
    } while (0)

// activations for up to `rows` rows: H_0 .. H_L, and two gradient buffers of the widest layer
static kfmm_status ensure_rows(kfmm_mlp *m, int64_t rows)
{
    if (rows <= m->cap_rows) return KFMM_OK;
    int64_t tot = 0, wmax = 0;
    for (int l = 0; l <= m->L; ++l) {
        tot += m->d[l];
        wmax = std::max<int64_t>(wmax, m->d[l]);
    }
    MK_CUDA(m->acts.ensure(sizeof(float) * (size_t)(tot * rows)));
    MK_CUDA(m->dacts.ensure(sizeof(float) * (size_t)(2 * wmax * rows)));
    MK_CUDA(m->batch_x.ensure(sizeof(float) * (size_t)(m->d[0] * rows)));
    MK_CUDA(m->batch_y.ensure(sizeof(float) * (size_t)(m->d[m->L] * rows)));
    m->cap_rows = rows;
    return KFMM_OK;
}

static float *act(kfmm_mlp *m, int l, int64_t rows)
{
    int64_t off = 0;
    for (int k = 0; k < l; ++k) off += m->d[k] * rows;
    return m->acts.as<float>() + off;
}

// forward of `rows` standardised rows already in H_0; output in H_L
static kfmm_status forward(kfmm_mlp *m, int64_t rows)
{
    const float *W = m->rounded.as<float>();
    for (int l = 1; l <= m->L; ++l) {
        const int din = m->d[l - 1], dout = m->d[l];
        const float *X = act(m, l - 1, rows);
        float *Y = act(m, l, rows);
        const float *Wl = W + m->w_off[l - 1], *bl = W + m->b_off[l - 1];
        // Y[i][j] = sum_k X[i][k] W[j][k] + b[j]
        if (l < m->L)
            gemm<EPI_BIAS_RELU>(m->stream, (int)rows, dout, din, X, din, 1, Wl, 1, din, Y, dout, bl);
        else
            gemm<EPI_BIAS>(m->stream, (int)rows, dout, din, X, din, 1, Wl, 1, din, Y, dout, bl);
        MK_LAUNCH();
    }
    return KFMM_OK;
}

// gradient of the mean squared error of H_L against `ys` (rows x d_L) into m->grad (zeroed
// here); adds the loss to *dloss (device double)
static kfmm_status backward(kfmm_mlp *m, int64_t rows, const float *ys, double *dloss)
{
    const int L = m->L;
    MK_CUDA(cudaMemsetAsync(m->grad.p, 0, sizeof(float) * (size_t)m->n_params, m->stream));
    int64_t wmax = 0;
    for (int l = 0; l <= L; ++l) wmax = std::max<int64_t>(wmax, m->d[l]);
    float *dcur = m->dacts.as<float>(), *dnext = dcur + wmax * rows;
    mse_kernel<<<g1(rows * m->d[L]), 256, 0, m->stream>>>(rows, m->d[L], act(m, L, rows), ys, dcur, dloss);
    MK_LAUNCH();
    const float *W = m->rounded.as<float>();
    float *G = m->grad.as<float>();
    for (int l = L; l >= 1; --l) {
        const int din = m->d[l - 1], dout = m->d[l];
        const float *X = act(m, l - 1, rows);
        // dW[j][k] = sum_i dY[i][j] X[i][k]  (M = dout, N = din, K = rows)
        gemm<EPI_ATOMIC>(m->stream, dout, din, (int)rows, dcur, 1, dout, X, din, 1, G + m->w_off[l - 1], din);
        MK_LAUNCH();
        colsum_kernel<<<dout, 256, 0, m->stream>>>(rows, dout, dcur, G + m->b_off[l - 1]);
        MK_LAUNCH();
        if (l > 1) {
            // dX[i][k] = (sum_j dY[i][j] W[j][k]) * (X[i][k] > 0)
            gemm<EPI_RELU_MASK>(m->stream, (int)rows, din, dout, dcur, dout, 1, W + m->w_off[l - 1], din, 1, dnext,
                                din, nullptr, X, din);
            MK_LAUNCH();
            std::swap(dcur, dnext);
        }
    }
    return KFMM_OK;
}

// device copy of a possibly-host array
static kfmm_status to_device(kfmm_mlp *m, DevBuf &buf, const float *p, int64_t count, const float **out)
{
    if (is_device_ptr(p)) {
        *out = p;
        return KFMM_OK;
    }
    MK_CUDA(buf.ensure(sizeof(float) * (size_t)count));
    MK_CUDA(cudaMemcpyAsync(buf.p, p, sizeof(float) * (size_t)count, cudaMemcpyHostToDevice, m->stream));
    *out = buf.as<float>();
    return KFMM_OK;
}

extern "C" {

void mlp_default_train_opts(mlp_train_opts *o)
{
    if (!o) return;
    o->epochs = 200;
    o->batch = 4096;
    o->lr = 1e-3;
    o->seed = 1612;
}

kfmm_status mlp_create(kfmm_mlp **out, int n_in, int n_hidden, int n_layers, int n_out, uint64_t seed)
{
    if (!out || n_in < 1 || n_hidden < 1 || n_layers < 1 || n_out < 1 || n_in > 4096 || n_hidden > 4096 ||
        n_out > 4096 || n_layers > 16)
        return KFMM_ERR_INVALID_ARG;
    *out = nullptr;
    kfmm_mlp *m = new (std::nothrow) kfmm_mlp();
    if (!m) return KFMM_ERR_OOM;
    m->L = n_layers;
    m->d.push_back(n_in);
    for (int l = 1; l < n_layers; ++l) m->d.push_back(n_hidden);
    m->d.push_back(n_out);
    int64_t off = 0;
    for (int l = 1; l <= m->L; ++l) {
        m->w_off.push_back(off);
        off += (int64_t)m->d[l] * m->d[l - 1];
        m->b_off.push_back(off);
        off += m->d[l];
    }
    m->n_params = off;
    // He-uniform weights, zero biases
    std::vector<float> p((size_t)off, 0.f);
    std::mt19937_64 rng(seed);
    for (int l = 1; l <= m->L; ++l) {
        const double a = std::sqrt(6.0 / m->d[l - 1]);
        std::uniform_real_distribution<double> U(-a, a);
        for (int64_t k = 0; k < (int64_t)m->d[l] * m->d[l - 1]; ++k) p[(size_t)(m->w_off[l - 1] + k)] = (float)U(rng);
    }
    const size_t bytes = sizeof(float) * (size_t)off;
    bool ok = m->master.ensure(bytes) == cudaSuccess && m->rounded.ensure(bytes) == cudaSuccess &&
              m->grad.ensure(bytes) == cudaSuccess && m->m1.ensure(bytes) == cudaSuccess &&
              m->m2.ensure(bytes) == cudaSuccess && m->x_mu.ensure(sizeof(float) * n_in) == cudaSuccess &&
              m->x_sd.ensure(sizeof(float) * n_in) == cudaSuccess && m->y_mu.ensure(sizeof(float) * n_out) == cudaSuccess &&
              m->y_sd.ensure(sizeof(float) * n_out) == cudaSuccess && m->loss.ensure(sizeof(double)) == cudaSuccess;
    if (!ok) {
        delete m;
        return KFMM_ERR_OOM;
    }
    cudaMemcpy(m->master.p, p.data(), bytes, cudaMemcpyHostToDevice);
    cudaMemset(m->m1.p, 0, bytes);
    cudaMemset(m->m2.p, 0, bytes);
    std::vector<float> zeros(std::max(n_in, n_out), 0.f), ones(std::max(n_in, n_out), 1.f);
    cudaMemcpy(m->x_mu.p, zeros.data(), sizeof(float) * n_in, cudaMemcpyHostToDevice);
    cudaMemcpy(m->x_sd.p, ones.data(), sizeof(float) * n_in, cudaMemcpyHostToDevice);
    cudaMemcpy(m->y_mu.p, zeros.data(), sizeof(float) * n_out, cudaMemcpyHostToDevice);
    cudaMemcpy(m->y_sd.p, ones.data(), sizeof(float) * n_out, cudaMemcpyHostToDevice);
    round_kernel<<<g1(off), 256>>>(off, m->master.as<float>(), m->bf16, m->rounded.as<float>());
    if (cudaDeviceSynchronize() != cudaSuccess) {
        delete m;
        return KFMM_ERR_CUDA;
    }
    *out = m;
    return KFMM_OK;
}

kfmm_status mlp_destroy(kfmm_mlp *m)
{
    if (!m) return KFMM_ERR_INVALID_ARG;
    cudaStreamSynchronize(m->stream);
    delete m;
    return KFMM_OK;
}

kfmm_status mlp_set_stream(kfmm_mlp *m, void *stream)
{
    if (!m) return KFMM_ERR_INVALID_ARG;
    m->stream = (cudaStream_t)stream;
    return KFMM_OK;
}

int64_t mlp_num_params(const kfmm_mlp *m) { return m ? m->n_params : 0; }

kfmm_status mlp_set_bf16(kfmm_mlp *m, int on)
{
    if (!m) return KFMM_ERR_INVALID_ARG;
    m->bf16 = on ? 1 : 0;
    round_kernel<<<g1(m->n_params), 256, 0, m->stream>>>(m->n_params, m->master.as<float>(), m->bf16,
                                                         m->rounded.as<float>());
    MK_LAUNCH();
    return KFMM_OK;
}

kfmm_status mlp_get_params(const kfmm_mlp *cm, float *p)
{
    kfmm_mlp *m = const_cast<kfmm_mlp *>(cm);
    if (!m || !p) return KFMM_ERR_INVALID_ARG;
    MK_CUDA(cudaMemcpyAsync(p, m->master.p, sizeof(float) * (size_t)m->n_params, cudaMemcpyDefault, m->stream));
    MK_CUDA(cudaStreamSynchronize(m->stream));
    return KFMM_OK;
}

kfmm_status mlp_set_params(kfmm_mlp *m, const float *p)
{
    if (!m || !p) return KFMM_ERR_INVALID_ARG;
    MK_CUDA(cudaMemcpyAsync(m->master.p, p, sizeof(float) * (size_t)m->n_params, cudaMemcpyDefault, m->stream));
    round_kernel<<<g1(m->n_params), 256, 0, m->stream>>>(m->n_params, m->master.as<float>(), m->bf16,
                                                         m->rounded.as<float>());
    MK_LAUNCH();
    MK_CUDA(cudaStreamSynchronize(m->stream));
    return KFMM_OK;
}

kfmm_status mlp_get_normalizers(const kfmm_mlp *cm, float *x_mu, float *x_sd, float *y_mu, float *y_sd)
{
    kfmm_mlp *m = const_cast<kfmm_mlp *>(cm);
    if (!m) return KFMM_ERR_INVALID_ARG;
    const int di = m->d[0], dd = m->d[m->L];
    if (x_mu) MK_CUDA(cudaMemcpyAsync(x_mu, m->x_mu.p, sizeof(float) * di, cudaMemcpyDefault, m->stream));
    if (x_sd) MK_CUDA(cudaMemcpyAsync(x_sd, m->x_sd.p, sizeof(float) * di, cudaMemcpyDefault, m->stream));
    if (y_mu) MK_CUDA(cudaMemcpyAsync(y_mu, m->y_mu.p, sizeof(float) * dd, cudaMemcpyDefault, m->stream));
    if (y_sd) MK_CUDA(cudaMemcpyAsync(y_sd, m->y_sd.p, sizeof(float) * dd, cudaMemcpyDefault, m->stream));
    MK_CUDA(cudaStreamSynchronize(m->stream));
    return KFMM_OK;
}

kfmm_status mlp_forward(kfmm_mlp *m, const float *X, int64_t n, float *Y)
{
    if (!m || !X || !Y || n < 1) return KFMM_ERR_INVALID_ARG;
    const int di = m->d[0], dd = m->d[m->L];
    const float *dX;
    if (to_device(m, m->tmpx, X, n * di, &dX) != KFMM_OK) return KFMM_ERR_CUDA;
    const bool host_out = !is_device_ptr(Y);
    float *dY = Y;
    if (host_out) {
        MK_CUDA(m->tmpy.ensure(sizeof(float) * (size_t)(n * dd)));
        dY = m->tmpy.as<float>();
    }
    const int64_t chunk = 1 << 16;
    kfmm_status s = ensure_rows(m, std::min(n, chunk));
    if (s != KFMM_OK) return s;
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t rows = std::min(chunk, n - r0);
        affine_kernel<<<g1(rows * di), 256, 0, m->stream>>>(rows, di, dX + r0 * di, nullptr, m->x_mu.as<float>(),
                                                            m->x_sd.as<float>(), 0, act(m, 0, rows));
        MK_LAUNCH();
        if ((s = forward(m, rows)) != KFMM_OK) return s;
        affine_kernel<<<g1(rows * dd), 256, 0, m->stream>>>(rows, dd, act(m, m->L, rows), nullptr, m->y_mu.as<float>(),
                                                            m->y_sd.as<float>(), 1, dY + r0 * dd);
        MK_LAUNCH();
    }
    if (host_out) MK_CUDA(cudaMemcpyAsync(Y, dY, sizeof(float) * (size_t)(n * dd), cudaMemcpyDeviceToHost, m->stream));
    MK_CUDA(cudaStreamSynchronize(m->stream));
    return KFMM_OK;
}

kfmm_status mlp_loss_grad(kfmm_mlp *m, const float *X, const float *Y, int64_t n, double *loss, float *grad)
{
    if (!m || !X || !Y || n < 1 || n > (1 << 20)) return KFMM_ERR_INVALID_ARG;
    const int di = m->d[0], dd = m->d[m->L];
    const float *dX, *dYt;
    if (to_device(m, m->tmpx, X, n * di, &dX) != KFMM_OK) return KFMM_ERR_CUDA;
    if (to_device(m, m->tmpy, Y, n * dd, &dYt) != KFMM_OK) return KFMM_ERR_CUDA;
    kfmm_status s = ensure_rows(m, n);
    if (s != KFMM_OK) return s;
    affine_kernel<<<g1(n * di), 256, 0, m->stream>>>(n, di, dX, nullptr, m->x_mu.as<float>(), m->x_sd.as<float>(), 0,
                                                     act(m, 0, n));
    MK_LAUNCH();
    affine_kernel<<<g1(n * dd), 256, 0, m->stream>>>(n, dd, dYt, nullptr, m->y_mu.as<float>(), m->y_sd.as<float>(), 0,
                                                     m->batch_y.as<float>());
    MK_LAUNCH();
    if ((s = forward(m, n)) != KFMM_OK) return s;
    MK_CUDA(cudaMemsetAsync(m->loss.p, 0, sizeof(double), m->stream));
    if ((s = backward(m, n, m->batch_y.as<float>(), m->loss.as<double>())) != KFMM_OK) return s;
    if (loss) MK_CUDA(cudaMemcpyAsync(loss, m->loss.p, sizeof(double), cudaMemcpyDefault, m->stream));
    if (grad) MK_CUDA(cudaMemcpyAsync(grad, m->grad.p, sizeof(float) * (size_t)m->n_params, cudaMemcpyDefault, m->stream));
    MK_CUDA(cudaStreamSynchronize(m->stream));
    return KFMM_OK;
}

kfmm_status mlp_train(kfmm_mlp *m, const float *X, const float *Y, int64_t n, const mlp_train_opts *opts,
                      mlp_train_stats *st)
{
    if (!m || !X || !Y || n < 1) return KFMM_ERR_INVALID_ARG;
    mlp_train_opts o;
    mlp_default_train_opts(&o);
    if (opts) o = *opts;
    if (o.epochs < 1 || o.batch < 1 || !(o.lr > 0)) return m->fail(KFMM_ERR_INVALID_ARG, "mlp_train: bad options");
    const int di = m->d[0], dd = m->d[m->L];
    const float *dX, *dYt;
    if (to_device(m, m->tmpx, X, n * di, &dX) != KFMM_OK) return KFMM_ERR_CUDA;
    if (to_device(m, m->tmpy, Y, n * dd, &dYt) != KFMM_OK) return KFMM_ERR_CUDA;
    // standardisation from the training set
    colstats_kernel<<<di, 256, 0, m->stream>>>(n, di, dX, m->x_mu.as<float>(), m->x_sd.as<float>());
    MK_LAUNCH();
    colstats_kernel<<<dd, 256, 0, m->stream>>>(n, dd, dYt, m->y_mu.as<float>(), m->y_sd.as<float>());
    MK_LAUNCH();
    const int64_t B = std::min<int64_t>(o.batch, n);
    kfmm_status s = ensure_rows(m, B);
    if (s != KFMM_OK) return s;
    MK_CUDA(m->idx.ensure(sizeof(int64_t) * (size_t)n));
    std::vector<int64_t> perm((size_t)n);
    for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = i;
    std::mt19937_64 rng(o.seed);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double last = 0.0;
    MK_CUDA(cudaMemsetAsync(m->loss.p, 0, sizeof(double), m->stream));
    int64_t steps = 0;
    for (int ep = 0; ep < o.epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        MK_CUDA(cudaMemcpyAsync(m->idx.p, perm.data(), sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice, m->stream));
        if (ep == o.epochs - 1) MK_CUDA(cudaMemsetAsync(m->loss.p, 0, sizeof(double), m->stream));
        int64_t nb = 0;
        for (int64_t r0 = 0; r0 + B <= n || (r0 < n && nb == 0); r0 += B, ++nb) {
            const int64_t rows = std::min(B, n - r0);
            const int64_t *idx = m->idx.as<int64_t>() + r0;
            affine_kernel<<<g1(rows * di), 256, 0, m->stream>>>(rows, di, dX, idx, m->x_mu.as<float>(),
                                                                m->x_sd.as<float>(), 0, act(m, 0, rows));
            MK_LAUNCH();
            affine_kernel<<<g1(rows * dd), 256, 0, m->stream>>>(rows, dd, dYt, idx, m->y_mu.as<float>(),
                                                                m->y_sd.as<float>(), 0, m->batch_y.as<float>());
            MK_LAUNCH();
            if ((s = forward(m, rows)) != KFMM_OK) return s;
            if ((s = backward(m, rows, m->batch_y.as<float>(), m->loss.as<double>())) != KFMM_OK) return s;
            ++m->adam_t;
            ++steps;
            const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
            adam_kernel<<<g1(m->n_params), 256, 0, m->stream>>>(m->n_params, m->master.as<float>(), m->grad.as<float>(),
                                                               m->m1.as<float>(), m->m2.as<float>(), (float)o.lr, b1,
                                                               b2, eps, c1, c2, m->bf16, m->rounded.as<float>());
            MK_LAUNCH();
        }
        if (ep == o.epochs - 1) {
            double h = 0.0;
            MK_CUDA(cudaMemcpyAsync(&h, m->loss.p, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
            MK_CUDA(cudaStreamSynchronize(m->stream));
            last = h / (double)std::max<int64_t>(1, nb);
        }
    }
    MK_CUDA(cudaStreamSynchronize(m->stream));
    if (st) {
        st->final_loss = last;
        st->steps = steps;
    }
    return KFMM_OK;
}

const char *mlp_last_error(const kfmm_mlp *m) { return m ? m->err.c_str() : "null context"; }

}  // extern "C"
