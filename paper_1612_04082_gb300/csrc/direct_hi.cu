// direct_hi.cu -- the all-pairs displacement sum of Eq. fmm_summation (single layer Eq. disp_1
// plus double layer Eq. disp_2) to FP64-grade accuracy at FP32 arithmetic rate.
//
// Why: the outer residual of the mixed-precision GMRES (Sec. "Numerical solution", the
// system of Eq. num2) is a difference b - A x whose terms cancel by a factor ||A| |x|| / ||b||
// of ~100 on a clamped cantilever, so a residual of 1e-6 needs the operator to ~1e-9 of its
// terms.  FP64 arithmetic on this GPU runs at 1/64 of the FP32 rate; an FP32 sum done the
// usual way is off by ~1e-7 of its terms.  This sum keeps FP32 arithmetic for almost every
// pair and removes the three error sources that do not average out over many pairs:
//  1. Positions: every coordinate is first shifted by one offset per axis into a single
//     binade [2^k, 2^(k+1)) (2^k >= twice the extent of all points), then carried as an FP32
//     pair hi + lo of its FP64 value.  Any two hi parts then lie within a factor 2, so
//     x_hi - y_hi is exact (Sterbenz) and d = (x_hi - y_hi) + (x_lo - y_lo) is rounded once:
//     its error is the FP32 rounding of d itself, of either sign.  Without the shift, a far
//     pair's x_hi - y_hi rounds to the grid of d and the target's lo part, a fixed offset
//     below that grid, is lost for every such pair -- a systematic shift of the target
//     (measured: a bias of 4e-8 of the sum for a target 10 units from its sources).
//     Before that, every point and vector is rotated by a fixed rotation of generic angles:
//     on a surface made of axis-aligned faces (voxel boundaries) a target's difference to
//     all the sources of one face shares a coordinate, whose single FP32 rounding would
//     otherwise repeat over the whole face (measured: 4x less error on a cantilever).
//  2. Constants: no material constant enters the pair loop.  The sum is carried as four
//     nu-free partial sums (A, B single layer; C, E double layer),
//        U t = c_sl [(3 - 4 nu) A + B],   A = t / r,   B = d (d.t) / r^3
//        P u = c_dl [(1 - 2 nu) C + 3 E], C = [(d.n) u + (d.u) n - (n.u) d] / r^3,
//                                         E = (d.n)(d.u) d / r^5
//     and the FP64 constants are applied once per target (an FP32 constant would scale
//     every pair by the same relative error).
//  3. Accumulation: FP32 partial sums over one tile of sources are folded into FP64.
// 1/r is rsqrtf refined by one Newton-Raphson step formed so that its remaining error is
// rounding of either sign (rsqrt_nr below).  Pairs closer than `near_radius` (their terms
// are the largest, and their FP32 rounding would not average out) are evaluated wholly in
// FP64 from the caller's FP64 arrays; the exactly coincident pair (r = 0) is skipped there.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kelvin.cuh"

namespace kfmm {

namespace {

constexpr int kHiThreads = 128;  // threads per CTA
constexpr int kHiTpt = 2;        // targets per thread
constexpr int kHiTile = 128;     // sources per shared-memory tile (and per FP64 fold)

// The frame the FP32 pairs are evaluated in: x' = R x + off, with R a fixed rotation of
// generic angles and off the per-axis shift into a single binade.  Vectors (densities,
// normals) are rotated by R; the result is rotated back by R^T in FP64.
struct HiFrame {
    double r[9];  // row-major R
    double off[3];
};

__device__ __forceinline__ void rot3(const HiFrame &F, const double *v, double *w)
{
    for (int a = 0; a < 3; ++a) w[a] = F.r[3 * a] * v[0] + F.r[3 * a + 1] * v[1] + F.r[3 * a + 2] * v[2];
}

// One source, 64 bytes: a = (y_hi, n.u), b = (y_lo, t.x), c = (t.y, t.z, u.x, u.y),
// e = (u.z, n) -- in the rotated frame; densities and normal rounded to FP32, n.u formed in
// FP64.
struct HiRec {
    float4 a, b, c, e;
};

// Per-block minimum and maximum of each coordinate over the targets and the sources:
// part[block][0..2] = min, part[block][3..5] = max.
constexpr int kBoundThreads = 256;
__global__ void hi_bounds_kernel(const double *__restrict__ trg, int64_t ntrg, const double *__restrict__ src,
                                 int64_t nsrc, HiFrame F, double *__restrict__ part)
{
    __shared__ double sh[6][kBoundThreads];
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ntrg + nsrc; e += stride) {
        double p[3];
        rot3(F, e < ntrg ? trg + 3 * e : src + 3 * (e - ntrg), p);
        for (int c = 0; c < 3; ++c) {
            lo[c] = fmin(lo[c], p[c]);
            hi[c] = fmax(hi[c], p[c]);
        }
    }
    for (int c = 0; c < 3; ++c) {
        sh[c][threadIdx.x] = lo[c];
        sh[3 + c][threadIdx.x] = hi[c];
    }
    __syncthreads();
    for (int h = kBoundThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int c = 0; c < 3; ++c) {
                sh[c][threadIdx.x] = fmin(sh[c][threadIdx.x], sh[c][threadIdx.x + h]);
                sh[3 + c][threadIdx.x] = fmax(sh[3 + c][threadIdx.x], sh[3 + c][threadIdx.x + h]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[6 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

// hi + lo FP32 parts of v + off (the shifted coordinate)
__device__ __forceinline__ void split_shifted(double v, double off, float &h, float &l)
{
    const double w = v + off;
    h = (float)w;
    l = (float)(w - (double)h);
}

__global__ void hi_pack_kernel(int64_t ns, const double *__restrict__ y, const double *__restrict__ nrm,
                               const double *__restrict__ sl, const double *__restrict__ dl, HiFrame F,
                               HiRec *__restrict__ rec)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ns; j += stride) {
        double yr[3];
        rot3(F, y + 3 * j, yr);
        float yh[3], yl[3];
        for (int c = 0; c < 3; ++c) split_shifted(yr[c], F.off[c], yh[c], yl[c]);
        double t[3] = {0, 0, 0}, u[3] = {0, 0, 0}, n[3] = {0, 0, 0}, nu = 0.0;
        if (sl) rot3(F, sl + 3 * j, t);
        if (dl) {
            const double *uo = dl + 3 * j, *no = nrm + 3 * j;
            nu = no[0] * uo[0] + no[1] * uo[1] + no[2] * uo[2];
            rot3(F, uo, u);
            rot3(F, no, n);
        }
        HiRec r;
        r.a = make_float4(yh[0], yh[1], yh[2], (float)nu);
        r.b = make_float4(yl[0], yl[1], yl[2], (float)t[0]);
        r.c = make_float4((float)t[1], (float)t[2], (float)u[0], (float)u[1]);
        r.e = make_float4((float)u[2], (float)n[0], (float)n[1], (float)n[2]);
        rec[j] = r;
    }
}

// 1/sqrt(a) for a > 0, within about half an ulp and without a sign bias: rsqrtf, then one
// Newton-Raphson step y + y (1 - a y^2) / 2 whose residual 1 - a y^2 is formed with FMAs from
// the exact square y^2 = p_hi + p_lo, so the correction is not rounded away.  (The textbook
// form y (1.5 - 0.5 a y^2) rounds its factor near 1, where floats are twice as dense below 1
// as above it: an estimate short by less than an ulp is then never corrected while one long
// by as much is, and 1/r comes out short on average -- a bias of ~1e-8 that does not average
// out over a sum.)  a = 0 gives NaN; callers select 0 for it.
__device__ __forceinline__ float rsqrt_nr(float a)
{
    const float y = rsqrtf(a);
    const float p_hi = y * y;
    const float p_lo = fmaf(y, y, -p_hi);
    float res = fmaf(-a, p_hi, 1.0f);
    res = fmaf(-a, p_lo, res);
    return fmaf(0.5f * y, res, y);
}

// FP64 evaluation of one near pair into the nu-free sums, in the rotated frame (d, t, u, n
// rotated by R from the caller's FP64 arrays).
template <bool SL, bool DL>
__device__ __noinline__ void near_pair64(const double *x, int64_t j, const double *__restrict__ y,
                                         const double *__restrict__ nrm, const double *__restrict__ sl,
                                         const double *__restrict__ dl, const HiFrame &F, double *A, double *B,
                                         double *C, double *E)
{
    const double d0[3] = {x[0] - y[3 * j], x[1] - y[3 * j + 1], x[2] - y[3 * j + 2]};
    const double r2 = d0[0] * d0[0] + d0[1] * d0[1] + d0[2] * d0[2];
    if (r2 == 0.0) return;  // the coincident point: kernel 0
    double d[3];
    rot3(F, d0, d);
    const double ir = rsqrt(r2), ir2 = ir * ir, ir3 = ir2 * ir;
    if (SL) {
        double t[3];
        rot3(F, sl + 3 * j, t);
        const double bt = (d[0] * t[0] + d[1] * t[1] + d[2] * t[2]) * ir3;
        for (int c = 0; c < 3; ++c) {
            A[c] += ir * t[c];
            B[c] += bt * d[c];
        }
    }
    if (DL) {
        double u[3], n[3];
        rot3(F, dl + 3 * j, u);
        rot3(F, nrm + 3 * j, n);
        const double dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
        const double du = d[0] * u[0] + d[1] * u[1] + d[2] * u[2];
        const double nu = n[0] * u[0] + n[1] * u[1] + n[2] * u[2];
        const double ee = dn * du * ir3 * ir2;
        for (int c = 0; c < 3; ++c) {
            C[c] += (dn * u[c] + du * n[c] - nu * d[c]) * ir3;
            E[c] += ee * d[c];
        }
    }
}

// out[3 i + c] += this CTA's source slice, combined with the FP64 constants.  Each thread
// holds kHiTpt targets (i, i + kHiThreads, ...), so one read of a staged source record serves
// kHiTpt independent pairs.
template <bool SL, bool DL>
__global__ void __launch_bounds__(kHiThreads)
direct_hi_kernel(const double *__restrict__ trg, int64_t ntrg, const HiRec *__restrict__ rec,
                 const double *__restrict__ src, const double *__restrict__ nrm, const double *__restrict__ sl,
                 const double *__restrict__ dl, int64_t nsrc, int64_t chunk, HiFrame F, float near2, double cA,
                 double cB, double cC, double cE, double *__restrict__ out)
{
    constexpr int T = kHiTpt;
    __shared__ float4 sh[4][kHiTile];
    const int64_t s_begin = (int64_t)blockIdx.y * chunk;
    const int64_t s_end = min(nsrc, s_begin + chunk);
    const int64_t i0 = (int64_t)blockIdx.x * kHiThreads * T + threadIdx.x;
    bool active[T];
    double x[T][3];
    float xh[T][3], xl[T][3];
    bool any = false;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t i = i0 + (int64_t)t * kHiThreads;
        active[t] = i < ntrg;
        any = any || active[t];
        for (int c = 0; c < 3; ++c) {
            x[t][c] = active[t] ? trg[3 * i + c] : 0.0;
            xh[t][c] = xl[t][c] = 0.f;
        }
        if (active[t]) {
            double xr[3];
            rot3(F, x[t], xr);
            for (int c = 0; c < 3; ++c) split_shifted(xr[c], F.off[c], xh[t][c], xl[t][c]);
        }
    }
    double A[T][3], B[T][3], C[T][3], E[T][3];
#pragma unroll
    for (int t = 0; t < T; ++t)
        for (int c = 0; c < 3; ++c) A[t][c] = B[t][c] = C[t][c] = E[t][c] = 0.0;
    for (int64_t base = s_begin; base < s_end; base += kHiTile) {
        const int cnt = (int)min((int64_t)kHiTile, s_end - base);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kHiThreads) {
            const HiRec r = rec[base + k];
            sh[0][k] = r.a;
            sh[1][k] = r.b;
            sh[2][k] = r.c;
            sh[3][k] = r.e;
        }
        __syncthreads();
        if (!any) continue;
        float a[T][3], b[T][3], c[T][3], e[T][3];
#pragma unroll
        for (int t = 0; t < T; ++t)
            for (int q = 0; q < 3; ++q) a[t][q] = b[t][q] = c[t][q] = e[t][q] = 0.f;
        for (int s = 0; s < cnt; ++s) {
            const float4 ra = sh[0][s], rb = sh[1][s], rc = sh[2][s], re = sh[3][s];
            const float tx = rb.w, ty = rc.x, tz = rc.y;
            const float ux = rc.z, uy = rc.w, uz = re.x, nx = re.y, ny = re.z, nz = re.w;
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const float dx = (xh[t][0] - ra.x) + (xl[t][0] - rb.x);
                const float dy = (xh[t][1] - ra.y) + (xl[t][1] - rb.y);
                const float dz = (xh[t][2] - ra.z) + (xl[t][2] - rb.z);
                const float r2 = dx * dx + dy * dy + dz * dz;
                const bool nearp = r2 < near2;
                const float ir = nearp ? 0.f : rsqrt_nr(r2);  // near pairs go to the FP64 path below
                const float ir2 = ir * ir, ir3 = ir2 * ir;
                if (SL) {
                    const float bt = (dx * tx + dy * ty + dz * tz) * ir3;
                    a[t][0] += ir * tx;
                    a[t][1] += ir * ty;
                    a[t][2] += ir * tz;
                    b[t][0] += bt * dx;
                    b[t][1] += bt * dy;
                    b[t][2] += bt * dz;
                }
                if (DL) {
                    const float dn = dx * nx + dy * ny + dz * nz;
                    const float du = dx * ux + dy * uy + dz * uz;
                    const float c1 = dn * ir3, c2 = du * ir3, c3 = ra.w * ir3;
                    const float ee = dn * du * ir3 * ir2;
                    c[t][0] += c1 * ux + c2 * nx - c3 * dx;
                    c[t][1] += c1 * uy + c2 * ny - c3 * dy;
                    c[t][2] += c1 * uz + c2 * nz - c3 * dz;
                    e[t][0] += ee * dx;
                    e[t][1] += ee * dy;
                    e[t][2] += ee * dz;
                }
                if (nearp && active[t]) near_pair64<SL, DL>(x[t], base + s, src, nrm, sl, dl, F, A[t], B[t], C[t], E[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < T; ++t)
            for (int q = 0; q < 3; ++q) {
                A[t][q] += a[t][q];
                B[t][q] += b[t][q];
                C[t][q] += c[t][q];
                E[t][q] += e[t][q];
            }
    }
    // back from the rotated frame: out = R^T v
#pragma unroll
    for (int t = 0; t < T; ++t) {
        if (!active[t]) continue;
        const int64_t i = i0 + (int64_t)t * kHiThreads;
        double v[3];
        for (int q = 0; q < 3; ++q) v[q] = cA * A[t][q] + cB * B[t][q] + cC * C[t][q] + cE * E[t][q];
        for (int k = 0; k < 3; ++k)
            atomicAdd(out + 3 * i + k, F.r[k] * v[0] + F.r[3 + k] * v[1] + F.r[6 + k] * v[2]);
    }
}

}  // namespace

kfmm_status direct_hi_sum(kfmm_ctx *ctx, const double *trg, int64_t ntrg, const double *src, const double *nrm,
                          int64_t nsrc, const double *sl, const double *dl, double near_radius, double *out)
{
    // a fixed rotation of generic angles (Euler z-y-x: 0.7, 1.1, 2.3 rad), then one offset per
    // axis that moves every rotated coordinate into [2^k, 2^(k+1)), 2^k >= twice the extent
    HiFrame F;
    {
        const double a = 0.7, b = 1.1, c = 2.3;
        const double ca = std::cos(a), sa = std::sin(a), cb = std::cos(b), sb = std::sin(b), cc = std::cos(c),
                     sc = std::sin(c);
        const double Rz[9] = {ca, -sa, 0, sa, ca, 0, 0, 0, 1}, Ry[9] = {cb, 0, sb, 0, 1, 0, -sb, 0, cb},
                     Rx[9] = {1, 0, 0, 0, cc, -sc, 0, sc, cc};
        double Ryx[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                Ryx[3 * i + j] = 0.0;
                for (int k = 0; k < 3; ++k) Ryx[3 * i + j] += Ry[3 * i + k] * Rx[3 * k + j];
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                F.r[3 * i + j] = 0.0;
                for (int k = 0; k < 3; ++k) F.r[3 * i + j] += Rz[3 * i + k] * Ryx[3 * k + j];
            }
    }
    const int nb = std::max(1, std::min<int>((int)((ntrg + nsrc + kBoundThreads - 1) / kBoundThreads), 2 * ctx->n_sms));
    KF_CUDA(ctx->work.hi_part.ensure(sizeof(double) * 6 * nb));
    hi_bounds_kernel<<<nb, kBoundThreads, 0, ctx->stream>>>(trg, ntrg, src, nsrc, F, ctx->work.hi_part.as<double>());
    KF_LAUNCH();
    std::vector<double> part((size_t)6 * nb);
    KF_CUDA(cudaMemcpyAsync(part.data(), ctx->work.hi_part.p, sizeof(double) * 6 * nb, cudaMemcpyDeviceToHost, ctx->stream));
    KF_CUDA(cudaStreamSynchronize(ctx->stream));
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, width = 0.0;
    for (int b = 0; b < nb; ++b)
        for (int c = 0; c < 3; ++c) {
            lo[c] = std::min(lo[c], part[6 * b + c]);
            hi[c] = std::max(hi[c], part[6 * b + 3 + c]);
        }
    for (int c = 0; c < 3; ++c) width = std::max(width, hi[c] - lo[c]);
    if (!std::isfinite(width)) return ctx->fail(KFMM_ERR_INVALID_ARG, "direct_hi: non-finite coordinates");
    const double base = std::ldexp(1.0, std::max(-60, (int)std::ceil(std::log2(std::max(2.0 * width, 1e-18)))));
    for (int c = 0; c < 3; ++c) F.off[c] = base - lo[c];
    KF_CUDA(ctx->work.hi_rec.ensure(sizeof(HiRec) * (size_t)nsrc));
    HiRec *rec = ctx->work.hi_rec.as<HiRec>();
    hi_pack_kernel<<<(unsigned)std::min<int64_t>((nsrc + 255) / 256, 32LL * ctx->n_sms), 256, 0, ctx->stream>>>(
        nsrc, src, nrm, sl, dl, F, rec);
    KF_LAUNCH();
    KF_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * 3 * ntrg, ctx->stream));
    // source slices: enough CTAs for ~8 per SM, at least 8 tiles of sources per slice
    const int64_t tb = (ntrg + kHiThreads * kHiTpt - 1) / (kHiThreads * kHiTpt);
    int64_t ns = (8 * (int64_t)ctx->n_sms + tb - 1) / tb;
    ns = std::min<int64_t>(ns, (nsrc + 8 * kHiTile - 1) / (8 * kHiTile));
    ns = std::max<int64_t>(1, std::min<int64_t>(ns, 65535));
    int64_t chunk = (nsrc + ns - 1) / ns;
    chunk = (chunk + kHiTile - 1) / kHiTile * kHiTile;
    ns = std::max<int64_t>(1, (nsrc + chunk - 1) / chunk);
    const double pi = 3.14159265358979323846, nu = ctx->nu, G = ctx->G;
    const double c_sl = 1.0 / (16.0 * pi * (1.0 - nu) * G), c_dl = 1.0 / (8.0 * pi * (1.0 - nu));
    const double cA = c_sl * (3.0 - 4.0 * nu), cB = c_sl, cC = c_dl * (1.0 - 2.0 * nu), cE = 3.0 * c_dl;
    // FLT_MIN keeps the exactly coincident pair (r2 = 0) on the FP64 path, which skips it
    const float near2 = (float)std::max(near_radius * near_radius, (double)FLT_MIN);
    dim3 grid((unsigned)tb, (unsigned)ns);
    if (sl && dl)
        direct_hi_kernel<true, true><<<grid, kHiThreads, 0, ctx->stream>>>(trg, ntrg, rec, src, nrm, sl, dl, nsrc,
                                                                           chunk, F, near2, cA, cB, cC, cE, out);
    else if (sl)
        direct_hi_kernel<true, false><<<grid, kHiThreads, 0, ctx->stream>>>(trg, ntrg, rec, src, nrm, sl, dl, nsrc,
                                                                            chunk, F, near2, cA, cB, cC, cE, out);
    else
        direct_hi_kernel<false, true><<<grid, kHiThreads, 0, ctx->stream>>>(trg, ntrg, rec, src, nrm, sl, dl, nsrc,
                                                                            chunk, F, near2, cA, cB, cC, cE, out);
    KF_LAUNCH();
    return KFMM_OK;
}

}  // namespace kfmm
