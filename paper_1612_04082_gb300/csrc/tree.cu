// tree.cu -- octree build and interaction lists on the device (Sec. "Kernel-independent fast
// multipole method": "generation of an octree partitioning of the domain into boxes";
// U/V/W/X lists as in the kernel-independent FMM the paper builds on).
//
// Steps: bounding cube -> 3L-bit Morton keys -> LSD radix sort (8-bit digits, stable,
// written here) -> level-by-level split of every box holding more than leaf_cap sources or
// targets -> colleagues (same-level neighbours) -> U, V, W, X lists as CSR.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "util.cuh"

namespace kfmm {

// ------------------------------------------------------------------------------------
// scan
// ------------------------------------------------------------------------------------
namespace {
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 2;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void scan_tile_kernel(const int *__restrict__ in, int *__restrict__ out, int n,
                                 int *__restrict__ tile_sums)
{
    __shared__ int warp_tot[kScanThreads / 32];
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int incl = warp_incl_scan(s);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int t = warp_tot[lane];
        t = warp_incl_scan(t);
        warp_tot[lane] = t;
    }
    __syncthreads();
    int excl = incl - s + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = excl;
        excl += v[k];
    }
    if (threadIdx.x == kScanThreads - 1 && tile_sums) tile_sums[blockIdx.x] = excl;
}

__global__ void scan_add_kernel(int *__restrict__ out, int n, const int *__restrict__ tile_off)
{
    const int i = blockIdx.x * kScanTile + threadIdx.x;
    const int add = tile_off[blockIdx.x];
    for (int k = i; k < min(n, (int)(blockIdx.x + 1) * kScanTile); k += kScanThreads) out[k] += add;
}

__global__ void scan_total_kernel(const int *last_in, const int *out, int n, int *total)
{
    *total = (n > 0) ? out[n - 1] + last_in[0] : 0;
}

__global__ void copy_last_kernel(const int *in, int n, int *dst) { *dst = n > 0 ? in[n - 1] : 0; }
}  // namespace

// Temporaries live in the context's scan scratch (grow-only, one slot per recursion level),
// so a scan neither allocates nor synchronises in steady state.
static kfmm_status scan_level(kfmm_ctx *ctx, const int *in, int *out, int n, int *total, int depth)
{
    if (n <= 0) {
        if (total) KF_CUDA(cudaMemsetAsync(total, 0, sizeof(int), ctx->stream));
        return KFMM_OK;
    }
    if (depth >= 4) return ctx->fail(KFMM_ERR_INTERNAL, "scan: too many levels");
    const int tiles = (n + kScanTile - 1) / kScanTile;
    DevBuf &slot = ctx->work.scan_tmp[depth];
    KF_CUDA(slot.ensure(sizeof(int) * (size_t)(tiles + 1)));
    int *last = slot.as<int>() + tiles;  // in[n-1], kept because in may alias out
    if (total) {
        copy_last_kernel<<<1, 1, 0, ctx->stream>>>(in, n, last);
        KF_LAUNCH();
    }
    if (tiles == 1) {
        scan_tile_kernel<<<1, kScanThreads, 0, ctx->stream>>>(in, out, n, nullptr);
        KF_LAUNCH();
    } else {
        int *sums = slot.as<int>();
        scan_tile_kernel<<<tiles, kScanThreads, 0, ctx->stream>>>(in, out, n, sums);
        KF_LAUNCH();
        KF_TRY(scan_level(ctx, sums, sums, tiles, nullptr, depth + 1));
        scan_add_kernel<<<tiles, kScanThreads, 0, ctx->stream>>>(out, n, sums);
        KF_LAUNCH();
    }
    if (total) {
        scan_total_kernel<<<1, 1, 0, ctx->stream>>>(last, out, n, total);
        KF_LAUNCH();
    }
    return KFMM_OK;
}

kfmm_status scan_exclusive(kfmm_ctx *ctx, const int *in, int *out, int n, int *total)
{
    return scan_level(ctx, in, out, n, total, 0);
}

kfmm_status sync_stream(kfmm_ctx *ctx)
{
    KF_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->staging.reset();
    return KFMM_OK;
}

kfmm_status upload_async(kfmm_ctx *ctx, void *dst, const void *src, size_t bytes)
{
    if (bytes == 0) return KFMM_OK;
    void *h = ctx->staging.take(bytes);
    if (!h) return ctx->fail(KFMM_ERR_OOM, "pinned staging for a table upload");
    std::memcpy(h, src, bytes);
    KF_CUDA(cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return KFMM_OK;
}

namespace {

// ------------------------------------------------------------------------------------
// bounding box and input checks
// ------------------------------------------------------------------------------------
constexpr int kBBoxBlocks = 2 * kNumSMs;
constexpr int kBBoxThreads = 256;

// Per point set (blockIdx.y) and partial block (blockIdx.x): bounds of the set's sources and
// targets, and a count of non-finite coordinates or normals.
__global__ void bbox_kernel(const int64_t *__restrict__ soff, const float *__restrict__ a,
                            const int64_t *__restrict__ toff, const float *__restrict__ b,
                            const float *__restrict__ nrm, float *__restrict__ part)
{
    const int set = blockIdx.y;
    const int64_t a0 = soff[set], na = soff[set + 1] - a0, b0 = toff[set], nb = toff[set + 1] - b0;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float bad = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += stride) {
        const float *p = i < na ? a + 3 * (a0 + i) : b + 3 * (b0 + i - na);
        for (int c = 0; c < 3; ++c) {
            float v = p[c];
            if (!isfinite(v)) bad += 1.f;
            lo[c] = fminf(lo[c], v);
            hi[c] = fmaxf(hi[c], v);
        }
        if (nrm && i < na)
            for (int c = 0; c < 3; ++c)
                if (!isfinite(nrm[3 * (a0 + i) + c])) bad += 1.f;
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int c = 0; c < 3; ++c) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    __shared__ float sh[kBBoxThreads / 32][7];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        for (int c = 0; c < 3; ++c) {
            sh[warp][c] = lo[c];
            sh[warp][3 + c] = hi[c];
        }
        sh[warp][6] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float r[7];
        for (int c = 0; c < 7; ++c) r[c] = sh[0][c];
        for (int w = 1; w < kBBoxThreads / 32; ++w) {
            for (int c = 0; c < 3; ++c) {
                r[c] = fminf(r[c], sh[w][c]);
                r[3 + c] = fmaxf(r[3 + c], sh[w][3 + c]);
            }
            r[6] += sh[w][6];
        }
        for (int c = 0; c < 7; ++c) part[7 * ((size_t)set * gridDim.x + blockIdx.x) + c] = r[c];
    }
}

// ------------------------------------------------------------------------------------
// Morton keys
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;  // 21 bits
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

// x in the most significant position of each 3-bit digit: octant = 4 bx + 2 by + bz.
__device__ __forceinline__ uint64_t morton3(uint32_t ix, uint32_t iy, uint32_t iz)
{
    return (spread3(ix) << 2) | (spread3(iy) << 1) | spread3(iz);
}

// Keys of the points of several sets: point i belongs to the last set s with off[s] <= i;
// its key is s followed by the 3L-bit Morton code of its cell in the set's root cube
// (roots: 8 doubles per set, lower corner x, y, z, side, 1 / side).
__global__ void keys_kernel(const float *__restrict__ xyz, int64_t n, const int64_t *__restrict__ off, int n_sets,
                            const double *__restrict__ roots, int L, uint64_t *__restrict__ key,
                            int *__restrict__ idx)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const double scale = (double)(1u << L);
    const int top = (1 << L) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int lo = 0, hi = n_sets - 1;
        while (lo < hi) {
            const int m = (lo + hi + 1) >> 1;
            if (off[m] <= i) lo = m;
            else hi = m - 1;
        }
        const double *r = roots + 8 * lo;
        int q[3];
        for (int c = 0; c < 3; ++c) {
            double t = ((double)xyz[3 * i + c] - r[c]) * r[4] * scale;
            int v = (int)floor(t);
            q[c] = v < 0 ? 0 : (v > top ? top : v);
        }
        key[i] = ((uint64_t)lo << (3 * L)) | morton3(q[0], q[1], q[2]);
        idx[i] = (int)i;
    }
}

// ------------------------------------------------------------------------------------
// LSD radix sort of (uint64 key, int value), 8-bit digits, stable
// ------------------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void radix_hist_kernel(const uint64_t *__restrict__ key, int n, int shift,
                                  int *__restrict__ hist, int ntiles)
{
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortTile;
    for (int k = 0; k < kSortItems; ++k) {
        int i = base + k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(key[i] >> shift) & 0xff], 1);
    }
    __syncthreads();
    hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void radix_scatter_kernel(const uint64_t *__restrict__ kin, const int *__restrict__ vin,
                                     uint64_t *__restrict__ kout, int *__restrict__ vout, int n,
                                     int shift, const int *__restrict__ off, int ntiles)
{
    __shared__ int run[256];
    __shared__ int wcnt[kSortThreads / 32][256];
    __shared__ int tot[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    run[tid] = off[tid * ntiles + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    const int base = blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        for (int w = 0; w < kSortThreads / 32; ++w) wcnt[w][tid] = 0;
        const int i = base + r * kSortThreads + tid;
        const bool valid = i < n;
        uint64_t k = valid ? kin[i] : 0;
        int v = valid ? vin[i] : 0;
        int d = valid ? (int)((k >> shift) & 0xff) : 256;
        __syncthreads();
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            int s = 0;
            for (int w = 0; w < kSortThreads / 32; ++w) {
                int c = wcnt[w][tid];
                wcnt[w][tid] = s;
                s += c;
            }
            tot[tid] = s;
        }
        __syncthreads();
        if (valid) {
            int pos = run[d] + wcnt[warp][d] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        run[tid] += tot[tid];
        __syncthreads();
    }
}

kfmm_status radix_sort(kfmm_ctx *ctx, DevBuf &key, DevBuf &val, int n, int bits)
{
    if (n <= 1) return KFMM_OK;
    const int ntiles = (n + kSortTile - 1) / kSortTile;
    DevBuf &k2 = ctx->work.tree_tmp[0], &v2 = ctx->work.tree_tmp[1], &hist = ctx->work.tree_tmp[2];
    KF_CUDA(k2.ensure(sizeof(uint64_t) * n));
    KF_CUDA(v2.ensure(sizeof(int) * n));
    KF_CUDA(hist.ensure(sizeof(int) * 256 * (size_t)ntiles));
    uint64_t *ka = key.as<uint64_t>(), *kb = k2.as<uint64_t>();
    int *va = val.as<int>(), *vb = v2.as<int>();
    const int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        radix_hist_kernel<<<ntiles, kSortThreads, 0, ctx->stream>>>(ka, n, 8 * p, hist.as<int>(), ntiles);
        KF_LAUNCH();
        KF_TRY(scan_exclusive(ctx, hist.as<int>(), hist.as<int>(), 256 * ntiles, nullptr));
        radix_scatter_kernel<<<ntiles, kSortThreads, 0, ctx->stream>>>(ka, va, kb, vb, n, 8 * p,
                                                                        hist.as<int>(), ntiles);
        KF_LAUNCH();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != key.as<uint64_t>()) {
        KF_CUDA(cudaMemcpyAsync(key.p, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        KF_CUDA(cudaMemcpyAsync(val.p, va, sizeof(int) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return KFMM_OK;
}

__global__ void gather_points_kernel(const float *__restrict__ xyz, const int *__restrict__ perm,
                                     int64_t n, float4 *__restrict__ out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int j = perm[i];
        out[i] = make_float4(xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2], 0.f);
    }
}

// ------------------------------------------------------------------------------------
// level-by-level split
// ------------------------------------------------------------------------------------
__device__ __forceinline__ int lower_bound_u64(const uint64_t *a, int lo, int hi, uint64_t v)
{
    while (lo < hi) {
        int m = (lo + hi) >> 1;
        if (a[m] < v) lo = m + 1;
        else hi = m;
    }
    return lo;
}

// ------------------------------------------------------------------------------------
// The level-by-level split and the leaf list in one cooperative launch: per level, every
// block finds the child ranges of a contiguous chunk of the level's boxes (8 lanes per box,
// one binary search per child boundary in the sorted keys), a grid barrier, the level's total
// and the block's first child from the per-block counts, then the block writes its children
// in box order; a last pass lists the leaves.  One launch and one read-back replace a
// launch sequence and a host round trip per level.
// ------------------------------------------------------------------------------------
constexpr int kSplitThreads = 256;
constexpr unsigned kBarrierSpin = 1u << 24;  // polls, ~64 ns apart, before a barrier gives up

// Written by the split kernel, read back once by the host.
struct SplitState {
    int n_boxes, n_levels, n_leaves;
    int err;  // 1: box capacity too small (the host grows it and runs again); 2: barrier time-out
    int deep;  // a box at the deepest level still holds more than leaf_cap points
    unsigned bar_count, bar_gen;
};

struct SplitArgs {
    int L, cap, capb;
    int n_sets;                       // roots: one per point set, box s at level 0
    const int64_t *soff, *toff;       // [n_sets + 1] sorted source / target ranges of the sets
    const uint64_t *skey, *tkey;  // sorted Morton keys of sources and targets
    uint64_t *bkey;
    int4 *banchor;
    int *bparent, *bchild;
    int2 *bsrc, *btrg;
    int *bleaf, *leaves;
    int4 *crange;    // [8 capb]: child ranges of the current level's boxes
    int *ccount;     // [capb]: their non-empty children
    int *block_sum;  // [gridDim.x]
    int *level_off;  // [L + 2]
    SplitState *st;
};

// Grid-wide barrier of a cooperative launch (all blocks resident).  Polls are bounded; a
// time-out is recorded in st->err and makes the caller return.
__device__ __forceinline__ bool grid_barrier(SplitState *st)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &st->bar_gen;
        const unsigned g = *gen;
        int good = 1;
        __threadfence();
        if (atomicAdd(&st->bar_count, 1u) == gridDim.x - 1) {
            atomicExch(&st->bar_count, 0u);
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            for (unsigned it = 0; *gen == g; ++it) {
                if (it >= kBarrierSpin) {
                    good = 0;
                    atomicExch(&st->err, 2);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Exclusive scan of one int per thread over the block; *total receives the block sum.
__device__ __forceinline__ int block_excl_scan(int v, int &total)
{
    __shared__ int wsum[kSplitThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int incl = warp_incl_scan(v);
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int x = lane < kSplitThreads / 32 ? wsum[lane] : 0;
        x = warp_incl_scan(x);
        if (lane < kSplitThreads / 32) wsum[lane] = x;
    }
    __syncthreads();
    const int excl = incl - v + (w > 0 ? wsum[w - 1] : 0);
    total = wsum[kSplitThreads / 32 - 1];
    __syncthreads();
    return excl;
}

// Sum over all blocks of block_sum (all) and over the blocks before this one (pre).
__device__ __forceinline__ void block_prefix(const int *block_sum, int &pre, int &all)
{
    int p = 0, t = 0;
    for (int j = threadIdx.x; j < (int)gridDim.x; j += kSplitThreads) {
        const int v = __ldcg(&block_sum[j]);
        t += v;
        if (j < (int)blockIdx.x) p += v;
    }
    block_excl_scan(p, pre);
    block_excl_scan(t, all);
}

__device__ __forceinline__ uint64_t ldcg_u64(const uint64_t *p)
{
    return (uint64_t)__ldcg(reinterpret_cast<const unsigned long long *>(p));
}

__global__ void __launch_bounds__(kSplitThreads) split_tree_kernel(SplitArgs a)
{
    const unsigned full = 0xffffffffu;
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
    SplitState *st = a.st;
    if (g == 0) {
        for (int r = tid; r < a.n_sets; r += kSplitThreads) {
            a.bkey[r] = (uint64_t)r;  // the set index leads every key of the set
            a.banchor[r] = make_int4(0, 0, 0, 0);
            a.bparent[r] = -1;
            a.bsrc[r] = make_int2((int)a.soff[r], (int)a.soff[r + 1]);
            a.btrg[r] = make_int2((int)a.toff[r], (int)a.toff[r + 1]);
        }
        if (tid == 0) {
            a.level_off[0] = 0;
            a.level_off[1] = a.n_sets;
        }
    }
    if (!grid_barrier(st)) return;
    int first = 0, nb = a.n_sets, n_boxes = a.n_sets, level = 0;
    for (;;) {
        // ---- child ranges and counts of this block's boxes (boxes written by any block at
        //      the previous level: read through L2)
        const int chunk = (nb + G - 1) / G;
        const int b0 = min(nb, g * chunk), b1 = min(nb, b0 + chunk);
        int mine = 0;
        for (int base = b0; base < b1; base += kSplitThreads / 8) {
            const int i = base + (tid >> 3), o = tid & 7;
            const bool valid = i < b1;
            const int b = first + (valid ? i : b0);
            const int2 s = __ldcg(&a.bsrc[b]), t = __ldcg(&a.btrg[b]);
            const bool over = valid && (s.y - s.x > a.cap || t.y - t.x > a.cap);
            const bool split = over && level < a.L;
            if (over && !split && o == 0) atomicExch(&st->deep, 1);
            int sb = s.x, tb = t.x;
            if (split && o > 0) {
                const int sh = 3 * (a.L - level - 1);
                const uint64_t lo = ((ldcg_u64(&a.bkey[b]) << 3) | (uint64_t)o) << sh;
                sb = lower_bound_u64(a.skey, s.x, s.y, lo);
                tb = lower_bound_u64(a.tkey, t.x, t.y, lo);
            }
            int se = __shfl_down_sync(full, sb, 1, 8), te = __shfl_down_sync(full, tb, 1, 8);
            if (o == 7) {
                se = s.y;
                te = t.y;
            }
            const bool nonempty = split && (se > sb || te > tb);
            const unsigned m = __ballot_sync(full, nonempty);
            if (valid) {
                a.crange[8 * (size_t)i + o] = make_int4(sb, se, tb, te);
                if (o == 0) {
                    const int c = __popc((m >> (tid & 24)) & 0xffu);
                    a.ccount[i] = c;
                    mine += c;
                }
            }
        }
        int bsum;
        block_excl_scan(mine, bsum);
        if (tid == 0) a.block_sum[g] = bsum;
        if (!grid_barrier(st)) return;
        int prefix, total;
        block_prefix(a.block_sum, prefix, total);
        if (n_boxes + total > a.capb) {  // the same decision in every block
            if (g == 0 && tid == 0) atomicExch(&st->err, 1);
            return;
        }
        // ---- this block's children, in box order, from n_boxes + prefix on
        int run = n_boxes + prefix;
        for (int base = b0; base < b1; base += kSplitThreads) {
            const int i = base + tid;
            const bool valid = i < b1;
            const int c = valid ? __ldcg(&a.ccount[i]) : 0;
            int tot;
            const int ex = block_excl_scan(c, tot);
            if (valid) {
                const int b = first + i;
                int k = run + ex;
                const int4 an = __ldcg(&a.banchor[b]);
                const uint64_t key = ldcg_u64(&a.bkey[b]);
                for (int o = 0; o < 8; ++o) {
                    int child = -1;
                    if (c > 0) {
                        const int4 r = __ldcg(&a.crange[8 * (size_t)i + o]);
                        if (r.y > r.x || r.w > r.z) {
                            a.bkey[k] = (key << 3) | (uint64_t)o;
                            a.banchor[k] = make_int4(2 * an.x + ((o >> 2) & 1), 2 * an.y + ((o >> 1) & 1),
                                                     2 * an.z + (o & 1), an.w + 1);
                            a.bparent[k] = b;
                            a.bsrc[k] = make_int2(r.x, r.y);
                            a.btrg[k] = make_int2(r.z, r.w);
                            child = k++;
                        }
                    }
                    a.bchild[8 * (size_t)b + o] = child;
                }
            }
            run += tot;
        }
        if (!grid_barrier(st)) return;
        if (total == 0) break;
        first = n_boxes;
        nb = total;
        n_boxes += total;
        ++level;
        if (g == 0 && tid == 0) a.level_off[level + 1] = n_boxes;
    }
    // ---- leaves (no children), listed in box order
    const int chunk = (n_boxes + G - 1) / G;
    const int b0 = min(n_boxes, g * chunk), b1 = min(n_boxes, b0 + chunk);
    int mine = 0;
    for (int b = b0 + tid; b < b1; b += kSplitThreads) {
        bool leaf = true;
        for (int o = 0; o < 8; ++o)
            if (__ldcg(&a.bchild[8 * (size_t)b + o]) >= 0) leaf = false;
        a.bleaf[b] = leaf;
        mine += leaf;
    }
    int bsum;
    block_excl_scan(mine, bsum);
    if (tid == 0) a.block_sum[g] = bsum;
    if (!grid_barrier(st)) return;
    int prefix, total;
    block_prefix(a.block_sum, prefix, total);
    int run = prefix;
    for (int base = b0; base < b1; base += kSplitThreads) {
        const int b = base + tid;
        const int f = b < b1 ? a.bleaf[b] : 0;  // written by this thread above
        int tot;
        const int ex = block_excl_scan(f, tot);
        if (f) a.leaves[run + ex] = b;
        run += tot;
    }
    if (g == 0 && tid == 0) {
        st->n_boxes = n_boxes;
        st->n_levels = level + 1;
        st->n_leaves = total;
    }
}

// ------------------------------------------------------------------------------------
// colleagues and lists
// ------------------------------------------------------------------------------------
struct TreeView {
    int L;
    int n_boxes;
    const uint64_t *key;
    const int4 *anchor;
    const int *parent;
    const int *child;
    const int *leaf;
    const int *colleague;
    const int *level_off;  // device copy, n_levels + 1
    int n_levels;
    int periodic;  // colleagues wrap around the root cell (entries carry the image)
};

// the box of set `set` at (level, ix, iy, iz), or -1
__device__ __forceinline__ int find_box(const TreeView &tv, int level, uint64_t set, int ix, int iy, int iz)
{
    const int side = 1 << level;
    if (ix < 0 || iy < 0 || iz < 0 || ix >= side || iy >= side || iz >= side) return -1;
    if (level >= tv.n_levels) return -1;
    const uint64_t k = (set << (3 * level)) | morton3(ix, iy, iz);
    int lo = tv.level_off[level], hi = tv.level_off[level + 1];
    while (lo < hi) {
        int m = (lo + hi) >> 1;
        if (tv.key[m] < k) lo = m + 1;
        else hi = m;
    }
    if (lo < tv.level_off[level + 1] && tv.key[lo] == k) return lo;
    return -1;
}

// The 27 boxes at the box's level around it (slot 13: itself), -1 where there is none.  In a
// periodic tree a position outside the root cell wraps around it: the entry is the box at the
// wrapped position, moved back by one cell (its image code, see ent_make).
__global__ void colleague_kernel(TreeView tv, int *__restrict__ coll)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= tv.n_boxes) return;
    const int4 a = tv.anchor[b];
    const uint64_t set = tv.key[b] >> (3 * a.w);  // colleagues come from the box's own set
    const int side = 1 << a.w;
    int c = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz, ++c) {
                if (c == 13) {
                    coll[27 * b + c] = b;
                    continue;
                }
                int x = a.x + dx, y = a.y + dy, z = a.z + dz, img = 13;
                if (tv.periodic) {
                    const int sx = x < 0 ? -1 : (x >= side ? 1 : 0), sy = y < 0 ? -1 : (y >= side ? 1 : 0),
                              sz = z < 0 ? -1 : (z >= side ? 1 : 0);
                    x -= sx * side;
                    y -= sy * side;
                    z -= sz * side;
                    img = 9 * (sx + 1) + 3 * (sy + 1) + (sz + 1);
                }
                const int f = find_box(tv, a.w, set, x, y, z);
                coll[27 * b + c] = f < 0 ? -1 : ent_make(f, img);
            }
}

// The image of entry e and the (unmoved) box with anchor b, at possibly different levels, touch
// or overlap as closed boxes.
__device__ __forceinline__ bool adjacent(const TreeView &tv, int e, const int4 &b)
{
    const int4 a = tv.anchor[ent_box(e)];
    int sx, sy, sz;
    ent_shift(e, sx, sy, sz);
    const int L = tv.L, sa = L - a.w, sb = L - b.w, full = 1 << L;
    const int ax0 = a.x * (1 << sa) + sx * full, ay0 = a.y * (1 << sa) + sy * full,
              az0 = a.z * (1 << sa) + sz * full, la = 1 << sa;
    const int bx0 = b.x << sb, by0 = b.y << sb, bz0 = b.z << sb, lb = 1 << sb;
    return ax0 <= bx0 + lb && bx0 <= ax0 + la && ay0 <= by0 + lb && by0 <= ay0 + la &&
           az0 <= bz0 + lb && bz0 <= az0 + la;
}

// the image of child o of the box of entry e (the child moves with its parent), or -1
__device__ __forceinline__ int child_ent(const TreeView &tv, int e, int o)
{
    const int ch = tv.child[8 * ent_box(e) + o];
    return ch < 0 ? -1 : ent_make(ch, ent_image(e));
}

// One warp per box, lanes over the candidates of each list, ballots to place them in
// candidate order.  mode 0: count into cnt[4][n_boxes] (U, V, W, X); mode 1: fill.  The
// descendants of the non-leaf colleagues (U (ii), W) are walked through a frontier in shared
// memory, 32 boxes per step, last in first out (so it stays about 8 x 32 per remaining
// level); a frontier that would exceed Q entries sets *overflow and stops the walk.  The
// small frontier (4 KB per warp) keeps ~56 warps per SM resident; the host falls back to
// the large one after an overflow.  Every candidate is a list entry (box and image): in a
// periodic tree the same box can enter a list as several images.
template <int WARPS, int Q>
__global__ void __launch_bounds__(32 * WARPS)
lists_kernel(TreeView tv, int mode, int *__restrict__ cnt, const int *__restrict__ uo, int *__restrict__ ui,
             const int *__restrict__ vo, int *__restrict__ vi, const int *__restrict__ wo, int *__restrict__ wi,
             const int *__restrict__ xo, int *__restrict__ xi, int *__restrict__ overflow)
{
    __shared__ int frontier[WARPS][Q];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    const int b = blockIdx.x * WARPS + wid;
    if (b >= tv.n_boxes) return;  // the whole warp
    int *q = frontier[wid];
    const int4 ab = tv.anchor[b];
    const int level = ab.w;
    const bool is_leaf = tv.leaf[b] != 0;
    const int par = tv.parent[b];
    int nu = 0, nv = 0, nw = 0, nx = 0;
    const int pu = mode ? uo[b] : 0, pv = mode ? vo[b] : 0, pw = mode ? wo[b] : 0, px = mode ? xo[b] : 0;
    // append the lanes with `pred` set, in lane order, to a list
    auto emit = [&](bool pred, int val, int *dst, int base, int &n) {
        const unsigned m = __ballot_sync(full, pred);
        if (mode && pred) dst[base + n + __popc(m & below)] = val;
        n += __popc(m);
    };

    // V: children of the parent's colleagues that are not adjacent to b (from level 1 on in a
    // periodic tree, whose root has its images as colleagues)
    if (level >= (tv.periodic ? 1 : 2)) {
        for (int t0 = 0; t0 < 27 * 8; t0 += 32) {
            const int t = t0 + lane;
            int D = -1;
            if (t < 27 * 8) {
                const int C = tv.colleague[27 * par + (t >> 3)];
                if (C >= 0 && !tv.leaf[ent_box(C)]) D = child_ent(tv, C, t & 7);
            }
            emit(D >= 0 && !adjacent(tv, D >= 0 ? D : 0, ab), D, vi, pv, nv);
        }
    }
    // X: coarser leaves adjacent to the parent but not to b (b lies in their W list)
    if (level >= 1) {
        const int4 ap = tv.anchor[par];
        for (int A = par; A >= 0; A = tv.parent[A]) {
            bool ok = false;
            int C = -1;
            if (lane < 27) {
                C = tv.colleague[27 * A + lane];
                if (C >= 0 && C != A && tv.leaf[ent_box(C)]) ok = adjacent(tv, C, ap) && !adjacent(tv, C, ab);
            }
            emit(ok, C, xi, px, nx);
        }
    }
    if (is_leaf) {
        // U (i): leaves at this or coarser levels adjacent to b
        for (int A = b; A >= 0; A = tv.parent[A]) {
            bool ok = false;
            int C = -1;
            if (lane < 27) {
                C = tv.colleague[27 * A + lane];
                if (C >= 0 && tv.leaf[ent_box(C)] && !(A != b && C == A)) ok = A == b || adjacent(tv, C, ab);
            }
            emit(ok, C, ui, pu, nu);
        }
        // U (ii) and W: descendants of non-leaf colleagues; the frontier starts with their
        // children
        int qn = 0;
        for (int t0 = 0; t0 < 27 * 8; t0 += 32) {
            const int t = t0 + lane;
            int D = -1;
            if (t < 27 * 8 && (t >> 3) != 13) {
                const int C = tv.colleague[27 * b + (t >> 3)];
                if (C >= 0 && !tv.leaf[ent_box(C)]) D = child_ent(tv, C, t & 7);
            }
            const unsigned m = __ballot_sync(full, D >= 0);
            if (D >= 0) q[qn + __popc(m & below)] = D;
            qn += __popc(m);
        }
        __syncwarp();
        while (qn > 0) {
            const int take = min(32, qn);
            qn -= take;
            const int D = lane < take ? q[qn + lane] : -1;
            __syncwarp();
            bool adj = false, lf = false;
            if (D >= 0) {
                adj = adjacent(tv, D, ab);
                lf = tv.leaf[ent_box(D)] != 0;
            }
            emit(D >= 0 && adj && lf, D, ui, pu, nu);
            emit(D >= 0 && !adj, D, wi, pw, nw);
            // adjacent non-leaf boxes: push their children
            int kids[8], nk = 0;
            if (D >= 0 && adj && !lf) {
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    const int E = child_ent(tv, D, o);
                    if (E >= 0) kids[nk++] = E;
                }
            }
            int incl = nk;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int v = __shfl_up_sync(full, incl, d);
                if (lane >= d) incl += v;
            }
            const int total = __shfl_sync(full, incl, 31);
            if (qn + total > Q) {
                if (lane == 0) atomicExch(overflow, 1);
                break;
            }
            for (int k = 0; k < nk; ++k) q[qn + incl - nk + k] = kids[k];
            qn += total;
            __syncwarp();
        }
    }
    if (!mode && lane == 0) {
        cnt[b] = nu;
        cnt[tv.n_boxes + b] = nv;
        cnt[2 * tv.n_boxes + b] = nw;
        cnt[3 * tv.n_boxes + b] = nx;
    }
}

// Offsets of the four lists from one exclusive scan S of their concatenated counts:
// off_l[b] = S[l n + b] - S[l n] for b <= n (S[4 n] is the grand total); tot[l] = list sizes.
__global__ void list_offsets_kernel(int n, const int *__restrict__ S, int *__restrict__ o0, int *__restrict__ o1,
                                    int *__restrict__ o2, int *__restrict__ o3, int *__restrict__ tot)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    int *outs[4] = {o0, o1, o2, o3};
#pragma unroll
    for (int l = 0; l < 4; ++l) outs[l][i] = S[(size_t)l * n + i] - S[(size_t)l * n];
    if (i == n)
        for (int l = 0; l < 4; ++l) tot[l] = S[(size_t)(l + 1) * n] - S[(size_t)l * n];
}

__global__ void compact_kernel(int n, const int *__restrict__ flag, const int *__restrict__ pos,
                               int *__restrict__ out)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n && flag[b]) out[pos[b]] = b;
}

// Per box: X list non-empty and more targets than x_direct_max (xflag: P2L through the
// downward check surface); in some W list with more sources than w_direct_max (wflag; a box is
// in some W list exactly when its X list is non-empty).
__global__ void box_flags_kernel(int n, const int *__restrict__ xcnt, const int2 *__restrict__ bsrc,
                                 const int2 *__restrict__ btrg, int w_direct_max, int x_direct_max,
                                 int *__restrict__ xflag, int *__restrict__ wflag)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const bool x = xcnt[b] > 0;
    xflag[b] = x && btrg[b].y - btrg[b].x > x_direct_max;
    wflag[b] = x && bsrc[b].y - bsrc[b].x > w_direct_max;
}

// X lists summed directly (the dual of the direct W boxes): a box B with an X list and at most
// x_direct_max targets skips P2L (n_surf check points per source) and each leaf L under B sums
// the sources of X(B) at its own targets instead.  Per leaf: the X lists of the leaf and its
// ancestors that take this path, counted (FILL false) or written at off[L] (FILL true).
template <bool FILL>
__global__ void xd_list_kernel(int n_leaves, const int *__restrict__ leaves, const int *__restrict__ parent,
                               const int2 *__restrict__ btrg, const int *__restrict__ xo,
                               const int *__restrict__ xi, int x_direct_max, int *__restrict__ cnt,
                               const int *__restrict__ off, int *__restrict__ idx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_leaves) return;
    const int leaf = leaves[i];
    int n = 0, at = FILL ? off[leaf] : 0;
    for (int b = leaf; b >= 0; b = parent[b]) {
        const int nx = xo[b + 1] - xo[b];
        if (nx == 0 || btrg[b].y - btrg[b].x > x_direct_max) continue;
        if (FILL)
            for (int k = 0; k < nx; ++k) idx[at++] = xi[xo[b] + k];
        n += nx;
    }
    if (!FILL) cnt[leaf] = n;
}

// V pairs grouped by direction (dx, dy, dz) in [-3,3]^3 minus [-1,1]^3: 316 groups.
__device__ __forceinline__ int dir_index(int dx, int dy, int dz)
{
    // index into 7^3 then compress by removing the 27 inner ones
    int full = ((dx + 3) * 7 + (dy + 3)) * 7 + (dz + 3);
    // minus the inner cells (components -1..1, indices 2..4 on each axis) with a smaller index
    int inner_before = 0;
    for (int a = 2; a <= 4; ++a)
        for (int bb = 2; bb <= 4; ++bb)
            for (int c = 2; c <= 4; ++c)
                if (((a * 7 + bb) * 7 + c) < full) ++inner_before;
    return full - inner_before;
}

constexpr int kVdirBox = 128;  // target boxes per block when grouping V pairs by direction

// Direction of every V pair and the per-block direction counts, bhist[d * nblk + block].
__global__ void vdir_hist_kernel(int n_boxes, const int *__restrict__ vo, const int *__restrict__ vi,
                                 const int4 *__restrict__ anchor, int *__restrict__ pair_dir, int *__restrict__ bhist,
                                 int nblk)
{
    __shared__ int h[316];
    for (int i = threadIdx.x; i < 316; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n_boxes) {
        const int4 ab = anchor[b];
        for (int k = vo[b]; k < vo[b + 1]; ++k) {
            const int e = vi[k];
            const int4 as = anchor[ent_box(e)];
            int sx, sy, sz;
            ent_shift(e, sx, sy, sz);  // an image moved by whole cells: 2^level boxes each
            const int side = 1 << as.w;
            // in [-3, 3] for every V pair by construction; clamped so that no index can leave h
            const int dx = min(3, max(-3, as.x + sx * side - ab.x)), dy = min(3, max(-3, as.y + sy * side - ab.y)),
                      dz = min(3, max(-3, as.z + sz * side - ab.z));
            const int d = dir_index(dx, dy, dz);
            pair_dir[k] = d;
            atomicAdd(&h[d], 1);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 316; i += blockDim.x) bhist[(size_t)i * nblk + blockIdx.x] = h[i];
}

// Place the pairs of this block from its scanned offsets (order within a block arbitrary).
__global__ void vdir_place_kernel(int n_boxes, const int *__restrict__ vo, const int *__restrict__ vi,
                                  const int *__restrict__ pair_dir, const int *__restrict__ boff, int nblk,
                                  int *__restrict__ psrc, int *__restrict__ ptrg)
{
    __shared__ int cur[316];
    for (int i = threadIdx.x; i < 316; i += blockDim.x) cur[i] = boff[(size_t)i * nblk + blockIdx.x];
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_boxes) return;
    for (int k = vo[b]; k < vo[b + 1]; ++k) {
        const int pos = atomicAdd(&cur[pair_dir[k]], 1);
        psrc[pos] = ent_box(vi[k]);  // the translation carries the image's offset
        ptrg[pos] = b;
    }
}

__global__ void oct_count_kernel(int n_boxes, const int4 *__restrict__ anchor, int *__restrict__ cnt)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_boxes || b == 0) return;
    const int4 a = anchor[b];
    const int o = ((a.x & 1) << 2) | ((a.y & 1) << 1) | (a.z & 1);
    atomicAdd(&cnt[8 * a.w + o], 1);
}

__global__ void oct_scatter_kernel(int n_boxes, const int4 *__restrict__ anchor, int *__restrict__ cursor,
                                   int *__restrict__ out)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_boxes || b == 0) return;
    const int4 a = anchor[b];
    const int o = ((a.x & 1) << 2) | ((a.y & 1) << 1) | (a.z & 1);
    out[atomicAdd(&cursor[8 * a.w + o], 1)] = b;
}

// Work counts for roofline accounting (one thread per box).
__global__ void work_count_kernel(int n_boxes, const int *__restrict__ leaf, const int2 *__restrict__ bsrc,
                                  const int2 *__restrict__ btrg, const int *__restrict__ uo,
                                  const int *__restrict__ ui, const int *__restrict__ wo,
                                  const int *__restrict__ wi, int w_direct_max, const int *__restrict__ xo,
                                  const int *__restrict__ xi, int x_direct_max, unsigned long long *__restrict__ acc)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_boxes) return;
    unsigned long long p2p = 0, l2p = 0, p2l = 0;
    if (leaf[b]) {
        const int nt = btrg[b].y - btrg[b].x;
        long long ns = 0, n_eq = 1;  // the leaf's own downward density
        for (int k = uo[b]; k < uo[b + 1]; ++k) ns += bsrc[ent_box(ui[k])].y - bsrc[ent_box(ui[k])].x;
        for (int k = wo[b]; k < wo[b + 1]; ++k) {
            const int w = bsrc[ent_box(wi[k])].y - bsrc[ent_box(wi[k])].x;
            if (w > w_direct_max) ++n_eq;
            else ns += w;
        }
        p2p = (unsigned long long)nt * ns;
        l2p = (unsigned long long)nt * n_eq;
    }
    unsigned long long xs = 0;
    for (int k = xo[b]; k < xo[b + 1]; ++k) xs += bsrc[ent_box(xi[k])].y - bsrc[ent_box(xi[k])].x;
    const int ntb = btrg[b].y - btrg[b].x;
    if (ntb > x_direct_max) p2l = xs;                       // through the check surface
    else p2p += (unsigned long long)ntb * xs;               // summed at the targets
    if (p2p) atomicAdd(&acc[0], p2p);
    if (l2p) atomicAdd(&acc[1], l2p);
    if (p2l) atomicAdd(&acc[2], p2l);
}

}  // namespace

kfmm_status build_tree(kfmm_ctx *ctx, const float *src_xyz, const float *src_nrm, int64_t nsrc,
                       const float *trg_xyz, int64_t ntrg)
{
    const int64_t so[2] = {0, nsrc}, to[2] = {0, ntrg};
    return build_forest(ctx, 1, so, src_xyz, src_nrm, to, trg_xyz);
}

kfmm_status build_forest(kfmm_ctx *ctx, int n_sets, const int64_t *src_off, const float *src_xyz,
                         const float *src_nrm, const int64_t *trg_off, const float *trg_xyz)
{
    Tree &T = ctx->tree;
    T.built = false;
    const cudaStream_t st = ctx->stream;
    const int cap = ctx->opt.leaf_cap;
    if (n_sets < 1) return ctx->fail(KFMM_ERR_INVALID_ARG, "need at least one point set");
    if (ctx->periodic && n_sets != 1)
        return ctx->fail(KFMM_ERR_INVALID_ARG, "a periodic tree holds one point set (one cell)");
    const int64_t nsrc = src_off[n_sets], ntrg = trg_off[n_sets];
    if (nsrc + ntrg > (int64_t)1 << 30) return ctx->fail(KFMM_ERR_INVALID_ARG, "too many points (limit 2^30)");
    // keys: the set index above 3 L Morton bits, within 64 bits
    int set_bits = 0;
    while ((1LL << set_bits) < n_sets) ++set_bits;
    const int L_full = std::min(ctx->opt.max_depth, (64 - set_bits) / 3);
    if (L_full < 1) return ctx->fail(KFMM_ERR_INVALID_ARG, "too many point sets");
    // keys first at a shallow depth (fewer sort passes); a leaf that would need more levels
    // sends the build back to the keys with the full depth
    constexpr int kShallowDepth = 10;
    int L = std::min(L_full, kShallowDepth);

    // ---- bounding cube of every set and NaN check
    DevBuf *tmp = ctx->work.tree_tmp;  // persistent scratch: slots 0-2 sort, 3-15 below
    DevBuf &set_off = tmp[15], &roots = T.set_root_dev;
    KF_CUDA(set_off.ensure(sizeof(int64_t) * 2 * (n_sets + 1)));
    int64_t *d_soff = set_off.as<int64_t>(), *d_toff = d_soff + n_sets + 1;
    KF_TRY(upload_async(ctx, d_soff, src_off, sizeof(int64_t) * (n_sets + 1)));
    KF_TRY(upload_async(ctx, d_toff, trg_off, sizeof(int64_t) * (n_sets + 1)));
    const int bx = std::max(1, kBBoxBlocks / n_sets);
    DevBuf &part = tmp[3];
    KF_CUDA(part.ensure(sizeof(float) * 7 * (size_t)bx * n_sets));
    bbox_kernel<<<dim3(bx, n_sets), kBBoxThreads, 0, st>>>(d_soff, src_xyz, d_toff, trg_xyz, src_nrm,
                                                           part.as<float>());
    KF_LAUNCH();
    std::vector<float> hp(7 * (size_t)bx * n_sets);
    KF_CUDA(cudaMemcpyAsync(hp.data(), part.p, sizeof(float) * hp.size(), cudaMemcpyDeviceToHost, st));
    KF_TRY(sync_stream(ctx));
    std::vector<double> hr(8 * (size_t)n_sets, 0.0);
    for (int k = 0; k < n_sets; ++k) {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        double bad = 0;
        for (int b = 0; b < bx; ++b) {
            const float *q = &hp[7 * ((size_t)k * bx + b)];
            for (int c = 0; c < 3; ++c) {
                lo[c] = std::min(lo[c], (double)q[c]);
                hi[c] = std::max(hi[c], (double)q[3 + c]);
            }
            bad += q[6];
        }
        if (bad > 0) return ctx->fail(KFMM_ERR_INVALID_ARG, "non-finite coordinate or normal");
        if (ctx->periodic) {
            // the root is the cell itself (a point on its upper faces joins the last boxes)
            const double side = ctx->cell_side, tol = 1e-6 * side;
            for (int c = 0; c < 3; ++c)
                if (lo[c] < ctx->cell_lo[c] - tol || hi[c] > ctx->cell_lo[c] + side + tol)
                    return ctx->fail(KFMM_ERR_INVALID_ARG, "periodic tree: a point lies outside the cell");
            for (int c = 0; c < 3; ++c) hr[8 * k + c] = ctx->cell_lo[c];
            hr[8 * k + 3] = side;
            hr[8 * k + 4] = 1.0 / side;
            continue;
        }
        double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
        double w = ext > 0 ? ext * (1.0 + 1e-6) : 1.0;
        for (int c = 0; c < 3; ++c) hr[8 * k + c] = 0.5 * (lo[c] + hi[c]) - 0.5 * w;
        hr[8 * k + 3] = w;
        hr[8 * k + 4] = 1.0 / w;
    }
    KF_CUDA(roots.ensure(sizeof(double) * hr.size()));
    KF_TRY(upload_async(ctx, roots.p, hr.data(), sizeof(double) * hr.size()));
    T.set_roots.assign(hr.begin(), hr.end());
    T.n_sets = n_sets;
    for (int c = 0; c < 3; ++c) T.root_lo[c] = hr[c];
    T.root_w = hr[3];
    T.nsrc = nsrc;
    T.ntrg = ntrg;
    T.has_nrm = src_nrm != nullptr;
    T.periodic = ctx->periodic;
    T.cell = ctx->periodic ? (float)ctx->cell_side : 0.f;

    SplitState hs{};
    size_t capb = std::max<size_t>(1024, (size_t)(4 * (nsrc + ntrg) / std::max(1, cap)) + 64 + (size_t)n_sets);
    DevBuf &crange = tmp[4], &ccount = tmp[5], &bsum = tmp[6], &sstate = tmp[7], &loff = tmp[9];
    for (;;) {  // depth attempts: kShallowDepth, then L_full if needed
        ctx->phase(KFMM_PH_TREE);
        // ---- keys and sort
        KF_CUDA(T.src_key.ensure(sizeof(uint64_t) * nsrc));
        KF_CUDA(T.trg_key.ensure(sizeof(uint64_t) * ntrg));
        KF_CUDA(T.src_perm.ensure(sizeof(int) * nsrc));
        KF_CUDA(T.trg_perm.ensure(sizeof(int) * ntrg));
        keys_kernel<<<grid_for(nsrc, 256), 256, 0, st>>>(src_xyz, nsrc, d_soff, n_sets, roots.as<double>(), L,
                                                          T.src_key.as<uint64_t>(), T.src_perm.as<int>());
        KF_LAUNCH();
        // targets given as the very array of the sources: one set of keys, one sort, then copies
        bool same = trg_xyz == src_xyz;
        for (int k = 0; k <= n_sets && same; ++k) same = src_off[k] == trg_off[k];
        if (!same) {
            keys_kernel<<<grid_for(ntrg, 256), 256, 0, st>>>(trg_xyz, ntrg, d_toff, n_sets, roots.as<double>(), L,
                                                              T.trg_key.as<uint64_t>(), T.trg_perm.as<int>());
            KF_LAUNCH();
        }
        KF_TRY(radix_sort(ctx, T.src_key, T.src_perm, (int)nsrc, 3 * L + set_bits));
        if (!same) KF_TRY(radix_sort(ctx, T.trg_key, T.trg_perm, (int)ntrg, 3 * L + set_bits));
        KF_CUDA(T.src_xyz.ensure(sizeof(float4) * nsrc));
        KF_CUDA(T.trg_xyz.ensure(sizeof(float4) * ntrg));
        gather_points_kernel<<<grid_for(nsrc, 256), 256, 0, st>>>(src_xyz, T.src_perm.as<int>(), nsrc,
                                                                   T.src_xyz.as<float4>());
        KF_LAUNCH();
        if (same) {
            KF_CUDA(cudaMemcpyAsync(T.trg_key.p, T.src_key.p, sizeof(uint64_t) * ntrg, cudaMemcpyDeviceToDevice, st));
            KF_CUDA(cudaMemcpyAsync(T.trg_perm.p, T.src_perm.p, sizeof(int) * ntrg, cudaMemcpyDeviceToDevice, st));
            KF_CUDA(cudaMemcpyAsync(T.trg_xyz.p, T.src_xyz.p, sizeof(float4) * ntrg, cudaMemcpyDeviceToDevice, st));
        } else {
            gather_points_kernel<<<grid_for(ntrg, 256), 256, 0, st>>>(trg_xyz, T.trg_perm.as<int>(), ntrg,
                                                                       T.trg_xyz.as<float4>());
            KF_LAUNCH();
        }
        if (src_nrm) {
            KF_CUDA(T.src_nrm.ensure(sizeof(float4) * nsrc));
            gather_points_kernel<<<grid_for(nsrc, 256), 256, 0, st>>>(src_nrm, T.src_perm.as<int>(), nsrc,
                                                                       T.src_nrm.as<float4>());
            KF_LAUNCH();
        }

        // ---- boxes, level by level, and the leaves: one cooperative launch
        ctx->phase(KFMM_PH_TREE_SPLIT);
        if (!T.split_grid) {
            int per_sm = 0, n_sm = 0;
            KF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, split_tree_kernel, kSplitThreads, 0));
            KF_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->opt.device));
            if (per_sm < 1) return ctx->fail(KFMM_ERR_INTERNAL, "tree split kernel cannot be resident");
            T.split_grid = std::min(per_sm, 2) * n_sm;
        }
        KF_CUDA(bsum.ensure(sizeof(int) * T.split_grid));
        KF_CUDA(sstate.ensure(sizeof(SplitState)));
        KF_CUDA(loff.ensure(sizeof(int) * (L + 2)));
        for (;;) {
            if (capb > (size_t)INT32_MAX / 8) return ctx->fail(KFMM_ERR_INVALID_ARG, "too many boxes");
            KF_CUDA(T.box_key.ensure(sizeof(uint64_t) * capb));
            KF_CUDA(T.box_anchor.ensure(sizeof(int4) * capb));
            KF_CUDA(T.box_parent.ensure(sizeof(int) * capb));
            KF_CUDA(T.box_child.ensure(sizeof(int) * 8 * capb));
            KF_CUDA(T.box_src.ensure(sizeof(int2) * capb));
            KF_CUDA(T.box_trg.ensure(sizeof(int2) * capb));
            KF_CUDA(T.box_leaf.ensure(sizeof(int) * capb));
            KF_CUDA(T.leaves.ensure(sizeof(int) * capb));
            KF_CUDA(crange.ensure(sizeof(int4) * 8 * capb));
            KF_CUDA(ccount.ensure(sizeof(int) * capb));
            KF_CUDA(cudaMemsetAsync(sstate.p, 0, sizeof(SplitState), st));
            SplitArgs sa{L, cap, (int)capb, n_sets, d_soff, d_toff, T.src_key.as<uint64_t>(), T.trg_key.as<uint64_t>(),
                         T.box_key.as<uint64_t>(), T.box_anchor.as<int4>(), T.box_parent.as<int>(),
                         T.box_child.as<int>(), T.box_src.as<int2>(), T.box_trg.as<int2>(), T.box_leaf.as<int>(),
                         T.leaves.as<int>(), crange.as<int4>(), ccount.as<int>(), bsum.as<int>(), loff.as<int>(),
                         sstate.as<SplitState>()};
            void *args[] = {&sa};
            KF_CUDA(cudaLaunchCooperativeKernel((const void *)split_tree_kernel, dim3(T.split_grid), dim3(kSplitThreads),
                                                args, 0, st));
            KF_LAUNCH();
            T.level_off.assign(L + 2, 0);
            KF_CUDA(cudaMemcpyAsync(&hs, sstate.p, sizeof(SplitState), cudaMemcpyDeviceToHost, st));
            KF_CUDA(cudaMemcpyAsync(T.level_off.data(), loff.p, sizeof(int) * (L + 2), cudaMemcpyDeviceToHost, st));
            KF_TRY(sync_stream(ctx));
            if (hs.err == 2) return ctx->fail(KFMM_ERR_DEVICE_TIMEOUT, "tree split: a grid barrier gave up");
            if (hs.err != 1) break;
            capb *= 2;  // more boxes than the estimate: run again with twice the room
        }
        if (!hs.deep || L >= L_full) break;
        L = L_full;  // clustered points: all over again with the full depth
    }
    T.max_depth = L;
    const int n_boxes = hs.n_boxes;
    if (n_boxes > kEntMask) return ctx->fail(KFMM_ERR_INVALID_ARG, "too many boxes (limit 2^26)");
    T.n_boxes = n_boxes;
    T.n_levels = hs.n_levels;
    T.n_leaves = hs.n_leaves;
    T.level_off.resize(T.n_levels + 1);

    // ---- colleagues (level offsets on the device as the split kernel left them)
    KF_CUDA(T.colleague.ensure(sizeof(int) * 27 * n_boxes));
    TreeView tv{L,
                n_boxes,
                T.box_key.as<uint64_t>(),
                T.box_anchor.as<int4>(),
                T.box_parent.as<int>(),
                T.box_child.as<int>(),
                T.box_leaf.as<int>(),
                T.colleague.as<int>(),
                loff.as<int>(),
                T.n_levels,
                T.periodic ? 1 : 0};
    colleague_kernel<<<grid_for(n_boxes, 128, 1 << 30), 128, 0, st>>>(tv, T.colleague.as<int>());
    KF_LAUNCH();

    // ---- lists: a count pass; then every size the host needs (list sizes, X and W boxes,
    //      octant groups) is counted on the device and read back in one go
    ctx->phase(KFMM_PH_TREE_LISTS);
    const int ng = 8 * T.n_levels;
    DevBuf &cnt = tmp[10], &hdr = tmp[11];
    // hdr (ints): 0-3 sizes of the U, V, W, X lists; 4 X boxes; 5 W boxes; 6 traversal
    // overflow; 8 on: octant-group sizes, 8 per level
    if (4 * (int64_t)n_boxes >= INT32_MAX) return ctx->fail(KFMM_ERR_INVALID_ARG, "too many boxes");
    KF_CUDA(cnt.ensure(sizeof(int) * (4 * (size_t)n_boxes + 1)));
    KF_CUDA(hdr.ensure(sizeof(int) * (8 + (size_t)ng)));
    int *H = hdr.as<int>();
    // list passes with the small frontier (attempt 0) or, after an overflow, the large one
    auto lists = [&](int attempt, int mode) {
        if (attempt == 0)
            lists_kernel<4, 1024><<<(n_boxes + 3) / 4, 128, 0, st>>>(
                tv, mode, mode ? nullptr : cnt.as<int>(), T.u_off.as<int>(), T.u_idx.as<int>(), T.v_off.as<int>(),
                T.v_idx.as<int>(), T.w_off.as<int>(), T.w_idx.as<int>(), T.x_off.as<int>(), T.x_idx.as<int>(), H + 6);
        else
            lists_kernel<2, 4096><<<(n_boxes + 1) / 2, 64, 0, st>>>(
                tv, mode, mode ? nullptr : cnt.as<int>(), T.u_off.as<int>(), T.u_idx.as<int>(), T.v_off.as<int>(),
                T.v_idx.as<int>(), T.w_off.as<int>(), T.w_idx.as<int>(), T.x_off.as<int>(), T.x_idx.as<int>(), H + 6);
    };
    std::vector<int> hh(8 + (size_t)ng);
    DevBuf *offs[4] = {&T.u_off, &T.v_off, &T.w_off, &T.x_off};
    DevBuf *idxs[4] = {&T.u_idx, &T.v_idx, &T.w_idx, &T.x_idx};
    DevBuf &scn = tmp[12];
    DevBuf &xflag = tmp[3], &xpos = tmp[8], &wflag = tmp[13], &wpos = tmp[14];
    int attempt = 0;
    for (;; ++attempt) {
        KF_CUDA(cudaMemsetAsync(H, 0, sizeof(int) * (8 + (size_t)ng), st));
        lists(attempt, 0);
        KF_LAUNCH();
        // offsets of the four lists from one scan over their concatenated counts
        KF_CUDA(scn.ensure(sizeof(int) * (4 * (size_t)n_boxes + 1)));
        int *S = scn.as<int>();
        KF_TRY(scan_exclusive(ctx, cnt.as<int>(), S, 4 * n_boxes, S + 4 * (size_t)n_boxes));
        for (int l = 0; l < 4; ++l) KF_CUDA(offs[l]->ensure(sizeof(int) * (n_boxes + 1)));
        list_offsets_kernel<<<grid_for(n_boxes + 1, 256, 1 << 30), 256, 0, st>>>(
            n_boxes, S, T.u_off.as<int>(), T.v_off.as<int>(), T.w_off.as<int>(), T.x_off.as<int>(), H);
        KF_LAUNCH();
        // X boxes (non-empty X list) and the W boxes whose upward densities are evaluated at the
        // targets.  A box lies in some W list exactly when its X list is non-empty (b is in W(C)
        // iff C is in X(b)); those with more sources than half the surface points take the M2P
        // path, the others are evaluated directly.
        T.w_direct_max = surface_points(ctx->opt.p) / 2;
        T.x_direct_max = surface_points(ctx->opt.p) / 2;
        KF_CUDA(xflag.ensure(sizeof(int) * n_boxes));
        KF_CUDA(xpos.ensure(sizeof(int) * n_boxes));
        KF_CUDA(wflag.ensure(sizeof(int) * n_boxes));
        KF_CUDA(wpos.ensure(sizeof(int) * n_boxes));
        box_flags_kernel<<<grid_for(n_boxes, 256, 1 << 30), 256, 0, st>>>(
            n_boxes, cnt.as<int>() + 3 * (size_t)n_boxes, T.box_src.as<int2>(), T.box_trg.as<int2>(),
            T.w_direct_max, T.x_direct_max, xflag.as<int>(), wflag.as<int>());
        KF_LAUNCH();
        KF_TRY(scan_exclusive(ctx, xflag.as<int>(), xpos.as<int>(), n_boxes, H + 4));
        KF_TRY(scan_exclusive(ctx, wflag.as<int>(), wpos.as<int>(), n_boxes, H + 5));
        oct_count_kernel<<<grid_for(n_boxes, 256, 1 << 30), 256, 0, st>>>(n_boxes, T.box_anchor.as<int4>(), H + 8);
        KF_LAUNCH();
        KF_CUDA(cudaMemcpyAsync(hh.data(), H, sizeof(int) * hh.size(), cudaMemcpyDeviceToHost, st));
        KF_TRY(sync_stream(ctx));
        if (!hh[6]) break;
        if (attempt == 1) return ctx->fail(KFMM_ERR_INTERNAL, "interaction-list traversal frontier overflow");
    }
    T.n_u = hh[0];
    T.n_v = hh[1];
    T.n_w = hh[2];
    T.n_x = hh[3];
    T.n_xboxes = hh[4];
    T.n_wboxes = hh[5];
    for (int l = 0; l < 4; ++l) KF_CUDA(idxs[l]->ensure(sizeof(int) * std::max(1, hh[l])));
    lists(attempt, 1);
    KF_LAUNCH();
    KF_CUDA(T.xboxes.ensure(sizeof(int) * std::max(1, T.n_xboxes)));
    compact_kernel<<<grid_for(n_boxes, 256, 1 << 30), 256, 0, st>>>(n_boxes, xflag.as<int>(), xpos.as<int>(),
                                                                     T.xboxes.as<int>());
    KF_LAUNCH();
    KF_CUDA(T.wboxes.ensure(sizeof(int) * std::max(1, T.n_wboxes)));
    compact_kernel<<<grid_for(n_boxes, 256, 1 << 30), 256, 0, st>>>(n_boxes, wflag.as<int>(), wpos.as<int>(),
                                                                     T.wboxes.as<int>());
    KF_LAUNCH();
    // ---- X lists summed directly at the leaves (per box; zero counts off the leaves)
    {
        DevBuf &xc = tmp[6];
        KF_CUDA(xc.ensure(sizeof(int) * (n_boxes + 1)));
        KF_CUDA(cudaMemsetAsync(xc.p, 0, sizeof(int) * (n_boxes + 1), st));
        KF_CUDA(T.xd_off.ensure(sizeof(int) * (n_boxes + 1)));
        const int nl = T.n_leaves;
        xd_list_kernel<false><<<grid_for(nl, 128, 1 << 30), 128, 0, st>>>(
            nl, T.leaves.as<int>(), T.box_parent.as<int>(), T.box_trg.as<int2>(), T.x_off.as<int>(), T.x_idx.as<int>(),
            T.x_direct_max, xc.as<int>(), nullptr, nullptr);
        KF_LAUNCH();
        KF_TRY(scan_exclusive(ctx, xc.as<int>(), T.xd_off.as<int>(), n_boxes + 1, H + 7));
        int nxd = 0;
        KF_CUDA(cudaMemcpyAsync(&nxd, H + 7, sizeof(int), cudaMemcpyDeviceToHost, st));
        KF_TRY(sync_stream(ctx));
        T.n_xd = nxd;
        KF_CUDA(T.xd_idx.ensure(sizeof(int) * std::max(1, nxd)));
        xd_list_kernel<true><<<grid_for(nl, 128, 1 << 30), 128, 0, st>>>(
            nl, T.leaves.as<int>(), T.box_parent.as<int>(), T.box_trg.as<int2>(), T.x_off.as<int>(), T.x_idx.as<int>(),
            T.x_direct_max, nullptr, T.xd_off.as<int>(), T.xd_idx.as<int>());
        KF_LAUNCH();
    }
    // ---- octant groups per level (M2M / L2L)
    {
        DevBuf &gc = tmp[6];
        KF_CUDA(gc.ensure(sizeof(int) * (ng + 1)));
        T.oct_off.assign(ng + 1, 0);
        for (int g = 0; g < ng; ++g) T.oct_off[g + 1] = T.oct_off[g] + hh[8 + g];
        KF_TRY(upload_async(ctx, gc.p, T.oct_off.data(), sizeof(int) * ng));
        KF_CUDA(T.oct_child.ensure(sizeof(int) * std::max(1, n_boxes)));
        oct_scatter_kernel<<<grid_for(n_boxes, 256, 1 << 30), 256, 0, st>>>(n_boxes, T.box_anchor.as<int4>(),
                                                                             gc.as<int>(), T.oct_child.as<int>());
        KF_LAUNCH();
    }
    // ---- V pairs grouped by direction
    {
        // per-block direction histograms in shared memory, one scan over (direction, block),
        // then each block scatters its pairs from its own offsets (no contended atomics)
        const int nblk = (n_boxes + kVdirBox - 1) / kVdirBox;
        DevBuf &bhist = tmp[4], &pair_dir = tmp[5];
        KF_CUDA(bhist.ensure(sizeof(int) * (316 * (size_t)nblk + 1)));
        KF_CUDA(pair_dir.ensure(sizeof(int) * std::max<int64_t>(1, T.n_v)));
        vdir_hist_kernel<<<nblk, kVdirBox, 0, st>>>(n_boxes, T.v_off.as<int>(), T.v_idx.as<int>(),
                                                    T.box_anchor.as<int4>(), pair_dir.as<int>(), bhist.as<int>(), nblk);
        KF_LAUNCH();
        KF_TRY(scan_exclusive(ctx, bhist.as<int>(), bhist.as<int>(), 316 * nblk, nullptr));
        // direction offsets for the host: the scanned value at each direction's first block
        std::vector<int> hoff(316);
        KF_CUDA(cudaMemcpy2DAsync(hoff.data(), sizeof(int), bhist.p, sizeof(int) * nblk, sizeof(int), 316,
                                  cudaMemcpyDeviceToHost, st));
        KF_TRY(sync_stream(ctx));
        T.vdir_off.assign(317, 0);
        for (int d = 0; d < 316; ++d) T.vdir_off[d] = hoff[d];
        T.vdir_off[316] = (int)T.n_v;
        KF_CUDA(T.vp_src.ensure(sizeof(int) * std::max<int64_t>(1, T.n_v)));
        KF_CUDA(T.vp_trg.ensure(sizeof(int) * std::max<int64_t>(1, T.n_v)));
        vdir_place_kernel<<<nblk, kVdirBox, 0, st>>>(n_boxes, T.v_off.as<int>(), T.v_idx.as<int>(), pair_dir.as<int>(),
                                                     bhist.as<int>(), nblk, T.vp_src.as<int>(), T.vp_trg.as<int>());
        KF_LAUNCH();
    }
    T.counts_valid = false;  // work counts for the statistics: made on request
    T.built = true;
    return KFMM_OK;
}

// Interaction counts of the built tree (P2P, L2P/M2P, P2L pairs) for the statistics.
kfmm_status tree_work_counts(kfmm_ctx *ctx)
{
    Tree &T = ctx->tree;
    if (T.counts_valid) return KFMM_OK;
    const cudaStream_t st = ctx->stream;
    DevBuf &acc = ctx->work.tree_tmp[4];
    KF_CUDA(acc.ensure(sizeof(unsigned long long) * 3));
    KF_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long) * 3, st));
    work_count_kernel<<<grid_for(T.n_boxes, 128, 1 << 30), 128, 0, st>>>(
        T.n_boxes, T.box_leaf.as<int>(), T.box_src.as<int2>(), T.box_trg.as<int2>(), T.u_off.as<int>(),
        T.u_idx.as<int>(), T.w_off.as<int>(), T.w_idx.as<int>(), T.w_direct_max, T.x_off.as<int>(),
        T.x_idx.as<int>(), T.x_direct_max, acc.as<unsigned long long>());
    KF_LAUNCH();
    unsigned long long h[3];
    KF_CUDA(cudaMemcpyAsync(h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    KF_TRY(sync_stream(ctx));
    T.p2p_pairs = (int64_t)h[0];
    T.l2p_pairs = (int64_t)h[1];
    T.p2l_pairs = (int64_t)h[2];
    T.counts_valid = true;
    return KFMM_OK;
}

}  // namespace kfmm
