// tc_gemm.cuh -- grouped gather-GEMM on the 5th-generation tensor cores (tcgen05, sm_103a)
// with BF16 split pairs and FP32 accumulation in tensor memory.
//
//   for each work item (matrix g, row tile mt, columns c0..c1):
//     Y[dst_j][mt*128 + i] += sum_k A_g[mt*128 + i][k] * X[src_j][k]     (atomic add)
//
// Split pairs: a = a_hi + a_lo with a_hi = bf16(a), a_lo = bf16(a - a_hi) (16 mantissa
// bits); each product is accumulated as a_hi b_hi + a_hi b_lo + a_lo b_hi in FP32 (the
// dropped a_lo b_lo is ~2^-16 of the product).
//
// Shared-memory operands use the canonical no-swizzle K-major layout of the UMMA
// descriptors: 8 x 16-byte core matrices; core (i = row / 8, j = k / 8) of an R-row tile sits
// at byte j * (R / 8) * 128 + i * 128, so the leading-dimension offset (next core along K)
// is (R / 8) * 128 and the stride-dimension offset (next core along rows) is 128.
//
// One CTA per work item (a translation, a row tile, up to 1024 columns).  The A tile (both
// halves, pre-laid-out in global memory) arrives by cp.async.bulk and stays resident; the B
// tiles are gathered from pre-split pairs by 16-byte asynchronous copies; producer, MMA and
// epilogue warps hand tiles and accumulators to one another through mbarriers.  Every
// mbarrier wait is bounded: on time-out the kernel records the error, waits (bounded) for its
// own copies and MMAs, frees its tensor memory and returns.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace kfmm {
namespace tc {

constexpr int BM = 128;       // rows per tile (UMMA M)
constexpr int BN = 64;        // columns per N step (UMMA N)
constexpr int TMEM_COLS = 128; // two FP32 accumulators of BN columns (double buffered)
constexpr long long WAIT_LIMIT = 1LL << 22;  // try_wait polls before giving up

__host__ __device__ inline uint32_t core_offset(int row, int k, int R)
{
    return (uint32_t)((k >> 3) * (R >> 3) * 128 + (row >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// bytes of one operand half (R rows x Kp columns of bf16)
__host__ __device__ inline uint32_t half_bytes(int R, int Kp) { return (uint32_t)R * (uint32_t)Kp * 2u; }

// instruction descriptor of tcgen05.mma kind::f16: D = F32, A = B = BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of sm_100-class tensor cores
    return d;                // base offset 0, no swizzle
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// true when the phase with parity `phase` has completed; false after `limit` polls
__device__ __forceinline__ bool mbar_wait_n(uint64_t *bar, uint32_t phase, long long limit)
{
    const uint32_t a = smem_u32(bar);
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// the same with the kernels' limit, WAIT_LIMIT polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase) { return mbar_wait_n(bar, phase, WAIT_LIMIT); }

// bulk copy global -> shared, completion counted on `bar` (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
    const uint16_t *A;     // [n_mat][n_mtile][2][half_bytes/2] pre-laid-out bf16 (hi then lo)
    int n_mat;             // item.x = column * n_mat + matrix (density columns batched)
    int64_t col_rows;      // rows of one density column in X2 and Y
    int n_mtile;           // row tiles per matrix
    int M;                 // valid rows (outputs at rows >= M are dropped)
    int Kp;                // padded K (multiple of 16), also the row length of X
    const int4 *items;     // {matrix, mtile, c0, c1}
    const int *src_idx;    // column j reads X[src_idx[j]]
    const int *dst_idx;    // column j adds into Y[dst_idx[j]]
    const uint16_t *X2;    // split pairs of the X rows (split_pairs_kernel), [rows][2][Kp]
    float *Y;
    int ldy;
    int *err;              // set to 1 if a bounded wait gave up
};


// X2[box] = the BF16 split pair of X[box] (Kp values).  Each 8-value chunk of K is 16
// contiguous bytes, one row of a core matrix.  Layout 0: hi at [0, Kp), lo at [Kp, 2 Kp);
// interleaved: chunk c of hi at [16 c, 16 c + 8), of lo at [16 c + 8, 16 c + 16).
__global__ void split_pairs_kernel(const float *__restrict__ X, int64_t n_rows, int Kp, uint16_t *__restrict__ X2,
                                   int interleaved)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // one thread per 8 values
    const int chunks = Kp / 8;
    if (e >= n_rows * chunks) return;
    const int64_t row = e / chunks;
    const int kb = (int)(e % chunks);
    const float *x = X + row * Kp + kb * 8;
    const float4 v0 = *reinterpret_cast<const float4 *>(x);
    const float4 v1 = *reinterpret_cast<const float4 *>(x + 4);
    const float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);  // low half = first value
        const uint32_t hb = *reinterpret_cast<const uint32_t *>(&hh);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * q] - __uint_as_float(hb << 16),
                                                        v[2 * q + 1] - __uint_as_float(hb & 0xffff0000u));
        h[q] = hb;
        l[q] = *reinterpret_cast<const uint32_t *>(&ll);
    }
    uint16_t *dst = X2 + row * 2 * Kp + (interleaved ? kb * 16 : kb * 8);
    *reinterpret_cast<uint4 *>(dst) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(dst + (interleaved ? 8 : Kp)) = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}

// The split-pair products of one N step into accumulator `d` (one thread).
__device__ __forceinline__ void issue_mmas(uint32_t a0, uint32_t a_half, uint32_t b0, uint32_t b_half, int Kp,
                                           uint32_t tmem_d)
{
    const uint32_t idesc = idesc_bf16(BM, BN);
    const uint32_t a_lbo = (BM / 8) * 128, b_lbo = (BN / 8) * 128;
    for (int ks = 0; ks < Kp / 16; ++ks) {
        const uint32_t ao = (uint32_t)(2 * ks) * a_lbo, bo = (uint32_t)(2 * ks) * b_lbo;
        const uint64_t ah = smem_desc(a0 + ao, a_lbo, 128), al = smem_desc(a0 + a_half + ao, a_lbo, 128);
        const uint64_t bh = smem_desc(b0 + bo, b_lbo, 128), bl = smem_desc(b0 + b_half + bo, b_lbo, 128);
        mma_bf16(tmem_d, ah, bh, idesc, ks > 0 ? 1u : 0u);
        mma_bf16(tmem_d, ah, bl, idesc, 1u);
        mma_bf16(tmem_d, al, bh, idesc, 1u);
    }
}

// Warp-specialised pipeline, N steps s of BN columns, buffers b = s % 2:
//   warps 0-7   epilogue: wait for accumulator b, read it (warp w: TMEM lanes 32 (w % 4) ..,
//               columns (w / 4) * 32 ..), release it, then add to the output (RED)
//   warps 8-15  producers, two groups of 128 threads; group b gathers the B tiles of the steps
//               with s % 2 == b (two threads per column, source indices fetched a round
//               ahead) once the MMAs of step s - 2 are done
//   warp 16     lane 0 loads the A tile and issues the MMAs of step s into accumulator b once
//               B(s) is in and accumulator b is released; warp 16 owns the tensor memory
// Every wait is bounded; a time-out sets the error flag and the shared fail flag, every role
// then leaves its loop, and in-flight copies and products are waited for (bounded) before the
// tensor memory is freed.
constexpr int M2L_EPI_WARPS = 8;
constexpr int M2L_PROD_THREADS = 128;  // per producer group
constexpr int M2L_MMA_WARP = M2L_EPI_WARPS + 2 * M2L_PROD_THREADS / 32;
constexpr int M2L_THREADS = 32 * (M2L_MMA_WARP + 1);

// dynamic shared memory: [A hi | A lo | B0 hi | B0 lo | B1 hi | B1 lo | barriers + flags]
__host__ __device__ inline uint32_t smem_bytes(int Kp) { return 2 * half_bytes(BM, Kp) + 4 * half_bytes(BN, Kp) + 128; }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool fail_set(const int *f) { return *(volatile const int *)f != 0; }

__global__ void __launch_bounds__(M2L_THREADS, 1) tc_gather_gemm_kernel(TcArgs g)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const int Kp = g.Kp;
    const uint32_t a_half = half_bytes(BM, Kp), b_half = half_bytes(BN, Kp);
    unsigned char *sA = sm;
    unsigned char *sB0 = sm + 2 * a_half;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 2 * a_half + 4 * b_half);
    uint64_t *barA = bar, *fullB = bar + 1, *emptyB = bar + 3, *fullAcc = bar + 5, *emptyAcc = bar + 7;
    uint32_t *holder = reinterpret_cast<uint32_t *>(bar + 9);
    int *s_fail = reinterpret_cast<int *>(holder + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int4 item = g.items[blockIdx.x];
    const int nsteps = (item.w - item.z + BN - 1) / BN;
    const int mat = item.x % g.n_mat;
    const int64_t crow = (int64_t)(item.x / g.n_mat) * g.col_rows;  // first row of this column

    if (warp == M2L_MMA_WARP) tmem_alloc(holder, TMEM_COLS);
    if (tid == 0) {
        mbar_init(barA, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&fullB[i], M2L_PROD_THREADS);
            mbar_init(&emptyB[i], 1);
            mbar_init(&fullAcc[i], 1);
            mbar_init(&emptyAcc[i], M2L_EPI_WARPS);
        }
        *s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder;
    auto fail = [&]() {
        atomicExch(s_fail, 1);
        atomicExch(g.err, 1);
    };

    if (warp < M2L_EPI_WARPS) {
        // ---------------- epilogue
        const int quad = warp & 3, chalf = warp >> 2;
        const int row = item.y * BM + quad * 32 + lane;
        for (int s = 0; s < nsteps; ++s) {
            const int b = s & 1;
            const uint32_t u = (uint32_t)(s >> 1);
            const int c0 = item.z + s * BN + chalf * (BN / 2);
            const int myd = c0 + lane < item.w ? (int)(g.dst_idx[c0 + lane] + crow) : -1;
            // warp-uniform decisions: the tensor-memory loads below are warp-collective
            if (__any_sync(0xffffffffu, fail_set(s_fail))) break;
            if (!__all_sync(0xffffffffu, mbar_wait(&fullAcc[b], u & 1u))) {
                if (lane == 0) fail();
                break;
            }
            tc_fence_after();
            float v[BN / 2];
            tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * BN + chalf * (BN / 2)), v);
            tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * BN + chalf * (BN / 2) + 16), v + 16);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&emptyAcc[b]);
#pragma unroll
            for (int k = 0; k < BN / 2; ++k) {
                const int d = __shfl_sync(0xffffffffu, myd, k);
                if (d >= 0 && row < g.M) atomicAdd(g.Y + (size_t)d * g.ldy + row, v[k]);
            }
        }
    } else if (warp < M2L_MMA_WARP) {
        // ---------------- producers: group pg fills buffer pg for steps s = pg, pg + 2, ...
        const int pt = tid - 32 * M2L_EPI_WARPS;
        const int pg = pt / M2L_PROD_THREADS, q = pt % M2L_PROD_THREADS;
        const int col = q % BN, kh = q / BN;  // column, and which half of its K chunks
        unsigned char *sB = sB0 + (size_t)pg * 2 * b_half;
        auto src_of = [&](int s) {
            const int c = item.z + s * BN + col;
            return (s < nsteps && c < item.w) ? (int)(g.src_idx[c] + crow) : -1;
        };
        int src_next = src_of(pg);
        for (int s = pg; s < nsteps; s += 2) {
            const uint32_t u = (uint32_t)(s >> 1);
            const int src = src_next;
            src_next = src_of(s + 2);  // in flight while this step waits and copies
            if (fail_set(s_fail)) break;
            // buffer pg was read by the MMAs of step s - 2
            if (u >= 1 && !mbar_wait(&emptyB[pg], (u - 1) & 1u)) {
                fail();
                break;
            }
            const uint16_t *xs = src >= 0 ? g.X2 + (size_t)src * 2 * Kp : nullptr;
            for (int kb = kh; kb < Kp / 8; kb += M2L_PROD_THREADS / BN) {
                const uint32_t off = core_offset(col, kb * 8, BN);
                if (xs) {
                    cp_async16(sB + off, xs + kb * 8);
                    cp_async16(sB + b_half + off, xs + Kp + kb * 8);
                } else {
                    *reinterpret_cast<uint4 *>(sB + off) = make_uint4(0, 0, 0, 0);
                    *reinterpret_cast<uint4 *>(sB + b_half + off) = make_uint4(0, 0, 0, 0);
                }
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
            fence_proxy_async();  // the tile is read by the tensor cores (async proxy)
            mbar_arrive(&fullB[pg]);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (lane == 0) {
        // ---------------- MMA issuer
        const unsigned char *src =
            reinterpret_cast<const unsigned char *>(g.A) + ((size_t)mat * g.n_mtile + item.y) * 2 * (size_t)a_half;
        mbar_expect_tx(barA, 2 * a_half);
        for (uint32_t off = 0; off < 2 * a_half; off += 16384) {
            const uint32_t n = (2 * a_half - off) < 16384u ? (2 * a_half - off) : 16384u;
            bulk_g2s(sA + off, src + off, n, barA);
        }
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB0);
        int issued = 0;
        bool have_a = false;
        for (int s = 0; s < nsteps; ++s) {
            const int b = s & 1;
            const uint32_t u = (uint32_t)(s >> 1);
            if (fail_set(s_fail)) break;
            bool ok = mbar_wait(&fullB[b], u & 1u);
            if (ok && !have_a) ok = have_a = mbar_wait(barA, 0);
            if (ok && u >= 1) ok = mbar_wait(&emptyAcc[b], (u - 1) & 1u);
            if (!ok) {
                fail();
                break;
            }
            tc_fence_after();
            issue_mmas(a0, a_half, b0 + (uint32_t)b * 2 * b_half, b_half, Kp, tmem + (uint32_t)(b * BN));
            mma_commit(&emptyB[b]);
            mma_commit(&fullAcc[b]);
            ++issued;
        }
        // on failure: let the issued products and the A copy finish before the memory goes
        if (fail_set(s_fail)) {
            if (issued > 0) {
                const int sl = issued - 1;
                mbar_wait(&fullAcc[sl & 1], (uint32_t)(sl >> 1) & 1u);
            }
            if (!have_a) mbar_wait(barA, 0);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == M2L_MMA_WARP) tmem_dealloc(tmem, TMEM_COLS);
}

// ======================================================================================
// M2L with the translation pairs as rows (rank rp <= 208):
//
//   for each work item (direction v, pairs p0..p1 of v, in tiles of 128 pairs):
//     D[j][i] = sum_k psi[src_j][k] C_v[i][k],   Y[dst_j][i] += D[j][i]
//
// The translation C_v (both BF16 halves, rp x rp, 4 rp^2 bytes) arrives once per item by bulk
// copy and stays resident as the B operand (N = rp output rows); the gathered split pairs of
// the source vectors stream through MT_STAGES stages of 16 K values as the A operand
// (M = 128 pairs).  Every gathered vector thus meets all rp output rows in one pass (no row
// tiles, no padded rows), and each MMA is 128 x rp x 16.  The accumulator is 128 lanes x rp
// FP32 columns, double buffered in tensor memory, so the epilogue of one tile overlaps the
// products of the next.
//
// The split pairs are read from the interleaved layout of split_pairs_kernel (per 8 K
// values: 16 bytes of hi, then 16 bytes of lo), so the 64 bytes of one vector that a K step
// needs are one piece that four lanes copy (a warp's copy touches 8 vectors, not 32).  The
// epilogue adds each lane's 16 columns into its target's row with 16-byte vector reductions.
// Measured at 1e6 points (1.98M pairs), the reductions set the pace: 0.95 ms per launch,
// 0.60 ms with them left out, 0.78 ms without the gathers, 0.89 ms without the products.
// Passing the columns through a shared-memory transpose for 64-byte reductions, or more
// copies in flight per thread, measured slower.
//
//   warps 0-7   epilogue: warp w reads lanes 32 (w % 4) .. (its 32 pairs) and the 16-column
//               blocks w / 4, w / 4 + 2, ... of an accumulator
//   warps 8-11  producers: thread q copies piece q % 4 of pairs q / 4 + 32 i (i < 4) of every
//               stage; groups of copies complete MT_LAG stages behind the issue and are then
//               published to the MMA thread
//   warp 12     owns the tensor memory; lane 0 loads the translation and issues the MMAs
// Every wait is bounded as in the kernel above.
// ======================================================================================
constexpr int MT_STAGES = 7;
constexpr int MT_LAG = 5;  // stages of copies in flight per producer thread (< MT_STAGES)
constexpr int MT_EPI_WARPS = 8;
constexpr int MT_PROD_THREADS = BM;
constexpr int MT_MMA_WARP = MT_EPI_WARPS + MT_PROD_THREADS / 32;
constexpr int MT_THREADS = 32 * (MT_MMA_WARP + 1);
constexpr uint32_t MT_A_HALF = BM * 16 * 2;   // one BF16 half of a 128 x 16 stage
constexpr uint32_t MT_STAGE = 2 * MT_A_HALF;
constexpr int MT_ACC_STRIDE = 256;             // tensor-memory columns between the accumulators
constexpr int MT_TMEM_COLS = 2 * MT_ACC_STRIDE;

__host__ __device__ inline uint32_t mt_smem_bytes(int rp)
{
    return 4u * rp * rp + MT_STAGES * MT_STAGE + 256;
}
__host__ __device__ inline bool mt_rank_ok(int rp)
{
    return rp % 16 == 0 && rp >= 16 && rp <= MT_ACC_STRIDE && mt_smem_bytes(rp) <= 227u * 1024u;
}

struct TcM2lArgs {
    const uint16_t *C;     // [n_dir][2][rp x rp] core-matrix images (hi, lo): row i = output index
    int n_dir;             // item.x = column * n_dir + direction (density columns batched)
    int64_t col_rows;      // rows of one density column in X2 and Y
    int rp;                // padded rank: K, N, and the row length of Y
    const int4 *items;     // {column * n_dir + direction, 0, p0, p1}
    const int *src_idx;    // pair j reads X2[src_idx[j]]
    const int *dst_idx;    // pair j adds into Y[dst_idx[j]]
    const uint16_t *X2;    // interleaved split pairs [rows][rp / 8][hi 8 | lo 8]
    float *Y;              // [rows][rp]
    int *err;              // set to 1 if a bounded wait gave up
};

// y[0..3] += (a, b, c, d): one 16-byte vector reduction (no return value)
__device__ __forceinline__ void red_add4(float *y, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(y), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

__global__ void __launch_bounds__(MT_THREADS, 1) tc_m2l_kernel(TcM2lArgs g)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const int rp = g.rp;
    const uint32_t c_half = (uint32_t)rp * (uint32_t)rp * 2u;
    unsigned char *sC = sm;                                  // [hi | lo] of the translation
    unsigned char *sA = sm + 2 * c_half;                     // MT_STAGES x [hi | lo] of 128 x 16
    uint64_t *bar = reinterpret_cast<uint64_t *>(sA + MT_STAGES * MT_STAGE);
    uint64_t *barC = bar, *full = bar + 1, *empty = full + MT_STAGES, *fullAcc = empty + MT_STAGES,
             *emptyAcc = fullAcc + 2;
    uint32_t *holder = reinterpret_cast<uint32_t *>(emptyAcc + 2);
    int *s_fail = reinterpret_cast<int *>(holder + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int4 item = g.items[blockIdx.x];
    const int ntiles = (item.w - item.z + BM - 1) / BM;
    const int nks = rp / 16;
    const int dir = item.x % g.n_dir;
    const int64_t crow = (int64_t)(item.x / g.n_dir) * g.col_rows;

    if (warp == MT_MMA_WARP) tmem_alloc(holder, MT_TMEM_COLS);
    if (tid == 0) {
        mbar_init(barC, 1);
        for (int i = 0; i < MT_STAGES; ++i) {
            mbar_init(&full[i], MT_PROD_THREADS);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&fullAcc[i], 1);
            mbar_init(&emptyAcc[i], MT_EPI_WARPS);
        }
        *s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder;
    auto fail = [&]() {
        atomicExch(s_fail, 1);
        atomicExch(g.err, 1);
    };

    if (warp < MT_EPI_WARPS) {
        // ---------------- epilogue
        const int quad = warp & 3, chalf = warp >> 2;
        const int nblk = rp / 16, my_blk = (nblk - chalf + 1) / 2;
        for (int t = 0; t < ntiles; ++t) {
            const int b = t & 1;
            const uint32_t u = (uint32_t)(t >> 1);
            const int pj = item.z + t * BM + quad * 32 + lane;
            float *y = pj < item.w ? g.Y + (size_t)(g.dst_idx[pj] + crow) * rp : nullptr;  // this lane's target
            if (__any_sync(0xffffffffu, fail_set(s_fail))) break;
            if (!__all_sync(0xffffffffu, mbar_wait(&fullAcc[b], u & 1u))) {
                if (lane == 0) fail();
                break;
            }
            tc_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * MT_ACC_STRIDE);
            for (int i = 0; i < my_blk; ++i) {
                const int c = 16 * (2 * i + chalf);
                float v[16];
                tmem_ld16(ta + (uint32_t)c, v);
                if (i + 1 == my_blk) {  // the last columns are in registers: release the accumulator
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&emptyAcc[b]);
                }
                if (y) {
#pragma unroll
                    for (int e = 0; e < 16; e += 4) red_add4(y + c + e, v[e], v[e + 1], v[e + 2], v[e + 3]);
                }
            }
            if (my_blk == 0) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&emptyAcc[b]);
            }
        }
    } else if (warp < MT_MMA_WARP) {
        // ---------------- producers
        const int q = tid - 32 * MT_EPI_WARPS;
        const int piece = q & 3, p0 = q >> 2;  // piece: (k half of the step) * 2 + (lo ? 1 : 0)
        const uint32_t half_off = (piece & 1) ? MT_A_HALF : 0u;
        const int kk = (piece >> 1) * 8;
        int64_t src[4], nxt[4];
        auto load_src = [&](int t, int64_t *s) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int pj = item.z + t * BM + p0 + 32 * i;
                s[i] = (t < ntiles && pj < item.w) ? (int64_t)g.src_idx[pj] + crow : (int64_t)-1;
            }
        };
        load_src(0, src);
        load_src(1, nxt);
        int gs = 0;  // global stage counter over the tiles
        bool ok = true;
        for (int t = 0; t < ntiles && ok; ++t) {
            for (int ks = 0; ks < nks; ++ks, ++gs) {
                const int st = gs % MT_STAGES;
                if (fail_set(s_fail)) {
                    ok = false;
                    break;
                }
                // stage st was read by the products of stage gs - MT_STAGES
                if (gs >= MT_STAGES && !mbar_wait(&empty[st], (uint32_t)(gs / MT_STAGES - 1) & 1u)) {
                    fail();
                    ok = false;
                    break;
                }
                unsigned char *base = sA + (size_t)st * MT_STAGE + half_off;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    unsigned char *d = base + core_offset(p0 + 32 * i, kk, BM);
                    if (src[i] >= 0) cp_async16(d, g.X2 + (size_t)src[i] * 2 * rp + ks * 32 + piece * 8);
                    else *reinterpret_cast<uint4 *>(d) = make_uint4(0, 0, 0, 0);
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
                if (gs >= MT_LAG) {
                    // the copies of stage gs - MT_LAG are complete: hand them to the async proxy
                    asm volatile("cp.async.wait_group %0;" ::"n"(MT_LAG) : "memory");
                    fence_proxy_async();
                    mbar_arrive(&full[(gs - MT_LAG) % MT_STAGES]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) src[i] = nxt[i];
            load_src(t + 2, nxt);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        fence_proxy_async();
        if (ok)
            for (int s = gs - MT_LAG < 0 ? 0 : gs - MT_LAG; s < gs; ++s) mbar_arrive(&full[s % MT_STAGES]);
    } else if (lane == 0) {
        // ---------------- translation load and MMA issue
        const unsigned char *csrc = reinterpret_cast<const unsigned char *>(g.C) + (size_t)dir * 2 * c_half;
        mbar_expect_tx(barC, 2 * c_half);
        for (uint32_t off = 0; off < 2 * c_half; off += 16384) {
            const uint32_t n = (2 * c_half - off) < 16384u ? (2 * c_half - off) : 16384u;
            bulk_g2s(sC + off, csrc + off, n, barC);
        }
        const uint32_t idesc = idesc_bf16(BM, rp);
        const uint32_t c0 = smem_u32(sC), a0 = smem_u32(sA);
        const uint32_t a_lbo = (BM / 8) * 128, c_lbo = (uint32_t)(rp / 8) * 128;
        bool have_c = false;
        int gs = 0, committed = 0;
        for (int t = 0; t < ntiles; ++t) {
            const int b = t & 1;
            if (fail_set(s_fail)) break;
            bool ok = t < 2 || mbar_wait(&emptyAcc[b], (uint32_t)((t >> 1) - 1) & 1u);
            if (ok && !have_c) ok = have_c = mbar_wait(barC, 0);
            if (!ok) {
                fail();
                break;
            }
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(b * MT_ACC_STRIDE);
            for (int ks = 0; ks < nks; ++ks, ++gs) {
                const int st = gs % MT_STAGES;
                if (!mbar_wait(&full[st], (uint32_t)(gs / MT_STAGES) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t as = a0 + (uint32_t)st * MT_STAGE, co = (uint32_t)(2 * ks) * c_lbo;
                const uint64_t ah = smem_desc(as, a_lbo, 128), al = smem_desc(as + MT_A_HALF, a_lbo, 128);
                const uint64_t ch = smem_desc(c0 + co, c_lbo, 128), cl = smem_desc(c0 + c_half + co, c_lbo, 128);
                mma_bf16(d, ah, ch, idesc, ks > 0 ? 1u : 0u);
                mma_bf16(d, ah, cl, idesc, 1u);
                mma_bf16(d, al, ch, idesc, 1u);
                mma_commit(&empty[st]);
                ++committed;
            }
            if (!ok) {
                fail();
                break;
            }
            mma_commit(&fullAcc[b]);
        }
        // before the memory goes: the products in flight (commits complete in order) and the
        // translation copy
        if (fail_set(s_fail) && committed > 0) {
            const int l = committed - 1;
            mbar_wait(&empty[l % MT_STAGES], (uint32_t)(l / MT_STAGES) & 1u);
        }
        if (!have_c) mbar_wait(barC, 0);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == MT_MMA_WARP) tmem_dealloc(tmem, MT_TMEM_COLS);
}

// ======================================================================================
// K-streamed variant for the box operators (check-to-equivalent factors, M2M, L2L, basis
// changes), whose K does not fit shared memory and whose products feed GMRES: FP32-grade
// accuracy is needed there, so both operands are split into THREE BF16 terms
// (a = a_h + a_m + a_l exactly for FP32 input; the operator's terms are taken from its FP64
// value) and each product is accumulated as hh + hm + mh + hl + lh + mm (the dropped terms
// are ~2^-26 of the product).  The tensor cores round their sums toward zero, and these
// products cancel heavily (high singular modes), so the rounding bias would add up over K:
// the leading term hh goes to a main accumulator restarted every FB chunks (two buffers,
// alternating) whose block sums are added in FP32 registers with round-to-nearest; the five
// small terms go to a third accumulator kept over the whole K range.
//
// One work item = one matrix, one row tile of 128, up to BN = 64 gathered columns.  K runs in
// chunks of KC = 32 through three pipeline stages: the operator chunk (3 terms, 24 KB)
// arrives by bulk copy two chunks ahead; the FP32 source rows are loaded into registers two
// chunks ahead, split, and stored in the core-matrix layout.  Output modes: store, add
// (exclusive rows), atomic add; each column may be scaled by alpha * geom[dst].w.
// ======================================================================================
constexpr int KC = 32;
constexpr int NTERM = 3;
constexpr int BOX_STAGES = 3;
constexpr int BOX_THREADS = 256;  // = BN * KC / 8: one 8-value group of one column per thread
constexpr int BOX_FB = 4;               // chunks per block of the main accumulator (>= BOX_STAGES - 1)
constexpr int BOX_TMEM_COLS = 4 * BN;  // main x2 | small terms | unused (power of two)

constexpr uint32_t A_TERM = BM * KC * 2;  // bytes of one term of an operator chunk
constexpr uint32_t B_TERM = BN * KC * 2;  // bytes of one term of a source chunk
constexpr uint32_t A_CHUNK = NTERM * A_TERM;
constexpr uint32_t STAGE_BYTES = NTERM * (A_TERM + B_TERM);

struct TcBoxArgs {
    const uint16_t *A;     // [n_mat][n_mtile][n_kc][term][BM x KC] core-matrix images
    int n_mat;             // item.x = column * n_mat + matrix (density columns batched)
    int64_t x_col_rows, y_col_rows;  // rows of one density column in X and Y
    int n_mtile, n_kc;
    int M;                 // valid rows
    const int4 *items;     // {matrix, mtile, c0, c1} with c1 - c0 <= BN
    const int *src_idx, *dst_idx, *parent;
    int src_par, dst_par;  // map the index through parent[] first
    const float *X;        // FP32 source rows; values past K must be finite (the operator is 0 there)
    int ldx;               // row length of X, a multiple of 8
    float *Y;
    int ldy;
    const float4 *geom;    // column scale alpha * geom[dst].w when non-null
    float alpha;
    int mode;              // 0 store, 1 add, 2 atomic add
    int *err;
};

__host__ __device__ inline uint32_t box_smem_bytes() { return BOX_STAGES * STAGE_BYTES + 128 + 2 * BN * 4; }

// three-term BF16 split of 8 FP32 values, stored as three 16-byte core-matrix rows.  Two
// values at a time: one packed round-to-nearest conversion gives both BF16 terms (low half =
// the first value), and each term is widened back by a shift or a mask (BF16 is the top half
// of an FP32), so a = h + m + l exactly with 11 instructions per pair of values.
__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void store_split3(unsigned char *dst, uint32_t term_stride, const float4 &x0,
                                             const float4 &x1)
{
    const float v[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
    uint32_t h[4], m[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float a = v[2 * q], b = v[2 * q + 1];
        const uint32_t th = bf16x2_rn(a, b);
        const float ra = a - __uint_as_float(th << 16), rb = b - __uint_as_float(th & 0xffff0000u);
        const uint32_t tm = bf16x2_rn(ra, rb);
        const float sa = ra - __uint_as_float(tm << 16), sb = rb - __uint_as_float(tm & 0xffff0000u);
        h[q] = th;
        m[q] = tm;
        l[q] = bf16x2_rn(sa, sb);
    }
    *reinterpret_cast<uint4 *>(dst) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(dst + term_stride) = make_uint4(m[0], m[1], m[2], m[3]);
    *reinterpret_cast<uint4 *>(dst + 2 * term_stride) = make_uint4(l[0], l[1], l[2], l[3]);
}

__global__ void __launch_bounds__(BOX_THREADS, 2) tc_box_gemm_kernel(TcBoxArgs g)
{
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *barA = reinterpret_cast<uint64_t *>(sm + BOX_STAGES * STAGE_BYTES);  // [BOX_STAGES]
    uint64_t *barM = barA + BOX_STAGES;                                             // [BOX_STAGES]
    uint32_t *holder = reinterpret_cast<uint32_t *>(barM + BOX_STAGES);
    int *s_fail = reinterpret_cast<int *>(holder + 1);
    int *s_src = reinterpret_cast<int *>(sm + BOX_STAGES * STAGE_BYTES + 128);
    int *s_dst = s_src + BN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, chalf = warp >> 2;
    const int4 item = g.items[blockIdx.x];
    const int ncols = min(BN, item.w - item.z);
    const int n_kc = g.n_kc;
    const int mat = item.x % g.n_mat, dcol = item.x / g.n_mat;

    if (warp == 0) tmem_alloc(holder, BOX_TMEM_COLS);
    if (tid < BN) {
        int sidx = -1, didx = -1;
        if (tid < ncols) {
            sidx = g.src_idx ? g.src_idx[item.z + tid] : item.z + tid;
            didx = g.dst_idx ? g.dst_idx[item.z + tid] : item.z + tid;
            if (g.src_par) sidx = g.parent[sidx];
            if (g.dst_par) didx = g.parent[didx];
        }
        s_src[tid] = sidx;
        s_dst[tid] = didx;
    }
    if (tid == 0) {
        for (int i = 0; i < 2 * BOX_STAGES; ++i) mbar_init(&barA[i], 1);
        *s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder;
    const uint32_t idesc = idesc_bf16(BM, BN);
    const unsigned char *Abase = reinterpret_cast<const unsigned char *>(g.A) +
                                 ((size_t)mat * g.n_mtile + item.y) * n_kc * (size_t)A_CHUNK;

    // this thread's piece of every source chunk: column col, values kb*8 .. kb*8 + 7
    const int col = tid % BN, kb = tid / BN;
    const int xrow = s_src[col];
    const float *xp = xrow >= 0 ? g.X + ((size_t)xrow + (size_t)dcol * g.x_col_rows) * g.ldx + kb * 8 : nullptr;
    const uint32_t boff = core_offset(col, kb * 8, BN);
    auto load_x = [&](int kc, float4 &x0, float4 &x1) {
        if (xp && kc * KC + kb * 8 + 8 <= g.ldx) {
            x0 = __ldg(reinterpret_cast<const float4 *>(xp + kc * KC));
            x1 = __ldg(reinterpret_cast<const float4 *>(xp + kc * KC + 4));
        } else {
            x0 = make_float4(0.f, 0.f, 0.f, 0.f);
            x1 = x0;
        }
    };
    auto issue_a = [&](int kc, int s) {  // one thread
        unsigned char *st = sm + (size_t)s * STAGE_BYTES;
        const unsigned char *src = Abase + (size_t)kc * A_CHUNK;
        mbar_expect_tx(&barA[s], A_CHUNK);
#pragma unroll
        for (int t = 0; t < NTERM; ++t) bulk_g2s(st + t * A_TERM, src + t * A_TERM, A_TERM, &barA[s]);
    };
    auto issue_mmas = [&](int s, int kc) {  // one thread
        const unsigned char *st = sm + (size_t)s * STAGE_BYTES;
        const uint32_t a0 = smem_u32(st), b0 = smem_u32(st + NTERM * A_TERM);
        const uint32_t a_lbo = (BM / 8) * 128, b_lbo = (BN / 8) * 128;
#pragma unroll
        for (int ks = 0; ks < KC / 16; ++ks) {
            const uint32_t ao = (uint32_t)(2 * ks) * a_lbo, bo = (uint32_t)(2 * ks) * b_lbo;
            uint64_t ad[NTERM], bd[NTERM];
#pragma unroll
            for (int t = 0; t < NTERM; ++t) {
                ad[t] = smem_desc(a0 + t * A_TERM + ao, a_lbo, 128);
                bd[t] = smem_desc(b0 + t * B_TERM + bo, b_lbo, 128);
            }
            const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
            const uint32_t acc_main = (kc % BOX_FB > 0 || ks > 0) ? 1u : 0u;
            const uint32_t t_main = tmem + (uint32_t)(((kc / BOX_FB) & 1) * BN);
            const uint32_t t_small = tmem + (uint32_t)(2 * BN);
            mma_bf16(t_small, ad[1], bd[1], idesc, acc);
            mma_bf16(t_small, ad[0], bd[2], idesc, 1u);
            mma_bf16(t_small, ad[2], bd[0], idesc, 1u);
            mma_bf16(t_small, ad[0], bd[1], idesc, 1u);
            mma_bf16(t_small, ad[1], bd[0], idesc, 1u);
            mma_bf16(t_main, ad[0], bd[0], idesc, acc_main);
        }
    };

    // this thread's output row (TMEM lane) and 32 columns; block sums of the main accumulator
    const uint32_t t_lane = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(chalf * (BN / 2));
    float racc[BN / 2];
#pragma unroll
    for (int i = 0; i < BN / 2; ++i) racc[i] = 0.f;
    auto add_acc = [&](uint32_t col0) {
#pragma unroll
        for (int h = 0; h < BN / 2; h += 16) {
            float t[16];
            tmem_ld16(t_lane + col0 + (uint32_t)h, t);
#pragma unroll
            for (int i = 0; i < 16; ++i) racc[h + i] += t[i];
        }
    };

    int loadsA = 0, commits = 0;  // operator chunks requested (thread 0), MMA groups committed
    // one K chunk; returns false (uniformly) after a failed wait
    auto step = [&](int kc, float4 &x0, float4 &x1) -> bool {
        const int s = kc % BOX_STAGES;
        bool w = true;
        // stage s was last read by the MMAs of chunk kc - 3
        if (kc >= BOX_STAGES) w = mbar_wait(&barM[s], (uint32_t)((kc - BOX_STAGES) / BOX_STAGES) & 1u);
        // the MMAs of chunk kc - 3 are complete: block b, whose last chunk that is, can be
        // folded into the registers; block b + 2 reuses its buffer no earlier than chunk kc
        if (w && kc >= BOX_FB + 2 && (kc - 2) % BOX_FB == 0) {
            tc_fence_after();
            add_acc((uint32_t)((((kc - 2) / BOX_FB - 1) & 1) * BN));
        }
        if (w) store_split3(sm + (size_t)s * STAGE_BYTES + NTERM * A_TERM + boff, B_TERM, x0, x1);
        if (kc + 2 < n_kc) load_x(kc + 2, x0, x1);
        if (tid == 0 && kc + 2 < n_kc && !*s_fail) {
            // the operator chunk two ahead goes to the stage last read by the MMAs of chunk
            // kc - 1 (committed at the end of the previous step)
            const int ns = (kc + 2) % BOX_STAGES;
            const bool w2 = kc + 2 < BOX_STAGES ||
                            mbar_wait(&barM[ns], (uint32_t)((kc + 2 - BOX_STAGES) / BOX_STAGES) & 1u);
            if (w2) {
                issue_a(kc + 2, ns);
                ++loadsA;
            } else {
                w = false;
            }
        }
        fence_proxy_async();
        tc_fence_before();
        const bool bad = __syncthreads_or(!w || (tid == 0 && *s_fail)) != 0;
        tc_fence_after();
        if (bad) return false;
        if (tid == 0) {
            if (mbar_wait(&barA[s], (uint32_t)(kc / BOX_STAGES) & 1u)) issue_mmas(s, kc);
            else *s_fail = 1;
            mma_commit(&barM[s]);
        }
        ++commits;
        return true;
    };

    float4 xa0, xa1, xb0, xb1;
    load_x(0, xa0, xa1);
    if (n_kc > 1) load_x(1, xb0, xb1);
    if (tid == 0) {
        issue_a(0, 0);
        loadsA = 1;
        if (n_kc > 1) {
            issue_a(1, 1);
            loadsA = 2;
        }
    }
    bool ok = true;
    for (int kc = 0; kc < n_kc && ok; kc += 2) {
        ok = step(kc, xa0, xa1);
        if (ok && kc + 1 < n_kc) ok = step(kc + 1, xb0, xb1);
    }
    if (ok) {
        // all products: wait for the last commit, then the epilogue
        const int kl = n_kc - 1;
        const bool w = mbar_wait(&barM[kl % BOX_STAGES], (uint32_t)(kl / BOX_STAGES) & 1u);
        ok = __syncthreads_or(!w || (tid == 0 && *s_fail)) == 0;
        tc_fence_after();
    }
    if (ok) {
        // blocks not folded in the loop (flush step kc = (b + 1) FB + 2 >= n_kc), then the
        // small terms
        const int nblk = (n_kc + BOX_FB - 1) / BOX_FB;
        for (int b = max(0, nblk - 2); b < nblk; ++b)
            if ((b + 1) * BOX_FB + 2 >= n_kc) add_acc((uint32_t)((b & 1) * BN));
        add_acc((uint32_t)(2 * BN));
        const int row = item.y * BM + quad * 32 + lane;
        if (row < g.M) {
#pragma unroll
            for (int k = 0; k < BN / 2; ++k) {
                const int d = s_dst[chalf * (BN / 2) + k];
                if (d < 0) continue;
                const float a = g.geom ? g.alpha * g.geom[d].w : g.alpha;
                float *y = g.Y + ((size_t)d + (size_t)dcol * g.y_col_rows) * g.ldy + row;
                if (g.mode == 0) *y = a * racc[k];
                else if (g.mode == 1) *y += a * racc[k];
                else atomicAdd(y, a * racc[k]);
            }
        }
    } else if (tid == 0) {
        // record the failure, then wait (bounded) for the products and operator copies still
        // in flight before the shared and tensor memory are released
        atomicExch(g.err, 1);
        if (commits > 0) mbar_wait(&barM[(commits - 1) % BOX_STAGES], (uint32_t)((commits - 1) / BOX_STAGES) & 1u);
        for (int c = max(0, loadsA - BOX_STAGES); c < loadsA; ++c)
            mbar_wait(&barA[c % BOX_STAGES], (uint32_t)(c / BOX_STAGES) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, BOX_TMEM_COLS);
}

}  // namespace tc
}  // namespace kfmm
