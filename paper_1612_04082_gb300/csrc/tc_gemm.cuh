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
// One CTA of 4 warps per work item.  The A tile (both halves, pre-laid-out in global
// memory) arrives by cp.async.bulk; the B tile is gathered, split and stored by all threads;
// one thread issues the MMAs and commits them to an mbarrier; every warp then reads its 32
// TMEM lanes and adds them to the output.  Every mbarrier wait is bounded: on time-out the
// kernel records the error, waits (bounded) for its own copies and MMAs, frees its tensor
// memory and returns.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace kfmm {
namespace tc {

constexpr int BM = 128;       // rows per tile (UMMA M)
constexpr int BN = 64;        // columns per N step (UMMA N)
constexpr int THREADS = 256;  // 8 warps: warp w reads TMEM lanes 32 (w % 4) .. + 31, column half w / 4
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

// true when the phase with parity `phase` has completed; false after WAIT_LIMIT polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase)
{
    const uint32_t a = smem_u32(bar);
    for (long long i = 0; i < WAIT_LIMIT; ++i) {
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

// dynamic shared memory: [A hi | A lo | B0 hi | B0 lo | B1 hi | B1 lo | mbar x3 + flags | dst x2]
__host__ __device__ inline uint32_t smem_bytes(int Kp)
{
    return 2 * half_bytes(BM, Kp) + 4 * half_bytes(BN, Kp) + 64 + 3 * 4 * BN;
}

// X2[box] = the BF16 split pair of X[box] (Kp values): hi at [0, Kp), lo at [Kp, 2 Kp).  Each
// 8-value chunk of K is then 16 contiguous bytes, one row of a core matrix.
__global__ void split_pairs_kernel(const float *__restrict__ X, int64_t n_rows, int Kp, uint16_t *__restrict__ X2)
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
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * q]), h1 = __float2bfloat16_rn(v[2 * q + 1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * q] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * q + 1] - __bfloat162float(h1));
        h[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        l[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    uint16_t *dst = X2 + row * 2 * Kp + kb * 8;
    *reinterpret_cast<uint4 *>(dst) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(dst + Kp) = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}

// Gather columns [c0, c0 + ncols) of the split pairs as the B operand (rows = columns of the
// product) in the core-matrix layout by 16-byte asynchronous copies; record destinations.
// THREADS is a multiple of BN, so each thread keeps one column (one index load).
__device__ __forceinline__ void gather_b(const TcArgs &g, int c0, int ncols, unsigned char *sB, uint32_t b_half,
                                         int *s_dst)
{
    const int Kp = g.Kp;
    const int col = threadIdx.x % BN;
    if (threadIdx.x < BN) s_dst[col] = col < ncols ? g.dst_idx[c0 + col] : -1;
    const uint16_t *xs = col < ncols ? g.X2 + (size_t)g.src_idx[c0 + col] * 2 * Kp : nullptr;
    for (int kb = threadIdx.x / BN; kb < Kp / 8; kb += THREADS / BN) {
        const uint32_t off = core_offset(col, kb * 8, BN);
        if (xs) {
            cp_async16(sB + off, xs + kb * 8);
            cp_async16(sB + b_half + off, xs + Kp + kb * 8);
        } else {
            *reinterpret_cast<uint4 *>(sB + off) = make_uint4(0, 0, 0, 0);
            *reinterpret_cast<uint4 *>(sB + b_half + off) = make_uint4(0, 0, 0, 0);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void gather_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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

// Pipeline per N step s (buffers b = s % 2): gather B(s+1) while MMA(s) runs; issue
// MMA(s+1) into the other accumulator; then wait for MMA(s) and add accumulator b to the
// output while MMA(s+1) runs.
__global__ void __launch_bounds__(THREADS, 1) tc_gather_gemm_kernel(TcArgs g)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const int Kp = g.Kp;
    const uint32_t a_half = half_bytes(BM, Kp), b_half = half_bytes(BN, Kp);
    unsigned char *sA = sm;
    unsigned char *sB[2] = {sm + 2 * a_half, sm + 2 * a_half + 2 * b_half};
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 2 * a_half + 4 * b_half);  // [0] A, [1] [2] MMA
    uint32_t *holder = reinterpret_cast<uint32_t *>(bar + 3);
    int *s_fail = reinterpret_cast<int *>(bar + 3) + 1;
    // destination indices of steps s - 1, s, s + 1 are live at once (the epilogue of s - 1 may
    // still be reading while step s + 1 is gathered), hence three buffers indexed by s % 3
    int *s_dst0 = reinterpret_cast<int *>(sm + 2 * a_half + 4 * b_half + 64);
    int *s_dst[3] = {s_dst0, s_dst0 + BN, s_dst0 + 2 * BN};
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, chalf = warp >> 2;
    const int4 item = g.items[blockIdx.x];
    const int nsteps = (item.w - item.z + BN - 1) / BN;

    if (warp == 0) tmem_alloc(holder, TMEM_COLS);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        *s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *holder;
    const uint32_t a0 = smem_u32(sA), bs0 = smem_u32(sB[0]), bs1 = smem_u32(sB[1]);

    // A tile (both halves) by bulk copy
    if (tid == 0) {
        const unsigned char *src = reinterpret_cast<const unsigned char *>(g.A) +
                                   ((size_t)item.x * g.n_mtile + item.y) * 2 * (size_t)a_half;
        mbar_expect_tx(&bar[0], 2 * a_half);
        const uint32_t chunk = 16384;
        for (uint32_t off = 0; off < 2 * a_half; off += chunk) {
            const uint32_t n = (2 * a_half - off) < chunk ? (2 * a_half - off) : chunk;
            bulk_g2s(sA + off, src + off, n, &bar[0]);
        }
    }
    // prologue: B(0), then MMA(0)
    gather_b(g, item.z, min(BN, item.w - item.z), sB[0], b_half, s_dst[0]);
    gather_wait();
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        if (mbar_wait(&bar[0], 0)) {
            issue_mmas(a0, a_half, bs0, b_half, Kp, tmem);
        } else {
            *s_fail = 1;
            atomicExch(g.err, 1);
        }
        mma_commit(&bar[1]);
    }
    uint32_t phase[2] = {0u, 0u};
    bool issued_next = false;
    int s = 0;
    for (; s < nsteps; ++s) {
        const int b = s & 1, nb = b ^ 1;
        issued_next = false;
        if (s + 1 < nsteps) {
            const int c0 = item.z + (s + 1) * BN;
            gather_b(g, c0, min(BN, item.w - c0), sB[nb], b_half, s_dst[(s + 1) % 3]);
            gather_wait();
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (s + 1 < nsteps) {
            if (tid == 0) {
                if (!*s_fail) issue_mmas(a0, a_half, nb ? bs1 : bs0, b_half, Kp, tmem + (uint32_t)(nb * BN));
                mma_commit(&bar[1 + nb]);
            }
            issued_next = true;
        }
        bool ok = mbar_wait(&bar[1 + b], phase[b]);
        phase[b] ^= 1u;
        if (!ok) atomicExch(g.err, 1);
        ok = __syncthreads_or(!ok || *s_fail) == 0;  // one decision for the whole CTA
        tc_fence_after();
        if (!ok) break;
        // epilogue of step s: this warp's lane quadrant, its half of the BN columns
        const int row = item.y * BM + quad * 32 + lane;
#pragma unroll
        for (int cb = 0; cb < BN / 2; cb += 16) {
            const int col = chalf * (BN / 2) + cb;
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * BN + col), v);
            if (row < g.M) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int d = s_dst[s % 3][col + q];
                    if (d >= 0) atomicAdd(g.Y + (size_t)d * g.ldy + row, v[q]);
                }
            }
        }
        tc_fence_before();
    }
    // after a failure, let the products already issued finish before freeing tensor memory
    if (s < nsteps && tid == 0) {
        const int b = s & 1;
        mbar_wait(&bar[1 + b], phase[b] ^ 1u);  // the step that failed (returns at once if done)
        if (issued_next) mbar_wait(&bar[1 + (b ^ 1)], phase[b ^ 1]);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace tc
}  // namespace kfmm
