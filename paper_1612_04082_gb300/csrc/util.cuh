// util.cuh -- device helpers shared by the tree and FMM translation units: exclusive scan
// of int arrays, grid sizing, warp reductions.
#pragma once

#include "common.cuh"

namespace kfmm {

constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs (grids are sized in multiples of this)

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 152LL * 32) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// Exclusive scan of n ints: out[i] = sum_{j<i} in[j]; if total != nullptr, *total (device)
// receives sum of all.  in and out may alias.  Temporaries come from `scratch`.
kfmm_status scan_exclusive(kfmm_ctx *ctx, const int *in, int *out, int n, int *total);

// Synchronises the context stream; the pinned staging of earlier uploads is free again.
kfmm_status sync_stream(kfmm_ctx *ctx);

// Copies `bytes` of host memory to device memory in stream order through pinned staging:
// no synchronisation, and `src` may be reused as soon as the call returns.
kfmm_status upload_async(kfmm_ctx *ctx, void *dst, const void *src, size_t bytes);

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

}  // namespace kfmm
