// rank.cuh -- stable block-local ranking of radix digits.
//
// The technique is the published one of the Onesweep radix sort (Adinets and
// Merrill, "Onesweep: a faster least significant digit radix sort for GPUs",
// 2022): find the lanes of a warp that hold the same digit, rank each item
// among its earlier peers, keep running counts per (warp, digit).  The code
// below is written for this library, with its own peer and counter protocol.
//
// Items are held warp-striped: item i of lane l in warp w sits at block
// position w*32*ITEMS + i*32 + l, so visiting (warp, i, lane) in order
// visits positions in order.  For every item the warp finds its peers (the
// lanes holding the same digit), ranks the
// item among its earlier peers, and keeps a running count per (warp, digit)
// in shared memory.  A block-wide pass then turns the counts into exclusive
// offsets ordered by (digit, warp), which makes the whole ranking stable.
// (Finding peers with warp ballots takes one ballot per digit bit; a shared
// atomicOr per item measured about four times faster on GB300, and the full
// bucket kernel ran 9% slower with __match_any_sync in its place.)
#pragma once

#include "common.cuh"

namespace fsp {

// Rank ITEMS digits per thread inside the warp.  `wc` points at this warp's
// RADIX counters and `wm` at its RADIX peer masks (both zeroed).  rnk[i]
// receives the rank among earlier items of the same digit in this warp.
// Peers are found by OR-ing each lane's bit into the mask of its digit in
// shared memory and reading the mask back (one atomic and one load per item,
// instead of one ballot per digit bit); the highest peer then advances the
// counter and clears the mask for the next item.
template <int R, int ITEMS>
__device__ __forceinline__ void warp_rank(const uint32_t (&digit)[ITEMS], const bool (&valid)[ITEMS],
                                          uint32_t *wc, uint32_t *wm, uint32_t (&rnk)[ITEMS]) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t d = digit[i];
        if (valid[i]) atomicOr(&wm[d], 1u << lane);
        __syncwarp();
        uint32_t peers = 0, before = 0;
        if (valid[i]) {
            peers = wm[d];
            before = wc[d];
        }
        __syncwarp();
        if (valid[i] && lane == 31 - __clz(peers)) {
            wc[d] = before + __popc(peers);
            wm[d] = 0;
        }
        __syncwarp();
        rnk[i] = before + __popc(peers & lt);
    }
}

// After warp_rank in every warp (and a __syncthreads): turn the per-warp
// counts s_wcnt[WARPS][RADIX] into exclusive offsets across warps and write
// the block-local start of every digit into s_local[RADIX].  Requires
// THREADS >= RADIX.  Ends with __syncthreads.
template <int R, int THREADS>
__device__ __forceinline__ void digit_offsets(uint32_t *s_wcnt, uint32_t *s_local, uint32_t *s_scan) {
    constexpr int RADIX = 1 << R, WARPS = THREADS / 32;
    static_assert(THREADS >= RADIX, "one thread per digit");
    const int tid = threadIdx.x;
    uint32_t total = 0;
    if (tid < RADIX) {
        for (int w = 0; w < WARPS; ++w) {
            const uint32_t c = s_wcnt[w * RADIX + tid];
            s_wcnt[w * RADIX + tid] = total;
            total += c;
        }
    }
    uint32_t sum;
    const uint32_t local = block_exclusive_scan<THREADS>(tid < RADIX ? total : 0u, s_scan, &sum);
    if (tid < RADIX) s_local[tid] = local;
    __syncthreads();
}

}  // namespace fsp
