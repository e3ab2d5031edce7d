// common.cuh -- device-side building blocks shared by the fsparse kernels.
//
// * DevStatus: the single status block every symbolic call writes on the
//   device and reads back once on the host (bad indices, bounded-wait
//   expiry, bucket overflow, implicit dimensions, nnz).
// * Decoupled look-back words: 32-bit, two flag bits + a 30-bit count.
//   Every wait on a predecessor is bounded; on expiry the kernel records
//   FSPARSE_ERR_TIMEOUT in DevStatus and carries on with a zero
//   contribution, so no launch can hang.
// * Small warp/block helpers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fsp {

constexpr uint32_t kHeadBit = 0x80000000u;   // perm[p] | kHeadBit marks the first triplet of a run
constexpr uint32_t kIndexMask = 0x7fffffffu;
// The numeric fold works on chunks of kChunk sorted positions; the plan keeps
// one slot base per chunk.
constexpr int kChunk = 16;
constexpr int kChunkShift = 4;

// Look-back word layout: [31:30] flag, [29:0] value.
constexpr uint32_t kFlagAgg = 1u << 30;      // tile aggregate only
constexpr uint32_t kFlagInc = 2u << 30;      // inclusive prefix through this tile
constexpr uint32_t kFlagMask = 3u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1;
constexpr int64_t kMaxLookbackValue = (int64_t(1) << 30) - 1;

// Polls of one predecessor word before giving up (each poll sleeps up to
// ~0.25 us after the first few): roughly half a second per predecessor.
constexpr int kSpinLimit = 1 << 21;

struct DevStatus {
    uint32_t bad_index;   // some index < 1 or beyond its dimension
    uint32_t timeout;     // a bounded wait expired
    uint32_t overflow;    // a column bucket exceeded shared-memory capacity
    int32_t max_i;        // largest row index seen (implicit m)
    int32_t max_j;        // largest column index seen (implicit n)
    uint32_t nnz;         // unique (row, column) pairs
    uint32_t oob;         // an internal index check failed (access skipped)
    uint32_t pad;
};

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive prefix of all tiles before `tile` for one bin: walk back over
// the words word[t * stride], t = tile-1, tile-2, ..., adding aggregates
// until an inclusive prefix is found.  Tiles are numbered by an atomic
// ticket, so every predecessor belongs to a block that is already running
// and will publish; the bound below only guards against the impossible.
__device__ __forceinline__ uint32_t lookback_exclusive(const uint32_t *word, int64_t stride,
                                                       int64_t tile, DevStatus *st) {
    uint32_t excl = 0;
    for (int64_t t = tile - 1; t >= 0; --t) {
        const uint32_t *w = word + t * stride;
        uint32_t v = ld_acquire(w);
        int spins = 0;
        while ((v & kFlagMask) == 0) {
            if (++spins > kSpinLimit) {
                atomicOr(&st->timeout, 1u);
                v = kFlagInc;   // treat as a zero inclusive prefix and stop
                break;
            }
            if (spins > 8) __nanosleep(spins > 64 ? 256 : 32);
            v = ld_acquire(w);
        }
        excl += v & kValueMask;
        if ((v & kFlagMask) == kFlagInc) break;
    }
    return excl;
}

// Warp-cooperative version of lookback_exclusive: all 32 lanes of the calling
// warp take part and inspect 32 predecessors per step (lane i looks at
// tile-1-i), so a walk over many aggregate-only predecessors costs one load
// latency per 32 of them.  Every lane returns the same value.  Bounded like
// lookback_exclusive.
__device__ __forceinline__ uint32_t warp_lookback_exclusive(const uint32_t *word, int64_t stride,
                                                            int64_t tile, DevStatus *st) {
    const int lane = threadIdx.x & 31;
    uint32_t excl = 0;
    for (int64_t hi = tile - 1; hi >= 0; hi -= 32) {
        const int64_t t = hi - lane;
        const bool have = t >= 0;
        uint32_t v = have ? ld_acquire(word + t * stride) : kFlagInc;
        int spins = 0;
        uint32_t need;
        while (true) {
            const uint32_t inc = __ballot_sync(0xffffffffu, have && (v & kFlagMask) == kFlagInc);
            const uint32_t ready = __ballot_sync(0xffffffffu, !have || (v & kFlagMask) != 0);
            need = inc ? ((inc & (0u - inc)) << 1) - 1u : 0xffffffffu;   // lanes up to the nearest inclusive
            if (need == 0) need = 0xffffffffu;                              // (inclusive in lane 31: all lanes)
            if ((ready & need) == need) break;
            if (++spins > kSpinLimit) {
                if (lane == 0) atomicOr(&st->timeout, 1u);
                return excl;
            }
            if (spins > 8) __nanosleep(spins > 64 ? 256 : 32);
            if (have && (v & kFlagMask) == 0) v = ld_acquire(word + t * stride);
        }
        const uint32_t inc = __ballot_sync(0xffffffffu, have && (v & kFlagMask) == kFlagInc);
        uint32_t part = ((need >> lane) & 1u) && have ? (v & kValueMask) : 0u;
#pragma unroll
        for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        excl += part;
        if (inc) break;
    }
    return excl;
}

// Runs of equal keys in consecutive lanes of a warp (all 32 lanes call it):
// *head is the first lane of this lane's run, *count (valid in head lanes)
// the run's length.  One shared-memory atomic per run instead of one per
// lane removes the same-address serialisation when neighbouring lanes hold
// the same key (triplets of one element share columns).  Give lanes without
// an item a key no real item has, e.g. 0xffff0000 | lane.
__device__ __forceinline__ void lane_runs(uint32_t key, int *head, uint32_t *count) {
    const int lane = threadIdx.x & 31;
    const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    const uint32_t hm = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
    *head = 31 - __clz(hm & ((2u << lane) - 1u));
    const uint32_t after = hm & ~((2u << lane) - 1u);   // heads above this lane
    *count = (after ? (uint32_t)(__ffs(after) - 1) : 32u) - (uint32_t)lane;
}

// Block-wide exclusive scan of one uint32 per thread; returns the total in
// *total.  `scratch` needs THREADS/32 + 1 words of shared memory.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *scratch, uint32_t *total) {
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < WARPS ? scratch[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < WARPS) scratch[lane] = wi - w;
        if (lane == WARPS - 1) scratch[WARPS] = wi;
    }
    __syncthreads();
    uint32_t out = scratch[warp] + inc - x;
    *total = scratch[WARPS];
    __syncthreads();
    return out;
}

// Defensive bound on every computed scatter/gather index: a value that a
// correct kernel never produces is recorded and the access is skipped, so a
// bug shows up as FSPARSE_ERR_INTERNAL instead of a memory fault.
__device__ __forceinline__ bool in_range(int64_t v, int64_t bound, DevStatus *st) {
    if (v >= 0 && v < bound) return true;
    if (st) atomicOr(&st->oob, 1u);
    return false;
}

// +0.0 + v, exactly, without an FP64 add (FP64 adds are scarce on GB300):
// equal to v for every v except -0.0, which becomes +0.0 (a NaN stays NaN).
// Every fold starts a run with it: the App. A insert adds into zeroed storage.
__device__ __forceinline__ double plus_zero(double v) {
    const unsigned long long b = __double_as_longlong(v);
    return __longlong_as_double(b == 0x8000000000000000ull ? 0ull : b);
}

// Value of triplet x (head bit ignored); an index beyond len, which a valid
// plan never holds, reads as 0 instead of faulting.
__device__ __forceinline__ double gather(const double *__restrict__ sr, uint32_t x, int64_t len) {
    const uint32_t k = x & kIndexMask;
    return k < len ? __ldg(sr + k) : 0.0;
}

// Index validation shared by every kernel that reads ii/jj: an index outside
// [1, dim] is reported and replaced by 1, so nothing downstream can address
// out of bounds; the host then returns FSPARSE_ERR_INDEX.
__device__ __forceinline__ int32_t checked_index(int32_t v, int32_t dim, DevStatus *st) {
    if (v < 1 || v > dim) {
        atomicOr(&st->bad_index, 1u);
        return 1;
    }
    return v;
}

}  // namespace fsp
