// scan.cu -- single-pass exclusive scan with decoupled look-back.
//
// Used for the column pointer (Part 4 of §2.3: jcS is the running sum of
// unique counts per column, jcS[0] = 0, jcS[n] = nnz) and for the bucket
// offsets of the hybrid path.  Tiles are taken by atomic ticket; each tile
// publishes its aggregate, then its inclusive prefix, in 32-bit look-back
// words (values below 2^30).
#include <algorithm>

#include "common.cuh"
#include "internal.hpp"

namespace fsp {

// From this many tiles on, reduce-then-scan replaces the single pass.
constexpr int64_t kReduceScanTiles = 256;

template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS)
    scan_kernel(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t count,
                uint32_t *look, uint32_t *ticket, DevStatus *st, int withhold_first) {
    constexpr int TILE = THREADS * ITEMS;
    __shared__ uint32_t s_scan[THREADS / 32 + 1];
    __shared__ uint32_t s_tile, s_excl;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t p0 = tile * TILE + (int64_t)tid * ITEMS;
    static_assert(ITEMS % 4 == 0, "16-byte groups");
    uint32_t v[ITEMS];
    uint32_t sum = 0;
    const bool whole = p0 + ITEMS <= count;
    if (whole && (reinterpret_cast<uintptr_t>(in) & 15) == 0) {
#pragma unroll
        for (int q = 0; q < ITEMS / 4; ++q) {
            const uint4 x = reinterpret_cast<const uint4 *>(in + p0)[q];
            v[4 * q] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) v[i] = p0 + i < count ? in[p0 + i] : 0u;
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) sum += v[i];
    uint32_t tile_sum;
    const uint32_t mine = block_exclusive_scan<THREADS>(sum, s_scan, &tile_sum);
    if (tid < 32) {
        uint32_t *word = look + tile;
        uint32_t excl = 0;
        // (withhold_first: injected failure -- tile 0 never publishes, so the
        // bounded waits of the following tiles run out)
        if (tid == 0 && !(withhold_first && tile == 0)) st_release(word, (tile == 0 ? kFlagInc : kFlagAgg) | tile_sum);
        if (tile > 0) {
            excl = warp_lookback_exclusive(look, 1, tile, st);
            if (tid == 0) st_release(word, kFlagInc | (excl + tile_sum));
        }
        if (tid == 0) s_excl = excl;
    }
    __syncthreads();
    uint32_t run = s_excl + mine;
    if (whole && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
#pragma unroll
        for (int q = 0; q < ITEMS / 4; ++q) {
            uint4 y;
            y.x = run;
            run += v[4 * q];
            y.y = run;
            run += v[4 * q + 1];
            y.z = run;
            run += v[4 * q + 2];
            y.w = run;
            run += v[4 * q + 3];
            reinterpret_cast<uint4 *>(out + p0)[q] = y;
        }
        if (p0 + ITEMS == count) out[count] = run;
    } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int64_t p = p0 + i;
            if (p < count) {
                out[p] = run;
                run += v[i];
                if (p == count - 1) out[count] = run;
            }
        }
    }
}

// Long inputs: reduce, then scan.  Each tile's sum first (one read), the
// tile sums scanned by the single-pass kernel above, then every tile scanned
// again from its offset (a second read and the write).  Tiles never wait on
// each other, which the single pass does once thousands of tiles are in
// flight at once.
template <int THREADS, int ITEMS>
__device__ __forceinline__ bool load_tile(const uint32_t *__restrict__ in, int64_t count, int64_t p0,
                                          uint32_t (&v)[ITEMS]) {
    const bool whole = p0 + ITEMS <= count;
    if (whole && (reinterpret_cast<uintptr_t>(in) & 15) == 0) {
#pragma unroll
        for (int q = 0; q < ITEMS / 4; ++q) {
            const uint4 x = __ldg(reinterpret_cast<const uint4 *>(in + p0) + q);
            v[4 * q] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) v[i] = p0 + i < count ? __ldg(in + p0 + i) : 0u;
    }
    return whole;
}

template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS)
    tile_sum_kernel(const uint32_t *__restrict__ in, int64_t count, uint32_t *__restrict__ tsum) {
    constexpr int TILE = THREADS * ITEMS;
    __shared__ uint32_t s_scan[THREADS / 32 + 1];
    uint32_t v[ITEMS];
    load_tile<THREADS, ITEMS>(in, count, blockIdx.x * (int64_t)TILE + (int64_t)threadIdx.x * ITEMS, v);
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) sum += v[i];
    uint32_t total;
    block_exclusive_scan<THREADS>(sum, s_scan, &total);
    if (threadIdx.x == 0) tsum[blockIdx.x] = total;
}

template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS)
    tile_scan_kernel(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t count,
                     const uint32_t *__restrict__ toff) {
    constexpr int TILE = THREADS * ITEMS;
    __shared__ uint32_t s_scan[THREADS / 32 + 1];
    const int64_t p0 = blockIdx.x * (int64_t)TILE + (int64_t)threadIdx.x * ITEMS;
    uint32_t v[ITEMS];
    const bool whole = load_tile<THREADS, ITEMS>(in, count, p0, v);
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) sum += v[i];
    uint32_t total;
    uint32_t run = __ldg(toff + blockIdx.x) + block_exclusive_scan<THREADS>(sum, s_scan, &total);
    if (whole && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
#pragma unroll
        for (int q = 0; q < ITEMS / 4; ++q) {
            uint4 y;
            y.x = run;
            run += v[4 * q];
            y.y = run;
            run += v[4 * q + 1];
            y.z = run;
            run += v[4 * q + 2];
            y.w = run;
            run += v[4 * q + 3];
            reinterpret_cast<uint4 *>(out + p0)[q] = y;
        }
        if (p0 + ITEMS == count) out[count] = run;
    } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int64_t p = p0 + i;
            if (p < count) {
                out[p] = run;
                run += v[i];
                if (p == count - 1) out[count] = run;
            }
        }
    }
}

fsparse_status exclusive_scan_u32(const uint32_t *counts, uint32_t *out, int64_t count,
                                  DevStatus *st, Scratch &scratch, cudaStream_t s) {
    constexpr int THREADS = 256, ITEMS = 16, TILE = THREADS * ITEMS;
    if (count == 0) {
        FSP_CUDA(cudaMemsetAsync(out, 0, 4, s));
        return FSPARSE_OK;
    }
    const int64_t ntiles = (count + TILE - 1) / TILE;
    fsparse_status e;
    const int withhold = injected_fault() == FAULT_TIMEOUT ? 1 : 0;
    // (an injected timeout keeps the single pass, whose waits it exercises)
    if (ntiles >= kReduceScanTiles && !withhold) {
        uint32_t *tsum, *toff;
        if ((e = scratch.get(&tsum, (size_t)ntiles)) != FSPARSE_OK) return e;
        if ((e = scratch.get(&toff, (size_t)ntiles + 1)) != FSPARSE_OK) return e;
        tile_sum_kernel<THREADS, ITEMS><<<(unsigned)ntiles, THREADS, 0, s>>>(counts, count, tsum);
        FSP_LAUNCHED();
        if ((e = exclusive_scan_u32(tsum, toff, ntiles, st, scratch, s)) != FSPARSE_OK) return e;
        tile_scan_kernel<THREADS, ITEMS><<<(unsigned)ntiles, THREADS, 0, s>>>(counts, out, count, toff);
        FSP_LAUNCHED();
        return FSPARSE_OK;
    }
    uint32_t *look, *ticket;
    if ((e = scratch.get(&look, (size_t)ntiles)) != FSPARSE_OK) return e;
    if ((e = scratch.get(&ticket, 1)) != FSPARSE_OK) return e;
    FSP_CUDA(cudaMemsetAsync(look, 0, (size_t)ntiles * 4, s));
    FSP_CUDA(cudaMemsetAsync(ticket, 0, 4, s));
    scan_kernel<THREADS, ITEMS><<<(unsigned)ntiles, THREADS, 0, s>>>(counts, out, count, look, ticket, st, withhold);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

}  // namespace fsp
