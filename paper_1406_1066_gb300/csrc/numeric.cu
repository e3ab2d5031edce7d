// numeric.cu -- the value side of the assembly.
//
// Numeric fold (Eq. (2.3) with the App. A insert order): the plan stores the
// sorted order perm[p] = k, with kHeadBit on the first triplet of every run
// (one run per CCS slot), and tile_slot0[q] = number of runs that start
// before numeric tile q.  ONE thread folds each run from +0.0 in ascending
// position order -- which is ascending k, the paper's order -- so the result
// is identical to the serial insert, bit for bit, for any launch shape.  No
// atomics touch values.
//
// Adjoint: ds[k] = dprS[irank[k]], the transpose of the fold (the map is
// linear in sr); 128-bit loads of irank and stores of ds.
#include <algorithm>

#include "common.cuh"
#include "internal.hpp"

namespace fsp {

// Value of triplet x (head bit ignored); an index beyond len, which a valid
// plan never holds, reads as 0 instead of faulting.
__device__ __forceinline__ double gather(const double *__restrict__ sr, uint32_t x, int64_t len) {
    const uint32_t k = x & kIndexMask;
    return k < len ? __ldg(sr + k) : 0.0;
}

// Register-blocked fold.  Thread t of a tile owns IPT consecutive positions:
// it loads their perm entries with 128-bit loads, issues all IPT value
// gathers at once, and folds every run that starts in its chunk in
// registers.  A run that crosses the chunk end continues through the leading
// segments (positions before the first run head) of the following threads,
// which are published in shared memory column-major (conflict-free), and,
// at the tile end, through a prefetched halo of the next tile.
template <int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS)
    numeric_kernel(const uint32_t *__restrict__ perm, const double *__restrict__ sr,
                   const uint32_t *__restrict__ tile_slot0, double *__restrict__ prS, int64_t len,
                   int64_t ntiles, int64_t nnz) {
    constexpr int NT = THREADS * IPT, HALO = 32;
    __shared__ double s_lead[NT + HALO];     // [j * THREADS + t]: leading values of thread t
    __shared__ uint8_t s_nlead[THREADS];     // leading-segment length of each thread
    __shared__ uint8_t s_ends[THREADS];      // 1 if a run head lies in the thread's chunk
    __shared__ uint32_t s_scan[THREADS / 32 + 1];
    __shared__ int s_halo;                   // halo positions before the next head (HALO+1: none)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(perm) & 15) == 0;
    for (int64_t q = blockIdx.x; q < ntiles; q += gridDim.x) {
        const int64_t P0 = q * NT;
        const int cnt = (int)min64(NT, len - P0);
        const int first = tid * IPT;
        const int nval = max(0, min(IPT, cnt - first));
        uint32_t pm[IPT];
        if (nval == IPT && vec) {
#pragma unroll
            for (int v = 0; v < IPT / 4; ++v) {
                const uint4 x = reinterpret_cast<const uint4 *>(perm + P0 + first)[v];
                pm[4 * v] = x.x;
                pm[4 * v + 1] = x.y;
                pm[4 * v + 2] = x.z;
                pm[4 * v + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < IPT; ++i) pm[i] = i < nval ? perm[P0 + first + i] : kHeadBit;
        }
        double v[IPT];
#pragma unroll
        for (int i = 0; i < IPT; ++i) v[i] = i < nval ? gather(sr, pm[i], len) : 0.0;
        uint32_t hmask = 0;
#pragma unroll
        for (int i = 0; i < IPT; ++i)
            if (i < nval && (pm[i] & kHeadBit)) hmask |= 1u << i;
        const int lead = hmask ? __ffs(hmask) - 1 : nval;
#pragma unroll
        for (int i = 0; i < IPT; ++i)
            if (i < lead) s_lead[i * THREADS + tid] = v[i];
        s_nlead[tid] = (uint8_t)lead;
        s_ends[tid] = hmask != 0 || nval < IPT;   // a short chunk is the end of the data
        // The last warp prefetches the halo: where the tile's last run may go on.
        if (warp == THREADS / 32 - 1) {
            const int64_t hp = P0 + cnt + lane;
            const bool in = cnt == NT && hp < len;
            const uint32_t x = in ? perm[hp] : kHeadBit;
            const uint32_t hm = __ballot_sync(0xffffffffu, x & kHeadBit);
            const int end = hm ? __ffs(hm) - 1 : HALO + 1;   // HALO+1: the run goes past the halo
            if (lane < (end > HALO ? HALO : end)) s_lead[NT + lane] = gather(sr, x, len);
            if (lane == 0) s_halo = end;
        }
        uint32_t tile_heads;
        const uint32_t excl = block_exclusive_scan<THREADS>(__popc(hmask), s_scan, &tile_heads);

        // Runs that start in this chunk, folded in registers from +0.0.
        int64_t slot = (int64_t)tile_slot0[q] + excl;
        double acc = 0.0;
        bool open = false;
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            if ((hmask >> i) & 1u) {
                if (open && slot < nnz) prS[slot] = acc;
                slot += open;
                acc = 0.0;   // +0.0: the insert adds into zeroed storage
                open = true;
            }
            if (open && i < nval) acc += v[i];
        }
        if (open) {
            // Continue through the leading segments of the following threads.
            bool done = nval < IPT;
            int t = tid + 1;
            for (; !done && t < THREADS; ++t) {
                const int nl = s_nlead[t];
                for (int j = 0; j < nl; ++j) acc += s_lead[j * THREADS + t];
                done = s_ends[t];
            }
            if (!done) {
                const int h = s_halo;
                const int take = h > HALO ? HALO : h;
                for (int j = 0; j < take; ++j) acc += s_lead[NT + j];
                if (h > HALO) {
                    // Longer than the halo: stream the rest, eight at a time, in order.
                    int64_t g = P0 + cnt + HALO;
                    while (g < len) {
                        uint32_t x[8];
                        int c = 0;
#pragma unroll
                        for (int u = 0; u < 8; ++u) x[u] = g + u < len ? perm[g + u] : kHeadBit;
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (c == u && !(x[u] & kHeadBit)) ++c;
                        double w[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) w[u] = u < c ? gather(sr, x[u], len) : 0.0;
                        for (int u = 0; u < c; ++u) acc += w[u];
                        if (c < 8) break;
                        g += 8;
                    }
                }
            }
            if (slot < nnz) prS[slot] = acc;
        }
        __syncthreads();   // s_lead / s_nlead are reused by the next tile
    }
}

template <int THREADS, int IPT>
static fsparse_status run_numeric(const uint32_t *perm, const uint32_t *tile_slot0, int64_t len,
                                  int64_t ntiles, const double *sr, double *prS, int64_t nnz,
                                  cudaStream_t s) {
    auto kern = numeric_kernel<THREADS, IPT>;
    int per_sm = 0;
    FSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, 0));
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sm_count(0) * std::max(per_sm, 1) * 8);
    kern<<<(unsigned)grid, THREADS, 0, s>>>(perm, sr, tile_slot0, prS, len, ntiles, nnz);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

fsparse_status launch_numeric(const uint32_t *perm, const uint32_t *tile_slot0, int64_t len,
                              int64_t ntiles, int tile, const double *sr, double *prS,
                              int64_t nnz, int64_t cap, cudaStream_t s) {
    fsparse_status e = FSPARSE_OK;
    // Writes are bounded by the output capacity (nnz is unknown to the host when
    // the fold is fused into the symbolic call; then the caller passes cap = len).
    const int64_t nnz_bound = cap > 0 ? cap : len;
    if (len > 0) {
        if (tile == 1024) e = run_numeric<128, 8>(perm, tile_slot0, len, ntiles, sr, prS, nnz_bound, s);
        else if (tile == 2048) e = run_numeric<128, 16>(perm, tile_slot0, len, ntiles, sr, prS, nnz_bound, s);
        else if (tile == 4096) e = run_numeric<256, 16>(perm, tile_slot0, len, ntiles, sr, prS, nnz_bound, s);
        else return set_error(FSPARSE_ERR_ARG, "unsupported numeric tile");
        if (e != FSPARSE_OK) return e;
    }
    if (cap > nnz) return launch_fill(nullptr, prS, nnz, cap, s);
    return FSPARSE_OK;
}

__global__ void adjoint_kernel(const int32_t *__restrict__ irank, int64_t len,
                               const double *__restrict__ dprS, double *__restrict__ ds, int vec,
                               int64_t nnz) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t done = 0;
    if (vec) {
        const int64_t n4 = len / 4;
        for (int64_t v = t0; v < n4; v += stride) {
            const int4 r = reinterpret_cast<const int4 *>(irank)[v];
            const double2 a = make_double2(r.x < nnz ? __ldg(dprS + r.x) : 0.0, r.y < nnz ? __ldg(dprS + r.y) : 0.0);
            const double2 b = make_double2(r.z < nnz ? __ldg(dprS + r.z) : 0.0, r.w < nnz ? __ldg(dprS + r.w) : 0.0);
            reinterpret_cast<double2 *>(ds)[2 * v] = a;
            reinterpret_cast<double2 *>(ds)[2 * v + 1] = b;
        }
        done = n4 * 4;
    }
    for (int64_t k = done + t0; k < len; k += stride) {
        const int32_t r = irank[k];
        ds[k] = (r >= 0 && r < nnz) ? __ldg(dprS + r) : 0.0;
    }
}

fsparse_status launch_adjoint(const int32_t *irank, int64_t len, const double *dprS, double *ds,
                              int64_t nnz, cudaStream_t s) {
    if (len == 0) return FSPARSE_OK;
    const int vec = ((reinterpret_cast<uintptr_t>(irank) | reinterpret_cast<uintptr_t>(ds)) & 15) == 0;
    const int64_t work = vec ? (len + 3) / 4 : len;
    const int grid = (int)std::min<int64_t>((work + 255) / 256, (int64_t)sm_count(0) * 8);
    adjoint_kernel<<<std::max(grid, 1), 256, 0, s>>>(irank, len, dprS, ds, vec, nnz);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

__global__ void fill_kernel(int32_t *irS, double *prS, int64_t from, int64_t to) {
    for (int64_t p = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < to;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (irS) irS[p] = 0;
        if (prS) prS[p] = 0.0;
    }
}

fsparse_status launch_fill(int32_t *irS, double *prS, int64_t from, int64_t to, cudaStream_t s) {
    if (to <= from) return FSPARSE_OK;
    const int grid = (int)std::min<int64_t>((to - from + 255) / 256, (int64_t)sm_count(0) * 4);
    fill_kernel<<<std::max(grid, 1), 256, 0, s>>>(irS, prS, from, to);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

__global__ void iota_kernel(uint32_t *perm, int64_t len) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < len;
         p += (int64_t)gridDim.x * blockDim.x)
        perm[p] = (uint32_t)p;
}

fsparse_status launch_iota(uint32_t *perm, int64_t len, cudaStream_t s) {
    if (len == 0) return FSPARSE_OK;
    const int grid = (int)std::min<int64_t>((len + 255) / 256, (int64_t)sm_count(0) * 4);
    iota_kernel<<<std::max(grid, 1), 256, 0, s>>>(perm, len);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

__global__ void batch_concat_kernel(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                    int64_t len, uint32_t offset) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < len;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = src[p];
        dst[p] = ((x & kIndexMask) + offset) | (x & kHeadBit);
    }
}

fsparse_status launch_batch_concat(const uint32_t *src, uint32_t *dst, int64_t len,
                                   uint32_t offset, cudaStream_t s) {
    if (len == 0) return FSPARSE_OK;
    const int grid = (int)std::min<int64_t>((len + 255) / 256, (int64_t)sm_count(0) * 4);
    batch_concat_kernel<<<std::max(grid, 1), 256, 0, s>>>(src, dst, len, offset);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

// Run heads per numeric tile (their exclusive scan is tile_slot0).
__global__ void tile_heads_kernel(const uint32_t *__restrict__ perm, int64_t len, int tile,
                                  uint32_t *counts, int64_t ntiles) {
    const int lane = threadIdx.x & 31;
    const int64_t warp_id = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = warp_id; q < ntiles; q += nwarps) {
        const int64_t p0 = q * tile, p1 = min64(p0 + tile, len);
        uint32_t c = 0;
        for (int64_t p = p0 + lane; p < p1; p += 32) c += (perm[p] >> 31);
#pragma unroll
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) counts[q] = c;
    }
}

fsparse_status launch_tile_heads(const uint32_t *perm, int64_t len, int tile, uint32_t *counts,
                                 int64_t ntiles, cudaStream_t s) {
    if (ntiles == 0) return FSPARSE_OK;
    const int grid = (int)std::min<int64_t>((ntiles * 32 + 255) / 256, (int64_t)sm_count(0) * 8);
    tile_heads_kernel<<<std::max(grid, 1), 256, 0, s>>>(perm, len, tile, counts, ntiles);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

}  // namespace fsp
