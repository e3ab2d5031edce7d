// numeric.cu -- the value side of the assembly.
//
// Numeric fold (Eq. (2.3) with the App. A insert order): the plan stores the
// sorted order perm[p] = k, with kHeadBit on the first triplet of every run
// (one run per CCS slot), and tile_slot0[q] = number of runs that start
// before numeric tile q.  A block takes a tile of NT positions, stages the
// perm entries and the gathered values sr[k] in shared memory (plus a halo
// for the run that crosses the tile end), lists the run heads in position
// order with warp ballots, and lets ONE thread fold each run from +0.0 in
// ascending position order -- which is ascending k, the paper's order --
// so the result is identical to the serial insert, bit for bit, for any
// launch shape.  No atomics touch values.
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

template <int NT, int THREADS>
struct NumericSmem {
    static constexpr int HALO = 64;
    static constexpr int ROWS = NT / THREADS, WARPS = THREADS / 32;
    static constexpr size_t bytes =
        (size_t)(NT + HALO) * 8 + (size_t)(NT + HALO) * 4 + (size_t)NT * 2 + (ROWS * WARPS + 4) * 4;
};

template <int NT, int THREADS>
__global__ void __launch_bounds__(THREADS)
    numeric_kernel(const uint32_t *__restrict__ perm, const double *__restrict__ sr,
                   const uint32_t *__restrict__ tile_slot0, double *__restrict__ prS, int64_t len,
                   int64_t ntiles, int64_t nnz) {
    using S = NumericSmem<NT, THREADS>;
    constexpr int HALO = S::HALO, ROWS = S::ROWS, WARPS = S::WARPS;
    extern __shared__ __align__(16) unsigned char smem[];
    double *s_val = reinterpret_cast<double *>(smem);
    uint32_t *s_perm = reinterpret_cast<uint32_t *>(s_val + NT + HALO);
    uint16_t *s_head = reinterpret_cast<uint16_t *>(s_perm + NT + HALO);
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(s_head + NT);   // [ROWS*WARPS] + nheads + halo_end
    uint32_t *s_misc = s_cnt + ROWS * WARPS;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(perm) & 15) == 0;
    for (int64_t q = blockIdx.x; q < ntiles; q += gridDim.x) {
        const int64_t P0 = q * NT;
        const int cnt = (int)min64(NT, len - P0);
        const int ext = (int)min64(HALO, len - P0 - cnt);
        if (cnt == NT && vec) {
            for (int v = tid; v < NT / 4; v += THREADS)
                reinterpret_cast<uint4 *>(s_perm)[v] = reinterpret_cast<const uint4 *>(perm + P0)[v];
        } else {
            for (int j = tid; j < cnt; j += THREADS) s_perm[j] = perm[P0 + j];
        }
        for (int j = tid; j < ext; j += THREADS) s_perm[cnt + j] = perm[P0 + cnt + j];
        __syncthreads();

        // Gather the tile's values; warp 0 also finds where the halo's first run starts.
#pragma unroll 4
        for (int j = tid; j < cnt; j += THREADS) s_val[j] = gather(sr, s_perm[j], len);
        if (warp == 0) {
            int end = ext;
            for (int b = 0; b < ext; b += 32) {
                const bool h = b + lane < ext && (s_perm[cnt + b + lane] & kHeadBit);
                const uint32_t m = __ballot_sync(0xffffffffu, h);
                if (m) {
                    end = b + __ffs(m) - 1;
                    break;
                }
            }
            if (lane == 0) s_misc[1] = (uint32_t)end;
        }
        // Run heads in position order: row r covers positions r*THREADS + tid.
        uint32_t hm[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int j = r * THREADS + tid;
            hm[r] = __ballot_sync(0xffffffffu, j < cnt && (s_perm[j] & kHeadBit));
            if (lane == 0) s_cnt[r * WARPS + warp] = __popc(hm[r]);
        }
        __syncthreads();
        const int halo_end = (int)s_misc[1];
        for (int j = tid; j < halo_end; j += THREADS)
            s_val[cnt + j] = gather(sr, s_perm[cnt + j], len);
        if (warp == 0) {
            uint32_t carry = 0;
            for (int b = 0; b < ROWS * WARPS; b += 32) {
                const uint32_t x = b + lane < ROWS * WARPS ? s_cnt[b + lane] : 0u;
                uint32_t inc = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += y;
                }
                if (b + lane < ROWS * WARPS) s_cnt[b + lane] = carry + inc - x;
                carry += __shfl_sync(0xffffffffu, inc, 31);
            }
            if (lane == 0) s_misc[0] = carry;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < ROWS; ++r)
            if ((hm[r] >> lane) & 1u)
                s_head[s_cnt[r * WARPS + warp] + __popc(hm[r] & lanemask_lt())] =
                    (uint16_t)(r * THREADS + tid);
        __syncthreads();

        const int nh = (int)s_misc[0];
        const int64_t base = tile_slot0[q];
        for (int h = tid; h < nh; h += THREADS) {
            const int start = s_head[h];
            const bool last = h + 1 == nh;
            const int end = last ? cnt + halo_end : s_head[h + 1];
            double acc = 0.0;   // +0.0: the insert adds into zeroed storage
            for (int p = start; p < end; ++p) acc += s_val[p];
            if (last && halo_end == ext) {
                // A run longer than the halo: continue through global memory,
                // eight triplets at a time, still in ascending order.
                int64_t g = P0 + cnt + ext;
                while (g < len) {
                    uint32_t x[8];
                    int c = 0;
#pragma unroll
                    for (int u = 0; u < 8; ++u) x[u] = g + u < len ? perm[g + u] : kHeadBit;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (c == u && !(x[u] & kHeadBit)) ++c;
                    }
                    double v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = u < c ? gather(sr, x[u], len) : 0.0;
                    for (int u = 0; u < c; ++u) acc += v[u];
                    if (c < 8) break;
                    g += 8;
                }
            }
            if (base + h < nnz) prS[base + h] = acc;
        }
        __syncthreads();
    }
}

template <int NT, int THREADS>
static fsparse_status run_numeric(const uint32_t *perm, const uint32_t *tile_slot0, int64_t len,
                                  int64_t ntiles, const double *sr, double *prS, int64_t nnz,
                                  cudaStream_t s) {
    using S = NumericSmem<NT, THREADS>;
    auto kern = numeric_kernel<NT, THREADS>;
    FSP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes));
    int per_sm = 0;
    FSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, S::bytes));
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sm_count(0) * std::max(per_sm, 1));
    kern<<<(unsigned)grid, THREADS, S::bytes, s>>>(perm, sr, tile_slot0, prS, len, ntiles, nnz);
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
        if (tile == 1024) e = run_numeric<1024, 256>(perm, tile_slot0, len, ntiles, sr, prS, nnz_bound, s);
        else if (tile == 2048) e = run_numeric<2048, 256>(perm, tile_slot0, len, ntiles, sr, prS, nnz_bound, s);
        else if (tile == 4096) e = run_numeric<4096, 256>(perm, tile_slot0, len, ntiles, sr, prS, nnz_bound, s);
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
