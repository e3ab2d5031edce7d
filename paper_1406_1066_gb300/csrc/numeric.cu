// numeric.cu -- the value side of the assembly.
//
// Numeric fold (Eq. (2.3) with the App. A insert order): the plan stores the
// sorted order perm[p] = k, with kHeadBit on the first triplet of every run
// (one run per CCS slot), and chunk_slot0[q] = number of runs that start
// before position q*kChunk.  ONE thread folds each run from +0.0 in ascending
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

// Chunked fold.  Positions are cut into chunks of kChunk = 16; the plan keeps,
// per chunk, the number of runs that start before it (chunk_slot0), so every
// chunk is processed by one thread with no communication at all:
//   * 128-bit loads of the chunk's perm entries;
//   * positions before the chunk's first run head belong to a run that an
//     earlier thread owns: skipped;
//   * every run that starts in the chunk is folded in registers from +0.0 in
//     ascending position order (= ascending k);
//   * the chunk's last run continues past the chunk: the thread keeps reading
//     perm (eight entries at a time, L1-resident since the neighbouring thread
//     loaded them) and gathering values until the next run head.
// Every value is gathered exactly once; no shared memory, no barriers.
template <int THREADS>
__global__ void __launch_bounds__(THREADS)
    numeric_kernel(const uint32_t *__restrict__ perm, const double *__restrict__ sr,
                   const uint32_t *__restrict__ chunk_slot0, double *__restrict__ prS, int64_t len,
                   int64_t nchunks, int64_t nnz) {
    constexpr int C = kChunk;
    const bool vec = (reinterpret_cast<uintptr_t>(perm) & 15) == 0;
    for (int64_t q = blockIdx.x * (int64_t)THREADS + threadIdx.x; q < nchunks;
         q += (int64_t)gridDim.x * THREADS) {
        const int64_t p0 = q * C;
        const int nval = (int)min64(C, len - p0);
        uint32_t pm[C];
        if (nval == C && vec) {
#pragma unroll
            for (int v = 0; v < C / 4; ++v) {
                const uint4 x = __ldg(reinterpret_cast<const uint4 *>(perm + p0) + v);
                pm[4 * v] = x.x;
                pm[4 * v + 1] = x.y;
                pm[4 * v + 2] = x.z;
                pm[4 * v + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < C; ++i) pm[i] = i < nval ? __ldg(perm + p0 + i) : 0u;
        }
        uint32_t hmask = 0;
#pragma unroll
        for (int i = 0; i < C; ++i)
            if (i < nval && (pm[i] & kHeadBit)) hmask |= 1u << i;
        if (hmask == 0) continue;   // the whole chunk lies inside an earlier thread's run
        const int lead = __ffs(hmask) - 1;
        int64_t slot = __ldg(chunk_slot0 + q);
        double v[C];
#pragma unroll
        for (int i = 0; i < C; ++i) v[i] = (i >= lead && i < nval) ? gather(sr, pm[i], len) : 0.0;
        // Each run: (((+0.0 + v0) + v1) + ...), the first add done as plus_zero.
        double acc = 0.0;
        bool open = false;
#pragma unroll
        for (int i = 0; i < C; ++i) {
            if ((hmask >> i) & 1u) {
                if (open && slot < nnz) prS[slot] = acc;
                slot += open;
                acc = plus_zero(v[i]);
                open = true;
            } else if (open && i < nval) {
                acc += v[i];
            }
        }
        // Continue the last run past the chunk, in order, until the next head.
        int64_t g = p0 + C;
        while (nval == C && g < len) {
            uint32_t x[8];
            if (g + 8 <= len && vec) {   // g is a multiple of 8: two aligned 16-byte loads
                const uint4 a0 = __ldg(reinterpret_cast<const uint4 *>(perm + g));
                const uint4 a1 = __ldg(reinterpret_cast<const uint4 *>(perm + g) + 1);
                x[0] = a0.x; x[1] = a0.y; x[2] = a0.z; x[3] = a0.w;
                x[4] = a1.x; x[5] = a1.y; x[6] = a1.z; x[7] = a1.w;
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) x[u] = g + u < len ? __ldg(perm + g + u) : kHeadBit;
            }
            int c = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (c == u && !(x[u] & kHeadBit)) ++c;
            double w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) w[u] = u < c ? gather(sr, x[u], len) : 0.0;
            // A warp-wide FP64 add costs the same issue time on GB300 however
            // few lanes take part, so the adds stop at the largest count of
            // the lanes still here (after the first batch usually one or two).
            const int cmax = __reduce_max_sync(__activemask(), c);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (u >= cmax) break;
                if (u < c) acc += w[u];
            }
            if (c < 8) break;
            g += 8;
        }
        if (slot < nnz) prS[slot] = acc;
    }
}

template <int THREADS>
static fsparse_status run_numeric(const uint32_t *perm, const uint32_t *chunk_slot0, int64_t len,
                                  const double *sr, double *prS, int64_t nnz, cudaStream_t s) {
    auto kern = numeric_kernel<THREADS>;
    const int64_t nchunks = (len + kChunk - 1) / kChunk;
    int per_sm = 0;
    FSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, 0));
    const int64_t blocks = (nchunks + THREADS - 1) / THREADS;
    const int64_t grid = std::min<int64_t>(blocks, (int64_t)sm_count(0) * std::max(per_sm, 1) * 16);
    kern<<<(unsigned)grid, THREADS, 0, s>>>(perm, sr, chunk_slot0, prS, len, nchunks, nnz);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

fsparse_status launch_numeric(const uint32_t *perm, const uint32_t *chunk_slot0, int64_t len,
                              int block_positions, const double *sr, double *prS, int64_t nnz,
                              int64_t cap, cudaStream_t s) {
    fsparse_status e = FSPARSE_OK;
    // Writes are bounded by the output capacity (nnz is unknown to the host when
    // the fold is fused into the symbolic call; then the caller passes cap = len).
    const int64_t nnz_bound = cap > 0 ? cap : len;
    if (len > 0) {
        if (block_positions == 1024) e = run_numeric<64>(perm, chunk_slot0, len, sr, prS, nnz_bound, s);
        else if (block_positions == 2048) e = run_numeric<128>(perm, chunk_slot0, len, sr, prS, nnz_bound, s);
        else if (block_positions == 4096) e = run_numeric<256>(perm, chunk_slot0, len, sr, prS, nnz_bound, s);
        else return set_error(FSPARSE_ERR_ARG, "unsupported numeric block size");
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
    // Four 256-thread blocks per SM (half the resident threads): on the 100^3
    // cube 0.206 ms against 0.261 at eight, 0.225 at three and 0.219 at six;
    // with more threads the gathers from dprS ran slower, not faster.
    const int grid = (int)std::min<int64_t>((work + 255) / 256, (int64_t)sm_count(0) * 4);
    adjoint_kernel<<<std::max(grid, 1), 256, 0, s>>>(irank, len, dprS, ds, vec, nnz);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

// irank from the sorted order: irank[perm[p]] = slot of position p, where the
// slot of p is the number of run heads at positions <= p, minus one.  One
// thread per kChunk positions, starting from the chunk's slot base.
__global__ void irank_kernel(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ chunk_slot0,
                             int64_t len, int32_t *__restrict__ irank) {
    const int64_t nchunks = (len + kChunk - 1) / kChunk;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nchunks;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p0 = q * kChunk;
        uint32_t slot = chunk_slot0[q] - 1;
        const int nval = (int)min64(kChunk, len - p0);
        for (int i = 0; i < nval; ++i) {
            const uint32_t x = perm[p0 + i];
            slot += x >> 31;
            const uint32_t k = x & kIndexMask;
            if (k < len) irank[k] = (int32_t)slot;
        }
    }
}

fsparse_status launch_irank(const uint32_t *perm, const uint32_t *chunk_slot0, int64_t len,
                            int32_t *irank, cudaStream_t s) {
    if (len == 0) return FSPARSE_OK;
    const int64_t nchunks = (len + kChunk - 1) / kChunk;
    const int grid = (int)std::min<int64_t>((nchunks + 255) / 256, (int64_t)sm_count(0) * 16);
    irank_kernel<<<std::max(grid, 1), 256, 0, s>>>(perm, chunk_slot0, len, irank);
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

// App. A pre-processing of Matlab's double index arrays: a value below 1.0,
// not an integer (NaN included), or above 2^31 - 1 -- the reading for values
// the paper's int cannot hold -- becomes 0, which the symbolic pass then
// reports as a bad index; every other value becomes its int.
__device__ __forceinline__ int32_t getix_one(double x) {
    if (!(x >= 1.0 && x <= 2147483647.0)) return 0;
    const int32_t v = (int32_t)x;   // truncation: exact for integral x in range
    return (double)v == x ? v : 0;
}

__global__ void getix_kernel(const double *__restrict__ ival, int64_t len, int32_t *__restrict__ out,
                             int vec) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t done = 0;
    if (vec) {
        const int64_t n2 = len / 2;
        for (int64_t v = t0; v < n2; v += stride) {
            const double2 x = reinterpret_cast<const double2 *>(ival)[v];
            reinterpret_cast<int2 *>(out)[v] = make_int2(getix_one(x.x), getix_one(x.y));
        }
        done = n2 * 2;
    }
    for (int64_t k = done + t0; k < len; k += stride) out[k] = getix_one(ival[k]);
}

fsparse_status launch_getix(const double *ival, int64_t len, int32_t *out, cudaStream_t s) {
    if (len <= 0) return FSPARSE_OK;
    const int vec = ((reinterpret_cast<uintptr_t>(ival) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    const int64_t work = vec ? (len + 1) / 2 : len;
    const int grid = (int)std::min<int64_t>((work + 255) / 256, (int64_t)sm_count(0) * 8);
    getix_kernel<<<std::max(grid, 1), 256, 0, s>>>(ival, len, out, vec);
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

// Run heads per chunk of kChunk positions (their exclusive scan is chunk_slot0).
__global__ void chunk_heads_kernel(const uint32_t *__restrict__ perm, int64_t len,
                                   uint32_t *__restrict__ counts, int64_t nchunks) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nchunks;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p0 = q * kChunk, p1 = min64(p0 + kChunk, len);
        uint32_t c = 0;
        for (int64_t p = p0; p < p1; ++p) c += perm[p] >> 31;
        counts[q] = c;
    }
}

fsparse_status launch_chunk_heads(const uint32_t *perm, int64_t len, uint32_t *counts,
                                  int64_t nchunks, cudaStream_t s) {
    if (nchunks == 0) return FSPARSE_OK;
    const int grid = (int)std::min<int64_t>((nchunks + 255) / 256, (int64_t)sm_count(0) * 8);
    chunk_heads_kernel<<<std::max(grid, 1), 256, 0, s>>>(perm, len, counts, nchunks);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

}  // namespace fsp
