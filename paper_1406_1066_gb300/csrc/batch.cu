// batch.cu -- symbolic assembly of many independent instances at once.
//
// Re-assembly of many small patterns per time step is the setting of the
// paper's §1 (nonlinear PDE solvers) and of its "quasi assembly" (§2.1: the
// information kept between assemblies).  fsparse_batch_symbolic assembles
// `count` instances, given as one concatenation of their triplets, in ONE
// symbolic pass: instance b's columns are shifted by col_off[b] = n_0 + ... +
// n_{b-1}, which makes the whole batch the horizontal concatenation
// [S_0 S_1 ... S_{count-1}] of the instances' matrices (rows are left as they
// are; the tallest instance sets the row count).  In column-compressed order
// that matrix keeps every instance's columns, and hence its slots, together:
// instance b owns columns [col_off[b], col_off[b+1]) and slots
// [nnz_off[b], nnz_off[b+1]) with nnz_off[b] = jcS[col_off[b]], and its irS
// entries are its own rows.  The kernels here only translate between the
// per-instance and the concatenated numbering; the sort, runs, slots and
// fold are the single-problem path's.
#include <algorithm>

#include "common.cuh"
#include "internal.hpp"

namespace fsp {

// Instance that owns position x of a concatenation with offsets off[0..count]
// (off ascending, off[0] = 0): the largest b with off[b] <= x.
__device__ __forceinline__ int owner_of(const int64_t *__restrict__ off, int count, int64_t x) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Largest row and column index of every instance (implicit dimensions, §2.2).
__global__ void batch_dims_kernel(const int32_t *__restrict__ ii, const int32_t *__restrict__ jj,
                                  const int64_t *__restrict__ len_off, int count, int64_t total,
                                  int32_t *__restrict__ max_i, int32_t *__restrict__ max_j) {
    const int lane = threadIdx.x & 31;
    for (int64_t k0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~int64_t(31); k0 < total;
         k0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = k0 + lane;
        const bool have = k < total;
        const int b = have ? owner_of(len_off, count, k) : -1;
        int32_t i = have ? ii[k] : 0, j = have ? jj[k] : 0;
        const int b0 = __shfl_sync(0xffffffffu, b, 0);
        if (__all_sync(0xffffffffu, !have || b == b0)) {   // the usual case: one instance per warp
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                i = max(i, __shfl_xor_sync(0xffffffffu, i, o));
                j = max(j, __shfl_xor_sync(0xffffffffu, j, o));
            }
            if (lane == 0 && b0 >= 0) {
                atomicMax(max_i + b0, i);
                atomicMax(max_j + b0, j);
            }
        } else if (have) {
            atomicMax(max_i + b, i);
            atomicMax(max_j + b, j);
        }
    }
}

// Column of every triplet in the concatenated matrix: jj + col_off[b].  An
// index outside instance b's own [1, m_b] x [1, n_b] becomes column 0, which
// the symbolic pass that follows reports as a bad index.
__global__ void batch_remap_kernel(const int32_t *__restrict__ ii, const int32_t *__restrict__ jj,
                                   const int64_t *__restrict__ len_off, const int64_t *__restrict__ col_off,
                                   const int32_t *__restrict__ m, int count, int64_t total,
                                   int32_t *__restrict__ jj_out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int b = owner_of(len_off, count, k);
        const int32_t i = ii[k], j = jj[k];
        const int64_t nb = col_off[b + 1] - col_off[b];
        const bool ok = i >= 1 && i <= m[b] && j >= 1 && (int64_t)j <= nb;
        jj_out[k] = ok ? (int32_t)(col_off[b] + j) : 0;
    }
}

// Slot offset of every instance: nnz_off[b] = jcS[col_off[b]], b = 0..count.
__global__ void batch_nnz_off_kernel(const int32_t *__restrict__ jcS, const int64_t *__restrict__ col_off,
                                     int count, int64_t *__restrict__ nnz_off) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= count; b += gridDim.x * blockDim.x)
        nnz_off[b] = jcS[col_off[b]];
}

// Per-instance column pointers, concatenated: instance b's n_b + 1 entries
// start at col_off[b] + b and count from its own first slot.
__global__ void batch_jcs_kernel(const int32_t *__restrict__ jcS, const int64_t *__restrict__ col_off,
                                 const int64_t *__restrict__ jcs_off, const int64_t *__restrict__ nnz_off,
                                 int count, int64_t total, int32_t *__restrict__ out) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int b = owner_of(jcs_off, count, x);
        const int64_t c = x - jcs_off[b];   // 0..n_b
        out[x] = (int32_t)(jcS[col_off[b] + c] - nnz_off[b]);
    }
}

// Concatenated slots -> instance-local slots, in place.
__global__ void batch_irank_kernel(int32_t *__restrict__ irank, const int64_t *__restrict__ len_off,
                                   const int64_t *__restrict__ nnz_off, int count, int64_t total) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int b = owner_of(len_off, count, k);
        irank[k] = (int32_t)(irank[k] - nnz_off[b]);
    }
}

static int grid_for(int64_t work) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)sm_count(0) * 8));
}

fsparse_status launch_batch_dims(const int32_t *ii, const int32_t *jj, const int64_t *len_off, int count,
                                 int64_t total, int32_t *max_i, int32_t *max_j, cudaStream_t s) {
    if (total == 0) return FSPARSE_OK;
    batch_dims_kernel<<<grid_for(total), 256, 0, s>>>(ii, jj, len_off, count, total, max_i, max_j);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

fsparse_status launch_batch_remap(const int32_t *ii, const int32_t *jj, const int64_t *len_off,
                                  const int64_t *col_off, const int32_t *m, int count, int64_t total,
                                  int32_t *jj_out, cudaStream_t s) {
    if (total == 0) return FSPARSE_OK;
    batch_remap_kernel<<<grid_for(total), 256, 0, s>>>(ii, jj, len_off, col_off, m, count, total, jj_out);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

fsparse_status launch_batch_nnz_off(const int32_t *jcS, const int64_t *col_off, int count, int64_t *nnz_off,
                                    cudaStream_t s) {
    batch_nnz_off_kernel<<<grid_for(count + 1), 256, 0, s>>>(jcS, col_off, count, nnz_off);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

fsparse_status launch_batch_jcs(const int32_t *jcS, const int64_t *col_off, const int64_t *jcs_off,
                                const int64_t *nnz_off, int count, int64_t total, int32_t *out,
                                cudaStream_t s) {
    if (total == 0) return FSPARSE_OK;
    batch_jcs_kernel<<<grid_for(total), 256, 0, s>>>(jcS, col_off, jcs_off, nnz_off, count, total, out);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

fsparse_status launch_batch_irank(int32_t *irank, const int64_t *len_off, const int64_t *nnz_off, int count,
                                  int64_t total, cudaStream_t s) {
    if (total == 0) return FSPARSE_OK;
    batch_irank_kernel<<<grid_for(total), 256, 0, s>>>(irank, len_off, nnz_off, count, total);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

}  // namespace fsp
