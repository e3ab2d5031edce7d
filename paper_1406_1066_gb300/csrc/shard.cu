// shard.cu -- routing for the column-sharded assembly on several GPUs.
//
// The paper's multicore method (§3) splits the rows into one contiguous
// range per thread, so that every thread owns whole rows of the work; §2
// names a distributed output as an extension.  On several GPUs the natural
// unit is a contiguous range of COLUMNS per GPU: a column-compressed matrix
// cut by columns is a set of independent column-compressed blocks, and
// every (i, j) pair, hence every slot, belongs to exactly one block.
//
// Rank r holds an arbitrary slice of the triplets.  fsparse_shard_route
// sends every triplet to the owner of its column: a stable partition of the
// slice by destination rank (ascending triplet number inside every
// destination), with the column made local to the destination's block.
// After an all-to-all exchange (the caller's collective), each rank receives
// its triplets ordered by (source rank, source position) -- which is the
// global triplet order when the slices are taken in rank order -- so its
// local assembly sums every slot in ascending global k, as the serial
// insert of App. A does.  fsparse_shard_unroute brings the slots back to
// the source positions (irank of the source slice); fsparse_shard_gather
// routes new values along a kept route for numeric re-assembly.
//
// Three kernels: a per-tile destination histogram (destination-major, so one
// exclusive scan gives every (destination, tile) its output offset), the
// scan, and a scatter that ranks each tile's items per destination with the
// stable warp ranking of rank.cuh.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.hpp"
#include "rank.cuh"

namespace fsp {

constexpr int kShardThreads = 256;
constexpr int kShardItems = 8;
constexpr int kShardTile = kShardThreads * kShardItems;
constexpr int kShardRadixBits = 8;   // destination ranks < 256

// Destination of column j (unit offset): the rank r with col_lo[r] < j <= col_lo[r+1].
__device__ __forceinline__ int shard_dest(const int64_t *s_split, int nranks, int32_t j) {
    int lo = 0, hi = nranks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_split[mid] < j) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kShardThreads)
    shard_hist_kernel(const int32_t *__restrict__ ii, const int32_t *__restrict__ jj, int64_t len, int32_t m,
                      int32_t n, const int64_t *__restrict__ split, int nranks, int64_t ntiles,
                      uint32_t *__restrict__ hist, DevStatus *st) {
    __shared__ int64_t s_split[257];
    __shared__ uint32_t s_cnt[256];
    for (int r = threadIdx.x; r <= nranks; r += blockDim.x) s_split[r] = split[r];
    for (int r = threadIdx.x; r < nranks; r += blockDim.x) s_cnt[r] = 0;
    __syncthreads();
    const int64_t t = blockIdx.x;
    const int64_t base = t * kShardTile;
    for (int x = threadIdx.x; x < kShardTile; x += blockDim.x) {
        const int64_t k = base + x;
        if (k >= len) break;
        checked_index(ii[k], m, st);
        atomicAdd(&s_cnt[shard_dest(s_split, nranks, checked_index(jj[k], n, st))], 1u);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nranks; r += blockDim.x) hist[(int64_t)r * ntiles + t] = s_cnt[r];
}

__global__ void __launch_bounds__(kShardThreads)
    shard_scatter_kernel(const int32_t *__restrict__ ii, const int32_t *__restrict__ jj,
                         const double *__restrict__ sr, int64_t len, int32_t m, int32_t n,
                         const int64_t *__restrict__ split, int nranks, int64_t ntiles,
                         const uint32_t *__restrict__ offs, int32_t *__restrict__ out_i,
                         int32_t *__restrict__ out_j, double *__restrict__ out_s, int32_t *__restrict__ out_k,
                         DevStatus *st) {
    constexpr int RADIX = 1 << kShardRadixBits, WARPS = kShardThreads / 32;
    __shared__ int64_t s_split[RADIX + 1];
    __shared__ uint32_t s_wcnt[WARPS * RADIX];
    __shared__ uint32_t s_wm[WARPS * RADIX];
    __shared__ uint32_t s_local[RADIX];
    __shared__ uint32_t s_scan[WARPS + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int r = tid; r <= nranks; r += kShardThreads) s_split[r] = split[r];
    for (int x = tid; x < WARPS * RADIX; x += kShardThreads) {
        s_wcnt[x] = 0;
        s_wm[x] = 0;
    }
    __syncthreads();
    const int64_t t = blockIdx.x;
    // warp-striped items: visiting (warp, item, lane) in order visits k in order
    const int64_t wbase = t * kShardTile + (int64_t)warp * 32 * kShardItems + lane;
    uint32_t dig[kShardItems], rnk[kShardItems];
    bool valid[kShardItems];
    int32_t iv[kShardItems], jv[kShardItems];
#pragma unroll
    for (int x = 0; x < kShardItems; ++x) {
        const int64_t k = wbase + x * 32;
        valid[x] = k < len;
        iv[x] = valid[x] ? checked_index(ii[k], m, st) : 1;
        jv[x] = valid[x] ? checked_index(jj[k], n, st) : 1;
        dig[x] = valid[x] ? (uint32_t)shard_dest(s_split, nranks, jv[x]) : 0u;
    }
    warp_rank<kShardRadixBits, kShardItems>(dig, valid, s_wcnt + warp * RADIX, s_wm + warp * RADIX, rnk);
    __syncthreads();
    digit_offsets<kShardRadixBits, kShardThreads>(s_wcnt, s_local, s_scan);
    // s_wcnt now holds, per (warp, destination), the items of earlier warps
#pragma unroll
    for (int x = 0; x < kShardItems; ++x) {
        if (!valid[x]) continue;
        const uint32_t d = dig[x];
        const int64_t pos = (int64_t)offs[(int64_t)d * ntiles + t] + s_wcnt[warp * RADIX + d] + rnk[x];
        if (!in_range(pos, len, st)) continue;
        const int64_t k = wbase + x * 32;
        out_i[pos] = iv[x];
        out_j[pos] = (int32_t)(jv[x] - s_split[d]);   // column inside the destination's block
        if (out_s) out_s[pos] = sr[k];
        out_k[pos] = (int32_t)k;
    }
}

// Start of every destination's segment: starts[r] = offs[r * ntiles] (r < nranks), starts[nranks] = len.
__global__ void shard_starts_kernel(const uint32_t *__restrict__ offs, int64_t ntiles, int nranks,
                                    int64_t len, uint32_t *__restrict__ starts) {
    for (int r = threadIdx.x; r <= nranks; r += blockDim.x)
        starts[r] = r < nranks ? offs[(int64_t)r * ntiles] : (uint32_t)len;
}

__global__ void shard_unroute_kernel(const int32_t *__restrict__ back, const int32_t *__restrict__ send_k,
                                     int64_t len, int32_t *__restrict__ out, DevStatus *st) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < len; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = send_k[p];
        if (k >= 0 && k < len) out[k] = back[p];
        else if (st) atomicOr(&st->oob, 1u);
    }
}

__global__ void shard_gather_kernel(const double *__restrict__ sr, const int32_t *__restrict__ send_k, int64_t len,
                                    double *__restrict__ out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < len; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = send_k[p];
        out[p] = (k >= 0 && k < len) ? __ldg(sr + k) : 0.0;
    }
}

__global__ void shard_offset_kernel(const int32_t *__restrict__ in, int64_t len, int64_t add,
                                    int32_t *__restrict__ out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < len; p += (int64_t)gridDim.x * blockDim.x)
        out[p] = (int32_t)(in[p] + add);
}

static int shard_grid(int64_t work) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)sm_count(0) * 8));
}

}  // namespace fsp

using namespace fsp;

extern "C" {

fsparse_status fsparse_shard_route(const int32_t *ii, const int32_t *jj, const double *sr, int64_t len,
                                   int32_t m, int32_t n, int32_t nranks, const int64_t *h_col_split,
                                   int32_t *send_i, int32_t *send_j, double *send_s, int32_t *send_k,
                                   int64_t *h_counts, void *stream) {
    NvtxRange nvtx_("fsparse_shard_route");
    if (!h_col_split || !h_counts) return set_error(FSPARSE_ERR_ARG, "NULL host array");
    if (nranks < 1 || nranks > 256) return set_error(FSPARSE_ERR_ARG, "nranks must be in 1..256");
    if (len < 0 || m <= 0 || n <= 0) return set_error(FSPARSE_ERR_ARG, "needs len >= 0 and explicit m, n > 0");
    if (len > kMaxLookbackValue) return set_error(FSPARSE_ERR_SIZE, "len above 2^30 - 1");
    if (h_col_split[0] != 0 || h_col_split[nranks] != n)
        return set_error(FSPARSE_ERR_ARG, "column split must run from 0 to n");
    for (int r = 0; r < nranks; ++r)
        if (h_col_split[r + 1] < h_col_split[r]) return set_error(FSPARSE_ERR_ARG, "column split decreases");
    if (len > 0 && (!ii || !jj || !send_i || !send_j || !send_k || (sr && !send_s)))
        return set_error(FSPARSE_ERR_ARG, "NULL device array");
    for (int r = 0; r < nranks; ++r) h_counts[r] = 0;
    if (len == 0) return FSPARSE_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    FSP_CUDA(cudaGetDevice(&dev));
    Scratch scratch(s);
    const int64_t ntiles = (len + kShardTile - 1) / kShardTile;
    int64_t *d_split = nullptr;
    uint32_t *hist = nullptr, *offs = nullptr, *starts = nullptr;
    DevStatus *d_st = nullptr;
    fsparse_status e;
    if ((e = scratch.get(&d_split, (size_t)nranks + 1)) || (e = scratch.get(&hist, (size_t)nranks * ntiles)) ||
        (e = scratch.get(&offs, (size_t)nranks * ntiles + 1)) || (e = scratch.get(&starts, (size_t)nranks + 1)) ||
        (e = scratch.get(&d_st, 1)))
        return e;
    FSP_CUDA(cudaMemsetAsync(d_st, 0, sizeof(DevStatus), s));
    FSP_CUDA(cudaMemcpyAsync(d_split, h_col_split, ((size_t)nranks + 1) * 8, cudaMemcpyHostToDevice, s));
    shard_hist_kernel<<<(unsigned)ntiles, kShardThreads, 0, s>>>(ii, jj, len, m, n, d_split, nranks, ntiles, hist,
                                                                  d_st);
    FSP_LAUNCHED();
    if ((e = exclusive_scan_u32(hist, offs, (int64_t)nranks * ntiles, d_st, scratch, s)) != FSPARSE_OK) return e;
    shard_scatter_kernel<<<(unsigned)ntiles, kShardThreads, 0, s>>>(ii, jj, sr, len, m, n, d_split, nranks, ntiles,
                                                                     offs, send_i, send_j, sr ? send_s : nullptr,
                                                                     send_k, d_st);
    FSP_LAUNCHED();
    shard_starts_kernel<<<1, 256, 0, s>>>(offs, ntiles, nranks, len, starts);
    FSP_LAUNCHED();
    std::vector<uint32_t> h_starts((size_t)nranks + 1);
    DevStatus h_st{};
    FSP_CUDA(cudaMemcpyAsync(h_starts.data(), starts, ((size_t)nranks + 1) * 4, cudaMemcpyDeviceToHost, s));
    FSP_CUDA(cudaMemcpyAsync(&h_st, d_st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    FSP_CUDA(cudaStreamSynchronize(s));
    if (h_st.bad_index) return set_error(FSPARSE_ERR_INDEX, "index below 1 or above its dimension");
    if (h_st.timeout) return set_error(FSPARSE_ERR_TIMEOUT, "device look-back wait expired");
    if (h_st.oob) return set_error(FSPARSE_ERR_INTERNAL, "internal index check failed");
    for (int r = 0; r < nranks; ++r) h_counts[r] = (int64_t)h_starts[r + 1] - (int64_t)h_starts[r];
    return FSPARSE_OK;
}

fsparse_status fsparse_shard_unroute(const int32_t *back, const int32_t *send_k, int64_t len, int32_t *out,
                                     void *stream) {
    if (len < 0) return set_error(FSPARSE_ERR_ARG, "len < 0");
    if (len == 0) return FSPARSE_OK;
    if (!back || !send_k || !out) return set_error(FSPARSE_ERR_ARG, "NULL device array");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    shard_unroute_kernel<<<shard_grid(len), 256, 0, s>>>(back, send_k, len, out, nullptr);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

fsparse_status fsparse_shard_gather(const double *sr, const int32_t *send_k, int64_t len, double *send_s,
                                    void *stream) {
    if (len < 0) return set_error(FSPARSE_ERR_ARG, "len < 0");
    if (len == 0) return FSPARSE_OK;
    if (!sr || !send_k || !send_s) return set_error(FSPARSE_ERR_ARG, "NULL device array");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    shard_gather_kernel<<<shard_grid(len), 256, 0, s>>>(sr, send_k, len, send_s);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

fsparse_status fsparse_shard_offset(const int32_t *in, int64_t len, int64_t add, int32_t *out, void *stream) {
    if (len < 0) return set_error(FSPARSE_ERR_ARG, "len < 0");
    if (len == 0) return FSPARSE_OK;
    if (!in || !out) return set_error(FSPARSE_ERR_ARG, "NULL device array");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    shard_offset_kernel<<<shard_grid(len), 256, 0, s>>>(in, len, add, out);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

}  // extern "C"
