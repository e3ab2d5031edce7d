// append.cu -- delayed assembly: merge a plan with the plan of new triplets.
//
// The paper notes (§2, before §2.1's problem statement closes) that its
// counting scheme extends to input that is not all available at the first
// call.  Here the result of appending triplets (ii2, jj2) to a plan of
// (ii1, jj1) is defined as the assembly of the concatenation, with the new
// triplet numbers continuing at len1.  Both plans are already sorted by
// (column, row) with runs in ascending k, so the new plan is a merge:
//
//   * slot keys: key(s) = column << 32 | row for every CCS slot of each plan;
//   * ranks by a merge path over the two sorted key lists: for every slot of
//     one plan, the number of keys of the other plan below it and whether the
//     other plan holds the same key;
//   * merged slot of an old slot a = a + (new keys below it) - (shared keys
//     before it); of a new slot b = b + (old keys below it) - (shared keys
//     before it); a shared key is one slot;
//   * positions: an old run moves right by the number of new triplets with a
//     smaller key; a new run moves right by the number of old triplets with a
//     key not above its own, so inside a shared slot the old triplets (smaller
//     k) come first and the run stays in ascending k;
//   * jcS of the merge: old + new column starts minus the shared keys in
//     earlier columns.
#include <algorithm>

#include "common.cuh"
#include "internal.hpp"

namespace fsp {

// First position of every run: rs[slot] = p at run heads, rs[nnz] = len.
__global__ void run_starts_kernel(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ chunk_slot0,
                                  int64_t len, int64_t nchunks, uint32_t *__restrict__ rs) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nchunks;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p0 = q * kChunk, p1 = min64(p0 + kChunk, len);
        uint32_t slot = chunk_slot0[q];   // runs before the chunk = index of the next run
        for (int64_t p = p0; p < p1; ++p)
            if (perm[p] & kHeadBit) rs[slot++] = (uint32_t)p;
        if (q == nchunks - 1) rs[chunk_slot0[nchunks]] = (uint32_t)len;
    }
}

// key(s) = column << 32 | row, one thread per column writing its slots.
__global__ void slot_keys_kernel(const int32_t *__restrict__ jcS, int32_t n, const int32_t *__restrict__ irS,
                                 uint64_t *__restrict__ keys) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s0 = jcS[c], s1 = jcS[c + 1];
        for (int32_t s = s0; s < s1; ++s) keys[s] = ((uint64_t)(uint32_t)c << 32) | (uint32_t)irS[s];
    }
}

// Merge path over the two sorted key lists (old keys first on ties): thread t
// finds where merged position 8t falls by one binary search, then merges 8
// steps.  An old key met at merged position i + j (i old, j new before it)
// has lbA = j new keys below it; a new key has i old keys not above it, eqB
// telling whether the last of them is equal, and lbB = i - eqB.
constexpr int kMergeSteps = 8;

__global__ void merge_path_kernel(const uint64_t *__restrict__ a, int64_t na, const uint64_t *__restrict__ b,
                                  int64_t nb, uint32_t *__restrict__ lbA, uint32_t *__restrict__ eqA,
                                  uint32_t *__restrict__ lbB, uint32_t *__restrict__ eqB) {
    const int64_t total = na + nb;
    const int64_t nthreads = (total + kMergeSteps - 1) / kMergeSteps;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nthreads;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = t * kMergeSteps;
        int64_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
        while (lo < hi) {   // i = old keys among the first d merged
            const int64_t mid = (lo + hi) >> 1;
            if (a[mid] <= b[d - mid - 1]) lo = mid + 1; else hi = mid;
        }
        int64_t i = lo, j = d - lo;
        const int64_t end = min64(d + kMergeSteps, total);
        for (int64_t step = d; step < end; ++step) {
            if (j >= nb || (i < na && a[i] <= b[j])) {
                lbA[i] = (uint32_t)j;
                eqA[i] = (j < nb && b[j] == a[i]) ? 1u : 0u;
                ++i;
            } else {
                const uint32_t e = (i > 0 && a[i - 1] == b[j]) ? 1u : 0u;
                lbB[j] = (uint32_t)(i - e);
                eqB[j] = e;
                ++j;
            }
        }
    }
}

// irS of the merged plan from one side: slot i goes to i + lb[i] - shared[i].
__global__ void merge_irs_kernel(const int32_t *__restrict__ irS, int64_t nnz, const uint32_t *__restrict__ lb,
                                 const uint32_t *__restrict__ shared, int32_t *__restrict__ out,
                                 int64_t cap_out, DevStatus *st) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i + (int64_t)lb[i] - (int64_t)shared[i];
        if (in_range(t, cap_out, st)) out[t] = irS[i];
    }
}

// jcS of the merge: old + new column starts minus shared keys in earlier columns.
__global__ void merge_jcs_kernel(const int32_t *__restrict__ jc1, const int32_t *__restrict__ jc2,
                                 const uint32_t *__restrict__ shared1, int32_t n, int32_t *__restrict__ out) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= n;
         c += (int64_t)gridDim.x * blockDim.x)
        out[c] = (int32_t)((int64_t)jc1[c] + jc2[c] - shared1[jc1[c]]);
}

// Positions of one side's runs in the merged order.  For the old side
// (second_side = 0) a run moves by other_rs[lb]: the new triplets with a
// smaller key.  For the new side it moves by other_rs[lb + eq]: the old
// triplets with a key not above its own; its head bit is dropped when the old
// side holds the same key (the old run starts that slot).
__global__ void merge_positions_kernel(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ chunk_slot0,
                                       int64_t len, int64_t nchunks, const uint32_t *__restrict__ lb,
                                       const uint32_t *__restrict__ eq, const uint32_t *__restrict__ other_rs,
                                       int second_side, uint32_t kofs, uint32_t *__restrict__ out,
                                       int64_t len_out, DevStatus *st) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nchunks;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p0 = q * kChunk, p1 = min64(p0 + kChunk, len);
        int64_t slot = (int64_t)chunk_slot0[q] - 1;   // run of the position before the chunk
        for (int64_t p = p0; p < p1; ++p) {
            const uint32_t x = perm[p];
            bool head = (x & kHeadBit) != 0;
            slot += head;
            const uint32_t e = second_side ? eq[slot] : 0u;
            const int64_t t = p + other_rs[lb[slot] + e];
            if (second_side && e) head = false;
            if (in_range(t, len_out, st)) out[t] = ((x & kIndexMask) + kofs) | (head ? kHeadBit : 0u);
        }
    }
}

// nnz of the merge (shared keys counted once), for the host's status read.
__global__ void merged_nnz_kernel(int64_t na, int64_t nb, const uint32_t *shared_total, DevStatus *st) {
    st->nnz = (uint32_t)(na + nb - *shared_total);
}

static int grid_for(int64_t work) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)sm_count(0) * 8));
}

// Merge plan a (old triplets) and plan b (new triplets, numbered from a.len)
// into out, whose perm [a.len + b.len], irS [>= a.nnz + b.nnz], jcS [n + 1]
// and chunk_slot0 are allocated by the caller.  st->nnz receives the merged
// nnz; index checks that fail set st->oob.  No synchronisation.
fsparse_status append_merge(const Plan &a, const Plan &b, Plan &out, DevStatus *st, Scratch &scratch,
                            cudaStream_t s) {
    const int64_t na = a.nnz, nb = b.nnz;
    uint32_t *rsA, *rsB, *lbA, *eqA, *lbB, *eqB, *shA, *shB;
    uint64_t *keyA, *keyB;
    fsparse_status e;
    if ((e = scratch.get(&rsA, (size_t)na + 1)) || (e = scratch.get(&rsB, (size_t)nb + 1)) ||
        (e = scratch.get(&keyA, (size_t)std::max<int64_t>(na, 1))) ||
        (e = scratch.get(&keyB, (size_t)std::max<int64_t>(nb, 1))) ||
        (e = scratch.get(&lbA, (size_t)na + 1)) || (e = scratch.get(&eqA, (size_t)na + 1)) ||
        (e = scratch.get(&lbB, (size_t)nb + 1)) || (e = scratch.get(&eqB, (size_t)nb + 1)) ||
        (e = scratch.get(&shA, (size_t)na + 1)) || (e = scratch.get(&shB, (size_t)nb + 1)))
        return e;
    // run starts (an empty side has rs = {0})
    if (a.len > 0) {
        run_starts_kernel<<<grid_for(a.nchunks), 256, 0, s>>>(a.perm, a.chunk_slot0, a.len, a.nchunks, rsA);
        FSP_LAUNCHED();
    } else {
        FSP_CUDA(cudaMemsetAsync(rsA, 0, 4, s));
    }
    if (b.len > 0) {
        run_starts_kernel<<<grid_for(b.nchunks), 256, 0, s>>>(b.perm, b.chunk_slot0, b.len, b.nchunks, rsB);
        FSP_LAUNCHED();
    } else {
        FSP_CUDA(cudaMemsetAsync(rsB, 0, 4, s));
    }
    if (na > 0) {
        slot_keys_kernel<<<grid_for(a.n), 256, 0, s>>>(a.jcS, a.n, a.irS, keyA);
        FSP_LAUNCHED();
    }
    if (nb > 0) {
        slot_keys_kernel<<<grid_for(b.n), 256, 0, s>>>(b.jcS, b.n, b.irS, keyB);
        FSP_LAUNCHED();
    }
    if (na + nb > 0) {
        merge_path_kernel<<<grid_for((na + nb + kMergeSteps - 1) / kMergeSteps), 256, 0, s>>>(
            keyA, na, keyB, nb, lbA, eqA, lbB, eqB);
        FSP_LAUNCHED();
    }
    if ((e = exclusive_scan_u32(eqA, shA, na, st, scratch, s)) != FSPARSE_OK) return e;
    if ((e = exclusive_scan_u32(eqB, shB, nb, st, scratch, s)) != FSPARSE_OK) return e;
    if (na > 0) {
        merge_irs_kernel<<<grid_for(na), 256, 0, s>>>(a.irS, na, lbA, shA, out.irS, na + nb, st);
        FSP_LAUNCHED();
    }
    if (nb > 0) {
        merge_irs_kernel<<<grid_for(nb), 256, 0, s>>>(b.irS, nb, lbB, shB, out.irS, na + nb, st);
        FSP_LAUNCHED();
    }
    merge_jcs_kernel<<<grid_for((int64_t)a.n + 1), 256, 0, s>>>(a.jcS, b.jcS, shA, a.n, out.jcS);
    FSP_LAUNCHED();
    merged_nnz_kernel<<<1, 1, 0, s>>>(na, nb, shA + na, st);
    FSP_LAUNCHED();
    if (a.len > 0) {
        merge_positions_kernel<<<grid_for(a.nchunks), 256, 0, s>>>(a.perm, a.chunk_slot0, a.len, a.nchunks, lbA,
                                                                   eqA, rsB, 0, 0u, out.perm, out.len, st);
        FSP_LAUNCHED();
    }
    if (b.len > 0) {
        merge_positions_kernel<<<grid_for(b.nchunks), 256, 0, s>>>(b.perm, b.chunk_slot0, b.len, b.nchunks, lbB,
                                                                   eqB, rsA, 1, (uint32_t)a.len, out.perm,
                                                                   out.len, st);
        FSP_LAUNCHED();
    }
    // chunk slot bases of the merged order; nnz = na + nb - shared
    uint32_t *counts;
    if ((e = scratch.get(&counts, (size_t)out.nchunks + 1)) != FSPARSE_OK) return e;
    if ((e = launch_chunk_heads(out.perm, out.len, counts, out.nchunks, s)) != FSPARSE_OK) return e;
    return exclusive_scan_u32(counts, out.chunk_slot0, out.nchunks, st, scratch, s);
}

}  // namespace fsp
