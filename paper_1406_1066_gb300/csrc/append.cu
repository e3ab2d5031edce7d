// append.cu -- delayed assembly: merge a plan with the plan of new triplets.
//
// The paper notes (§2, before §2.1's problem statement closes) that its
// counting scheme extends to input that is not all available at the first
// call.  Here the result of appending triplets (ii2, jj2) to a plan of
// (ii1, jj1) is defined as the assembly of the concatenation, with the new
// triplet numbers continuing at len1.  Both plans are already sorted by
// (column, row) with runs in ascending k, so the new plan is a merge:
//
//   * ranks by a merge of the two plans' sorted rows, column by column (the
//     columns are aligned, so no search is needed): for every slot of one
//     plan, the number of keys of the other plan below it and whether the
//     other plan holds the same key;
//   * merged slot of an old slot a = a + (new keys below it) - (shared keys
//     before it); of a new slot b = b + (old keys below it) - (shared keys
//     before it); a shared key is one slot;
//   * positions: an old run moves right by the number of new triplets with a
//     smaller key; a new run moves right by the number of old triplets with a
//     key not above its own, so inside a shared slot the old triplets (smaller
//     k) come first and the run stays in ascending k; the shift is computed
//     once per run, then applied to every position of it;
//   * jcS of the merge: old + new column starts minus the shared keys in
//     earlier columns.
#include <algorithm>

#include "common.cuh"
#include "internal.hpp"

namespace fsp {

// The kChunk perm entries of chunk q (128-bit loads when the chunk is whole
// and aligned; entries past len read as 0).
__device__ __forceinline__ void load_chunk(const uint32_t *__restrict__ perm, int64_t len, int64_t q,
                                           uint32_t (&pm)[kChunk]) {
    const int64_t p0 = q * kChunk;
    if (p0 + kChunk <= len && (reinterpret_cast<uintptr_t>(perm) & 15) == 0) {
#pragma unroll
        for (int v = 0; v < kChunk / 4; ++v) {
            const uint4 x = __ldg(reinterpret_cast<const uint4 *>(perm + p0) + v);
            pm[4 * v] = x.x;
            pm[4 * v + 1] = x.y;
            pm[4 * v + 2] = x.z;
            pm[4 * v + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kChunk; ++i) pm[i] = p0 + i < len ? __ldg(perm + p0 + i) : 0u;
    }
}

// First position of every run: rs[slot] = p at run heads, rs[nnz] = len.
__global__ void run_starts_kernel(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ chunk_slot0,
                                  int64_t len, int64_t nchunks, uint32_t *__restrict__ rs) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nchunks;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p0 = q * kChunk;
        uint32_t pm[kChunk];
        load_chunk(perm, len, q, pm);
        uint32_t slot = chunk_slot0[q];   // runs before the chunk = index of the next run
#pragma unroll
        for (int i = 0; i < kChunk; ++i)
            if (p0 + i < len && (pm[i] & kHeadBit)) rs[slot++] = (uint32_t)(p0 + i);
        if (q == nchunks - 1) rs[chunk_slot0[nchunks]] = (uint32_t)len;
    }
}

// Ranks across the two plans, one thread per column: the column's old rows
// irA[jcA[c] .. jcA[c+1]) and new rows irB[jcB[c] .. jcB[c+1]) are both
// ascending, so one merge gives, for an old slot x, lbA[x] = new slots with
// a smaller key (all new slots of earlier columns plus the smaller rows of
// this one) and eqA[x] = the new plan holds the same key; and for a new slot
// y, lbB[y] = old slots with a smaller key and eqB[y] likewise.  Columns of
// up to kStage rows per side are first copied to the thread's own slice of
// shared memory with independent loads, so the merge does not wait on one
// global load per step.
constexpr int kStage = 16;
constexpr int kColThreads = 128;

__global__ void __launch_bounds__(kColThreads)
    merge_columns_kernel(const int32_t *__restrict__ jcA, const int32_t *__restrict__ irA,
                         const int32_t *__restrict__ jcB, const int32_t *__restrict__ irB, int32_t n,
                         uint32_t *__restrict__ lbA, uint32_t *__restrict__ eqA,
                         uint32_t *__restrict__ lbB, uint32_t *__restrict__ eqB) {
    __shared__ int32_t s_rows[2 * kStage][kColThreads];   // [row index][thread]: conflict-free
    const int tid = threadIdx.x;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + tid; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x0 = jcA[c], xe = jcA[c + 1], y0 = jcB[c], ye = jcB[c + 1];
        const int32_t na = xe - x0, nb = ye - y0;
        const bool staged = na <= kStage && nb <= kStage;
        if (staged) {
#pragma unroll
            for (int u = 0; u < kStage; ++u) {
                if (u < na) s_rows[u][tid] = __ldg(irA + x0 + u);
                if (u < nb) s_rows[kStage + u][tid] = __ldg(irB + y0 + u);
            }
        }
        int32_t x = x0, y = y0;
        while (x < xe || y < ye) {
            const int32_t rx = x < xe ? (staged ? s_rows[x - x0][tid] : irA[x]) : 0;
            const int32_t ry = y < ye ? (staged ? s_rows[kStage + y - y0][tid] : irB[y]) : 0;
            if (y >= ye || (x < xe && rx < ry)) {
                lbA[x] = (uint32_t)y;
                eqA[x] = 0u;
                ++x;
            } else if (x >= xe || ry < rx) {
                lbB[y] = (uint32_t)x;
                eqB[y] = 0u;
                ++y;
            } else {   // the same (i,j) in both plans: one slot of the merge
                lbA[x] = (uint32_t)y;
                eqA[x] = 1u;
                lbB[y] = (uint32_t)x;
                eqB[y] = 1u;
                ++x;
                ++y;
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

// Shift of every run of one side in the merged order, one thread per slot
// (lb is non-decreasing along the slots, so the lookups into the other
// side's run starts are nearly sequential).  For the old side (second_side
// = 0) a run moves by other_rs[lb]: the new triplets with a smaller key.
// For the new side it moves by other_rs[lb + eq]: the old triplets with a
// key not above its own, so inside a shared slot the old triplets come
// first.  Bit 31 marks a new run whose key the old side also holds: its
// head bit is dropped (the old run starts that slot).
__global__ void merge_shift_kernel(int64_t nnz, const uint32_t *__restrict__ lb, const uint32_t *__restrict__ eq,
                                   const uint32_t *__restrict__ other_rs, int second_side,
                                   uint32_t *__restrict__ shift) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nnz;
         x += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = second_side ? eq[x] : 0u;
        shift[x] = other_rs[lb[x] + e] | (e ? kHeadBit : 0u);
    }
}

// Start of run x of a plan (its first position in the sorted order), found
// from the plan's chunk slot bases instead of a pass over all its runs: the
// chunk q with chunk_slot0[q] <= x < chunk_slot0[q + 1] holds the head, as the
// (x - chunk_slot0[q])-th head of that chunk; x == nnz gives len.
__device__ __forceinline__ uint32_t run_start_of(const uint32_t *__restrict__ perm,
                                                 const uint32_t *__restrict__ chunk_slot0, int64_t len,
                                                 int64_t nchunks, int64_t nnz, uint32_t x) {
    if (x >= nnz) return (uint32_t)len;
    int64_t lo = 0, hi = nchunks - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(chunk_slot0 + mid) <= x) lo = mid; else hi = mid - 1;
    }
    uint32_t need = x - __ldg(chunk_slot0 + lo);
    const int64_t p1 = min64((lo + 1) * kChunk, len);
    for (int64_t p = lo * kChunk; p < p1; ++p) {
        if (__ldg(perm + p) & kHeadBit) {
            if (need == 0) return (uint32_t)p;
            --need;
        }
    }
    return (uint32_t)len;   // only for a damaged plan
}

// The new side's shifts when it has few runs: the old side's run starts are
// looked up where they are needed instead of being listed for all old runs.
__global__ void merge_shift_search_kernel(int64_t nnz, const uint32_t *__restrict__ lb,
                                          const uint32_t *__restrict__ eq, const uint32_t *__restrict__ other_perm,
                                          const uint32_t *__restrict__ other_cs0, int64_t other_len,
                                          int64_t other_nchunks, int64_t other_nnz, uint32_t *__restrict__ shift) {
    for (int64_t y = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; y < nnz;
         y += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = eq[y];
        shift[y] = run_start_of(other_perm, other_cs0, other_len, other_nchunks, other_nnz, lb[y] + e) |
                   (e ? kHeadBit : 0u);
    }
}

// Positions of one side's runs in the merged order, one thread per position
// (a warp takes 32 consecutive positions, two chunks, so loads and stores
// are coalesced and the lanes of one run share their lookups).  The slot of
// a position is the run before the warp's first chunk plus the heads up to
// it; the position moves by its slot's shift.  Each warp step handles
// kGroups such 32-position groups, whose dependent lookups (perm -> slot ->
// shift) overlap.
constexpr int kGroups = 4;

__global__ void merge_positions_kernel(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ chunk_slot0,
                                       int64_t len, int64_t nnz, const uint32_t *__restrict__ shift,
                                       uint32_t kofs, uint32_t *__restrict__ out, int64_t len_out,
                                       uint32_t *__restrict__ head_counts, int64_t nchunks_out, DevStatus *st) {
    const int lane = threadIdx.x & 31;
    const uint32_t le = lanemask_lt() | (1u << lane);
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t span = 32 * kGroups;
    for (int64_t w0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * span; w0 < len;
         w0 += warps * span) {
        uint32_t x[kGroups], base[kGroups];
#pragma unroll
        for (int g = 0; g < kGroups; ++g) {
            const int64_t p = w0 + 32 * g + lane;
            x[g] = p < len ? __ldg(perm + p) : 0u;
            base[g] = w0 + 32 * g < len ? __ldg(chunk_slot0 + ((w0 + 32 * g) >> kChunkShift)) : 0u;
        }
        uint32_t sh[kGroups];
        bool ok[kGroups];
#pragma unroll
        for (int g = 0; g < kGroups; ++g) {
            const uint32_t hm = __ballot_sync(0xffffffffu, (x[g] & kHeadBit) != 0);
            const int64_t slot = (int64_t)base[g] - 1 + __popc(hm & le);
            ok[g] = w0 + 32 * g + lane < len && slot >= 0 && slot < nnz;
            sh[g] = ok[g] ? __ldg(shift + slot) : 0u;
        }
#pragma unroll
        for (int g = 0; g < kGroups; ++g) {
            const int64_t p = w0 + 32 * g + lane;
            const int64_t t = p + (sh[g] & kIndexMask);
            const bool keep = ok[g] && (x[g] & kHeadBit) && !(sh[g] & kHeadBit);
            if (!ok[g]) {
                if (p < len) atomicOr(&st->oob, 1u);
            } else if (in_range(t, len_out, st)) {
                out[t] = ((x[g] & kIndexMask) + kofs) | (keep ? kHeadBit : 0u);
            }
            // Run heads per chunk of the merged order, counted here instead of
            // in a pass over the merged perm: the kept heads of the warp come
            // in ascending merged position, so heads that land in one chunk
            // are neighbours among them and add their count once.
            const uint32_t hm = __ballot_sync(0xffffffffu, keep);
            if (hm) {
                const uint32_t key = (uint32_t)(t >> kChunkShift);
                const uint32_t before = hm & lanemask_lt();
                const int prev = before ? 31 - __clz(before) : lane;
                const uint32_t prev_key = __shfl_sync(0xffffffffu, key, prev);
                const uint32_t lm = __ballot_sync(0xffffffffu, keep && (!before || prev_key != key));
                if (keep && ((lm >> lane) & 1u)) {
                    const uint32_t above = lm & ~((2u << lane) - 1u);
                    const uint32_t upto = above ? (1u << (__ffs(above) - 1)) - 1u : 0xffffffffu;
                    const uint32_t c = __popc(hm & upto & ~((1u << lane) - 1u));
                    if (in_range(key, nchunks_out, st)) atomicAdd(head_counts + key, c);
                }
            }
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
    fsparse_status e;
    uint32_t *mvA, *mvB;
    if ((e = scratch.get(&rsA, (size_t)na + 1)) || (e = scratch.get(&rsB, (size_t)nb + 1)) ||
        (e = scratch.get(&lbA, (size_t)na + 1)) || (e = scratch.get(&eqA, (size_t)na + 1)) ||
        (e = scratch.get(&lbB, (size_t)nb + 1)) || (e = scratch.get(&eqB, (size_t)nb + 1)) ||
        (e = scratch.get(&shA, (size_t)na + 1)) || (e = scratch.get(&shB, (size_t)nb + 1)) ||
        (e = scratch.get(&mvA, (size_t)na + 1)) || (e = scratch.get(&mvB, (size_t)nb + 1)))
        return e;
    // run starts (an empty side has rs = {0}); the old side's are listed only
    // when the new side has many runs, else looked up where needed
    const bool search_a = nb * 64 < na;
    phase_begin("merge_run_starts");
    if (a.len > 0 && !search_a) {
        run_starts_kernel<<<grid_for(a.nchunks), 256, 0, s>>>(a.perm, a.chunk_slot0, a.len, a.nchunks, rsA);
        FSP_LAUNCHED();
    } else if (a.len == 0) {
        FSP_CUDA(cudaMemsetAsync(rsA, 0, 4, s));
    }
    if (b.len > 0) {
        run_starts_kernel<<<grid_for(b.nchunks), 256, 0, s>>>(b.perm, b.chunk_slot0, b.len, b.nchunks, rsB);
        FSP_LAUNCHED();
    } else {
        FSP_CUDA(cudaMemsetAsync(rsB, 0, 4, s));
    }
    phase_mark("merge_run_starts");
    phase_begin("merge_columns");
    if (na + nb > 0) {
        const int cgrid = (int)std::max<int64_t>(
            1, std::min<int64_t>((a.n + kColThreads - 1) / kColThreads, (int64_t)sm_count(0) * 16));
        merge_columns_kernel<<<cgrid, kColThreads, 0, s>>>(a.jcS, a.irS, b.jcS, b.irS, a.n, lbA, eqA, lbB, eqB);
        FSP_LAUNCHED();
    }
    phase_mark("merge_columns");
    phase_begin("merge_slots");
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
    if (na > 0) {
        merge_shift_kernel<<<grid_for(na), 256, 0, s>>>(na, lbA, eqA, rsB, 0, mvA);
        FSP_LAUNCHED();
    }
    if (nb > 0 && search_a && a.len > 0) {
        merge_shift_search_kernel<<<grid_for(nb), 256, 0, s>>>(nb, lbB, eqB, a.perm, a.chunk_slot0, a.len,
                                                               a.nchunks, na, mvB);
        FSP_LAUNCHED();
    } else if (nb > 0) {
        merge_shift_kernel<<<grid_for(nb), 256, 0, s>>>(nb, lbB, eqB, rsA, 1, mvB);
        FSP_LAUNCHED();
    }
    phase_mark("merge_slots");
    phase_begin("merge_positions");
    // run heads per chunk of the merged order, counted by the position kernels
    uint32_t *counts;
    if ((e = scratch.get(&counts, (size_t)out.nchunks + 1)) != FSPARSE_OK) return e;
    FSP_CUDA(cudaMemsetAsync(counts, 0, ((size_t)out.nchunks + 1) * 4, s));
    if (a.len > 0) {
        merge_positions_kernel<<<grid_for((a.len + 8 * kGroups - 1) / (8 * kGroups)), 256, 0, s>>>(
            a.perm, a.chunk_slot0, a.len, na, mvA, 0u, out.perm, out.len, counts, out.nchunks, st);
        FSP_LAUNCHED();
    }
    if (b.len > 0) {
        merge_positions_kernel<<<grid_for((b.len + 8 * kGroups - 1) / (8 * kGroups)), 256, 0, s>>>(
            b.perm, b.chunk_slot0, b.len, nb, mvB, (uint32_t)a.len, out.perm, out.len, counts, out.nchunks, st);
        FSP_LAUNCHED();
    }
    phase_mark("merge_positions");
    phase_begin("merge_chunk_heads");
    // chunk slot bases of the merged order; nnz = na + nb - shared
    e = exclusive_scan_u32(counts, out.chunk_slot0, out.nchunks, st, scratch, s);
    phase_mark("merge_chunk_heads");
    return e;
}

}  // namespace fsp
