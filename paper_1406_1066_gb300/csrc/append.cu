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
//     earlier columns;
//   * chunk slot bases of the merge: every merged position is written once,
//     and the one that lands on a chunk's first position writes the chunk's
//     base (its run's merged slot, plus one when it is not the run's head).
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
// One thread per chunk of 16 positions.  (A warp per 32 positions with one
// ballot each measured slower: 0.17 against 0.14 ms for both halves of the
// 100^3 cube.)
__global__ void run_starts_kernel(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ chunk_slot0,
                                  int64_t len, int64_t nnz, uint32_t *__restrict__ rs, DevStatus *st) {
    const int64_t nchunks = (len + kChunk - 1) >> kChunkShift;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nchunks;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p0 = q * kChunk;
        uint32_t pm[kChunk];
        load_chunk(perm, len, q, pm);
        int64_t slot = __ldg(chunk_slot0 + q);   // runs before the chunk = index of the next run
#pragma unroll
        for (int i = 0; i < kChunk; ++i) {
            if (p0 + i < len && (pm[i] & kHeadBit)) {
                if (in_range(slot, nnz, st)) rs[slot] = (uint32_t)(p0 + i);
                ++slot;
            }
        }
        if (q == nchunks - 1) rs[nnz] = (uint32_t)len;
    }
}

// Ranks across the two plans, one lane per column: the column's old rows
// irA[jcA[c] .. jcA[c+1]) and new rows irB[jcB[c] .. jcB[c+1]) are both
// ascending, so one merge gives, for an old slot x, lbA[x] = new slots with
// a smaller key (all new slots of earlier columns plus the smaller rows of
// this one) and eqA[x] = the new plan holds the same key; and for a new slot
// y, lbB[y] = old slots with a smaller key and eqB[y] likewise.  A warp
// takes 32 neighbouring columns, whose rows are contiguous in irA and irB:
// when they fit, they are read into shared memory with coalesced loads, the
// lanes merge from there, and the ranks go back out coalesced too.  Larger
// column groups merge straight from global memory.
constexpr int kColWarps = 4;
constexpr int kColCap = 512;   // rows per side staged per warp

__global__ void __launch_bounds__(kColWarps * 32)
    merge_columns_kernel(const int32_t *__restrict__ jcA, const int32_t *__restrict__ irA,
                         const int32_t *__restrict__ jcB, const int32_t *__restrict__ irB, int32_t n,
                         uint32_t *__restrict__ lbA, uint32_t *__restrict__ eqA,
                         uint32_t *__restrict__ lbB, uint32_t *__restrict__ eqB) {
    __shared__ int32_t s_ra[kColWarps][kColCap], s_rb[kColWarps][kColCap];
    __shared__ uint32_t s_la[kColWarps][kColCap], s_lb[kColWarps][kColCap];   // rank | eq << 31
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t *ra = s_ra[w], *rb = s_rb[w];
    uint32_t *la = s_la[w], *lbs = s_lb[w];
    const int64_t warps = (int64_t)gridDim.x * kColWarps;
    for (int64_t c0 = ((int64_t)blockIdx.x * kColWarps + w) * 32; c0 < n; c0 += warps * 32) {
        const int64_t c = c0 + lane;
        const int64_t ce = min64(c0 + 32, (int64_t)n);
        const int32_t ga0 = __ldg(jcA + c0), ga1 = __ldg(jcA + ce);
        const int32_t gb0 = __ldg(jcB + c0), gb1 = __ldg(jcB + ce);
        int32_t x0 = 0, xe = 0, y0 = 0, ye = 0;
        if (c < n) {
            x0 = __ldg(jcA + c);
            xe = __ldg(jcA + c + 1);
            y0 = __ldg(jcB + c);
            ye = __ldg(jcB + c + 1);
        }
        const bool staged = ga1 - ga0 <= kColCap && gb1 - gb0 <= kColCap;
        if (staged) {
            for (int u = lane; u < ga1 - ga0; u += 32) ra[u] = __ldg(irA + ga0 + u);
            for (int u = lane; u < gb1 - gb0; u += 32) rb[u] = __ldg(irB + gb0 + u);
            __syncwarp();
        }
        int32_t x = x0, y = y0;
        while (x < xe || y < ye) {
            const int32_t rx = x < xe ? (staged ? ra[x - ga0] : __ldg(irA + x)) : 0;
            const int32_t ry = y < ye ? (staged ? rb[y - gb0] : __ldg(irB + y)) : 0;
            uint32_t va = 0xffffffffu, vb = 0xffffffffu;
            if (y >= ye || (x < xe && rx < ry)) {
                va = (uint32_t)y;
            } else if (x >= xe || ry < rx) {
                vb = (uint32_t)x;
            } else {   // the same (i,j) in both plans: one slot of the merge
                va = (uint32_t)y | kHeadBit;
                vb = (uint32_t)x | kHeadBit;
            }
            if (va != 0xffffffffu) {
                if (staged) {
                    la[x - ga0] = va;
                } else {
                    lbA[x] = va & kIndexMask;
                    eqA[x] = va >> 31;
                }
                ++x;
            }
            if (vb != 0xffffffffu) {
                if (staged) {
                    lbs[y - gb0] = vb;
                } else {
                    lbB[y] = vb & kIndexMask;
                    eqB[y] = vb >> 31;
                }
                ++y;
            }
        }
        if (staged) {
            __syncwarp();
            for (int u = lane; u < ga1 - ga0; u += 32) {
                lbA[ga0 + u] = la[u] & kIndexMask;
                eqA[ga0 + u] = la[u] >> 31;
            }
            for (int u = lane; u < gb1 - gb0; u += 32) {
                lbB[gb0 + u] = lbs[u] & kIndexMask;
                eqB[gb0 + u] = lbs[u] >> 31;
            }
            __syncwarp();
        }
    }
}

// jcS of the merge: old + new column starts minus shared keys in earlier columns.
__global__ void merge_jcs_kernel(const int32_t *__restrict__ jc1, const int32_t *__restrict__ jc2,
                                 const uint32_t *__restrict__ shared1, int32_t n, int32_t *__restrict__ out) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= n;
         c += (int64_t)gridDim.x * blockDim.x)
        out[c] = (int32_t)((int64_t)jc1[c] + jc2[c] - shared1[jc1[c]]);
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

// Every slot x of one side, one thread each: its merged slot
// ms = x + lb[x] - sh[x] (sh: shared keys before it), its row into the merged
// irS (a new slot whose key the old side also holds is the old slot's), and
// the shift of its run into the merged order.  For the old side (second_side
// = 0) a run moves by the new triplets with a smaller key, other_rs[lb]; for
// the new side by the old triplets with a key not above its own,
// other_rs[lb + eq], so inside a shared slot the old triplets (smaller k)
// come first.  Bit 31 of the shift marks a new run whose key the old side
// holds: its head bit is dropped (the old run starts that slot).  With
// other_rs == NULL the other side's run starts are looked up from its chunk
// slot bases (few runs on this side, many on the other).
__global__ void merge_slots_kernel(int64_t nnz, const int32_t *__restrict__ irS, const uint32_t *__restrict__ lb,
                                   const uint32_t *__restrict__ eq, const uint32_t *__restrict__ sh,
                                   int second_side, const uint32_t *__restrict__ other_rs,
                                   const uint32_t *__restrict__ other_perm, const uint32_t *__restrict__ other_cs0,
                                   int64_t other_len, int64_t other_nchunks, int64_t other_nnz,
                                   int32_t *__restrict__ irs_out, int64_t cap_out, uint32_t *__restrict__ shift,
                                   uint32_t *__restrict__ mslot, DevStatus *st) {
    constexpr int U = 4;   // slots per thread step, their loads in flight together
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x0 < nnz; x0 += stride * U) {
        uint32_t e[U], l[U], h[U], j[U], start[U];
        int32_t row[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t x = x0 + u * stride;
            const bool have = x < nnz;
            e[u] = have && second_side ? __ldg(eq + x) : 0u;
            l[u] = have ? __ldg(lb + x) : 0u;
            h[u] = have ? __ldg(sh + x) : 0u;
            row[u] = have ? __ldg(irS + x) : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            j[u] = l[u] + e[u];
            start[u] = 0;
            if (x0 + u * stride < nnz && other_rs && in_range(j[u], other_nnz + 1, st)) start[u] = __ldg(other_rs + j[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t x = x0 + u * stride;
            if (x >= nnz) continue;
            if (!other_rs) start[u] = run_start_of(other_perm, other_cs0, other_len, other_nchunks, other_nnz, j[u]);
            const int64_t ms = x + (int64_t)l[u] - (int64_t)h[u];
            if (!e[u] && in_range(ms, cap_out, st)) irs_out[ms] = row[u];
            shift[x] = start[u] | (e[u] ? kHeadBit : 0u);
            mslot[x] = (uint32_t)ms;
        }
    }
}

// Positions of one side's runs in the merged order, one thread per position
// (a warp takes 32 consecutive positions, two chunks, so loads and stores
// are coalesced and the lanes of one run share their lookups).  The slot of
// a position is the run before the warp's first chunk plus the heads up to
// it; the position moves by its slot's shift.  The position that lands on
// the first position of a merged chunk writes that chunk's slot base: the
// runs that start before it, i.e. its own run's merged slot, plus one when
// it is not that run's head.  Each warp step handles kGroups such
// 32-position groups, whose dependent lookups (perm -> slot -> shift)
// overlap.
constexpr int kGroups = 4;

__global__ void merge_positions_kernel(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ chunk_slot0,
                                       int64_t len, int64_t nnz, const uint32_t *__restrict__ shift,
                                       const uint32_t *__restrict__ mslot, uint32_t kofs,
                                       uint32_t *__restrict__ out, int64_t len_out,
                                       uint32_t *__restrict__ cs_out, DevStatus *st) {
    // positions and slots fit 32 bits (plans hold fewer than 2^30 triplets)
    const int lane = threadIdx.x & 31;
    const uint32_t le = lanemask_lt() | (1u << lane);
    const uint32_t n = (uint32_t)len, nz = (uint32_t)nnz, nout = (uint32_t)len_out;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    constexpr uint32_t span = 32 * kGroups;
    for (uint32_t w0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * span; w0 < n; w0 += warps * span) {
        uint32_t x[kGroups], base[kGroups];
#pragma unroll
        for (int g = 0; g < kGroups; ++g) {
            const uint32_t p = w0 + 32 * g + lane;
            x[g] = p < n ? __ldg(perm + p) : 0u;
            base[g] = w0 + 32 * g < n ? __ldg(chunk_slot0 + ((w0 + 32 * g) >> kChunkShift)) : 0u;
        }
        uint32_t sh[kGroups], slot[kGroups];
#pragma unroll
        for (int g = 0; g < kGroups; ++g) {
            const uint32_t hm = __ballot_sync(0xffffffffu, (x[g] & kHeadBit) != 0);
            slot[g] = base[g] - 1u + __popc(hm & le);   // wraps to ~0 before the first head: rejected below
            const bool ok = w0 + 32 * g + lane < n && slot[g] < nz;
            sh[g] = ok ? __ldg(shift + slot[g]) : 0xffffffffu;
            if (!ok) slot[g] = 0xffffffffu;
        }
#pragma unroll
        for (int g = 0; g < kGroups; ++g) {
            const uint32_t p = w0 + 32 * g + lane;
            if (p >= n) continue;
            if (slot[g] == 0xffffffffu) {
                atomicOr(&st->oob, 1u);
                continue;
            }
            const uint32_t t = p + (sh[g] & kIndexMask);
            const bool keep = (x[g] & kHeadBit) && !(sh[g] & kHeadBit);
            if (!in_range(t, nout, st)) continue;
            out[t] = ((x[g] & kIndexMask) + kofs) | (keep ? kHeadBit : 0u);
            if ((t & (kChunk - 1)) == 0) cs_out[t >> kChunkShift] = __ldg(mslot + slot[g]) + (keep ? 0u : 1u);
        }
    }
}

// nnz of the merge (shared keys counted once) for the host's status read,
// and the merged chunk slot bases' closing entry.
__global__ void merged_nnz_kernel(int64_t na, int64_t nb, const uint32_t *shared_total, uint32_t *cs_end,
                                  DevStatus *st) {
    const uint32_t nnz = (uint32_t)(na + nb - *shared_total);
    st->nnz = nnz;
    *cs_end = nnz;
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
    uint32_t *rsA, *rsB, *lbA, *eqA, *lbB, *eqB, *shA, *shB, *mvA, *mvB, *msA, *msB;
    fsparse_status e;
    if ((e = scratch.get(&rsA, (size_t)na + 1)) || (e = scratch.get(&rsB, (size_t)nb + 1)) ||
        (e = scratch.get(&lbA, (size_t)na + 1)) || (e = scratch.get(&eqA, (size_t)na + 1)) ||
        (e = scratch.get(&lbB, (size_t)nb + 1)) || (e = scratch.get(&eqB, (size_t)nb + 1)) ||
        (e = scratch.get(&shA, (size_t)na + 1)) || (e = scratch.get(&shB, (size_t)nb + 1)) ||
        (e = scratch.get(&mvA, (size_t)na + 1)) || (e = scratch.get(&mvB, (size_t)nb + 1)) ||
        (e = scratch.get(&msA, (size_t)na + 1)) || (e = scratch.get(&msB, (size_t)nb + 1)))
        return e;
    // run starts (an empty side has rs = {0}); the old side's are listed only
    // when the new side has many runs, else looked up where needed
    const bool search_a = nb * 64 < na;
    phase_begin("merge_run_starts");
    if (a.len > 0 && !search_a) {
        run_starts_kernel<<<grid_for((a.len + kChunk - 1) / kChunk), 256, 0, s>>>(a.perm, a.chunk_slot0, a.len, na, rsA, st);
        FSP_LAUNCHED();
    } else if (a.len == 0) {
        FSP_CUDA(cudaMemsetAsync(rsA, 0, 4, s));
    }
    if (b.len > 0) {
        run_starts_kernel<<<grid_for((b.len + kChunk - 1) / kChunk), 256, 0, s>>>(b.perm, b.chunk_slot0, b.len, nb, rsB, st);
        FSP_LAUNCHED();
    } else {
        FSP_CUDA(cudaMemsetAsync(rsB, 0, 4, s));
    }
    phase_mark("merge_run_starts");
    phase_begin("merge_columns");
    if (na + nb > 0) {
        const int64_t groups = ((int64_t)a.n + 31) / 32;
        const int cgrid = (int)std::max<int64_t>(
            1, std::min<int64_t>((groups + kColWarps - 1) / kColWarps, (int64_t)sm_count(0) * 16));
        merge_columns_kernel<<<cgrid, kColWarps * 32, 0, s>>>(a.jcS, a.irS, b.jcS, b.irS, a.n, lbA, eqA, lbB, eqB);
        FSP_LAUNCHED();
    }
    phase_mark("merge_columns");
    phase_begin("merge_slots");
    if ((e = exclusive_scan_u32(eqA, shA, na, st, scratch, s)) != FSPARSE_OK) return e;
    if ((e = exclusive_scan_u32(eqB, shB, nb, st, scratch, s)) != FSPARSE_OK) return e;
    merge_jcs_kernel<<<grid_for((int64_t)a.n + 1), 256, 0, s>>>(a.jcS, b.jcS, shA, a.n, out.jcS);
    FSP_LAUNCHED();
    merged_nnz_kernel<<<1, 1, 0, s>>>(na, nb, shA + na, out.chunk_slot0 + out.nchunks, st);
    FSP_LAUNCHED();
    if (na > 0) {
        merge_slots_kernel<<<grid_for((na + 3) / 4), 256, 0, s>>>(na, a.irS, lbA, eqA, shA, 0, rsB, nullptr, nullptr, 0, 0, nb,
                                                        out.irS, na + nb, mvA, msA, st);
        FSP_LAUNCHED();
    }
    if (nb > 0) {
        const bool search = search_a && a.len > 0;
        merge_slots_kernel<<<grid_for((nb + 3) / 4), 256, 0, s>>>(nb, b.irS, lbB, eqB, shB, 1, search ? nullptr : rsA, a.perm,
                                                        a.chunk_slot0, a.len, a.nchunks, na, out.irS, na + nb, mvB,
                                                        msB, st);
        FSP_LAUNCHED();
    }
    phase_mark("merge_slots");
    phase_begin("merge_positions");
    // every merged position is written once; the ones on chunk starts write
    // the merged chunk slot bases
    if (a.len > 0) {
        merge_positions_kernel<<<grid_for((a.len + 8 * kGroups - 1) / (8 * kGroups)), 256, 0, s>>>(
            a.perm, a.chunk_slot0, a.len, na, mvA, msA, 0u, out.perm, out.len, out.chunk_slot0, st);
        FSP_LAUNCHED();
    }
    if (b.len > 0) {
        merge_positions_kernel<<<grid_for((b.len + 8 * kGroups - 1) / (8 * kGroups)), 256, 0, s>>>(
            b.perm, b.chunk_slot0, b.len, nb, mvB, msB, (uint32_t)a.len, out.perm, out.len, out.chunk_slot0, st);
        FSP_LAUNCHED();
    }
    phase_mark("merge_positions");
    return FSPARSE_OK;
}

}  // namespace fsp
