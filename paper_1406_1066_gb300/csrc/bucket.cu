// bucket.cu -- the hybrid path: one partition by high column bits, then one
// shared-memory sort per column bucket with everything else fused.
//
// The paper (§2.3) orders the triplets with counting passes whose tables are
// as long as the matrix is wide or tall.  On a GPU the cheap counting pass is
// the one whose table fits in shared memory, so the column index is split:
//
//   bucket = (j-1) >> cs            (up to 131072 buckets, 2^cs columns each)
//
//   1. count:    every block counts bucket sizes over its contiguous slice of
//                jj in a shared-memory table (above 32768 buckets, one pass
//                per range of 32768 buckets, each skipping the others);
//   2. offsets:  every non-empty (block, bucket) count reserves its range
//                inside the bucket by one atomic add on the bucket's total,
//                then an exclusive scan over buckets gives the bucket starts;
//   3. scatter:  every block re-reads its slice of ii/jj and appends packed
//                words  (j-1 low bits | i-1 | k)  to its ranges -- one 8-byte
//                write per triplet, the only global reordering pass;
//   4. emit:     one CTA per bucket (taken by atomic ticket) loads the bucket
//                and ranks its rows densely.  When the (column, row rank)
//                key space fits a 2^16-bit map, every triplet sets its key's
//                bit: the set bits are the bucket's unique (i,j) pairs in CCS
//                order (the collision detection of Part 3), a prefix
//                popcount numbers them and counts each column (Part 4), and
//                one counting scatter groups the triplets by slot.  Other
//                buckets sort (column, row) with a stable LSD radix sort in
//                shared memory (rank.cuh) and detect runs by comparing
//                neighbours.  Either way the slots are numbered across
//                buckets with one decoupled look-back, and the kernel writes
//                perm -- each run in ascending k, since the scatter keeps no
//                order inside a block: every triplet counts the triplets of
//                its run with a smaller k and lands that far into the run --,
//                irS, jcS and the numeric chunk slot bases (the values are
//                folded by the numeric kernel afterwards).
//
// A bucket above the kernel's capacity, or a run longer than kRunSortMax,
// sets DevStatus::overflow; the host then redoes the call with the global
// onesweep sort, which has no such limit.  Results are identical either way.
#include <algorithm>

#include "common.cuh"
#include "internal.hpp"
#include "rank.cuh"

namespace fsp {

constexpr int64_t kBucketsPerPass = 32768;   // shared-memory table of the count and scatter kernels
constexpr int kMaxBucketPasses = 4;           // more buckets: the count and scatter run once per range
constexpr int64_t kMaxBuckets = kBucketsPerPass * kMaxBucketPasses;
constexpr int kMaxColBits = 12;     // 2^cs column counters in shared memory
// Longest run put back into k order in the bucket kernel.  Each triplet of a
// run of length r reads the run once (r/4 shared loads), so the rank grows
// with r; a longer run makes the host redo the whole call with the onesweep
// sort.  On 2e7 triplets in runs of exactly r (20,000 x 20,000): onesweep
// alone 1.61 ms; ranked here 1.28 / 2.10 / 2.65 / 3.21 ms for r = 160 / 256 /
// 384 / 512; a bucket pass thrown away plus onesweep 2.5-2.8 ms.  384 sits
// at the crossover.  (The paper's first data set, pairs 50 times each and a
// few drawn two or three times, has runs of 150: 2.99 -> 1.05 ms.)
constexpr int kRunSortMax = 384;
constexpr int kRowBits = 1 << 16;   // row ranges up to this are compressed to dense ranks
constexpr int kKeyBits = 1 << 16;   // (column, row rank) key spaces up to this are counted in a bitmap

struct BucketShape {
    int cs = 0;        // low column bits kept inside a bucket
    int64_t nb = 0;    // number of buckets
    int kb = 1;        // bits of k in a packed word
    int grid = 1;      // blocks of the count/scatter kernels
};

// Bucket kernel shapes, smallest capacity first; the one used is the
// smallest whose capacity holds the largest bucket.
constexpr int kEmitCap[3] = {256 * 16, 512 * 12, 512 * 16};
constexpr int kMaxBucketCap = 512 * 16;

static bool bucket_shape(int64_t len, int32_t n, const KeyLayout &key, const fsparse_config &cfg,
                         BucketShape *out) {
    if (len <= 0 || n <= 0) return false;
    BucketShape sh;
    sh.kb = std::max(1, bits_for((uint64_t)len - 1));
    const double per_col = (double)len / (double)n;
    while (sh.cs < key.cb && per_col * (double)(1ll << (sh.cs + 1)) <= cfg.bucket_target) ++sh.cs;
    sh.nb = ((int64_t)(n - 1) >> sh.cs) + 1;
    while (sh.nb > kMaxBuckets && sh.cs < key.cb) {
        ++sh.cs;
        sh.nb = ((int64_t)(n - 1) >> sh.cs) + 1;
    }
    if (sh.nb > kMaxBuckets || sh.cs > kMaxColBits) return false;
    if (sh.cs + key.rb + sh.kb > 64) return false;
    if (out) *out = sh;
    return true;
}

bool bucket_supported(int64_t len, int32_t n, const KeyLayout &key, const fsparse_config &cfg) {
    return bucket_shape(len, n, key, cfg, nullptr);
}

// in_range for 32-bit values (one unsigned compare); the per-item checks of
// these kernels use it.
__device__ __forceinline__ bool in_range32(uint32_t v, uint32_t bound, DevStatus *st) {
    if (v < bound) return true;
    if (st) atomicOr(&st->oob, 1u);
    return false;
}

// Zero-based index, clamped into [0, dim); an index below 1 or above dim
// sets `bad` (reported once per thread).  The clamp keeps every address in
// range, and both kernels map a bad index the same way.
__device__ __forceinline__ uint32_t zero_based(int32_t v, int32_t dim, uint32_t &bad) {
    const uint32_t z = (uint32_t)v - 1u;
    bad |= (uint32_t)(z >= (uint32_t)dim);
    return min(z, (uint32_t)dim - 1u);
}

// ----------------------------------------------------------------------------
// 1+2. per-block bucket counts over a contiguous slice of jj (a shared-memory
//      table, 16-byte loads), then every non-empty (block, bucket) count
//      reserves its range inside the bucket with one atomic add on the
//      bucket's total: goff[g][b] is block g's offset inside bucket b, tot[b]
//      ends as the bucket's size, and *largest as the largest size (every
//      final total passes through some block's old + count).  The order of
//      the blocks inside a bucket is therefore arbitrary, as is the order
//      inside a block's range: the emit kernel restores ascending k.
template <bool RANGED>
__global__ void bucket_count_kernel(const int32_t *__restrict__ jj, int64_t len, int32_t n, int cs,
                                    int b_lo, int nb, uint32_t *__restrict__ goff, uint32_t *__restrict__ tot,
                                    uint32_t *largest, DevStatus *st) {
    extern __shared__ uint32_t s_h[];
    const int tid = threadIdx.x;
    for (int b = tid; b < nb; b += blockDim.x) s_h[b] = 0;
    __syncthreads();
    const int64_t g = blockIdx.x, G = gridDim.x;
    const int64_t c0 = len * g / G, c1 = len * (g + 1) / G;
    // (Counting runs of equal buckets across the lanes first, one add per
    // run, measured slower here: 0.18 against 0.13 ms on the 100^3 cube.)
    // buckets [b_lo, b_lo + nb) only; the others belong to another pass
    uint32_t bad = 0;
    auto count = [&](int32_t j) {
        const uint32_t b = (zero_based(j, n, bad) >> cs) - (uint32_t)b_lo;
        if (!RANGED || b < (uint32_t)nb) atomicAdd(&s_h[b], 1u);   // one pass: every bucket is in range
    };
    // scalar head up to a 16-byte boundary, int4 body, scalar tail
    const int64_t v0 = min64(c1, (c0 + 3) & ~int64_t(3)), v1 = max(v0, c1 & ~int64_t(3));
    if (((reinterpret_cast<uintptr_t>(jj)) & 15) == 0) {
        for (int64_t k = c0 + tid; k < v0; k += blockDim.x) count(jj[k]);
        for (int64_t q = v0 / 4 + tid; q < v1 / 4; q += blockDim.x) {
            const int4 x = __ldg(reinterpret_cast<const int4 *>(jj) + q);
            count(x.x);
            count(x.y);
            count(x.z);
            count(x.w);
        }
        for (int64_t k = v1 + tid; k < c1; k += blockDim.x) count(jj[k]);
    } else {
        for (int64_t k = c0 + tid; k < c1; k += blockDim.x) count(jj[k]);
    }
    if (bad) atomicOr(&st->bad_index, 1u);
    __syncthreads();
    uint32_t m = 0;
    for (int b = tid; b < nb; b += blockDim.x) {
        const uint32_t c = s_h[b];
        if (c) {
            const uint32_t old = atomicAdd(&tot[b_lo + b], c);
            goff[g * nb + b] = old;
            m = max(m, old + c);
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0 && m) atomicMax(largest, m);
}

// 3. scatter packed words into the buckets (order inside a block's range is
//    not kept; the emit kernel restores ascending k inside each run).
template <bool RANGED>
__global__ void __launch_bounds__(1024, 2) bucket_scatter_kernel(const int32_t *__restrict__ ii, const int32_t *__restrict__ jj,
                                      int64_t len, int32_t m, int32_t n, int rb, int cs, int kb,
                                      int b_lo, int nb, const uint32_t *__restrict__ goff,
                                      const uint32_t *__restrict__ bstart, uint64_t *__restrict__ words,
                                      const uint32_t *__restrict__ largest, DevStatus *st) {
    extern __shared__ uint32_t s_cur[];
    const int tid = threadIdx.x;
    // The host redoes count and scatter with narrower buckets when the
    // largest one is over the emit's capacity; this width's scatter is then
    // skipped (it was queued before the host knew).
    if (*largest > (uint32_t)kMaxBucketCap) return;
    const int64_t g = blockIdx.x, G = gridDim.x;
    for (int b = tid; b < nb; b += blockDim.x) s_cur[b] = bstart[b_lo + b] + goff[g * nb + b];
    __syncthreads();
    const int64_t c0 = len * g / G, c1 = len * (g + 1) / G;
    const uint64_t lowmask = (1ull << cs) - 1;
    const int lane = tid & 31;
    const int64_t B = blockDim.x;
    // One position reservation per run of equal buckets across the lanes of
    // a warp: the head lane adds the run's length, every lane of the run
    // takes head's base + its distance to the head (lane order).
    uint32_t bad = 0;
    auto put = [&](int32_t i, int32_t j, int64_t k, bool have) {
        const uint32_t i0 = have ? zero_based(i, m, bad) : 0u;
        const uint32_t j0 = have ? zero_based(j, n, bad) : 0u;
        const uint32_t bl = (j0 >> cs) - (uint32_t)b_lo;   // bucket inside this pass's range
        if (RANGED) have = have && bl < (uint32_t)nb;
        const uint32_t b = have ? bl : 0xffff0000u | (uint32_t)lane;
        int head;
        uint32_t c;
        lane_runs(b, &head, &c);
        uint32_t base = 0;
        if (have && head == lane) base = atomicAdd(&s_cur[b], c);
        const uint32_t pos = __shfl_sync(0xffffffffu, base, head) + (uint32_t)(lane - head);
        const uint64_t w = ((uint64_t)(j0 & lowmask) << (rb + kb)) | ((uint64_t)i0 << kb) | (uint64_t)k;
        if (have && in_range32(pos, (uint32_t)len, st)) words[pos] = w;
    };
    // 16-byte index loads (four consecutive triplets per thread) when both
    // arrays are 16-byte aligned; scalar head and tail around the aligned body
    // of the slice.  Loops run warp-uniformly.
    const int64_t v0 = min64(c1, (c0 + 3) & ~int64_t(3)), v1 = max(v0, c1 & ~int64_t(3));
    auto scalar = [&](int64_t from, int64_t to) {
        for (int64_t k0 = from; k0 < to; k0 += B) {
            const int64_t k = k0 + tid;
            const bool have = k < to;
            put(have ? ii[k] : 1, have ? jj[k] : 1, k, have);
        }
    };
    if (((reinterpret_cast<uintptr_t>(ii) | reinterpret_cast<uintptr_t>(jj)) & 15) == 0) {
        scalar(c0, v0);
        const int4 *i4 = reinterpret_cast<const int4 *>(ii), *j4 = reinterpret_cast<const int4 *>(jj);
        for (int64_t q0 = v0 / 4; q0 < v1 / 4; q0 += B) {
            const int64_t q = q0 + tid;
            const bool have = q < v1 / 4;
            const int4 ia = have ? __ldg(i4 + q) : make_int4(1, 1, 1, 1);
            const int4 ja = have ? __ldg(j4 + q) : make_int4(1, 1, 1, 1);
            put(ia.x, ja.x, 4 * q, have);
            put(ia.y, ja.y, 4 * q + 1, have);
            put(ia.z, ja.z, 4 * q + 2, have);
            put(ia.w, ja.w, 4 * q + 3, have);
        }
        scalar(v1, c1);
    } else {
        scalar(c0, c1);
    }
    if (bad) atomicOr(&st->bad_index, 1u);
}

// ----------------------------------------------------------------------------
// 4. per-bucket sort + emit (+ fold).
struct BucketEmitArgs {
    const uint64_t *words;
    const uint32_t *bstart;
    int64_t nb;
    int cs, rb, kb;
    int32_t n;
    int64_t len;
    uint32_t *perm;
    int32_t *irS, *jcS;
    uint32_t *chunk_slot0;
    int64_t nchunks;
    uint32_t *look;
    uint32_t *ticket;
    DevStatus *st;
    int bitmap;   // allow the bitmap counting path (else always the radix passes)
};

template <int THREADS, int IPT>
struct BucketSmem {
    static constexpr int CAP = THREADS * IPT, WARPS = THREADS / 32;
    // Region A: rank counters during the sort, then run head positions.
    static constexpr size_t bytes_a = std::max<size_t>((size_t)WARPS * 256 * 4, ((size_t)(CAP + 1) * 2 + 15) / 16 * 16);
    // Region B: peer masks during the sort, then per-column unique counts.
    static constexpr size_t bytes_b = std::max<size_t>((size_t)WARPS * 256 * 4, (size_t)(1 << kMaxColBits) * 4);
    static constexpr size_t off_a = (size_t)CAP * 8;
    static constexpr size_t off_b = off_a + bytes_a;
    // Region C: row bitmap (kRowBits bits) and its u16 prefix counts.
    static constexpr size_t off_bits = off_b + bytes_b;
    static constexpr size_t off_pref = off_bits + (size_t)(kRowBits / 32) * 4;
    static constexpr size_t off_local = off_pref + (size_t)(kRowBits / 32) * 2;
    static constexpr size_t off_scan = off_local + 256 * 4;
    static constexpr size_t off_misc = off_scan + (WARPS + 2) * 4;
    static constexpr size_t bytes = off_misc + 16 * 4;
};

__device__ __forceinline__ int bits_of(uint32_t v) { return v ? 32 - __clz(v) : 0; }

// Block-wide exclusive scan with one barrier: each warp scans its lanes,
// publishes its total, and after the barrier every warp sums the totals of
// the warps before it itself (no second barrier to hand the result back).
// The caller must pass a barrier between the reads of one call and the
// writes of the next call on the same scratch.
template <int THREADS>
__device__ __forceinline__ uint32_t block_scan_1b(uint32_t x, uint32_t *scratch, uint32_t *total) {
    constexpr int WARPS = THREADS / 32;
    static_assert(WARPS <= 32, "one warp of totals");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    const uint32_t t = lane < WARPS ? scratch[lane] : 0u;
    uint32_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += y;
    }
    const uint32_t before = __shfl_sync(0xffffffffu, ti - t, warp);
    *total = __shfl_sync(0xffffffffu, ti, WARPS - 1);
    return before + inc - x;
}

template <int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) bucket_emit_kernel(BucketEmitArgs a) {
    using S = BucketSmem<THREADS, IPT>;
    constexpr int CAP = S::CAP, WARPS = S::WARPS;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *s_w = reinterpret_cast<uint64_t *>(smem);
    uint32_t *s_wcnt = reinterpret_cast<uint32_t *>(smem + S::off_a);    // sort
    uint16_t *s_hpos = reinterpret_cast<uint16_t *>(smem + S::off_a);    // after the sort
    uint32_t *s_wm = reinterpret_cast<uint32_t *>(smem + S::off_b);      // sort
    uint32_t *s_col = reinterpret_cast<uint32_t *>(smem + S::off_b);     // after the sort
    uint32_t *s_bits = reinterpret_cast<uint32_t *>(smem + S::off_bits);
    uint16_t *s_pref = reinterpret_cast<uint16_t *>(smem + S::off_pref);
    uint32_t *s_local = reinterpret_cast<uint32_t *>(smem + S::off_local);
    uint32_t *s_scan = reinterpret_cast<uint32_t *>(smem + S::off_scan);
    uint32_t *s_misc = reinterpret_cast<uint32_t *>(smem + S::off_misc);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_misc[0] = atomicAdd(a.ticket, 1u);
        s_misc[1] = 0xffffffffu;   // row min
        s_misc[2] = 0;             // row max
    }
    __syncthreads();
    const int64_t x = s_misc[0];
    const int64_t b0 = a.bstart[x];
    const int nx = (int)((int64_t)a.bstart[x + 1] - b0);
    // The row bitmap, the key bitmap and the run-size counters are cleared
    // here, before the first barrier, instead of each behind a barrier of
    // its own later on (buckets that take the radix passes overwrite them):
    // emit 1.182 -> 1.157 ms on the 100^3 cube.
    for (int w = tid; w < kRowBits / 32; w += THREADS) s_bits[w] = 0;
    for (int w = tid; w < kKeyBits / 32; w += THREADS) reinterpret_cast<uint32_t *>(smem + S::off_b)[w] = 0;
    for (int q = tid; q < min(nx, CAP); q += THREADS) reinterpret_cast<uint32_t *>(smem)[q] = 0;
    const int64_t col0 = x << a.cs;
    const int ncols = (int)min64((int64_t)1 << a.cs, (int64_t)a.n - col0);
    const int kb = a.kb, rb = a.rb;
    const uint64_t kmask = (1ull << kb) - 1;

    if (nx > CAP || nx < 0) {   // does not fit: flag it, keep the look-back chain moving
        if (warp == 0) {
            if (lane == 0) {
                atomicOr(&a.st->overflow, 1u);
                st_release(a.look + x, x == 0 ? kFlagInc : kFlagAgg);
            }
            if (x > 0) {
                const uint32_t e = warp_lookback_exclusive(a.look, 1, x, a.st);
                if (lane == 0) st_release(a.look + x, kFlagInc | e);
            }
        }
        return;
    }
    if (nx == 0) {   // empty bucket: its columns start where the previous bucket ends
        if (warp == 0) {
            uint32_t e = 0;
            if (lane == 0) st_release(a.look + x, x == 0 ? kFlagInc : kFlagAgg);
            if (x > 0) {
                e = warp_lookback_exclusive(a.look, 1, x, a.st);
                if (lane == 0) st_release(a.look + x, kFlagInc | e);
            }
            if (lane == 0) s_misc[3] = e;
        }
        __syncthreads();
        const uint32_t E = s_misc[3];
        for (int c = tid; c < ncols; c += THREADS) a.jcS[col0 + c] = (int32_t)E;
        if (x == a.nb - 1 && tid == 0) {
            a.jcS[a.n] = (int32_t)E;
            a.st->nnz = E;
            a.chunk_slot0[a.nchunks] = E;
        }
        return;
    }

    // Load the bucket (warp-striped) and find its row range.
    uint64_t pk[IPT];
    bool valid[IPT];
    uint32_t rmin = 0xffffffffu, rmax = 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int p = warp * 32 * IPT + i * 32 + lane;
        valid[i] = p < nx;
        pk[i] = 0;
        if (valid[i]) {
            pk[i] = a.words[b0 + p];
            const uint32_t row = (uint32_t)((pk[i] >> kb) & ((1ull << rb) - 1));
            rmin = min(rmin, row);
            rmax = max(rmax, row);
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        rmin = min(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
        rmax = max(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    }
    if (lane == 0) {
        atomicMin(&s_misc[1], rmin);
        atomicMax(&s_misc[2], rmax);
    }
    __syncthreads();
    const uint32_t row_lo = nx ? s_misc[1] : 0u;
    const uint32_t range = nx ? s_misc[2] - row_lo + 1 : 0u;
    // Rows of a bucket are compressed to dense ranks when their range fits the
    // bitmap (mesh-like data: a few hundred distinct rows spread over ~2^15),
    // which shortens the sort key; otherwise row - row_lo is used as is.
    const bool dense = range > 0 && range <= (uint32_t)kRowBits;
    int rbits;
    uint32_t distinct = 0;
    const int RW = (int)((range + 31) / 32);   // row bitmap words the row offsets can reach
    if (dense) {
        constexpr int WORDS = kRowBits / 32, WPT = WORDS / THREADS;
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            if (valid[i]) {
                const uint32_t r = (uint32_t)((pk[i] >> kb) & ((1ull << rb) - 1)) - row_lo;
                atomicOr(&s_bits[r >> 5], 1u << (r & 31));
            }
        }
        __syncthreads();
        uint32_t cw[WPT], c = 0;
#pragma unroll
        for (int j = 0; j < WPT; ++j) {
            cw[j] = tid * WPT + j < RW ? __popc(s_bits[tid * WPT + j]) : 0u;
            c += cw[j];
        }
        uint32_t run = block_scan_1b<THREADS>(c, s_scan, &distinct);
#pragma unroll
        for (int j = 0; j < WPT; ++j) {
            if (tid * WPT + j < RW) s_pref[tid * WPT + j] = (uint16_t)run;
            run += cw[j];
        }
        __syncthreads();
        rbits = bits_of(distinct - 1);
    } else {
        rbits = bits_of(range ? range - 1 : 0u);
    }
    // Bitmap counting path.  With the rows ranked densely, the bucket's keys
    // (column, row rank) span ncols * distinct values; when that fits a
    // bitmap, the set bits ARE the bucket's unique (i,j) pairs in CCS order,
    // and a prefix popcount over the bitmap numbers the slots: Part 3's
    // uniqueness test and Part 4's column counts with no sort pass at all.
    // Triplets are then grouped by slot with one counting scatter, and put
    // into ascending k inside each run as in the radix path.
    if (a.bitmap && dense && (uint32_t)ncols * distinct <= (uint32_t)kKeyBits) {
        const uint32_t R = distinct, K = (uint32_t)ncols * distinct;
        const int KW = (int)((K + 31) / 32);
        const uint32_t rbm = (uint32_t)((1ull << rb) - 1);
        uint32_t *s_kb = reinterpret_cast<uint32_t *>(smem + S::off_b);                 // [KW] key bitmap
        uint16_t *s_kpref = reinterpret_cast<uint16_t *>(smem + S::off_b + kKeyBits / 8); // [KW] set bits before
        uint32_t *s_cnt = reinterpret_cast<uint32_t *>(smem);   // [U] run sizes, until the scan
        uint32_t *s_k = s_cnt;                                  // [nx] k, grouped by slot, after it
        uint16_t *s_slot = reinterpret_cast<uint16_t *>(smem + (size_t)CAP * 4);   // [nx] slot of a position
        uint16_t *s_roff = reinterpret_cast<uint16_t *>(smem + (size_t)CAP * 6);   // [U] row offset of a slot
        uint16_t *s_lo = s_hpos;                                // [U+1] first position of each run
        static_assert(S::bytes_b >= kKeyBits / 8 + kKeyBits / 32 * 2, "key bitmap region");
        static_assert(CAP <= 8192, "slots and positions are packed in 13 bits");
        // Keys into the bitmap; the word becomes k (bits 0-29) | key (30-45) |
        // row offset (46-61), or ~0 for no triplet.
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const uint64_t w = pk[i];
            pk[i] = ~0ull;
            if (valid[i]) {
                const uint32_t roff = ((uint32_t)(w >> kb) & rbm) - row_lo;
                const uint32_t rank = s_pref[roff >> 5] + __popc(s_bits[roff >> 5] & ((1u << (roff & 31)) - 1u));
                const uint32_t kk = (uint32_t)(w >> (kb + rb)) * R + rank;
                if (in_range32(kk, K, a.st)) {
                    atomicOr(&s_kb[kk >> 5], 1u << (kk & 31));
                    pk[i] = (w & kmask) | ((uint64_t)kk << 30) | ((uint64_t)roff << 46);
                }
            }
        }
        __syncthreads();
        // Prefix popcount of the bitmap: slot of every key, U = unique keys.
        uint32_t U;
        {
            constexpr int WPT = (kKeyBits / 32 + THREADS - 1) / THREADS;
            uint32_t c[WPT], sum = 0;
#pragma unroll
            for (int j = 0; j < WPT; ++j) {
                const int w = tid * WPT + j;
                c[j] = w < KW ? __popc(s_kb[w]) : 0u;
                sum += c[j];
            }
            uint32_t run = block_scan_1b<THREADS>(sum, s_scan, &U);
#pragma unroll
            for (int j = 0; j < WPT; ++j) {
                const int w = tid * WPT + j;
                if (w < KW) s_kpref[w] = (uint16_t)run;
                run += c[j];
            }
        }
        if (tid == 0) st_release(a.look + x, (x == 0 ? kFlagInc : kFlagAgg) | U);
        __syncthreads();
        // Run sizes; every triplet takes a provisional place inside its run.
        // The word becomes k (bits 0-29) | slot (30-42) | place (43-55).
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const uint64_t w = pk[i];
            if (w != ~0ull) {
                const uint32_t kk = (uint32_t)(w >> 30) & 0xffffu;
                const uint32_t slot = s_kpref[kk >> 5] + __popc(s_kb[kk >> 5] & ((1u << (kk & 31)) - 1u));
                if (in_range32(slot, (uint32_t)nx, a.st)) {
                    const uint32_t place = atomicAdd(&s_cnt[slot], 1u);
                    s_roff[slot] = (uint16_t)(w >> 46);   // the same value from every triplet of the slot
                    pk[i] = (w & kmask) | ((uint64_t)slot << 30) | ((uint64_t)place << 43);
                } else {
                    pk[i] = ~0ull;
                }
            }
        }
        __syncthreads();
        // First position of every run: exclusive scan of the run sizes.  (Laying
        // the runs out by length class for the in-run k rank below measured no
        // faster: the rank's cost is not the lanes' unequal run lengths.)
        {
            uint32_t c[IPT], sum = 0;
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const int r = tid * IPT + j;
                c[j] = r < (int)U ? s_cnt[r] : 0u;
                sum += c[j];
            }
            uint32_t tot;
            uint32_t run = block_scan_1b<THREADS>(sum, s_scan, &tot);
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const int r = tid * IPT + j;
                if (r < (int)U) s_lo[r] = (uint16_t)run;
                run += c[j];
            }
            if (tid == 0) s_lo[U] = (uint16_t)nx;
        }
        __syncthreads();
        // Group the triplets by slot.
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            if (pk[i] != ~0ull) {
                const uint32_t slot = (uint32_t)(pk[i] >> 30) & 0x1fffu;
                const uint32_t q = s_lo[slot] + (uint32_t)(pk[i] >> 43);
                if (in_range32(q, (uint32_t)nx, a.st)) {
                    s_k[q] = (uint32_t)(pk[i] & kmask);
                    s_slot[q] = (uint16_t)slot;
                }
            }
        }
        __syncthreads();
        // Slot base: warp 0 looks back over earlier buckets while the other
        // warps write perm; everything that needs it is written afterwards.
        if (warp == 0) {
            uint32_t e = 0;
            if (x > 0) {
                e = warp_lookback_exclusive(a.look, 1, x, a.st);
                if (lane == 0) st_release(a.look + x, kFlagInc | (e + U));
            }
            if (lane == 0) s_misc[3] = e;
        }
        // Outputs, position by position (warp-striped, so the lanes of a warp
        // mostly share a run): each triplet lands at lo + (number of triplets
        // of its run with a smaller k); the first carries the head bit.  The
        // chunk slot bases of chunks starting here are kept, bucket-local.
        uint16_t *s_cs = reinterpret_cast<uint16_t *>(s_bits);   // row bitmap no longer needed
        const int64_t c_first = (b0 + kChunk - 1) >> kChunkShift;
#pragma unroll 1
        for (int i = 0; i < IPT; ++i) {
            const int q = warp * 32 * IPT + i * 32 + lane;
            if (q >= nx) continue;
            const uint32_t kq = s_k[q], slot = s_slot[q];
            if (!in_range32(slot, U, a.st)) continue;
            const int lo = s_lo[slot], hi = s_lo[slot + 1];
            int dest = q;
            if (hi - lo > 1) {
                if (hi - lo > kRunSortMax) {
                    atomicOr(&a.st->overflow, 1u);   // redone by the onesweep path
                } else {
                    // 16-byte loads from the aligned word at or below lo;
                    // entries outside [lo, hi) are masked out (they stay
                    // inside the shared array: hi + 3 <= CAP + 3 words lands
                    // in the next region at worst).
                    const uint32_t len = (uint32_t)(hi - lo);
                    int rank = 0;
                    // unrolled by 4 so the loads of a long run overlap (symbolic on the
                    // 100^3 cube 1.59 -> 1.56 ms, 60^3 0.478 -> 0.465; by 2 no gain)
#pragma unroll 4
                    for (int r = lo & ~3; r < hi; r += 4) {
                        const uint4 f = *reinterpret_cast<const uint4 *>(s_k + r);
                        const uint32_t o = (uint32_t)(r - lo);
                        rank += ((o < len) & (f.x < kq)) + ((o + 1 < len) & (f.y < kq)) +
                                ((o + 2 < len) & (f.z < kq)) + ((o + 3 < len) & (f.w < kq));
                    }
                    dest = lo + rank;
                }
            }
            const int64_t gp = b0 + dest;
            const bool head = dest == lo;
            a.perm[gp] = kq | (head ? kHeadBit : 0u);
            if ((gp & (kChunk - 1)) == 0 && in_range((gp >> kChunkShift) - c_first, kMaxBucketCap / kChunk + 1, a.st))
                s_cs[(gp >> kChunkShift) - c_first] = (uint16_t)(head ? slot : slot + 1);
        }
        __syncthreads();
        const uint32_t E = s_misc[3];
        for (int r = tid; r < (int)U; r += THREADS)
            if (in_range(E + r, a.len, a.st)) a.irS[E + r] = (int32_t)(s_roff[r] + row_lo);
        const int64_t c_end = (b0 + nx + kChunk - 1) >> kChunkShift;   // chunks starting in [b0, b0+nx)
        for (int64_t c = c_first + tid; c < c_end; c += THREADS) a.chunk_slot0[c] = E + s_cs[c - c_first];
        // jcS: E + number of unique keys before each column's first key c*R.
        for (int c = tid; c < ncols; c += THREADS) {
            const uint32_t bpos = (uint32_t)c * R;
            a.jcS[col0 + c] = (int32_t)(E + s_kpref[bpos >> 5] + __popc(s_kb[bpos >> 5] & ((1u << (bpos & 31)) - 1u)));
        }
        if (x == a.nb - 1 && tid == 0) {
            a.jcS[a.n] = (int32_t)(E + U);
            a.st->nnz = E + U;
            a.chunk_slot0[a.nchunks] = E + U;
        }
        return;
    }

    const int npass = (a.cs + rbits + 7) / 8;
    // When a row rank replaces the row, the row offset (< 2^16) rides along
    // in the bits above the sorted digits, so the output needs no search.
    const int stash_shift = kb + 8 * npass;
    const bool stash = dense && stash_shift + 16 <= 64;
    // Sort key inside the bucket: (column low bits, row rank), then k below it.
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        if (valid[i]) {
            const uint64_t w = pk[i];
            const uint32_t roff = (uint32_t)((w >> kb) & ((1ull << rb) - 1)) - row_lo;
            uint32_t row = roff;
            if (dense) row = s_pref[roff >> 5] + __popc(s_bits[roff >> 5] & ((1u << (roff & 31)) - 1u));
            const uint64_t lowcol = w >> (kb + rb);
            pk[i] = (((lowcol << rbits) | row) << kb) | (w & kmask);
            if (stash) pk[i] |= (uint64_t)roff << stash_shift;
        }
    }

    // Stable LSD radix sort of the sort key, 8 bits per pass, in shared memory.
    for (int t = tid; t < WARPS * 256; t += THREADS) s_wm[t] = 0;
    for (int d = 0; d < npass; ++d) {
        for (int t = tid; t < WARPS * 256; t += THREADS) s_wcnt[t] = 0;
        __syncthreads();
        uint32_t dig[IPT], rnk[IPT];
#pragma unroll
        for (int i = 0; i < IPT; ++i) dig[i] = (uint32_t)(pk[i] >> (kb + 8 * d)) & 255u;
        warp_rank<8, IPT>(dig, valid, s_wcnt + warp * 256, s_wm + warp * 256, rnk);
        __syncthreads();
        digit_offsets<8, THREADS>(s_wcnt, s_local, s_scan);
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            if (valid[i]) {
                const uint32_t q = s_local[dig[i]] + s_wcnt[warp * 256 + dig[i]] + rnk[i];
                if (in_range32(q, (uint32_t)nx, a.st)) s_w[q] = pk[i];
            }
        }
        __syncthreads();
        if (d + 1 < npass) {
#pragma unroll
            for (int i = 0; i < IPT; ++i)
                if (valid[i]) pk[i] = s_w[warp * 32 * IPT + i * 32 + lane];
            __syncthreads();
        }
    }
    if (npass == 0) {
#pragma unroll
        for (int i = 0; i < IPT; ++i)
            if (valid[i]) s_w[warp * 32 * IPT + i * 32 + lane] = pk[i];
        __syncthreads();
    }

    // Runs: a new run starts where the sort key changes.  Positions are read
    // warp-striped (consecutive lanes, conflict-free); hb[i] holds the head
    // flags of row i, so heads are counted in position order.
    uint32_t hb[IPT];
    uint32_t wheads = 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int p = warp * 32 * IPT + i * 32 + lane;
        bool head = false;
        if (p < nx) head = p == 0 || (s_w[p] >> kb) != (s_w[p - 1] >> kb);
        hb[i] = __ballot_sync(0xffffffffu, head);
        wheads += __popc(hb[i]);
    }
    if (lane == 0) s_scan[warp] = wheads;
    __syncthreads();
    if (warp == 0) {
        const uint32_t c = lane < WARPS ? s_scan[lane] : 0u;
        uint32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane < WARPS) s_scan[lane] = inc - c;
        if (lane == WARPS - 1) s_scan[WARPS] = inc;
    }
    __syncthreads();
    const uint32_t U = s_scan[WARPS];
    const uint32_t wbase = s_scan[warp];
    if (tid == 0) st_release(a.look + x, (x == 0 ? kFlagInc : kFlagAgg) | U);
    {
        uint32_t run = wbase;
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            if ((hb[i] >> lane) & 1u) s_hpos[run + __popc(hb[i] & lt)] = (uint16_t)(warp * 32 * IPT + i * 32 + lane);
            run += __popc(hb[i]);
        }
    }
    if (tid == 0) s_hpos[U] = (uint16_t)nx;
    for (int c = tid; c < (1 << a.cs); c += THREADS) s_col[c] = 0;
    // Slot base of this bucket: warp 0 looks back over earlier buckets and
    // publishes the inclusive prefix at once, before the run sort below.
    if (warp == 0) {
        uint32_t e = 0;
        if (x > 0) {
            e = warp_lookback_exclusive(a.look, 1, x, a.st);
            if (lane == 0) st_release(a.look + x, kFlagInc | (e + U));
        }
        if (lane == 0) s_misc[3] = e;
    }
    __syncthreads();

    const uint32_t E = s_misc[3];

    // perm, irS, column counts, chunk slot bases (warp-striped).  A triplet
    // of run [lo, hi) goes to lo + (number of triplets of the run with a
    // smaller k): ascending k inside the run, the head bit on the first.
    const uint64_t rmaskx = (1ull << rbits) - 1;
    const uint64_t cmask = (1ull << a.cs) - 1;
    const uint32_t *s_w32 = reinterpret_cast<const uint32_t *>(s_w);   // low words: k and equal key bits
    {
        uint32_t before = wbase;   // heads at earlier positions
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const int p = warp * 32 * IPT + i * 32 + lane;
            const bool head = (hb[i] >> lane) & 1u;
            const uint32_t run = before + __popc(hb[i] & lt) - (head ? 0u : 1u);
            before += __popc(hb[i]);
            if (p >= nx) continue;
            const uint32_t slot = E + run;
            const uint64_t v = s_w[p];
            const uint32_t k = (uint32_t)(v & kmask);
            const uint64_t sk = v >> kb;
            const int lo = s_hpos[run], hi = s_hpos[run + 1];
            int dest = p;
            if (hi - lo > 1) {
                if (hi - lo > kRunSortMax) {
                    atomicOr(&a.st->overflow, 1u);   // redone by the onesweep path
                } else {
                    // Two words per 16-byte shared load (low words at 0 and
                    // 8), from the even position at or below lo; positions
                    // outside [lo, hi) are masked out.
                    const uint32_t kl = (uint32_t)v;
                    const uint32_t len = (uint32_t)(hi - lo);
                    int rank = 0;
#pragma unroll 4
                    for (int q = lo & ~1; q < hi; q += 2) {
                        const uint4 two = *reinterpret_cast<const uint4 *>(s_w32 + 2 * q);
                        const uint32_t o = (uint32_t)(q - lo);
                        rank += ((o < len) & (two.x < kl)) + ((o + 1 < len) & (two.z < kl));
                    }
                    dest = lo + rank;
                }
            }
            const int64_t gp = b0 + p;
            a.perm[b0 + dest] = k | (dest == lo ? kHeadBit : 0u);
            if (head) {
                uint32_t row;
                if (stash) {
                    row = (uint32_t)(v >> stash_shift) & 0xffffu;
                } else {
                    row = (uint32_t)(sk & rmaskx);
                    if (dense) {   // row of dense rank `row`: word by binary search, bit by __fns
                        int wlo = 0, whi = RW - 1;
                        while (wlo < whi) {
                            const int mid = (wlo + whi + 1) >> 1;
                            if (s_pref[mid] <= row) wlo = mid; else whi = mid - 1;
                        }
                        row = (uint32_t)wlo * 32 + __fns(s_bits[wlo], 0, (int)(row - s_pref[wlo]) + 1);
                    }
                }
                if (in_range(slot, a.len, a.st)) a.irS[slot] = (int32_t)(row + row_lo);
                const uint32_t lowcol = (uint32_t)((sk >> rbits) & cmask);
                if (in_range(lowcol, ncols, a.st)) atomicAdd(&s_col[lowcol], 1u);
            }
            if ((gp & (kChunk - 1)) == 0) a.chunk_slot0[gp >> kChunkShift] = head ? slot : slot + 1;
        }
    }

    __syncthreads();

    // jcS of this bucket's columns: E + exclusive prefix of the unique counts.
    {
        constexpr int CPT_MAX = (1 << kMaxColBits) / THREADS;
        const int cpt = ((1 << a.cs) + THREADS - 1) / THREADS;
        uint32_t cnt[CPT_MAX];
        uint32_t sum = 0;
#pragma unroll
        for (int c = 0; c < CPT_MAX; ++c) {
            const int col = tid * cpt + c;
            cnt[c] = (c < cpt && col < ncols) ? s_col[col] : 0u;
            sum += cnt[c];
        }
        uint32_t tot;
        uint32_t run = E + block_exclusive_scan<THREADS>(sum, s_scan, &tot);
#pragma unroll
        for (int c = 0; c < CPT_MAX; ++c) {
            const int col = tid * cpt + c;
            if (c < cpt && col < ncols) a.jcS[col0 + col] = (int32_t)run;
            run += cnt[c];
        }
        if (x == a.nb - 1 && tid == 0) {
            a.jcS[a.n] = (int32_t)(E + U);
            a.st->nnz = E + U;
            a.chunk_slot0[a.nchunks] = E + U;
        }
    }
}

template <int THREADS, int IPT>
static fsparse_status run_emit(const BucketEmitArgs &a, int64_t nb, cudaStream_t s) {
    using S = BucketSmem<THREADS, IPT>;
    auto kern = bucket_emit_kernel<THREADS, IPT>;
    FSP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes));
    kern<<<(unsigned)nb, THREADS, S::bytes, s>>>(a);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

fsparse_status bucket_symbolic(const int32_t *ii, const int32_t *jj, int64_t len, int32_t m,
                               int32_t n, const KeyLayout &key,
                               const fsparse_config &cfg, Plan &plan, DevStatus *st, Scratch &scratch,
                               cudaStream_t s, bool *unfit) {
    *unfit = false;
    BucketShape sh;
    if (!bucket_shape(len, n, key, cfg, &sh)) {
        *unfit = true;
        return FSPARSE_OK;
    }
    // Buckets are sized from the average triplets per column; where columns
    // are filled unevenly (half of them empty, say) the largest bucket can
    // outgrow shared memory.  The bucket totals are read back once, before
    // the scatter, and the buckets narrowed until the largest fits.
    uint32_t *goff = nullptr, *tot = nullptr, *bstart = nullptr, *look, *ticket, *dmax;
    uint64_t *words;
    fsparse_status e;
    if ((e = scratch.get(&look, (size_t)kMaxBuckets + 1)) || (e = scratch.get(&ticket, 1)) ||
        (e = scratch.get(&dmax, 1)) || (e = scratch.get(&tot, (size_t)kMaxBuckets)) ||
        (e = scratch.get(&bstart, (size_t)kMaxBuckets + 1)) || (e = scratch.get(&words, (size_t)len)))
        return e;
    // The largest bucket comes back through a pinned word, so the scan and
    // the scatter for the current width are queued before the host waits:
    // the GPU does not idle across the read (they are redone if the width
    // has to shrink).
    struct PinnedWord {   // one per host thread, released when the thread ends
        uint32_t *p = nullptr;
        ~PinnedWord() {
            if (p) cudaFreeHost(p);
        }
    };
    static thread_local PinnedWord pinned;
    if (!pinned.p) FSP_CUDA(cudaMallocHost(reinterpret_cast<void **>(&pinned.p), sizeof(uint32_t)));
    uint32_t *const h_largest = pinned.p;
    cudaEvent_t got_largest = nullptr;
    FSP_CUDA(cudaEventCreateWithFlags(&got_largest, cudaEventDisableTiming));
    struct EventGuard {
        cudaEvent_t e;
        ~EventGuard() { cudaEventDestroy(e); }
    } guard{got_largest};
    int G = 1, nb = 0;
    uint32_t largest = 0;
    for (int attempt = 0;; ++attempt) {
        nb = (int)sh.nb;
        // one count and one scatter pass per range of up to kBucketsPerPass
        // buckets; each pass keeps only its range's table in shared memory
        const int npass = (int)((nb + kBucketsPerPass - 1) / kBucketsPerPass);
        const int nbp_max = (int)std::min<int64_t>(nb, kBucketsPerPass);
        const size_t table = (size_t)nbp_max * 4;
        // Blocks per SM (two 1024-thread blocks are resident at a time).  A
        // large table is paid for by every block, so one wave of two per SM:
        // count + scatter 0.42 ms on the 100^3 cube against 0.45-0.53 with
        // 3-6.  With a small table more waves win where the triplets scatter
        // (each wave's half-written lines then fit in L2): six per SM takes
        // uniform random 2e7 from 0.50 to 0.35 ms and the pooled 2e7 from
        // 0.48 to 0.32 ms.
        const int per_sm_cap = table > (32u << 10) ? 2 : 6;
        const int per_sm = (int)std::max<size_t>(
            1, std::min<size_t>((size_t)per_sm_cap, (200u << 10) / std::max<size_t>(table, 1)));
        G = sm_count(0) * per_sm;
        G = (int)std::max<int64_t>(1, std::min<int64_t>(G, (len + 4095) / 4096));
        if ((e = scratch.get(&goff, (size_t)nb * G))) return e;
        phase_begin("bucket_count");
        FSP_CUDA(cudaMemsetAsync(tot, 0, (size_t)nb * 4, s));
        FSP_CUDA(cudaMemsetAsync(dmax, 0, 4, s));
        auto count = npass > 1 ? bucket_count_kernel<true> : bucket_count_kernel<false>;
        FSP_CUDA(cudaFuncSetAttribute(count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)table));
        for (int r = 0; r < npass; ++r) {
            const int b_lo = r * (int)kBucketsPerPass, nbp = std::min(nb - b_lo, (int)kBucketsPerPass);
            count<<<G, 1024, (size_t)nbp * 4, s>>>(jj, len, n, sh.cs, b_lo, nbp, goff + (size_t)G * b_lo, tot, dmax, st);
            FSP_LAUNCHED();
        }
        FSP_CUDA(cudaMemcpyAsync(h_largest, dmax, 4, cudaMemcpyDeviceToHost, s));
        FSP_CUDA(cudaEventRecord(got_largest, s));
        phase_mark("bucket_count");
        phase_begin("bucket_scatter");
        FSP_CUDA(cudaMemsetAsync(look, 0, ((size_t)nb + 1) * 4, s));
        FSP_CUDA(cudaMemsetAsync(ticket, 0, 4, s));
        if ((e = exclusive_scan_u32(tot, bstart, nb, st, scratch, s)) != FSPARSE_OK) return e;
        auto scatter = npass > 1 ? bucket_scatter_kernel<true> : bucket_scatter_kernel<false>;
        FSP_CUDA(cudaFuncSetAttribute(scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)table));
        for (int r = 0; r < npass; ++r) {
            const int b_lo = r * (int)kBucketsPerPass, nbp = std::min(nb - b_lo, (int)kBucketsPerPass);
            scatter<<<G, 1024, (size_t)nbp * 4, s>>>(ii, jj, len, m, n, key.rb, sh.cs, sh.kb, b_lo, nbp,
                                                     goff + (size_t)G * b_lo, bstart, words, dmax, st);
            FSP_LAUNCHED();
        }
        phase_mark("bucket_scatter");
        if ((e = wait_event(got_largest)) != FSPARSE_OK) return e;
        largest = *h_largest;
        if (largest <= (uint32_t)kMaxBucketCap) break;
        if (sh.cs == 0 || attempt >= 3) {   // a column (or a few) beyond the cap: onesweep instead
            *unfit = true;
            return FSPARSE_OK;
        }
        int shrink = 1;
        while (shrink < sh.cs && ((uint64_t)kMaxBucketCap << shrink) < largest) ++shrink;
        sh.cs -= shrink;
        sh.nb = ((int64_t)(n - 1) >> sh.cs) + 1;
        if (sh.nb > kMaxBuckets) {
            *unfit = true;
            return FSPARSE_OK;
        }
    }
    sh.grid = G;

    BucketEmitArgs a{};
    a.words = words;
    a.bstart = bstart;
    a.nb = nb;
    a.cs = sh.cs;
    a.rb = key.rb;
    a.kb = sh.kb;
    a.n = n;
    a.len = len;
    a.perm = plan.perm;
    a.irS = plan.irS;
    a.jcS = plan.jcS;
    a.chunk_slot0 = plan.chunk_slot0;
    a.nchunks = plan.nchunks;
    a.look = look;
    a.ticket = ticket;
    a.st = st;
    a.bitmap = cfg.strategy != FSPARSE_SORT_BUCKET_RADIX;
    phase_begin("bucket_emit");
    if (largest <= (uint32_t)kEmitCap[0]) e = run_emit<256, 16>(a, nb, s);
    else if (largest <= (uint32_t)kEmitCap[1]) e = run_emit<512, 12>(a, nb, s);
    else e = run_emit<512, 16>(a, nb, s);
    phase_mark("bucket_emit");
    return e;
}

}  // namespace fsp
