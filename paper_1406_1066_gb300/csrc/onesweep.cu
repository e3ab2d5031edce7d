// onesweep.cu -- the general path: a stable LSD radix sort of the packed
// (column, row) keys, then run detection and slot numbering.
//
// The paper (§2.3) reaches the CCS order with two counting passes on a CPU
// (a stable placement by row, then a column sweep that recognises the
// first (row, column) sighting).  Here the same order -- columns, then
// rows, then ascending triplet number k -- comes from a stable least-
// significant-digit radix sort of key = ((j-1) << rb) | (i-1):
//
//   1. one read of ii/jj counts every digit of every pass at once;
//   2. one kernel per digit: each block takes a tile by atomic ticket,
//      ranks its items per digit inside every warp (rank.cuh), publishes
//      its digit counts, resolves its global offsets by decoupled
//      look-back over earlier tiles, and writes the tile out through shared
//      memory so that each digit's run is stored contiguously;
//   3. a pass consumes its digit: the stored key shrinks (64 -> 32 bits ->
//      nothing), and the last pass stores only k, which is the sorted
//      order `perm` itself;
//   4. the emit kernel gathers each sorted triplet's (i, j) back, compares
//      neighbours (a new run starts where the key changes: the collision
//      detection of Part 3), numbers the runs with a block scan plus
//      look-back, and writes irS, the per-column unique counts (scanned into
//      jcS, Part 4) and the numeric chunk slot bases; irank (Eq. (2.2)) is
//      derived from perm on first request.
#include <algorithm>

#include "common.cuh"
#include "internal.hpp"
#include "rank.cuh"

namespace fsp {

// ----------------------------------------------------------------------------
// Implicit dimensions (§2.2) and validation (App. A): max of i and j.
__global__ void minmax_kernel(const int32_t *__restrict__ ii, const int32_t *__restrict__ jj,
                              int64_t len, int32_t m, int32_t n, DevStatus *st) {
    int32_t mi = 0, mj = 0;
    bool bad = false;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < len;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = ii[k], j = jj[k];
        bad |= (i < 1) | (j < 1) | (m > 0 && i > m) | (n > 0 && j > n);
        mi = max(mi, i);
        mj = max(mj, j);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        mi = max(mi, __shfl_xor_sync(0xffffffffu, mi, o));
        mj = max(mj, __shfl_xor_sync(0xffffffffu, mj, o));
    }
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&st->max_i, mi);
        atomicMax(&st->max_j, mj);
        if (bad) atomicOr(&st->bad_index, 1u);
    }
}

fsparse_status launch_minmax(const int32_t *ii, const int32_t *jj, int64_t len, int32_t m,
                             int32_t n, DevStatus *st, cudaStream_t s) {
    if (len == 0) return FSPARSE_OK;
    int grid = (int)std::min<int64_t>((len + 255) / 256, (int64_t)sm_count(0) * 8);
    minmax_kernel<<<grid, 256, 0, s>>>(ii, jj, len, m, n, st);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

__device__ __forceinline__ uint64_t make_key(int32_t i, int32_t j, int rb) {
    return ((uint64_t)(uint32_t)(j - 1) << rb) | (uint32_t)(i - 1);
}

// ----------------------------------------------------------------------------
// All digit histograms in one read of ii/jj (validation fused).  Every warp
// counts into its own copy of the tables (fewer colliding shared atomics),
// and each thread takes four triplets per step (16-byte loads when aligned).
template <int R>
__device__ __forceinline__ void hist_add(uint32_t *my, uint64_t key, int npass) {
    constexpr int RADIX = 1 << R;
    for (int d = 0; d < npass; ++d) atomicAdd(&my[d * RADIX + (int)((key >> (d * R)) & (RADIX - 1))], 1u);
}

template <int R>
__global__ void digit_hist_kernel(const int32_t *__restrict__ ii, const int32_t *__restrict__ jj,
                                  int64_t len, int32_t m, int32_t n, int rb, int npass,
                                  uint32_t *hist, DevStatus *st) {
    constexpr int RADIX = 1 << R;
    extern __shared__ uint32_t s_hist[];   // [warps][npass * RADIX]
    const int nb = npass * RADIX, warps = blockDim.x >> 5;
    uint32_t *my = s_hist + (threadIdx.x >> 5) * nb;
    for (int t = threadIdx.x; t < warps * nb; t += blockDim.x) s_hist[t] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t done = 0;
    if (((reinterpret_cast<uintptr_t>(ii) | reinterpret_cast<uintptr_t>(jj)) & 15) == 0) {
        const int64_t n4 = len / 4;
        for (int64_t q = t0; q < n4; q += stride) {
            const int4 a = reinterpret_cast<const int4 *>(ii)[q];
            const int4 b = reinterpret_cast<const int4 *>(jj)[q];
            hist_add<R>(my, make_key(checked_index(a.x, m, st), checked_index(b.x, n, st), rb), npass);
            hist_add<R>(my, make_key(checked_index(a.y, m, st), checked_index(b.y, n, st), rb), npass);
            hist_add<R>(my, make_key(checked_index(a.z, m, st), checked_index(b.z, n, st), rb), npass);
            hist_add<R>(my, make_key(checked_index(a.w, m, st), checked_index(b.w, n, st), rb), npass);
        }
        done = n4 * 4;
    }
    for (int64_t k = done + t0; k < len; k += stride)
        hist_add<R>(my, make_key(checked_index(ii[k], m, st), checked_index(jj[k], n, st), rb), npass);
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        uint32_t c = 0;
        for (int w = 0; w < warps; ++w) c += s_hist[w * nb + t];
        if (c) atomicAdd(&hist[t], c);
    }
}

template <int R>
__global__ void digit_offsets_kernel(const uint32_t *hist, uint32_t *offs) {
    constexpr int RADIX = 1 << R;
    __shared__ uint32_t scratch[RADIX / 32 + 1];
    const int d = blockIdx.x;
    uint32_t total;
    uint32_t x = hist[d * RADIX + threadIdx.x];
    offs[d * RADIX + threadIdx.x] = block_exclusive_scan<RADIX>(x, scratch, &total);
}

// ----------------------------------------------------------------------------
// One digit pass.
enum KeyFmt : int { FMT_NONE = 0, FMT_U64 = 1, FMT_U32 = 2, FMT_IJ = 3 };

struct PassArgs {
    const int32_t *ii, *jj;
    int32_t m, n;
    int rb;
    const void *kin;
    const uint32_t *vin;
    int in_fmt;
    void *kout;
    uint32_t *vout;
    int out_fmt;
    int shift;                 // this pass's digit is (key >> shift) & (RADIX - 1)
    int64_t len;
    const uint32_t *bin_off;   // [RADIX] exclusive global offsets of this digit
    uint32_t *look;            // [ntiles][RADIX] look-back words
    uint32_t *ticket;
    DevStatus *st;
    int withhold_first;        // injected failure: tile 0 never publishes its counts
};

template <int R, int THREADS, int ITEMS>
struct PassSmem {
    static constexpr int RADIX = 1 << R, WARPS = THREADS / 32, TILE = THREADS * ITEMS;
    static constexpr size_t bytes = TILE * 8 + TILE * 4 + 2 * WARPS * RADIX * 4 + RADIX * 4 * 3 +
                                    (THREADS / 32 + 2) * 4 + 16;
};

template <int R, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS) onesweep_pass_kernel(PassArgs a) {
    using S = PassSmem<R, THREADS, ITEMS>;
    constexpr int RADIX = S::RADIX, WARPS = S::WARPS, TILE = S::TILE;
    constexpr uint32_t MASK = RADIX - 1;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *s_keys = reinterpret_cast<uint64_t *>(smem);
    uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_keys + TILE);
    uint32_t *s_wcnt = s_vals + TILE;                 // [WARPS][RADIX]
    uint32_t *s_wm = s_wcnt + WARPS * RADIX;          // [WARPS][RADIX] peer masks
    uint32_t *s_local = s_wm + WARPS * RADIX;         // [RADIX] tile-local digit start
    uint32_t *s_global = s_local + RADIX;             // [RADIX] global digit start of this tile
    uint32_t *s_total = s_global + RADIX;             // [RADIX]
    uint32_t *s_scan = s_total + RADIX;               // block scan scratch
    uint32_t *s_tile = s_scan + THREADS / 32 + 1;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) *s_tile = atomicAdd(a.ticket, 1u);
    for (int t = tid; t < WARPS * RADIX; t += THREADS) {
        s_wcnt[t] = 0;
        s_wm[t] = 0;
    }
    __syncthreads();
    const int64_t tile = *s_tile;
    const int64_t base = tile * TILE;
    const int count = (int)min64(TILE, a.len - base);

    // Warp-striped load: item i of lane l sits at base + warp*32*ITEMS + i*32 + l,
    // so visiting (i, lane) in order visits positions in order (stability).
    uint64_t key[ITEMS];
    uint32_t val[ITEMS];
    uint32_t rnk[ITEMS];
    const int64_t wbase = base + (int64_t)warp * 32 * ITEMS + lane;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int64_t p = wbase + i * 32;
        key[i] = 0;
        val[i] = 0;
        if (p < a.len) {
            if (a.in_fmt == FMT_IJ) {
                key[i] = make_key(checked_index(a.ii[p], a.m, a.st),
                                  checked_index(a.jj[p], a.n, a.st), a.rb);
                val[i] = (uint32_t)p;
            } else {
                key[i] = a.in_fmt == FMT_U64 ? static_cast<const uint64_t *>(a.kin)[p]
                                             : static_cast<const uint32_t *>(a.kin)[p];
                val[i] = a.vin[p];
            }
        }
    }

    // Warp-level stable ranking: peers = lanes holding the same digit.
    uint32_t dig[ITEMS];
    bool valid[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        valid[i] = wbase + i * 32 < a.len;
        dig[i] = (uint32_t)((key[i] >> a.shift) & MASK);
    }
    warp_rank<R, ITEMS>(dig, valid, s_wcnt + warp * RADIX, s_wm + warp * RADIX, rnk);
    __syncthreads();

    // Per digit: exclusive offsets across warps, tile total.  Each thread
    // owns DPT consecutive digits (more than one when the radix exceeds the
    // block: 9- and 10-bit digits in 256-thread passes).
    constexpr int DPT = RADIX > THREADS ? RADIX / THREADS : 1;
    static_assert(RADIX <= THREADS || RADIX % THREADS == 0, "digits split evenly over the threads");
    const int d0 = tid * DPT;
    const bool owner = d0 < RADIX;
    uint32_t tot[DPT];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
        tot[j] = 0;
        if (owner) {
            const int d = d0 + j;
            for (int w = 0; w < WARPS; ++w) {
                const uint32_t c = s_wcnt[w * RADIX + d];
                s_wcnt[w * RADIX + d] = tot[j];
                tot[j] += c;
            }
            s_total[d] = tot[j];
            sum += tot[j];
        }
    }
    uint32_t tile_sum;
    uint32_t local = block_exclusive_scan<THREADS>(owner ? sum : 0, s_scan, &tile_sum);
    if (owner) {
        // every aggregate is published before any wait, so the successors'
        // look-backs never wait on this thread's own waits
#pragma unroll
        for (int j = 0; j < DPT; ++j) {
            const int d = d0 + j;
            s_local[d] = local;
            local += tot[j];
            uint32_t *word = a.look + tile * RADIX + d;
            if (tile == 0) {
                s_global[d] = a.bin_off[d];
                if (!a.withhold_first) st_release(word, kFlagInc | (a.bin_off[d] + tot[j]));
            } else {
                st_release(word, kFlagAgg | tot[j]);
            }
        }
        if (tile > 0) {
#pragma unroll
            for (int j = 0; j < DPT; ++j) {
                const int d = d0 + j;
                const uint32_t excl = lookback_exclusive(a.look + d, RADIX, tile, a.st);
                st_release(a.look + tile * RADIX + d, kFlagInc | (excl + tot[j]));
                s_global[d] = excl;
            }
        }
    }
    __syncthreads();

    // Place items tile-locally in digit order, then stream them out.
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (wbase + i * 32 < a.len) {
            const uint32_t d = dig[i];
            const uint32_t q = s_local[d] + s_wcnt[warp * RADIX + d] + rnk[i];
            if (in_range(q, count, a.st)) {
                s_keys[q] = key[i];
                s_vals[q] = val[i];
            }
        }
    }
    __syncthreads();
    for (int j = tid; j < count; j += THREADS) {
        const uint64_t k = s_keys[j];
        const uint32_t d = (uint32_t)((k >> a.shift) & MASK);
        const int64_t g = (int64_t)s_global[d] + (j - (int64_t)s_local[d]);
        if (!in_range(g, a.len, a.st)) continue;
        if (a.out_fmt == FMT_U64)
            static_cast<uint64_t *>(a.kout)[g] = k;
        else if (a.out_fmt == FMT_U32)
            static_cast<uint32_t *>(a.kout)[g] = (uint32_t)k;
        a.vout[g] = s_vals[j];
    }
}

// ----------------------------------------------------------------------------
template <int R, int THREADS, int ITEMS>
static fsparse_status run_pass(const PassArgs &a, int64_t ntiles, cudaStream_t s) {
    using S = PassSmem<R, THREADS, ITEMS>;
    auto kern = onesweep_pass_kernel<R, THREADS, ITEMS>;
    FSP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes));
    kern<<<(unsigned)ntiles, THREADS, S::bytes, s>>>(a);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

template <int R>
static fsparse_status run_hist(const int32_t *ii, const int32_t *jj, int64_t len, int32_t m,
                               int32_t n, int rb, int npass, uint32_t *hist, uint32_t *offs,
                               DevStatus *st, cudaStream_t s) {
    constexpr int RADIX = 1 << R;
    int grid = (int)std::min<int64_t>((len + 4095) / 4096, (int64_t)sm_count(0) * 4);
    grid = std::max(grid, 1);
    const size_t smem = (size_t)(256 / 32) * npass * RADIX * 4;
    FSP_CUDA(cudaFuncSetAttribute(digit_hist_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    digit_hist_kernel<R><<<grid, 256, smem, s>>>(ii, jj, len, m, n, rb, npass, hist, st);
    FSP_LAUNCHED();
    digit_offsets_kernel<R><<<npass, RADIX, 0, s>>>(hist, offs);
    FSP_LAUNCHED();
    return FSPARSE_OK;
}

using PassFn = fsparse_status (*)(const PassArgs &, int64_t, cudaStream_t);

static PassFn pick_pass(int R, int threads, int items) {
#define FSP_PASS(r, t, i) \
    if (R == r && threads == t && items == i) return &run_pass<r, t, i>;
#define FSP_PASS_R(r) \
    FSP_PASS(r, 256, 8) FSP_PASS(r, 256, 12) FSP_PASS(r, 256, 16) \
    FSP_PASS(r, 512, 8) FSP_PASS(r, 512, 12) FSP_PASS(r, 512, 16)
#define FSP_PASS_R256(r) FSP_PASS(r, 256, 8) FSP_PASS(r, 256, 12) FSP_PASS(r, 256, 16)
    FSP_PASS_R(6)
    FSP_PASS_R(7)
    FSP_PASS_R(8)
    FSP_PASS_R256(9)
    FSP_PASS_R256(10)
#undef FSP_PASS_R256
#undef FSP_PASS_R
#undef FSP_PASS
    return nullptr;
}

fsparse_status onesweep_sort(const int32_t *ii, const int32_t *jj, int64_t len, int32_t m,
                             int32_t n, const KeyLayout &key, const fsparse_config &cfg,
                             uint32_t *perm_out, const void **keys_out, int *key_bytes, DevStatus *st,
                             Scratch &scratch, cudaStream_t s) {
    *keys_out = nullptr;
    *key_bytes = 0;
    const int KB = key.total();
    const int R = cfg.radix_bits;
    const int RADIX = 1 << R;
    const int npass = (KB + R - 1) / R;
    if (len == 0) return FSPARSE_OK;
    if (npass == 0) return launch_iota(perm_out, len, s);   // a single (1,1) key: identity order
    PassFn pass = pick_pass(R, cfg.sweep_threads, cfg.sweep_items);
    if (!pass) return set_error(FSPARSE_ERR_ARG, "unsupported onesweep configuration");

    uint32_t *hist, *offs;
    fsparse_status e;
    if ((e = scratch.get(&hist, (size_t)npass * RADIX)) != FSPARSE_OK) return e;
    if ((e = scratch.get(&offs, (size_t)npass * RADIX)) != FSPARSE_OK) return e;
    phase_begin("digit_hist");
    FSP_CUDA(cudaMemsetAsync(hist, 0, (size_t)npass * RADIX * 4, s));
    if (R == 6) e = run_hist<6>(ii, jj, len, m, n, key.rb, npass, hist, offs, st, s);
    else if (R == 7) e = run_hist<7>(ii, jj, len, m, n, key.rb, npass, hist, offs, st, s);
    else if (R == 8) e = run_hist<8>(ii, jj, len, m, n, key.rb, npass, hist, offs, st, s);
    else if (R == 9) e = run_hist<9>(ii, jj, len, m, n, key.rb, npass, hist, offs, st, s);
    else if (R == 10) e = run_hist<10>(ii, jj, len, m, n, key.rb, npass, hist, offs, st, s);
    else return set_error(FSPARSE_ERR_ARG, "unsupported digit width");
    if (e != FSPARSE_OK) return e;
    phase_mark("digit_hist");
    phase_begin("digit_passes");

    const int64_t tile = (int64_t)cfg.sweep_threads * cfg.sweep_items;
    const int64_t ntiles = (len + tile - 1) / tile;
    uint32_t *look, *tickets;
    if ((e = scratch.get(&look, (size_t)npass * ntiles * RADIX)) != FSPARSE_OK) return e;
    if ((e = scratch.get(&tickets, (size_t)npass)) != FSPARSE_OK) return e;
    FSP_CUDA(cudaMemsetAsync(look, 0, (size_t)npass * ntiles * RADIX * 4, s));
    FSP_CUDA(cudaMemsetAsync(tickets, 0, (size_t)npass * 4, s));

    // Every pass carries the whole key (digits are taken by shifting), so the
    // sorted keys come out beside perm and the emit reads them in order
    // instead of gathering ii/jj through perm.
    const int kfmt = KB > 32 ? FMT_U64 : FMT_U32;
    const size_t kbytes = KB > 32 ? 8 : 4;
    void *kbuf[2] = {nullptr, nullptr};
    uint32_t *vbuf[2] = {nullptr, nullptr};
    if ((e = scratch.alloc(&kbuf[0], (size_t)len * kbytes)) != FSPARSE_OK) return e;
    if (npass > 1) {
        if ((e = scratch.alloc(&kbuf[1], (size_t)len * kbytes)) != FSPARSE_OK) return e;
        if ((e = scratch.get(&vbuf[0], (size_t)len)) != FSPARSE_OK) return e;
    }
    if (npass > 2) {
        if ((e = scratch.get(&vbuf[1], (size_t)len)) != FSPARSE_OK) return e;
    }
    for (int d = 0; d < npass; ++d) {
        PassArgs a{};
        a.ii = ii;
        a.jj = jj;
        a.m = m;
        a.n = n;
        a.rb = key.rb;
        a.len = len;
        a.st = st;
        a.bin_off = offs + (size_t)d * RADIX;
        a.look = look + (size_t)d * ntiles * RADIX;
        a.ticket = tickets + d;
        a.withhold_first = d == 0 && injected_fault() == FAULT_TIMEOUT_SORT ? 1 : 0;
        a.shift = d * R;
        a.in_fmt = d == 0 ? FMT_IJ : kfmt;
        a.kin = d == 0 ? nullptr : kbuf[(d - 1) & 1];
        a.vin = d == 0 ? nullptr : vbuf[(d - 1) & 1];
        a.out_fmt = kfmt;
        a.kout = kbuf[d & 1];
        a.vout = d == npass - 1 ? perm_out : vbuf[d & 1];
        if ((e = pass(a, ntiles, s)) != FSPARSE_OK) return e;
    }
    *keys_out = kbuf[(npass - 1) & 1];
    *key_bytes = (int)kbytes;
    phase_mark("digit_passes");
    return FSPARSE_OK;
}

// ----------------------------------------------------------------------------
// Emit: runs, slots, irS, column counts and numeric chunk slot bases.
struct EmitArgs {
    const void *keys;        // sorted (column, row) keys, key_bytes wide; NULL: all equal
    int key_bytes;
    int rb;
    uint32_t *perm;          // in: sorted k, out: k | kHeadBit on run heads
    int32_t *irS;
    uint32_t *colcnt;        // [n] unique pairs per column (zeroed)
    int32_t n;               // columns (bound of every colcnt index)
    uint32_t *chunk_slot0;   // [nchunks + 1]
    int64_t nchunks;
    int64_t len;
    uint32_t *look;
    uint32_t *ticket;
    DevStatus *st;
};

__device__ __forceinline__ uint64_t sorted_key(const EmitArgs &a, int64_t p) {
    if (!a.keys) return 0;
    return a.key_bytes == 8 ? static_cast<const uint64_t *>(a.keys)[p]
                            : static_cast<const uint32_t *>(a.keys)[p];
}

template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS) emit_kernel(EmitArgs a) {
    constexpr int TILE = THREADS * ITEMS;
    __shared__ uint32_t s_scan[THREADS / 32 + 1];
    __shared__ uint32_t s_tile, s_excl;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) s_tile = atomicAdd(a.ticket, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t p0 = tile * TILE + (int64_t)tid * ITEMS;

    uint32_t k[ITEMS];
    uint64_t key[ITEMS];
    if (p0 + ITEMS <= a.len) {
#pragma unroll
        for (int v = 0; v < ITEMS / 4; ++v) {
            const uint4 q = reinterpret_cast<const uint4 *>(a.perm + p0)[v];
            k[4 * v] = q.x;
            k[4 * v + 1] = q.y;
            k[4 * v + 2] = q.z;
            k[4 * v + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) k[i] = p0 + i < a.len ? a.perm[p0 + i] : 0u;
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) key[i] = p0 + i < a.len ? sorted_key(a, p0 + i) : 0;
    // Key of the position just before this thread's first one.
    uint64_t prev = __shfl_up_sync(0xffffffffu, key[ITEMS - 1], 1);
    if (lane == 0 && p0 > 0 && p0 <= a.len) prev = sorted_key(a, p0 - 1);
    uint32_t heads = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int64_t p = p0 + i;
        const uint64_t before = i == 0 ? prev : key[i - 1];
        if (p < a.len && (p == 0 || key[i] != before)) heads |= 1u << i;
    }
    uint32_t tile_heads;
    const uint32_t mine = block_exclusive_scan<THREADS>(__popc(heads), s_scan, &tile_heads);
    if (tid < 32) {
        uint32_t *word = a.look + tile;
        uint32_t excl = 0;
        if (tid == 0) st_release(word, (tile == 0 ? kFlagInc : kFlagAgg) | tile_heads);
        if (tile > 0) {
            excl = warp_lookback_exclusive(a.look, 1, tile, a.st);
            if (tid == 0) st_release(word, kFlagInc | (excl + tile_heads));
        }
        if (tid == 0) s_excl = excl;
    }
    __syncthreads();

    uint32_t slot = s_excl + mine - 1;   // becomes the slot of each position after its head count
    uint32_t run_col = 0xffffffffu, run_cnt = 0;
    uint32_t out[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int64_t p = p0 + i;
        if (p >= a.len) {
            out[i] = 0;
            continue;
        }
        const bool head = (heads >> i) & 1u;
        slot += head;
        const uint32_t kk = k[i] & kIndexMask;
        out[i] = kk | (head ? kHeadBit : 0u);
        if (head) {
            const uint32_t row = (uint32_t)(key[i] & ((1ull << a.rb) - 1));
            const uint32_t col = (uint32_t)(key[i] >> a.rb);
            if (in_range(slot, a.len, a.st)) a.irS[slot] = (int32_t)row;
            if (col != run_col) {
                if (run_cnt && in_range(run_col, a.n, a.st)) atomicAdd(&a.colcnt[run_col], run_cnt);
                run_col = col;
                run_cnt = 0;
            }
            ++run_cnt;
        }
        if ((p & (kChunk - 1)) == 0) a.chunk_slot0[p >> kChunkShift] = head ? slot : slot + 1;
        if (p == a.len - 1) {
            a.st->nnz = slot + 1;
            a.chunk_slot0[a.nchunks] = slot + 1;
        }
    }
    // (sorted keys left over from an earlier call, after a digit pass whose
    // wait gave up, can name any column: the bound keeps the add in place)
    if (run_cnt && in_range(run_col, a.n, a.st)) atomicAdd(&a.colcnt[run_col], run_cnt);
    if (p0 + ITEMS <= a.len) {
#pragma unroll
        for (int v = 0; v < ITEMS / 4; ++v)
            reinterpret_cast<uint4 *>(a.perm + p0)[v] =
                make_uint4(out[4 * v], out[4 * v + 1], out[4 * v + 2], out[4 * v + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
            if (p0 + i < a.len) a.perm[p0 + i] = out[i];
    }
}

fsparse_status emit_from_perm(const void *keys, int key_bytes, int64_t len, int32_t n,
                              const KeyLayout &key, Plan &plan, DevStatus *st, Scratch &scratch,
                              cudaStream_t s) {
    constexpr int THREADS = 256, ITEMS = 8, TILE = THREADS * ITEMS;
    const int64_t ntiles = (len + TILE - 1) / TILE;
    uint32_t *colcnt, *look, *ticket;
    fsparse_status e;
    if ((e = scratch.get(&colcnt, (size_t)n + 1)) != FSPARSE_OK) return e;
    if ((e = scratch.get(&look, (size_t)ntiles + 1)) != FSPARSE_OK) return e;
    if ((e = scratch.get(&ticket, 1)) != FSPARSE_OK) return e;
    FSP_CUDA(cudaMemsetAsync(colcnt, 0, ((size_t)n + 1) * 4, s));
    FSP_CUDA(cudaMemsetAsync(look, 0, ((size_t)ntiles + 1) * 4, s));
    FSP_CUDA(cudaMemsetAsync(ticket, 0, 4, s));
    phase_begin("emit");
    if (len > 0) {
        EmitArgs a{};
        a.keys = keys;
        a.key_bytes = key_bytes;
        a.rb = key.rb;
        a.perm = plan.perm;
        a.irS = plan.irS;
        a.colcnt = colcnt;
        a.n = n;
        a.chunk_slot0 = plan.chunk_slot0;
        a.nchunks = plan.nchunks;
        a.len = len;
        a.look = look;
        a.ticket = ticket;
        a.st = st;
        emit_kernel<THREADS, ITEMS><<<(unsigned)ntiles, THREADS, 0, s>>>(a);
        FSP_LAUNCHED();
        phase_mark("emit");
    }
    phase_begin("jcS_scan");
    e = exclusive_scan_u32(colcnt, reinterpret_cast<uint32_t *>(plan.jcS), n, st, scratch, s);
    phase_mark("jcS_scan");
    return e;
}

}  // namespace fsp
