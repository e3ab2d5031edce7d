// internal.hpp -- host-side types shared by the fsparse translation units.
#pragma once

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/fsparse.h"

namespace fsp {

struct DevStatus;

// Streams on which a plan's (or batch's) arrays were read by launches that
// outlive the call (numeric, adjoint, irank derivation), each with an event
// recorded after its latest such launch.  The arrays are released only after
// these events, on a library stream: destroying never stalls the device.
// Launches captured into a CUDA graph are not recorded (an event recorded in
// a capture belongs to the graph); replays are the caller's to finish.
struct UseLog {
    static constexpr int kMax = 8;
    std::mutex mu;           // numeric calls on one plan may come from several host threads
    cudaStream_t stream[kMax] = {};
    cudaEvent_t event[kMax] = {};
    int n = 0;
    bool overflow = false;   // more streams than kMax: the release waits for the device
};
void note_use(UseLog &log, cudaStream_t s);

// Number of bits needed for the values 0..x (0 for x == 0).
inline int bits_for(uint64_t x) {
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

// Packed sort key of one triplet: ((j-1) << rb) | (i-1), column-major CCS order.
struct KeyLayout {
    int rb = 0;   // row bits, bits_for(m-1)
    int cb = 0;   // column bits, bits_for(n-1)
    int total() const { return rb + cb; }
};

// Everything the symbolic phase leaves behind (the reusable "quasi assembly"
// state): the CCS pattern, the triplet->slot map and the sorted-order map
// that drives the numeric fold.
struct Plan {
    int device = 0;
    int32_t m = 0, n = 0;
    int64_t len = 0, nnz = 0, cap = 0;
    KeyLayout key;
    int32_t *irank = nullptr;        // [len], filled on first request (irank_ready)
    bool irank_ready = false;
    int32_t *jcS = nullptr;          // [n+1]
    int32_t *irS = nullptr;          // [max(len, nzmax, 1)]
    uint32_t *perm = nullptr;        // [len] sorted position -> k, kHeadBit on run heads
    uint32_t *chunk_slot0 = nullptr; // [nchunks+1] runs that start before each kChunk positions
    int numeric_tile = 1024;         // positions per numeric block
    int64_t nchunks = 0;
    fsparse_config cfg{};            // configuration that built this plan
    UseLog uses;                     // streams whose launches may still read the arrays
};

struct Batch {
    int device = 0;
    int32_t count = 0;
    int64_t total_len = 0, total_nnz = 0;
    int64_t *h_len_off = nullptr;    // host [count+1]
    int64_t *h_nnz_off = nullptr;    // host [count+1]
    uint32_t *perm = nullptr;        // [total_len], k offset into the concatenation
    uint32_t *chunk_slot0 = nullptr; // [nchunks+1]
    int numeric_tile = 1024;
    int64_t nchunks = 0;
    UseLog uses;
    // Set only by fsparse_batch_symbolic (a batch made from plans leaves the
    // CCS arrays in its plans).
    bool symbolic = false;
    int32_t *irank = nullptr;        // [total_len] instance-local slots, derived on first request
    bool irank_ready = false;
    int32_t *jcS = nullptr;          // [sum(n_b + 1)] per-instance column pointers, concatenated
    int32_t *irS = nullptr;          // [total_nnz] per-instance rows, concatenated
    int64_t *d_len_off = nullptr;    // device copies of the offsets [count+1]
    int64_t *d_nnz_off = nullptr;
    int32_t *h_m = nullptr;          // host [count] resolved dimensions
    int32_t *h_n = nullptr;
};

// ---- errors ---------------------------------------------------------------
fsparse_status set_error(fsparse_status st, const std::string &msg);
fsparse_status cuda_error(cudaError_t e, const char *what);
// Host waits that poll briefly before blocking (api.cu).
fsparse_status wait_stream(cudaStream_t s);
fsparse_status wait_event(cudaEvent_t e);

// Host-side fault injection for the failure paths, read from the environment
// at each call: FSPARSE_FAULT=alloc makes every device allocation report
// out-of-memory; FSPARSE_FAULT=timeout makes the first tile of each
// look-back scan withhold its prefix, so the following tiles' bounded waits
// run out and the call returns FSPARSE_ERR_TIMEOUT; FSPARSE_FAULT=timeout_sort
// does the same in the first digit pass of the onesweep sort, so that pass
// leaves some positions unwritten and the kernels after it read stale keys;
// FSPARSE_FAULT=index seeds the device status word with a bad index after the
// symbolic kernels, so the call takes its bad-index return on valid input.
// Nothing faults, traps or hangs the GPU; unset, it costs one getenv per call.
enum InjectedFault { FAULT_NONE = 0, FAULT_ALLOC = 1, FAULT_TIMEOUT = 2, FAULT_TIMEOUT_SORT = 3, FAULT_INDEX = 4 };
int injected_fault();

// Per-phase timing of one symbolic call with CUDA events on its stream, on
// when FSPARSE_TIMING=1.  symbolic_impl owns the timer of the calling thread;
// the host launchers mark the end of each phase with phase_mark(name), which
// does nothing when timing is off.  The durations of the thread's last timed
// call are read with fsparse_last_timings.
void phase_mark(const char *name);
// NVTX range of the phase that starts here (closed by the next phase_mark,
// or at the end of the entry point).
void phase_begin(const char *name);

// NVTX range over a host scope (an entry point or one phase of it): tools
// such as Nsight Systems show it on the host timeline and tie the kernels
// launched inside it to it.  Header-only NVTX; a few ns when no tool listens.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define FSP_CUDA(call)                                                        \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return ::fsp::cuda_error(e_, #call);           \
    } while (0)

// ---- launch accounting -----------------------------------------------------
extern std::atomic<int64_t> g_launches;
inline void count_launch(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }
#define FSP_LAUNCHED()                                                        \
    do {                                                                      \
        ::fsp::count_launch();                                                \
        cudaError_t e_ = cudaGetLastError();                                  \
        if (e_ != cudaSuccess) return ::fsp::cuda_error(e_, "kernel launch"); \
    } while (0)

int sm_count(int device);

// ---- configuration ----------------------------------------------------------
fsparse_config resolve_config(int64_t len, const KeyLayout &key);
bool config_valid(const fsparse_config &c);
fsparse_config default_config(int64_t len, const KeyLayout &key);

// ---- stream-ordered scratch -------------------------------------------------
// Allocations made during a call and released (stream-ordered) at its end.
class Scratch {
  public:
    explicit Scratch(cudaStream_t s) : s_(s) {}
    // Bump allocation from caller-provided device memory instead of the pool
    // (nothing is allocated or freed; used by fsparse_assemble_noalloc).
    Scratch(cudaStream_t s, void *arena, size_t bytes) : s_(s), arena_(static_cast<char *>(arena)), arena_bytes_(bytes) {}
    ~Scratch();
    fsparse_status alloc(void **p, size_t bytes);
    // Queue the frees of everything allocated so far (stream-ordered after
    // the work already on the stream); the object can allocate again.
    void release();
    template <class T>
    fsparse_status get(T **p, size_t count) {
        return alloc(reinterpret_cast<void **>(p), count * sizeof(T));
    }

  private:
    cudaStream_t s_;
    void *ptrs_[32] = {};
    int n_ = 0;
    char *arena_ = nullptr;
    size_t arena_bytes_ = 0, arena_used_ = 0;
};

fsparse_status device_alloc(void **p, size_t bytes, cudaStream_t s);

// ---- kernel launchers (one per translation unit) ------------------------------
// All return FSPARSE_OK or an error status; none synchronises.

// Implicit dimensions and validation when m or n is zero.
fsparse_status launch_minmax(const int32_t *ii, const int32_t *jj, int64_t len, int32_t m,
                             int32_t n, DevStatus *st, cudaStream_t s);

// Global stable LSD radix sort (one kernel per digit) producing perm[len]
// (sorted position -> k) and the sorted (column, row) keys (*keys_out, in
// scratch, *key_bytes = 4 or 8; NULL when every key is equal).  Tile/radix
// from cfg.
fsparse_status onesweep_sort(const int32_t *ii, const int32_t *jj, int64_t len, int32_t m,
                             int32_t n, const KeyLayout &key, const fsparse_config &cfg,
                             uint32_t *perm_out, const void **keys_out, int *key_bytes, DevStatus *st,
                             Scratch &scratch, cudaStream_t s);

// Run detection + slots + irS + column counts + chunk slot bases from a
// sorted perm and its sorted keys.
fsparse_status emit_from_perm(const void *keys, int key_bytes, int64_t len, int32_t n,
                              const KeyLayout &key, Plan &plan, DevStatus *st, Scratch &scratch,
                              cudaStream_t s);

// Exclusive scan of counts[count] into out[count+1] (out[count] = total).
fsparse_status exclusive_scan_u32(const uint32_t *counts, uint32_t *out, int64_t count,
                                  DevStatus *st, Scratch &scratch, cudaStream_t s);

// Numeric fold prS[slot] over perm and the chunk slot bases; tail [nnz, cap)
// zero-filled.  block_positions: 1024, 2048 or 4096.
fsparse_status launch_numeric(const uint32_t *perm, const uint32_t *chunk_slot0, int64_t len,
                              int block_positions, const double *sr, double *prS, int64_t nnz,
                              int64_t cap, cudaStream_t s);
fsparse_status launch_adjoint(const int32_t *irank, int64_t len, const double *dprS, double *ds,
                              int64_t nnz, cudaStream_t s);
fsparse_status launch_irank(const uint32_t *perm, const uint32_t *chunk_slot0, int64_t len,
                            int32_t *irank, cudaStream_t s);
fsparse_status launch_fill(int32_t *irS, double *prS, int64_t from, int64_t to, cudaStream_t s);
fsparse_status launch_iota(uint32_t *perm, int64_t len, cudaStream_t s);
fsparse_status launch_getix(const double *ival, int64_t len, int32_t *out, cudaStream_t s);
// Delayed assembly: merge plan a with the plan b of appended triplets into out.
fsparse_status append_merge(const Plan &a, const Plan &b, Plan &out, DevStatus *st, Scratch &scratch,
                            cudaStream_t s);
fsparse_status launch_batch_concat(const uint32_t *src, uint32_t *dst, int64_t len,
                                   uint32_t offset, cudaStream_t s);
fsparse_status launch_chunk_heads(const uint32_t *perm, int64_t len, uint32_t *counts,
                                  int64_t nchunks, cudaStream_t s);

// Batched symbolic assembly (batch.cu): per-instance dimensions, the column
// shift into the concatenated matrix, and the per-instance views of its CCS
// arrays.  Offsets are ascending int64 arrays of count + 1 entries.
fsparse_status launch_batch_dims(const int32_t *ii, const int32_t *jj, const int64_t *len_off, int count,
                                 int64_t total, int32_t *max_i, int32_t *max_j, cudaStream_t s);
fsparse_status launch_batch_remap(const int32_t *ii, const int32_t *jj, const int64_t *len_off,
                                  const int64_t *col_off, const int32_t *m, int count, int64_t total,
                                  int32_t *jj_out, cudaStream_t s);
fsparse_status launch_batch_nnz_off(const int32_t *jcS, const int64_t *col_off, int count, int64_t *nnz_off,
                                    cudaStream_t s);
fsparse_status launch_batch_jcs(const int32_t *jcS, const int64_t *col_off, const int64_t *jcs_off,
                                const int64_t *nnz_off, int count, int64_t total, int32_t *out,
                                cudaStream_t s);
fsparse_status launch_batch_irank(int32_t *irank, const int64_t *len_off, const int64_t *nnz_off, int count,
                                  int64_t total, cudaStream_t s);

// Hybrid column-bucket path.  Synchronises once to read the largest bucket
// and narrows the buckets until it fits shared memory; sets *unfit (and does
// nothing else) when no width fits, so the caller takes the onesweep path.
// A run longer than the in-bucket limit sets DevStatus::overflow instead,
// and the caller redoes the call with onesweep.
fsparse_status bucket_symbolic(const int32_t *ii, const int32_t *jj, int64_t len, int32_t m,
                               int32_t n, const KeyLayout &key, const fsparse_config &cfg,
                               Plan &plan, DevStatus *st, Scratch &scratch, cudaStream_t s,
                               bool *unfit);
bool bucket_supported(int64_t len, int32_t n, const KeyLayout &key, const fsparse_config &cfg);

}  // namespace fsp
