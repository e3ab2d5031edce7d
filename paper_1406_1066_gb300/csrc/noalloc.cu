// noalloc.cu -- full assembly for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc or any allocating routine: code that
// runs inside another framework's memory manager or arena, real-time solver
// loops that forbid allocation after start-up, or plug-ins that only receive
// pre-allocated buffers.  fsparse_assemble_noalloc serves them: the caller
// passes inputs and every output, and the sort's working memory lives in the
// file-scope array below, which every GPU that loads this library holds
// until the process exits.
//
// In host code `g_noalloc_scratch` names a host-side stand-in, not a device
// address, so the device address is looked up on every call (with the
// caller's device current) and only that address is handed to the kernels.
// The lookup is cheap after the first one on a device, and a fresh lookup
// stays right when the device was reset (and the array loaded again) since
// the previous call.
#include <algorithm>

#include "common.cuh"
#include "internal.hpp"

namespace fsp {

constexpr size_t kNoallocBytes = (size_t)FSPARSE_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch on the current device.
static fsparse_status noalloc_scratch(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    *out = p;
    return FSPARSE_OK;
}

}  // namespace fsp

using namespace fsp;

extern "C" fsparse_status fsparse_assemble_noalloc(const int32_t *ii, const int32_t *jj,
                                                   const double *sr, int64_t len, int32_t m,
                                                   int32_t n, int32_t *irank, int32_t *jcS,
                                                   int32_t *irS, double *prS, int64_t *nnz_out,
                                                   void *stream) {
    if (!nnz_out) return set_error(FSPARSE_ERR_ARG, "nnz_out is NULL");
    *nnz_out = 0;
    if (len < 0 || m <= 0 || n <= 0) return set_error(FSPARSE_ERR_ARG, "needs len >= 0 and explicit m, n > 0");
    if (len > FSPARSE_NOALLOC_MAX_LEN || n > FSPARSE_NOALLOC_MAX_COLS)
        return set_error(FSPARSE_ERR_SIZE, "problem above the no-alloc limits (len <= 131072, n <= 131072)");
    if (!jcS || (len > 0 && (!ii || !jj || !sr || !irank || !irS || !prS)))
        return set_error(FSPARSE_ERR_ARG, "NULL array");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    void *base = nullptr;
    fsparse_status e = noalloc_scratch(&base);
    if (e != FSPARSE_OK) return e;

    Scratch scratch(s, base, kNoallocBytes);
    DevStatus *d_st = nullptr;
    if ((e = scratch.get(&d_st, 1)) != FSPARSE_OK) return e;
    FSP_CUDA(cudaMemsetAsync(d_st, 0, sizeof(DevStatus), s));

    // A plan whose arrays are the caller's outputs plus two arena buffers.
    Plan plan;
    plan.m = m;
    plan.n = n;
    plan.len = len;
    plan.key.rb = bits_for((uint64_t)m - 1);
    plan.key.cb = bits_for((uint64_t)n - 1);
    const fsparse_config cfg{FSPARSE_SORT_ONESWEEP, 8, 16, 256, 8192, 1024};
    plan.cfg = cfg;
    plan.numeric_tile = cfg.numeric_tile;
    plan.nchunks = (len + kChunk - 1) / kChunk;
    plan.irank = irank;
    plan.irS = irS;
    plan.jcS = jcS;
    if ((e = scratch.get(&plan.perm, (size_t)std::max<int64_t>(len, 1))) != FSPARSE_OK) return e;
    if ((e = scratch.get(&plan.chunk_slot0, (size_t)plan.nchunks + 1)) != FSPARSE_OK) return e;

    if (len == 0) {
        FSP_CUDA(cudaMemsetAsync(jcS, 0, ((size_t)n + 1) * 4, s));
    } else {
        const void *keys = nullptr;
        int key_bytes = 0;
        if ((e = onesweep_sort(ii, jj, len, m, n, plan.key, cfg, plan.perm, &keys, &key_bytes, d_st, scratch,
                               s)) != FSPARSE_OK)
            return e;
        if ((e = emit_from_perm(keys, key_bytes, len, n, plan.key, plan, d_st, scratch, s)) != FSPARSE_OK)
            return e;
        if ((e = launch_numeric(plan.perm, plan.chunk_slot0, len, plan.numeric_tile, sr, prS, 0, 0, s)) !=
            FSPARSE_OK)
            return e;
        if ((e = launch_irank(plan.perm, plan.chunk_slot0, len, irank, s)) != FSPARSE_OK) return e;
    }
    DevStatus h{};   // pageable stack copy: no pinned allocation
    FSP_CUDA(cudaMemcpyAsync(&h, d_st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    FSP_CUDA(cudaStreamSynchronize(s));
    if (h.bad_index) return set_error(FSPARSE_ERR_INDEX, "index below 1 or above its dimension");
    if (h.timeout) return set_error(FSPARSE_ERR_TIMEOUT, "device look-back wait expired");
    if (h.oob) return set_error(FSPARSE_ERR_INTERNAL, "internal index check failed");
    *nnz_out = len ? (int64_t)h.nnz : 0;
    return FSPARSE_OK;
}
