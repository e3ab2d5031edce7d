// api.cu -- the C ABI of libfsparse (declared in include/fsparse.h).
//
// Orchestration only: argument checks, plan allocation, choosing the sort
// strategy, and the single host synchronisation of the symbolic phase.
// Every step of the assembly itself runs in the kernels of onesweep.cu,
// bucket.cu, scan.cu and numeric.cu.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.hpp"

struct fsparse_plan_s {
    fsp::Plan p;
};
struct fsparse_batch_s {
    fsp::Batch b;
};

namespace fsp {

std::atomic<int64_t> g_launches{0};
static thread_local std::string g_err;

fsparse_status set_error(fsparse_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

fsparse_status cuda_error(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? FSPARSE_ERR_NOMEM : FSPARSE_ERR_CUDA;
}

int sm_count(int) {
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    if (!cache[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 152;
        cache[dev] = v;
    }
    return cache[dev];
}

// Stream-ordered allocations come from the device's default memory pool;
// keep freed blocks cached in the pool so repeated calls do not go back to
// the driver.
static fsparse_status ensure_pool(int dev) {
    static std::mutex mu;
    static bool done[64] = {false};
    if (dev < 0 || dev >= 64) return FSPARSE_OK;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return FSPARSE_OK;
    cudaMemPool_t pool;
    FSP_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t threshold = UINT64_MAX;
    FSP_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold));
    done[dev] = true;
    return FSPARSE_OK;
}

// ---- phase timing ----------------------------------------------------------------
namespace {
struct PhaseTimer {
    static constexpr int kMax = 24;
    cudaStream_t s = nullptr;
    int n = 0;
    cudaEvent_t ev[kMax];
    const char *name[kMax];
};
thread_local PhaseTimer *t_timer = nullptr;
thread_local std::vector<std::pair<const char *, double>> t_last;

bool timing_requested() {
    const char *t = std::getenv("FSPARSE_TIMING");
    return t && t[0] == '1';
}

// Starts a timer for the calling thread when FSPARSE_TIMING=1 (RAII: the
// durations are stored on finish(), the events always destroyed).
struct TimerScope {
    PhaseTimer timer;
    bool on = false;
    explicit TimerScope(cudaStream_t s) {
        if (t_timer) return;   // nested call: the outer call's timer keeps running
        t_last.clear();
        if (!timing_requested()) return;
        timer.s = s;
        if (cudaEventCreate(&timer.ev[0]) != cudaSuccess) return;
        cudaEventRecord(timer.ev[0], s);
        timer.name[0] = "start";
        timer.n = 1;
        t_timer = &timer;
        on = true;
    }
    void finish() {
        if (!on || timer.n < 2) return;
        cudaEventSynchronize(timer.ev[timer.n - 1]);
        t_last.clear();
        for (int i = 1; i < timer.n; ++i) {
            float ms = 0;
            cudaEventElapsedTime(&ms, timer.ev[i - 1], timer.ev[i]);
            t_last.emplace_back(timer.name[i], (double)ms);
        }
    }
    ~TimerScope() {
        if (!on) return;
        for (int i = 0; i < timer.n; ++i) cudaEventDestroy(timer.ev[i]);
        t_timer = nullptr;
    }
};
}  // namespace

namespace {
thread_local bool t_phase_open = false;
// Closes a phase range left open by an early return of the entry point.
struct PhaseRangeGuard {
    ~PhaseRangeGuard() {
        if (t_phase_open) nvtxRangePop();
        t_phase_open = false;
    }
};
}  // namespace

void phase_begin(const char *name) {
    if (t_phase_open) nvtxRangePop();
    nvtxRangePushA(name);
    t_phase_open = true;
}

void phase_mark(const char *name) {
    if (t_phase_open) nvtxRangePop();
    t_phase_open = false;
    PhaseTimer *t = t_timer;
    if (!t || t->n >= PhaseTimer::kMax) return;
    if (cudaEventCreate(&t->ev[t->n]) != cudaSuccess) return;
    cudaEventRecord(t->ev[t->n], t->s);
    t->name[t->n++] = name;
}

int injected_fault() {
    const char *f = std::getenv("FSPARSE_FAULT");
    if (!f || !*f) return FAULT_NONE;
    if (std::strcmp(f, "alloc") == 0) return FAULT_ALLOC;
    if (std::strcmp(f, "timeout") == 0) return FAULT_TIMEOUT;
    if (std::strcmp(f, "timeout_sort") == 0) return FAULT_TIMEOUT_SORT;
    if (std::strcmp(f, "index") == 0) return FAULT_INDEX;
    return FAULT_NONE;
}

fsparse_status device_alloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (injected_fault() == FAULT_ALLOC) return set_error(FSPARSE_ERR_NOMEM, "injected allocation failure (FSPARSE_FAULT=alloc)");
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return cuda_error(e, "cudaMallocAsync");
    }
    return FSPARSE_OK;
}

Scratch::~Scratch() { release(); }

void Scratch::release() {
    for (int i = 0; i < n_; ++i) cudaFreeAsync(ptrs_[i], s_);
    n_ = 0;
}

fsparse_status Scratch::alloc(void **p, size_t bytes) {
    if (arena_) {
        const size_t take = (std::max<size_t>(bytes, 16) + 255) & ~size_t(255);
        if (arena_used_ + take > arena_bytes_) {
            *p = nullptr;
            return set_error(FSPARSE_ERR_SIZE, "static scratch exhausted");
        }
        *p = arena_ + arena_used_;
        arena_used_ += take;
        return FSPARSE_OK;
    }
    if (n_ == 32) return set_error(FSPARSE_ERR_NOMEM, "too many scratch buffers");
    fsparse_status e = device_alloc(p, bytes, s_);
    if (e == FSPARSE_OK) ptrs_[n_++] = *p;
    return e;
}

// One pinned status block per host thread for the single readback.
static DevStatus *host_status() {
    static thread_local DevStatus *h = nullptr;
    if (!h && cudaMallocHost(reinterpret_cast<void **>(&h), sizeof(DevStatus)) != cudaSuccess) {
        cudaGetLastError();
        h = nullptr;
    }
    return h;
}

// Waits on the host: poll for up to kPollMs, then block.  A blocking wait
// returns some tens of microseconds after the GPU finishes (the thread has
// to be woken), which a caller pays at every synchronisation of a call;
// polling returns within a microsecond or two.  Longer waits block, so a
// long queue costs no more than kPollMs of host time.
constexpr double kPollMs = 10.0;

template <typename Query, typename Block>
static fsparse_status poll_then_block(Query query, Block block, const char *what) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t q = query();
        if (q == cudaSuccess) return FSPARSE_OK;
        if (q != cudaErrorNotReady) return cuda_error(q, what);
        if (std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() > kPollMs)
            break;
    }
    const cudaError_t b = block();
    return b == cudaSuccess ? FSPARSE_OK : cuda_error(b, what);
}

fsparse_status wait_stream(cudaStream_t s) {
    return poll_then_block([&] { return cudaStreamQuery(s); }, [&] { return cudaStreamSynchronize(s); },
                           "cudaStreamSynchronize");
}

fsparse_status wait_event(cudaEvent_t e) {
    return poll_then_block([&] { return cudaEventQuery(e); }, [&] { return cudaEventSynchronize(e); },
                           "cudaEventSynchronize");
}

// The status read in two halves: queue the copy, then wait for it (work
// such as freeing the status word's own scratch can be queued in between).
static fsparse_status post_status(DevStatus *d, cudaStream_t s) {
    DevStatus *h = host_status();
    if (!h) return set_error(FSPARSE_ERR_NOMEM, "cudaMallocHost failed");
    FSP_CUDA(cudaMemcpyAsync(h, d, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    return FSPARSE_OK;
}

static fsparse_status finish_status(DevStatus *out, cudaStream_t s) {
    fsparse_status e = wait_stream(s);
    if (e != FSPARSE_OK) return e;
    *out = *host_status();
    return FSPARSE_OK;
}

static fsparse_status read_status(DevStatus *d, DevStatus *out, cudaStream_t s) {
    fsparse_status e = post_status(d, s);
    if (e != FSPARSE_OK) return e;
    return finish_status(out, s);
}

void note_use(UseLog &log, cudaStream_t s) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lock(log.mu);
        log.overflow = true;
        return;
    }
    if (cap != cudaStreamCaptureStatusNone) return;   // graph replays are the caller's to finish
    std::lock_guard<std::mutex> lock(log.mu);
    int i = 0;
    while (i < log.n && log.stream[i] != s) ++i;
    if (i == log.n) {
        if (log.n == UseLog::kMax ||
            cudaEventCreateWithFlags(&log.event[i], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            log.overflow = true;
            return;
        }
        log.stream[i] = s;
        ++log.n;
    }
    if (cudaEventRecord(log.event[i], s) != cudaSuccess) {
        cudaGetLastError();
        log.overflow = true;
    }
}

// A non-blocking stream per device on which released arrays go back to the
// stream-ordered pool.
static cudaStream_t release_stream(int dev) {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
}

// Release arrays of a plan or batch whose launches may still be running,
// without blocking the host or the device as a whole: the library's release
// stream waits for the events of `log` (every stream a numeric, adjoint or
// irank launch used) and for the work queued so far on `after` (the caller's
// stream; the legacy default stream also orders every blocking stream), then
// frees in stream order.  Falls back to waiting for the device when a stream
// could not be recorded.
static void release_after(void *const *ptrs, int count, UseLog &log, cudaStream_t after) {
    bool any = false;
    for (int i = 0; i < count; ++i) any |= ptrs[i] != nullptr;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaStream_t rs = any ? release_stream(dev) : nullptr;
    cudaEvent_t tail = nullptr;
    const bool ordered = rs && !log.overflow &&
                         cudaEventCreateWithFlags(&tail, cudaEventDisableTiming) == cudaSuccess &&
                         cudaEventRecord(tail, after) == cudaSuccess &&
                         cudaStreamWaitEvent(rs, tail, 0) == cudaSuccess;
    if (any) {
        if (ordered) {
            for (int i = 0; i < log.n; ++i) cudaStreamWaitEvent(rs, log.event[i], 0);
            for (int i = 0; i < count; ++i)
                if (ptrs[i]) cudaFreeAsync(ptrs[i], rs);
        } else {
            cudaGetLastError();
            cudaDeviceSynchronize();
            for (int i = 0; i < count; ++i)
                if (ptrs[i]) cudaFreeAsync(ptrs[i], nullptr);
            cudaStreamSynchronize(nullptr);
        }
    }
    if (tail) cudaEventDestroy(tail);   // released by the driver once it has completed
    for (int i = 0; i < log.n; ++i) cudaEventDestroy(log.event[i]);
    log.n = 0;
    log.overflow = false;
    cudaGetLastError();
}

// Arrays of a plan that a failed call built: only that call's stream has
// touched them, so they go back to the pool in its order.
static void free_plan_arrays_on(Plan &p, cudaStream_t s) {
    void *ptrs[5] = {p.irank, p.jcS, p.irS, p.perm, p.chunk_slot0};
    for (void *q : ptrs)
        if (q) cudaFreeAsync(q, s);
    cudaGetLastError();
    p.irank = p.jcS = p.irS = nullptr;
    p.perm = p.chunk_slot0 = nullptr;
}

static void free_plan_arrays(Plan &p, cudaStream_t after) {
    void *ptrs[5] = {p.irank, p.jcS, p.irS, p.perm, p.chunk_slot0};
    release_after(ptrs, 5, p.uses, after);
    p.irank = p.jcS = p.irS = nullptr;
    p.perm = p.chunk_slot0 = nullptr;
}

constexpr int64_t kMaxLen = kMaxLookbackValue;   // 2^30 - 1

static fsparse_status check_dims_args(const int32_t *ii, const int32_t *jj, int64_t len, int32_t m,
                                      int32_t n, int64_t nzmax) {
    if (len < 0) return set_error(FSPARSE_ERR_ARG, "len < 0");
    if (m < 0 || n < 0) return set_error(FSPARSE_ERR_ARG, "negative dimension");
    if (nzmax < 0) return set_error(FSPARSE_ERR_ARG, "nzmax < 0");
    if (len > 0 && (!ii || !jj)) return set_error(FSPARSE_ERR_ARG, "NULL index array");
    if (len > kMaxLen) return set_error(FSPARSE_ERR_SIZE, "len above 2^30 - 1");
    if (nzmax > kMaxLen) return set_error(FSPARSE_ERR_SIZE, "nzmax above 2^30 - 1");
    return FSPARSE_OK;
}

// The sort + emit for one strategy; values folded into prS when given.
static fsparse_status run_symbolic(const int32_t *ii, const int32_t *jj, const double *sr,
                                   double *prS, int64_t len, Plan &plan, const fsparse_config &cfg,
                                   DevStatus *d_st, Scratch &scratch, cudaStream_t s, bool *folded) {
    *folded = false;
    fsparse_status e;
    bool unfit = true;
    const bool bucket = cfg.strategy == FSPARSE_SORT_BUCKET || cfg.strategy == FSPARSE_SORT_BUCKET_RADIX;
    if (bucket && bucket_supported(len, plan.n, plan.key, cfg)) {
        e = bucket_symbolic(ii, jj, len, plan.m, plan.n, plan.key, cfg, plan, d_st, scratch, s, &unfit);
        if (e != FSPARSE_OK) return e;
    }
    if (!unfit) {
        e = FSPARSE_OK;
    } else {
        const void *keys = nullptr;
        int key_bytes = 0;
        if ((e = onesweep_sort(ii, jj, len, plan.m, plan.n, plan.key, cfg, plan.perm, &keys, &key_bytes, d_st,
                               scratch, s)) != FSPARSE_OK)
            return e;
        e = emit_from_perm(keys, key_bytes, len, plan.n, plan.key, plan, d_st, scratch, s);
    }
    if (e != FSPARSE_OK) return e;
    if (sr) {
        phase_begin("numeric_fold");
        e = launch_numeric(plan.perm, plan.chunk_slot0, len, plan.numeric_tile, sr, prS, 0, 0, s);
        if (e == FSPARSE_OK) *folded = true;
        phase_mark("numeric_fold");
    }
    return e;
}

// Symbolic phase with an optional fused fold into prS (capacity >= max(len, nzmax)).
static fsparse_status symbolic_impl(const int32_t *ii, const int32_t *jj, const double *sr,
                                    double *prS, int64_t len, int32_t m, int32_t n, int64_t nzmax,
                                    cudaStream_t s, Plan **out, const fsparse_config *force) {
    NvtxRange nvtx_("fsparse_symbolic");
    PhaseRangeGuard phase_guard_;
    *out = nullptr;
    fsparse_status e = check_dims_args(ii, jj, len, m, n, nzmax);
    if (e != FSPARSE_OK) return e;
    int dev = 0;
    FSP_CUDA(cudaGetDevice(&dev));
    if ((e = ensure_pool(dev)) != FSPARSE_OK) return e;

    TimerScope timing(s);
    Scratch scratch(s);
    DevStatus *d_st = nullptr;
    DevStatus h_st{};
    if ((e = scratch.get(&d_st, 1)) != FSPARSE_OK) return e;
    FSP_CUDA(cudaMemsetAsync(d_st, 0, sizeof(DevStatus), s));

    if (m == 0 || n == 0) {   // implicit dimensions (§2.2): one extra synchronisation
        phase_begin("dims");
        if ((e = launch_minmax(ii, jj, len, m, n, d_st, s)) != FSPARSE_OK) return e;
        phase_mark("dims");
        if ((e = read_status(d_st, &h_st, s)) != FSPARSE_OK) return e;
        if (h_st.bad_index) return set_error(FSPARSE_ERR_INDEX, "index below 1 or above its dimension");
        if (m == 0) m = h_st.max_i;
        if (n == 0) n = h_st.max_j;
    }

    Plan *plan = new (std::nothrow) Plan();
    if (!plan) return set_error(FSPARSE_ERR_NOMEM, "host allocation");
    plan->device = dev;
    plan->m = m;
    plan->n = n;
    plan->len = len;
    plan->key.rb = m > 0 ? bits_for((uint64_t)m - 1) : 0;
    plan->key.cb = n > 0 ? bits_for((uint64_t)n - 1) : 0;
    fsparse_config cfg = force ? *force : resolve_config(len, plan->key);
    plan->cfg = cfg;
    plan->numeric_tile = cfg.numeric_tile;
    plan->nchunks = (len + kChunk - 1) / kChunk;
    const int64_t irs_cap = std::max<int64_t>(std::max<int64_t>(len, nzmax), 1);

    auto fail = [&](fsparse_status st) {
        free_plan_arrays_on(*plan, s);
        delete plan;
        return st;
    };
    if ((e = device_alloc(reinterpret_cast<void **>(&plan->irank), (size_t)std::max<int64_t>(len, 1) * 4, s)) ||
        (e = device_alloc(reinterpret_cast<void **>(&plan->perm), (size_t)std::max<int64_t>(len, 1) * 4, s)) ||
        (e = device_alloc(reinterpret_cast<void **>(&plan->irS), (size_t)irs_cap * 4, s)) ||
        (e = device_alloc(reinterpret_cast<void **>(&plan->jcS), ((size_t)n + 1) * 4, s)) ||
        (e = device_alloc(reinterpret_cast<void **>(&plan->chunk_slot0), ((size_t)plan->nchunks + 1) * 4, s)))
        return fail(e);

    bool folded = false;
    if (len == 0) {
        if (cudaMemsetAsync(plan->jcS, 0, ((size_t)n + 1) * 4, s) != cudaSuccess ||
            cudaMemsetAsync(plan->chunk_slot0, 0, 4, s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "cudaMemsetAsync"));
        folded = sr != nullptr;
    } else {
        e = run_symbolic(ii, jj, sr, prS, len, *plan, cfg, d_st, scratch, s, &folded);
        if (e != FSPARSE_OK) return fail(e);
    }
    if (injected_fault() == FAULT_INDEX) {   // seed the status word as a kernel finding a bad index would
        const uint32_t one = 1;
        if (cudaMemcpyAsync(&d_st->bad_index, &one, 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "cudaMemcpyAsync"));
    }
    // The scratch (status word included) is freed behind the status copy, so
    // the frees are queued before the host waits instead of after it.
    if ((e = post_status(d_st, s)) != FSPARSE_OK) return fail(e);
    scratch.release();
    if ((e = finish_status(&h_st, s)) != FSPARSE_OK) return fail(e);
    if (h_st.overflow && !h_st.bad_index && !h_st.timeout) {
        // A column bucket outgrew shared memory: same result through onesweep.
        fsparse_config os = cfg;
        os.strategy = FSPARSE_SORT_ONESWEEP;
        plan->cfg = os;
        if ((e = scratch.get(&d_st, 1)) != FSPARSE_OK) return fail(e);
        if (cudaMemsetAsync(d_st, 0, sizeof(DevStatus), s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "cudaMemsetAsync"));
        e = run_symbolic(ii, jj, sr, prS, len, *plan, os, d_st, scratch, s, &folded);
        if (e != FSPARSE_OK) return fail(e);
        if ((e = read_status(d_st, &h_st, s)) != FSPARSE_OK) return fail(e);
    }
    if (h_st.bad_index) return fail(set_error(FSPARSE_ERR_INDEX, "index below 1 or above its dimension"));
    if (h_st.timeout) return fail(set_error(FSPARSE_ERR_TIMEOUT, "device look-back wait expired"));
    if (h_st.oob) return fail(set_error(FSPARSE_ERR_INTERNAL, "internal index check failed"));
    const int64_t nnz = len ? (int64_t)h_st.nnz : 0;
    if (nzmax > 0 && nzmax < nnz) return fail(set_error(FSPARSE_ERR_NZMAX, "nzmax below nnz"));
    plan->nnz = nnz;
    plan->cap = std::max(nnz, nzmax);
    if (plan->cap > nnz) {
        phase_begin("nzmax_tail");
        if ((e = launch_fill(plan->irS, folded ? prS : nullptr, nnz, plan->cap, s)) != FSPARSE_OK) return fail(e);
        phase_mark("nzmax_tail");
    }
    timing.finish();
    *out = plan;
    return FSPARSE_OK;
}

}  // namespace fsp

using namespace fsp;

static inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

extern "C" {

fsparse_status fsparse_symbolic(const int32_t *ii, const int32_t *jj, int64_t len, int32_t m,
                                int32_t n, int64_t nzmax, void *stream, fsparse_plan *plan_out) {
    if (!plan_out) return set_error(FSPARSE_ERR_ARG, "plan_out is NULL");
    *plan_out = nullptr;
    Plan *p = nullptr;
    fsparse_status e = symbolic_impl(ii, jj, nullptr, nullptr, len, m, n, nzmax, as_stream(stream), &p, nullptr);
    if (e != FSPARSE_OK) return e;
    *plan_out = reinterpret_cast<fsparse_plan>(p);
    return FSPARSE_OK;
}

fsparse_status fsparse_plan_info(fsparse_plan plan, int32_t *m, int32_t *n, int64_t *len,
                                 int64_t *nnz, int64_t *cap) {
    if (!plan) return set_error(FSPARSE_ERR_ARG, "plan is NULL");
    const Plan &p = reinterpret_cast<fsparse_plan_s *>(plan)->p;
    if (m) *m = p.m;
    if (n) *n = p.n;
    if (len) *len = p.len;
    if (nnz) *nnz = p.nnz;
    if (cap) *cap = p.cap;
    return FSPARSE_OK;
}

// irank is derived from perm the first time it is needed.
static fsparse_status ensure_irank(Plan &p, cudaStream_t s, bool sync) {
    if (p.irank_ready) return FSPARSE_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p.device) cudaSetDevice(p.device);
    fsparse_status e = launch_irank(p.perm, p.chunk_slot0, p.len, p.irank, s);
    if (e == FSPARSE_OK && sync && cudaStreamSynchronize(s) != cudaSuccess)
        e = cuda_error(cudaGetLastError(), "cudaStreamSynchronize");
    if (cur != p.device) cudaSetDevice(cur);
    if (e == FSPARSE_OK) p.irank_ready = true;
    return e;
}

fsparse_status fsparse_plan_arrays(fsparse_plan plan, const int32_t **irank, const int32_t **jcS,
                                   const int32_t **irS) {
    if (!plan) return set_error(FSPARSE_ERR_ARG, "plan is NULL");
    Plan &p = reinterpret_cast<fsparse_plan_s *>(plan)->p;
    if (irank) {
        fsparse_status e = ensure_irank(p, nullptr, true);
        if (e != FSPARSE_OK) return e;
    }
    if (irank) *irank = p.irank;
    if (jcS) *jcS = p.jcS;
    if (irS) *irS = p.irS;
    return FSPARSE_OK;
}

static fsparse_status destroy_plan(fsparse_plan plan, cudaStream_t after) {
    if (!plan) return FSPARSE_OK;
    Plan *p = &reinterpret_cast<fsparse_plan_s *>(plan)->p;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    free_plan_arrays(*p, after);
    if (cur != p->device) cudaSetDevice(cur);
    delete p;
    return FSPARSE_OK;
}

fsparse_status fsparse_plan_destroy(fsparse_plan plan) { return destroy_plan(plan, nullptr); }

fsparse_status fsparse_plan_release(fsparse_plan plan, void *stream) {
    return destroy_plan(plan, as_stream(stream));
}

fsparse_status fsparse_numeric(fsparse_plan plan, const double *sr, double *prS, void *stream) {
    NvtxRange nvtx_("fsparse_numeric");
    if (!plan) return set_error(FSPARSE_ERR_ARG, "plan is NULL");
    const Plan &p = reinterpret_cast<fsparse_plan_s *>(plan)->p;
    if ((p.len > 0 && !sr) || (p.cap > 0 && !prS)) return set_error(FSPARSE_ERR_ARG, "NULL array");
    const fsparse_status e = launch_numeric(p.perm, p.chunk_slot0, p.len, p.numeric_tile, sr, prS, p.nnz,
                                            p.cap, as_stream(stream));
    if (e == FSPARSE_OK) note_use(reinterpret_cast<fsparse_plan_s *>(plan)->p.uses, as_stream(stream));
    return e;
}

fsparse_status fsparse_numeric_adjoint(fsparse_plan plan, const double *dprS, double *ds, void *stream) {
    NvtxRange nvtx_("fsparse_numeric_adjoint");
    if (!plan) return set_error(FSPARSE_ERR_ARG, "plan is NULL");
    Plan &p = reinterpret_cast<fsparse_plan_s *>(plan)->p;
    if (p.len > 0 && (!dprS || !ds)) return set_error(FSPARSE_ERR_ARG, "NULL array");
    fsparse_status e = ensure_irank(p, as_stream(stream), false);
    if (e != FSPARSE_OK) return e;
    e = launch_adjoint(p.irank, p.len, dprS, ds, p.nnz, as_stream(stream));
    if (e == FSPARSE_OK) note_use(p.uses, as_stream(stream));
    return e;
}

fsparse_status fsparse_assemble(const int32_t *ii, const int32_t *jj, const double *sr, int64_t len,
                                int32_t m, int32_t n, int64_t nzmax, double *prS,
                                int64_t prS_capacity, void *stream, fsparse_plan *plan_out) {
    if (!plan_out) return set_error(FSPARSE_ERR_ARG, "plan_out is NULL");
    *plan_out = nullptr;
    if (len > 0 && !sr) return set_error(FSPARSE_ERR_ARG, "NULL value array");
    if (prS_capacity < 0 || (prS_capacity > 0 && !prS)) return set_error(FSPARSE_ERR_ARG, "bad prS");
    cudaStream_t s = as_stream(stream);
    Plan *p = nullptr;
    fsparse_status e;
    if (prS_capacity >= std::max<int64_t>(len, nzmax) && prS_capacity > 0) {
        e = symbolic_impl(ii, jj, sr, prS, len, m, n, nzmax, s, &p, nullptr);
        if (e != FSPARSE_OK) return e;
        *plan_out = reinterpret_cast<fsparse_plan>(p);
        return FSPARSE_OK;
    }
    e = symbolic_impl(ii, jj, nullptr, nullptr, len, m, n, nzmax, s, &p, nullptr);
    if (e != FSPARSE_OK) return e;
    *plan_out = reinterpret_cast<fsparse_plan>(p);
    if (prS_capacity < p->cap) return set_error(FSPARSE_ERR_NZMAX, "prS capacity below the plan's cap");
    e = launch_numeric(p->perm, p->chunk_slot0, p->len, p->numeric_tile, sr, prS, p->nnz, p->cap, s);
    if (e == FSPARSE_OK) note_use(p->uses, s);
    return e;
}

// ---- Matlab-style double index arrays ----------------------------------------
// Converted once into int32 scratch (App. A pre-processing), then the int
// path runs; a bad value becomes index 0, so the int path's own check returns
// FSPARSE_ERR_INDEX at its usual synchronisation.
static fsparse_status check_f64_args(const double *ii, const double *jj, int64_t len, int32_t m,
                                     int32_t n, int64_t nzmax, void *plan_out) {
    if (!plan_out) return set_error(FSPARSE_ERR_ARG, "plan_out is NULL");
    if (len < 0) return set_error(FSPARSE_ERR_ARG, "len < 0");
    if (m < 0 || n < 0) return set_error(FSPARSE_ERR_ARG, "negative dimension");
    if (nzmax < 0) return set_error(FSPARSE_ERR_ARG, "nzmax < 0");
    if (len > kMaxLen) return set_error(FSPARSE_ERR_SIZE, "len above 2^30 - 1");
    if (nzmax > kMaxLen) return set_error(FSPARSE_ERR_SIZE, "nzmax above 2^30 - 1");
    if (len > 0 && (!ii || !jj)) return set_error(FSPARSE_ERR_ARG, "NULL index array");
    return FSPARSE_OK;
}

static fsparse_status getix_pair(const double *ii, const double *jj, int64_t len, Scratch &scratch,
                                 int32_t **i32, int32_t **j32, cudaStream_t s) {
    fsparse_status e;
    int dev = 0;
    FSP_CUDA(cudaGetDevice(&dev));
    if ((e = ensure_pool(dev)) != FSPARSE_OK) return e;
    const size_t n = (size_t)std::max<int64_t>(len, 1);
    if ((e = scratch.get(i32, n)) != FSPARSE_OK || (e = scratch.get(j32, n)) != FSPARSE_OK) return e;
    if ((e = launch_getix(ii, len, *i32, s)) != FSPARSE_OK) return e;
    return launch_getix(jj, len, *j32, s);
}

fsparse_status fsparse_symbolic_f64(const double *ii, const double *jj, int64_t len, int32_t m,
                                    int32_t n, int64_t nzmax, void *stream, fsparse_plan *plan_out) {
    fsparse_status e = check_f64_args(ii, jj, len, m, n, nzmax, plan_out);
    if (e != FSPARSE_OK) return e;
    *plan_out = nullptr;
    cudaStream_t s = as_stream(stream);
    Scratch scratch(s);
    int32_t *i32 = nullptr, *j32 = nullptr;
    if ((e = getix_pair(ii, jj, len, scratch, &i32, &j32, s)) != FSPARSE_OK) return e;
    return fsparse_symbolic(i32, j32, len, m, n, nzmax, stream, plan_out);
}

fsparse_status fsparse_assemble_f64(const double *ii, const double *jj, const double *sr, int64_t len,
                                    int32_t m, int32_t n, int64_t nzmax, double *prS,
                                    int64_t prS_capacity, void *stream, fsparse_plan *plan_out) {
    fsparse_status e = check_f64_args(ii, jj, len, m, n, nzmax, plan_out);
    if (e != FSPARSE_OK) return e;
    *plan_out = nullptr;
    if (len > 0 && !sr) return set_error(FSPARSE_ERR_ARG, "NULL value array");
    if (prS_capacity < 0 || (prS_capacity > 0 && !prS)) return set_error(FSPARSE_ERR_ARG, "bad prS");
    cudaStream_t s = as_stream(stream);
    Scratch scratch(s);
    int32_t *i32 = nullptr, *j32 = nullptr;
    if ((e = getix_pair(ii, jj, len, scratch, &i32, &j32, s)) != FSPARSE_OK) return e;
    return fsparse_assemble(i32, j32, sr, len, m, n, nzmax, prS, prS_capacity, stream, plan_out);
}

// ---- checkpoint: plan export / import -------------------------------------------
// Layout: PlanImage header, then perm[len] u32, chunk_slot0[nchunks + 1] u32,
// jcS[n + 1] i32, irS[cap] i32 (little-endian, as in device memory).  irank is
// not stored: it is derived again on first request.
struct PlanImage {
    char magic[8];          // "FSPPLAN1"
    int64_t m, n, len, nnz, cap, nchunks;
    int32_t strategy, radix_bits, sweep_items, sweep_threads, bucket_target, numeric_tile;
};

static int64_t image_bytes(const PlanImage &h) {
    return (int64_t)sizeof(PlanImage) + 4 * (h.len + (h.nchunks + 1) + (h.n + 1) + h.cap);
}

fsparse_status fsparse_plan_export(fsparse_plan plan, void *host_buf, int64_t capacity, int64_t *bytes_out) {
    if (!plan || !bytes_out) return set_error(FSPARSE_ERR_ARG, "plan or bytes_out is NULL");
    const Plan &p = reinterpret_cast<fsparse_plan_s *>(plan)->p;
    PlanImage h{};
    std::memcpy(h.magic, "FSPPLAN1", 8);
    h.m = p.m; h.n = p.n; h.len = p.len; h.nnz = p.nnz; h.cap = p.cap; h.nchunks = p.nchunks;
    h.strategy = p.cfg.strategy; h.radix_bits = p.cfg.radix_bits; h.sweep_items = p.cfg.sweep_items;
    h.sweep_threads = p.cfg.sweep_threads; h.bucket_target = p.cfg.bucket_target; h.numeric_tile = p.numeric_tile;
    *bytes_out = image_bytes(h);
    if (!host_buf) return FSPARSE_OK;   // size query
    if (capacity < *bytes_out) return set_error(FSPARSE_ERR_ARG, "host buffer smaller than the plan image");
    char *out = static_cast<char *>(host_buf);
    std::memcpy(out, &h, sizeof(h));
    size_t off = sizeof(h);
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p.device) cudaSetDevice(p.device);
    auto get = [&](const void *src, int64_t count) {
        const cudaError_t e = count > 0 ? cudaMemcpy(out + off, src, (size_t)count * 4, cudaMemcpyDeviceToHost)
                                        : cudaSuccess;
        off += (size_t)count * 4;
        return e;
    };
    cudaError_t e = get(p.perm, p.len);
    if (e == cudaSuccess) e = get(p.chunk_slot0, p.nchunks + 1);
    if (e == cudaSuccess) e = get(p.jcS, (int64_t)p.n + 1);
    if (e == cudaSuccess) e = get(p.irS, p.cap);
    if (cur != p.device) cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy (plan export)");
    return FSPARSE_OK;
}

fsparse_status fsparse_plan_import(const void *host_buf, int64_t bytes, void *stream, fsparse_plan *plan_out) {
    if (!plan_out) return set_error(FSPARSE_ERR_ARG, "plan_out is NULL");
    *plan_out = nullptr;
    if (!host_buf || bytes < (int64_t)sizeof(PlanImage)) return set_error(FSPARSE_ERR_ARG, "no plan image");
    PlanImage h;
    std::memcpy(&h, host_buf, sizeof(h));
    if (std::memcmp(h.magic, "FSPPLAN1", 8) != 0) return set_error(FSPARSE_ERR_ARG, "not a plan image");
    const bool sane = h.len >= 0 && h.len <= kMaxLen && h.m >= 0 && h.n >= 0 && h.m <= INT32_MAX &&
                      h.n <= INT32_MAX && h.nnz >= 0 && h.nnz <= h.len && h.cap >= h.nnz &&
                      h.cap <= std::max<int64_t>(kMaxLen, h.len) &&
                      h.nchunks == (h.len + kChunk - 1) / kChunk &&
                      (h.numeric_tile == 1024 || h.numeric_tile == 2048 || h.numeric_tile == 4096);
    if (!sane || bytes != image_bytes(h)) return set_error(FSPARSE_ERR_ARG, "inconsistent plan image");
    cudaStream_t s = as_stream(stream);
    int dev = 0;
    FSP_CUDA(cudaGetDevice(&dev));
    fsparse_status e;
    if ((e = ensure_pool(dev)) != FSPARSE_OK) return e;
    Plan *plan = new (std::nothrow) Plan();
    if (!plan) return set_error(FSPARSE_ERR_NOMEM, "host allocation");
    plan->device = dev;
    plan->m = (int32_t)h.m;
    plan->n = (int32_t)h.n;
    plan->len = h.len;
    plan->nnz = h.nnz;
    plan->cap = h.cap;
    plan->key.rb = plan->m > 0 ? bits_for((uint64_t)plan->m - 1) : 0;
    plan->key.cb = plan->n > 0 ? bits_for((uint64_t)plan->n - 1) : 0;
    plan->cfg = fsparse_config{h.strategy, h.radix_bits, h.sweep_items, h.sweep_threads, h.bucket_target, h.numeric_tile};
    plan->numeric_tile = h.numeric_tile;
    plan->nchunks = h.nchunks;
    auto fail = [&](fsparse_status st) {
        free_plan_arrays_on(*plan, s);
        delete plan;
        return st;
    };
    if ((e = device_alloc(reinterpret_cast<void **>(&plan->irank), (size_t)std::max<int64_t>(h.len, 1) * 4, s)) ||
        (e = device_alloc(reinterpret_cast<void **>(&plan->perm), (size_t)std::max<int64_t>(h.len, 1) * 4, s)) ||
        (e = device_alloc(reinterpret_cast<void **>(&plan->irS), (size_t)std::max<int64_t>(h.cap, 1) * 4, s)) ||
        (e = device_alloc(reinterpret_cast<void **>(&plan->jcS), ((size_t)h.n + 1) * 4, s)) ||
        (e = device_alloc(reinterpret_cast<void **>(&plan->chunk_slot0), ((size_t)h.nchunks + 1) * 4, s)))
        return fail(e);
    const char *in = static_cast<const char *>(host_buf) + sizeof(h);
    auto put = [&](void *dst, int64_t count) {
        const cudaError_t ce = count > 0 ? cudaMemcpyAsync(dst, in, (size_t)count * 4, cudaMemcpyHostToDevice, s)
                                         : cudaSuccess;
        in += (size_t)count * 4;
        return ce;
    };
    cudaError_t ce = put(plan->perm, h.len);
    if (ce == cudaSuccess) ce = put(plan->chunk_slot0, h.nchunks + 1);
    if (ce == cudaSuccess) ce = put(plan->jcS, h.n + 1);
    if (ce == cudaSuccess) ce = put(plan->irS, h.cap);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);   // the caller's buffer may go away
    if (ce != cudaSuccess) return fail(cuda_error(ce, "cudaMemcpyAsync (plan import)"));
    *plan_out = reinterpret_cast<fsparse_plan>(plan);
    return FSPARSE_OK;
}

// ---- phase timing ------------------------------------------------------------
int32_t fsparse_last_timings(const char **names, double *ms, int32_t max) {
    const int32_t n = (int32_t)t_last.size();
    for (int32_t i = 0; i < n && i < max; ++i) {
        if (names) names[i] = t_last[i].first;
        if (ms) ms[i] = t_last[i].second;
    }
    return n;
}

// ---- delayed assembly ---------------------------------------------------------
fsparse_status fsparse_plan_append(fsparse_plan plan, const int32_t *ii, const int32_t *jj, int64_t len,
                                   void *stream, fsparse_plan *plan_out) {
    NvtxRange nvtx_("fsparse_plan_append");
    if (!plan_out) return set_error(FSPARSE_ERR_ARG, "plan_out is NULL");
    *plan_out = nullptr;
    if (!plan) return set_error(FSPARSE_ERR_ARG, "plan is NULL");
    if (len < 0) return set_error(FSPARSE_ERR_ARG, "len < 0");
    if (len > 0 && (!ii || !jj)) return set_error(FSPARSE_ERR_ARG, "NULL index array");
    const Plan &a = reinterpret_cast<fsparse_plan_s *>(plan)->p;
    if (a.len + len > kMaxLen) return set_error(FSPARSE_ERR_SIZE, "appended len above 2^30 - 1");
    if (a.m == 0 || a.n == 0) {
        if (len > 0) return set_error(FSPARSE_ERR_INDEX, "the plan has a zero dimension");
    }
    cudaStream_t s = as_stream(stream);
    int cur = 0;
    FSP_CUDA(cudaGetDevice(&cur));
    if (cur != a.device) return set_error(FSPARSE_ERR_ARG, "the plan belongs to another device");

    // The new triplets alone, checked against the plan's dimensions.
    TimerScope timing(s);
    PhaseRangeGuard phase_guard_;
    Plan *b = nullptr;
    fsparse_status e = symbolic_impl(ii, jj, nullptr, nullptr, len, a.m, a.n, 0, s, &b, nullptr);
    if (e != FSPARSE_OK) return e;
    phase_mark("append_symbolic");

    Plan *out = new (std::nothrow) Plan();
    if (!out) {
        free_plan_arrays_on(*b, s);
        delete b;
        return set_error(FSPARSE_ERR_NOMEM, "host allocation");
    }
    auto fail = [&](fsparse_status st) {
        free_plan_arrays_on(*b, s);
        delete b;
        free_plan_arrays_on(*out, s);
        delete out;
        return st;
    };
    out->device = a.device;
    out->m = a.m;
    out->n = a.n;
    out->len = a.len + len;
    out->key = a.key;
    out->cfg = a.cfg;
    out->numeric_tile = a.numeric_tile;
    out->nchunks = (out->len + kChunk - 1) / kChunk;
    const int64_t irs = std::max<int64_t>(a.nnz + b->nnz, 1);
    if ((e = device_alloc(reinterpret_cast<void **>(&out->irank), (size_t)std::max<int64_t>(out->len, 1) * 4, s)) ||
        (e = device_alloc(reinterpret_cast<void **>(&out->perm), (size_t)std::max<int64_t>(out->len, 1) * 4, s)) ||
        (e = device_alloc(reinterpret_cast<void **>(&out->irS), (size_t)irs * 4, s)) ||
        (e = device_alloc(reinterpret_cast<void **>(&out->jcS), ((size_t)out->n + 1) * 4, s)) ||
        (e = device_alloc(reinterpret_cast<void **>(&out->chunk_slot0), ((size_t)out->nchunks + 1) * 4, s)))
        return fail(e);
    DevStatus h_st{};
    {
        Scratch scratch(s);
        DevStatus *d_st = nullptr;
        if ((e = scratch.get(&d_st, 1)) != FSPARSE_OK) return fail(e);
        if (cudaMemsetAsync(d_st, 0, sizeof(DevStatus), s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "cudaMemsetAsync"));
        if ((e = append_merge(a, *b, *out, d_st, scratch, s)) != FSPARSE_OK) return fail(e);
        if ((e = read_status(d_st, &h_st, s)) != FSPARSE_OK) return fail(e);
    }
    if (h_st.timeout) return fail(set_error(FSPARSE_ERR_TIMEOUT, "device look-back wait expired"));
    if (h_st.oob) return fail(set_error(FSPARSE_ERR_INTERNAL, "internal index check failed"));
    out->nnz = out->len ? (int64_t)h_st.nnz : 0;
    out->cap = out->nnz;
    timing.finish();
    free_plan_arrays_on(*b, s);
    delete b;
    *plan_out = reinterpret_cast<fsparse_plan>(out);
    return FSPARSE_OK;
}

// ---- batch ----------------------------------------------------------------
fsparse_status fsparse_batch_create(int32_t count, const fsparse_plan *h_plans, void *stream,
                                    fsparse_batch *batch_out) {
    NvtxRange nvtx_("fsparse_batch_create");
    if (!batch_out) return set_error(FSPARSE_ERR_ARG, "batch_out is NULL");
    *batch_out = nullptr;
    if (count < 0 || (count > 0 && !h_plans)) return set_error(FSPARSE_ERR_ARG, "bad plan list");
    cudaStream_t s = as_stream(stream);
    int64_t total_len = 0, total_nnz = 0;
    for (int32_t b = 0; b < count; ++b) {
        if (!h_plans[b]) return set_error(FSPARSE_ERR_ARG, "NULL plan in batch");
        const Plan &p = reinterpret_cast<fsparse_plan_s *>(h_plans[b])->p;
        total_len += p.len;
        total_nnz += p.nnz;
    }
    if (total_len > kMaxLen) return set_error(FSPARSE_ERR_SIZE, "batch total len above 2^30 - 1");
    Batch *bt = new (std::nothrow) Batch();
    if (!bt) return set_error(FSPARSE_ERR_NOMEM, "host allocation");
    cudaGetDevice(&bt->device);
    bt->count = count;
    bt->total_len = total_len;
    bt->total_nnz = total_nnz;
    bt->h_len_off = new (std::nothrow) int64_t[count + 1];
    bt->h_nnz_off = new (std::nothrow) int64_t[count + 1];
    {   // numeric tile of the concatenation's size class (tuned table, else default)
        KeyLayout key;
        bt->numeric_tile = resolve_config(total_len, key).numeric_tile;
    }
    bt->nchunks = (total_len + kChunk - 1) / kChunk;
    auto fail = [&](fsparse_status st) {
        for (void *q : {static_cast<void *>(bt->perm), static_cast<void *>(bt->chunk_slot0)})
            if (q) cudaFreeAsync(q, s);
        cudaGetLastError();
        delete[] bt->h_len_off;
        delete[] bt->h_nnz_off;
        delete bt;
        return st;
    };
    if (!bt->h_len_off || !bt->h_nnz_off) return fail(set_error(FSPARSE_ERR_NOMEM, "host allocation"));
    fsparse_status e;
    if ((e = device_alloc(reinterpret_cast<void **>(&bt->perm), (size_t)std::max<int64_t>(total_len, 1) * 4, s)) ||
        (e = device_alloc(reinterpret_cast<void **>(&bt->chunk_slot0), ((size_t)bt->nchunks + 1) * 4, s)))
        return fail(e);
    int64_t lo = 0, no = 0;
    for (int32_t b = 0; b < count; ++b) {
        const Plan &p = reinterpret_cast<fsparse_plan_s *>(h_plans[b])->p;
        bt->h_len_off[b] = lo;
        bt->h_nnz_off[b] = no;
        if ((e = launch_batch_concat(p.perm, bt->perm + lo, p.len, (uint32_t)lo, s)) != FSPARSE_OK) return fail(e);
        lo += p.len;
        no += p.nnz;
    }
    bt->h_len_off[count] = lo;
    bt->h_nnz_off[count] = no;
    {
        Scratch scratch(s);
        uint32_t *counts = nullptr;
        DevStatus *d_st = nullptr;
        DevStatus h_st{};
        if ((e = scratch.get(&counts, (size_t)bt->nchunks + 1)) != FSPARSE_OK) return fail(e);
        if ((e = scratch.get(&d_st, 1)) != FSPARSE_OK) return fail(e);
        if (cudaMemsetAsync(d_st, 0, sizeof(DevStatus), s) != cudaSuccess)
            return fail(cuda_error(cudaGetLastError(), "cudaMemsetAsync"));
        if ((e = launch_chunk_heads(bt->perm, total_len, counts, bt->nchunks, s)) != FSPARSE_OK)
            return fail(e);
        if ((e = exclusive_scan_u32(counts, bt->chunk_slot0, bt->nchunks, d_st, scratch, s)) != FSPARSE_OK)
            return fail(e);
        if ((e = read_status(d_st, &h_st, s)) != FSPARSE_OK) return fail(e);
        if (h_st.timeout) return fail(set_error(FSPARSE_ERR_TIMEOUT, "device look-back wait expired"));
    }
    *batch_out = reinterpret_cast<fsparse_batch>(bt);
    return FSPARSE_OK;
}

// Many instances in one symbolic pass (batch.cu explains the numbering):
// remap the columns into the concatenated matrix [S_0 ... S_{count-1}], run
// the single-problem symbolic phase on it, and keep its sorted order as the
// batch's numeric plan and its irS as the instances' rows.
fsparse_status fsparse_batch_symbolic(int32_t count, const int32_t *ii, const int32_t *jj,
                                      const int64_t *h_len_off, const int32_t *h_m, const int32_t *h_n,
                                      void *stream, fsparse_batch *batch_out) {
    NvtxRange nvtx_("fsparse_batch_symbolic");
    if (!batch_out) return set_error(FSPARSE_ERR_ARG, "batch_out is NULL");
    *batch_out = nullptr;
    if (count < 0 || (count > 0 && (!h_len_off || !h_m || !h_n)))
        return set_error(FSPARSE_ERR_ARG, "bad instance description");
    int64_t total = 0;
    if (count > 0) {
        if (h_len_off[0] != 0) return set_error(FSPARSE_ERR_ARG, "h_len_off[0] must be 0");
        for (int32_t b = 0; b < count; ++b) {
            if (h_len_off[b + 1] < h_len_off[b]) return set_error(FSPARSE_ERR_ARG, "h_len_off decreases");
            if (h_m[b] < 0 || h_n[b] < 0) return set_error(FSPARSE_ERR_ARG, "negative dimension");
        }
        total = h_len_off[count];
    }
    if (total > kMaxLen) return set_error(FSPARSE_ERR_SIZE, "batch total len above 2^30 - 1");
    if (total > 0 && (!ii || !jj)) return set_error(FSPARSE_ERR_ARG, "NULL index array");
    cudaStream_t s = as_stream(stream);
    int dev = 0;
    FSP_CUDA(cudaGetDevice(&dev));
    fsparse_status e;
    if ((e = ensure_pool(dev)) != FSPARSE_OK) return e;

    Batch *bt = new (std::nothrow) Batch();
    if (!bt) return set_error(FSPARSE_ERR_NOMEM, "host allocation");
    bt->device = dev;
    bt->count = count;
    bt->symbolic = true;
    bt->total_len = total;
    const int cn = std::max(count, 1);
    bt->h_len_off = new (std::nothrow) int64_t[cn + 1];
    bt->h_nnz_off = new (std::nothrow) int64_t[cn + 1];
    bt->h_m = new (std::nothrow) int32_t[cn];
    bt->h_n = new (std::nothrow) int32_t[cn];
    Plan *P = nullptr;
    auto fail = [&](fsparse_status st) {
        for (void *q : {static_cast<void *>(bt->perm), static_cast<void *>(bt->chunk_slot0),
                        static_cast<void *>(bt->irank), static_cast<void *>(bt->jcS), static_cast<void *>(bt->irS),
                        static_cast<void *>(bt->d_len_off), static_cast<void *>(bt->d_nnz_off)})
            if (q) cudaFreeAsync(q, s);
        if (P) {
            free_plan_arrays_on(*P, s);
            delete P;
        }
        cudaGetLastError();
        delete[] bt->h_len_off;
        delete[] bt->h_nnz_off;
        delete[] bt->h_m;
        delete[] bt->h_n;
        delete bt;
        return st;
    };
    if (!bt->h_len_off || !bt->h_nnz_off || !bt->h_m || !bt->h_n)
        return fail(set_error(FSPARSE_ERR_NOMEM, "host allocation"));
    bt->h_len_off[0] = 0;
    for (int32_t b = 0; b < count; ++b) {
        bt->h_len_off[b + 1] = h_len_off[b + 1];
        bt->h_m[b] = h_m[b];
        bt->h_n[b] = h_n[b];
    }
    if ((e = device_alloc(reinterpret_cast<void **>(&bt->d_len_off), (size_t)(cn + 1) * 8, s)) ||
        (e = device_alloc(reinterpret_cast<void **>(&bt->d_nnz_off), (size_t)(cn + 1) * 8, s)))
        return fail(e);
    if (cudaMemcpyAsync(bt->d_len_off, bt->h_len_off, (size_t)(count + 1) * 8, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return fail(cuda_error(cudaGetLastError(), "cudaMemcpyAsync"));

    std::vector<int64_t> col_off((size_t)count + 1, 0);
    int32_t m_all = 0;
    {
        Scratch scratch(s);
        bool implicit = false;
        for (int32_t b = 0; b < count; ++b) implicit |= bt->h_m[b] == 0 || bt->h_n[b] == 0;
        if (implicit && total > 0) {   // implicit dimensions of some instances (§2.2): one extra synchronisation
            int32_t *dmax = nullptr;
            if ((e = scratch.get(&dmax, (size_t)2 * cn)) != FSPARSE_OK) return fail(e);
            std::vector<int32_t> hmax((size_t)2 * cn, 0);
            if (cudaMemsetAsync(dmax, 0, (size_t)2 * cn * 4, s) != cudaSuccess)
                return fail(cuda_error(cudaGetLastError(), "cudaMemsetAsync"));
            if ((e = launch_batch_dims(ii, jj, bt->d_len_off, count, total, dmax, dmax + cn, s)) != FSPARSE_OK)
                return fail(e);
            if (cudaMemcpyAsync(hmax.data(), dmax, (size_t)2 * cn * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return fail(cuda_error(cudaGetLastError(), "reading instance dimensions"));
            for (int32_t b = 0; b < count; ++b) {
                if (bt->h_m[b] == 0) bt->h_m[b] = std::max(hmax[b], 0);
                if (bt->h_n[b] == 0) bt->h_n[b] = std::max(hmax[cn + b], 0);
            }
        }
        for (int32_t b = 0; b < count; ++b) {
            col_off[b + 1] = col_off[b] + bt->h_n[b];
            m_all = std::max(m_all, bt->h_m[b]);
        }
        if (col_off[count] > INT32_MAX)
            return fail(set_error(FSPARSE_ERR_SIZE, "the instances' columns add up beyond 2^31 - 1"));
        const int32_t n_all = (int32_t)col_off[count];
        int64_t *d_col_off = nullptr, *d_jcs_off = nullptr;
        int32_t *d_m = nullptr, *jj2 = nullptr;
        std::vector<int64_t> jcs_off((size_t)count + 1, 0);
        for (int32_t b = 0; b < count; ++b) jcs_off[b + 1] = jcs_off[b] + bt->h_n[b] + 1;
        if ((e = scratch.get(&d_col_off, (size_t)cn + 1)) || (e = scratch.get(&d_jcs_off, (size_t)cn + 1)) ||
            (e = scratch.get(&d_m, (size_t)cn)) || (e = scratch.get(&jj2, (size_t)std::max<int64_t>(total, 1))))
            return fail(e);
        if (cudaMemcpyAsync(d_col_off, col_off.data(), (size_t)(count + 1) * 8, cudaMemcpyHostToDevice, s) ||
            cudaMemcpyAsync(d_jcs_off, jcs_off.data(), (size_t)(count + 1) * 8, cudaMemcpyHostToDevice, s) ||
            (count > 0 && cudaMemcpyAsync(d_m, bt->h_m, (size_t)count * 4, cudaMemcpyHostToDevice, s)))
            return fail(cuda_error(cudaGetLastError(), "cudaMemcpyAsync"));
        if ((e = launch_batch_remap(ii, jj, bt->d_len_off, d_col_off, d_m, count, total, jj2, s)) != FSPARSE_OK)
            return fail(e);
        // The whole batch as one problem: bad indices of any instance arrive
        // as column 0 and are reported here.
        if ((e = symbolic_impl(ii, jj2, nullptr, nullptr, total, total > 0 ? std::max(m_all, 1) : m_all,
                               total > 0 ? std::max(n_all, 1) : n_all, 0, s, &P, nullptr)) != FSPARSE_OK)
            return fail(e);
        if ((e = launch_batch_nnz_off(P->jcS, d_col_off, count, bt->d_nnz_off, s)) != FSPARSE_OK) return fail(e);
        const int64_t jcs_total = jcs_off[count];
        if ((e = device_alloc(reinterpret_cast<void **>(&bt->jcS), (size_t)std::max<int64_t>(jcs_total, 1) * 4, s)))
            return fail(e);
        if ((e = launch_batch_jcs(P->jcS, d_col_off, d_jcs_off, bt->d_nnz_off, count, jcs_total, bt->jcS, s)))
            return fail(e);
        if (cudaMemcpyAsync(bt->h_nnz_off, bt->d_nnz_off, (size_t)(count + 1) * 8, cudaMemcpyDeviceToHost, s) ||
            cudaStreamSynchronize(s))
            return fail(cuda_error(cudaGetLastError(), "reading instance offsets"));
    }
    if (count == 0) bt->h_nnz_off[0] = 0;
    // The concatenated plan's arrays become the batch's.
    bt->total_nnz = P->nnz;
    bt->perm = P->perm;
    bt->chunk_slot0 = P->chunk_slot0;
    bt->irS = P->irS;
    bt->irank = P->irank;
    bt->numeric_tile = P->numeric_tile;
    bt->nchunks = P->nchunks;
    cudaFreeAsync(P->jcS, s);
    cudaGetLastError();
    P->perm = P->chunk_slot0 = nullptr;
    P->irS = P->irank = P->jcS = nullptr;
    delete P;
    *batch_out = reinterpret_cast<fsparse_batch>(bt);
    return FSPARSE_OK;
}

fsparse_status fsparse_batch_arrays(fsparse_batch batch, const int32_t **irank, const int32_t **jcS,
                                    const int32_t **irS, int32_t *h_m, int32_t *h_n) {
    if (!batch) return set_error(FSPARSE_ERR_ARG, "batch is NULL");
    Batch &b = reinterpret_cast<fsparse_batch_s *>(batch)->b;
    if (!b.symbolic) return set_error(FSPARSE_ERR_ARG, "a batch made from plans keeps its arrays in the plans");
    if (irank && !b.irank_ready) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != b.device) cudaSetDevice(b.device);
        fsparse_status e = launch_irank(b.perm, b.chunk_slot0, b.total_len, b.irank, nullptr);
        if (e == FSPARSE_OK)
            e = launch_batch_irank(b.irank, b.d_len_off, b.d_nnz_off, b.count, b.total_len, nullptr);
        if (e == FSPARSE_OK && cudaStreamSynchronize(nullptr) != cudaSuccess)
            e = cuda_error(cudaGetLastError(), "cudaStreamSynchronize");
        if (cur != b.device) cudaSetDevice(cur);
        if (e != FSPARSE_OK) return e;
        b.irank_ready = true;
    }
    if (irank) *irank = b.irank;
    if (jcS) *jcS = b.jcS;
    if (irS) *irS = b.irS;
    if (h_m) std::memcpy(h_m, b.h_m, sizeof(int32_t) * b.count);
    if (h_n) std::memcpy(h_n, b.h_n, sizeof(int32_t) * b.count);
    return FSPARSE_OK;
}

fsparse_status fsparse_batch_info(fsparse_batch batch, int32_t *count, int64_t *h_len_off,
                                  int64_t *h_nnz_off) {
    if (!batch) return set_error(FSPARSE_ERR_ARG, "batch is NULL");
    const Batch &b = reinterpret_cast<fsparse_batch_s *>(batch)->b;
    if (count) *count = b.count;
    if (h_len_off) std::memcpy(h_len_off, b.h_len_off, sizeof(int64_t) * (b.count + 1));
    if (h_nnz_off) std::memcpy(h_nnz_off, b.h_nnz_off, sizeof(int64_t) * (b.count + 1));
    return FSPARSE_OK;
}

fsparse_status fsparse_batch_numeric(fsparse_batch batch, const double *sr_concat, double *prS_concat,
                                     void *stream) {
    NvtxRange nvtx_("fsparse_batch_numeric");
    if (!batch) return set_error(FSPARSE_ERR_ARG, "batch is NULL");
    const Batch &b = reinterpret_cast<fsparse_batch_s *>(batch)->b;
    if (b.total_len > 0 && (!sr_concat || !prS_concat)) return set_error(FSPARSE_ERR_ARG, "NULL array");
    const fsparse_status e = launch_numeric(b.perm, b.chunk_slot0, b.total_len, b.numeric_tile, sr_concat,
                                            prS_concat, b.total_nnz, b.total_nnz, as_stream(stream));
    if (e == FSPARSE_OK) note_use(reinterpret_cast<fsparse_batch_s *>(batch)->b.uses, as_stream(stream));
    return e;
}

static fsparse_status destroy_batch(fsparse_batch batch, cudaStream_t after) {
    if (!batch) return FSPARSE_OK;
    Batch *b = &reinterpret_cast<fsparse_batch_s *>(batch)->b;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    void *ptrs[7] = {b->perm, b->chunk_slot0, b->irank, b->jcS, b->irS, b->d_len_off, b->d_nnz_off};
    release_after(ptrs, 7, b->uses, after);
    if (cur != b->device) cudaSetDevice(cur);
    delete[] b->h_len_off;
    delete[] b->h_nnz_off;
    delete[] b->h_m;
    delete[] b->h_n;
    delete b;
    return FSPARSE_OK;
}

fsparse_status fsparse_batch_destroy(fsparse_batch batch) { return destroy_batch(batch, nullptr); }

fsparse_status fsparse_batch_release(fsparse_batch batch, void *stream) {
    return destroy_batch(batch, as_stream(stream));
}

// ---- diagnostics ------------------------------------------------------------
const char *fsparse_last_error_string(void) { return g_err.c_str(); }

const char *fsparse_status_string(fsparse_status st) {
    switch (st) {
        case FSPARSE_OK: return "FSPARSE_OK";
        case FSPARSE_ERR_ARG: return "FSPARSE_ERR_ARG";
        case FSPARSE_ERR_INDEX: return "FSPARSE_ERR_INDEX";
        case FSPARSE_ERR_NZMAX: return "FSPARSE_ERR_NZMAX";
        case FSPARSE_ERR_SIZE: return "FSPARSE_ERR_SIZE";
        case FSPARSE_ERR_NOMEM: return "FSPARSE_ERR_NOMEM";
        case FSPARSE_ERR_CUDA: return "FSPARSE_ERR_CUDA";
        case FSPARSE_ERR_TIMEOUT: return "FSPARSE_ERR_TIMEOUT";
        case FSPARSE_ERR_INTERNAL: return "FSPARSE_ERR_INTERNAL";
    }
    return "FSPARSE_STATUS_UNKNOWN";
}

int64_t fsparse_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"

// ---- autotuning (needs the internals above) -----------------------------------
namespace fsp {
void tune_store(int64_t len, const KeyLayout &key, const fsparse_config &cfg);
std::vector<fsparse_config> tune_candidates(int64_t len, const KeyLayout &key);
}  // namespace fsp

extern "C" fsparse_status fsparse_autotune(const int32_t *ii, const int32_t *jj, const double *sr,
                                           int64_t len, int32_t m, int32_t n, int32_t reps,
                                           void *stream, fsparse_config *best) {
    if (reps < 1 || m <= 0 || n <= 0) return set_error(FSPARSE_ERR_ARG, "autotune needs reps >= 1 and explicit m, n");
    if (len <= 0 || !sr) return set_error(FSPARSE_ERR_ARG, "autotune needs a non-empty problem");
    cudaStream_t s = as_stream(stream);
    KeyLayout key;
    key.rb = bits_for((uint64_t)m - 1);
    key.cb = bits_for((uint64_t)n - 1);
    double *prS = nullptr;
    fsparse_status e;
    if ((e = device_alloc(reinterpret_cast<void **>(&prS), (size_t)len * 8, s)) != FSPARSE_OK) return e;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    float best_ms = 1e30f;
    fsparse_config best_cfg = resolve_config(len, key);
    // 1. The sort configuration, by the time of the symbolic call alone.
    for (const fsparse_config &c : tune_candidates(len, key)) {
        std::vector<float> times;
        bool ok = true;
        for (int r = 0; r < reps + 1 && ok; ++r) {   // first run warms the pool and caches
            Plan *p = nullptr;
            cudaEventRecord(t0, s);
            e = symbolic_impl(ii, jj, nullptr, nullptr, len, m, n, 0, s, &p, &c);
            cudaEventRecord(t1, s);
            cudaEventSynchronize(t1);
            if (e != FSPARSE_OK) {
                ok = false;
                break;
            }
            const bool fell_back = p->cfg.strategy != c.strategy;
            fsparse_plan_destroy(reinterpret_cast<fsparse_plan>(p));
            if (fell_back) {
                ok = false;
                break;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, t0, t1);
            if (r > 0) times.push_back(ms);
        }
        if (!ok) continue;
        std::sort(times.begin(), times.end());
        const float med = times[times.size() / 2];
        if (med < best_ms) {
            best_ms = med;
            best_cfg = c;
        }
    }
    // 2. The numeric tile, by repeated folds on the winner's plan (re-assembly
    //    is where the fold's speed counts).
    if (best_ms < 1e30f) {
        Plan *p = nullptr;
        if (symbolic_impl(ii, jj, nullptr, nullptr, len, m, n, 0, s, &p, &best_cfg) == FSPARSE_OK) {
            float best_fold = 1e30f;
            for (int tile : {1024, 2048, 4096}) {
                const int folds = 4 * reps + 2;
                bool ok = launch_numeric(p->perm, p->chunk_slot0, len, tile, sr, prS, p->nnz, p->cap, s) == FSPARSE_OK;
                cudaEventRecord(t0, s);
                for (int r = 0; r < folds && ok; ++r)
                    ok = launch_numeric(p->perm, p->chunk_slot0, len, tile, sr, prS, p->nnz, p->cap, s) == FSPARSE_OK;
                cudaEventRecord(t1, s);
                cudaEventSynchronize(t1);
                float ms = 0;
                cudaEventElapsedTime(&ms, t0, t1);
                if (ok && ms < best_fold) {
                    best_fold = ms;
                    best_cfg.numeric_tile = tile;
                }
            }
            fsparse_plan_destroy(reinterpret_cast<fsparse_plan>(p));
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFreeAsync(prS, s);
    cudaStreamSynchronize(s);
    if (best_ms >= 1e30f) return set_error(FSPARSE_ERR_CUDA, "no candidate configuration ran");
    tune_store(len, key, best_cfg);
    if (best) *best = best_cfg;
    return FSPARSE_OK;
}
