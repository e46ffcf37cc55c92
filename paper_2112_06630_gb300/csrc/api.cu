// api.cu -- the C ABI (include/knng.h): argument checks, the context and its
// device memory, and the order in which the kernels of an NN-Descent build are
// enqueued.  No computation of the method happens here; every step is a
// kernel launch on the caller's stream.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <array>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/knng.h"
#include "internal.h"
#include "join_common.cuh"

using namespace knng;

namespace {

constexpr int kMaxItersArg = 1000;

int rev_capacity(int s) { return 2 * s + 8; }

// s = ceil(rho K); the tolerance absorbs the float32 rounding of rho (0.3f x
// 10 = 3.0000001 must give 3), far below any fractional part of rho K
int sample_size(float rho, int K) {
    int s = (int)std::ceil((double)rho * (double)K - 1e-5);
    if (s < 1) s = 1;
    if (s > K) s = K;
    return s;
}

// Where a caller's buffer lives.  Host memory (pageable, pinned or registered)
// goes through a device copy; memory of the current device, and managed
// memory it can reach, is used in place; another device's memory is refused
// before anything is launched (the kernels would fault on it, or read it over
// the link without notice).
enum class Where { kHost, kDevice, kForeign };

Where where(const void *p) {
    if (!p) return Where::kHost;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return Where::kHost;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return Where::kHost;
    int dev = 0, cma = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return Where::kForeign;
    }
    if (cudaDeviceGetAttribute(&cma, cudaDevAttrConcurrentManagedAccess, dev) != cudaSuccess) {
        cudaGetLastError();
        cma = 0;
    }
    // test hook: classify as if another device were current (every device
    // pointer then belongs to a foreign device), with nothing launched
    if (std::getenv("KNNG_TEST_FOREIGN_DEVICE")) {
        dev += 1;
        cma = 0;
    }
    if (a.type == cudaMemoryTypeDevice) return a.device == dev ? Where::kDevice : Where::kForeign;
    return (a.device == dev || cma != 0) ? Where::kDevice : Where::kForeign;
}

bool is_device_ptr(const void *p) { return where(p) == Where::kDevice; }
bool is_foreign_ptr(const void *p) { return where(p) == Where::kForeign; }

// Maps a CUDA error to a return code and clears it as the thread's last error,
// so that a failed call does not fail the next, unrelated launch check.
int cuda_code(cudaError_t e) {
    if (e == cudaSuccess) return KNNG_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? KNNG_ERR_OOM : KNNG_ERR_CUDA;
}

#define KNNG_TRY(expr)                              \
    do {                                            \
        cudaError_t _e = (expr);                    \
        if (_e != cudaSuccess) return cuda_code(_e); \
    } while (0)

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device memory comes from a pool owned by the library (one per device) whose
// release threshold is unlimited: memory freed by one build stays mapped for
// the next, instead of being returned at every stream synchronisation (the
// default pool's behaviour), which made each build re-map its arena.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[256];

cudaError_t lib_malloc(void **p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaMallocAsync(p, bytes, s);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> g(g_pool_mu);
        if (!g_pool[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&g_pool[dev], &props);
            if (e != cudaSuccess) {
                g_pool[dev] = nullptr;
                return e;
            }
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        }
        pool = g_pool[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}


int check_args(int64_t n, int d, int K, float rho, float delta) {
    if (n < 2 || n >= (int64_t(1) << 30) - 1) return KNNG_ERR_INVALID_ARG;
    if (d < 1 || K < 1 || K > n - 1) return KNNG_ERR_INVALID_ARG;
    if (!(rho > 0.0f && rho <= 1.0f) || !(delta >= 0.0f)) return KNNG_ERR_INVALID_ARG;
    if (K > kMaxK) return KNNG_ERR_UNSUPPORTED;
    return KNNG_OK;
}

}  // namespace

struct knng_ctx {
    int64_t n = 0;
    int d = 0, dp = 0, nv = 0, K = 0, s = 0, R = 0, cap = 0, pool_chunks = 0;
    float rho = 0, delta = 0;
    uint64_t seed = 0;
    uint32_t flags = 0;
    cudaStream_t stream = nullptr;
    double thr = 0;
    int it_done = 0;    // absolute iterations done (selects the random streams)
    int li = 0;         // iterations launched by this context
    bool reordered = false;
    bool tune_pending = false;  // KNNG_FLAG_AUTOTUNE: the first iteration times the join kernels
    long long launches = 0;

    unsigned char *arena = nullptr;
    float *X = nullptr, *X2 = nullptr;
    uint64_t *keys = nullptr, *keys2 = nullptr;
    int *locks = nullptr, *ibuf = nullptr, *cand = nullptr, *err = nullptr, *pcursor = nullptr;
    bool heap = false;  // KNNG_FLAG_HEAP_SAMPLING
    unsigned char *rscratch = nullptr;  // KNNG_FLAG_REORDER_PARALLEL scratch
    int *hoff = nullptr, *hcursor = nullptr;
    uint64_t *hcsr = nullptr;
    int *pchunk = nullptr, *pool_next = nullptr;
    uint16_t *Xb = nullptr, *Xb2 = nullptr;
    float *xnorm = nullptr, *xnorm2 = nullptr;
    int dpb = 0;
    bool bf16 = false;
    bool fp8 = false;  // KNNG_FLAG_FP8 taken: e4m3 rows in Xb
    // precision of the join's rows: 0 float32, 1 bf16, 2 e4m3
    int kind() const { return fp8 ? 2 : bf16 ? 1 : 0; }
    int join_path = kJoinWarp;
    int *cset = nullptr, *cmeta = nullptr;
    uint64_t *pbucket = nullptr, *ppool = nullptr;
    int32_t *sigma = nullptr, *sigma_inv = nullptr, *total_perm = nullptr, *total_inv = nullptr;
    long long *stats = nullptr, *it_stats = nullptr;

    // batched mode
    int nds = 0;
    unsigned char *barena = nullptr;
    int *ds = nullptr, *ds_n = nullptr;
    long long *ds_off = nullptr, *ds_changes = nullptr;
    double *ds_thr = nullptr;

    std::vector<cudaGraphExec_t> graphs;  // captured iteration loops (KNNG_FLAG_GRAPH)
    cudaStream_t capture = nullptr;       // private stream the loops are captured on

    std::vector<cudaEvent_t> ev;  // per timed iteration: before the count, after the sampling
    std::vector<int> ev_li;       // iteration index of each pair
    struct PassEvents {
        int li;
        cudaEvent_t join0, join1, merge1;  // before and after a join pass, after its merge
    };
    std::vector<PassEvents> pev;  // per timed join pass
    std::vector<cudaEvent_t> rev; // start/stop pairs around relabellings (KNNG_FLAG_TIMING)

    DevState dev(bool gate) const {
        DevState st;
        st.X = X;
        st.Xb = Xb;
        st.xnorm = xnorm;
        st.keys = keys;
        st.locks = locks;
        st.pcursor = pcursor;
        st.pbucket = pbucket;
        st.pchunk = pchunk;
        st.ppool = ppool;
        st.pool_next = pool_next;
        st.pool_chunks = pool_chunks;
        st.rev_new = ibuf;
        st.rev_old = ibuf + n;
        st.fill_new = ibuf + 2 * n;
        st.fill_old = ibuf + 3 * n;
        st.fwd_new = ibuf + 4 * n;
        st.fwd_old = ibuf + 5 * n;
        st.cand_new = cand;
        st.cand_old = cand + (size_t)n * cap;
        st.hoff = hoff;
        st.hcsr = hcsr;
        st.hcursor = hcursor;
        st.stats = stats;
        st.it_stats = it_stats;
        st.n = n;
        st.d = d;
        st.dp = dp;
        st.dpb = dpb;
        st.bf16 = (bf16 || fp8) ? 1 : 0;
        st.fp8 = fp8 ? 1 : 0;
        st.nv = nv;
        st.K = K;
        st.s = s;
        st.R = R;
        st.cap = cap;
        st.thr = gate ? thr : -1.0;
        st.ds = ds;
        st.ds_off = ds_off;
        st.ds_n = ds_n;
        st.ds_thr = ds_thr;
        st.ds_changes = ds_changes;
        st.cset = cset;
        st.cmeta = cmeta;
        st.join_path = join_path;
        st.u_lo = 0;
        st.u_hi = n;
        return st;
    }
};

namespace {

// knng_bruteforce_last_fallbacks: this thread's last tensor-core brute force
thread_local int g_bf_fallbacks = -1;
thread_local float g_bf_prefilter_ms = -1.f;

// Join kernels chosen by the autotuner, per geometry (bf16, row width, K,
// reverse capacity), for the life of the process.
std::mutex g_tune_mu;
std::map<std::array<int, 4>, int> g_tune_cache;

std::array<int, 4> tune_key(const knng_ctx *c) { return {c->kind(), c->kind() ? c->dpb : c->dp, c->K, c->R}; }

int ctx_alloc(knng_ctx *c) {
    const int64_t n = c->n;
    const bool reorder = (c->flags & KNNG_FLAG_REORDER) != 0;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t oX = take(sizeof(float) * n * c->dp);
    const size_t oX2 = reorder ? take(sizeof(float) * n * c->dp) : 0;
    const size_t oK = take(sizeof(uint64_t) * n * c->K);
    const size_t oK2 = reorder ? take(sizeof(uint64_t) * n * c->K) : 0;
    // locks | bucket cursors | bucket chunk tables | pool cursor
    const size_t nint = (size_t)n * (2 + kBucketChunks) + 1;
    const size_t oL = take(sizeof(int) * nint);
    const size_t oB = take(sizeof(uint64_t) * (size_t)n * kBucketRun);
    const size_t oQ = take(sizeof(uint64_t) * (size_t)c->pool_chunks * kBucketRun);
    const size_t oI = take(sizeof(int) * 6 * n);
    const size_t oC = take(sizeof(int) * 2 * (size_t)n * c->cap);
    const size_t oP = reorder ? take(sizeof(int32_t) * 4 * n) : 0;
    const size_t oS = take(sizeof(long long) * kStatCount);
    const size_t oT = take(sizeof(long long) * kItCount * kMaxLocalIters);
    const size_t oE = take(sizeof(int));
    const size_t oXb = c->fp8 ? take((size_t)n * c->dpb) : c->bf16 ? take(sizeof(uint16_t) * n * c->dpb) : 0;
    const size_t oXn = (c->bf16 || c->fp8) ? take(sizeof(float) * n) : 0;
    const bool ring = c->join_path == kJoinRing || c->join_path == kJoinPipe || c->join_path == kJoinPipe8 ||
                      (c->tune_pending && (ring_join_fits(c->kind(), c->nv, c->dpb, c->K) ||
                                           pipe_join_fits(c->kind(), c->nv)));
    const size_t oCs = ring ? take(sizeof(int) * (size_t)n * kSetMax) : 0;
    const size_t oCm = ring ? take(sizeof(int) * (size_t)n) : 0;
    const bool prel = reorder && (c->flags & KNNG_FLAG_REORDER_PARALLEL);
    const size_t oR = prel ? take(parallel_relabel_scratch(n, c->K)) : 0;
    const size_t oHo = c->heap ? take(sizeof(int) * (2 * (size_t)n + 1)) : 0;
    const size_t oHc = c->heap ? take(sizeof(uint64_t) * (size_t)n * c->K) : 0;
    cudaError_t e = lib_malloc((void **)&c->arena, off, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_code(e);
    }
    unsigned char *a = c->arena;
    c->X = (float *)(a + oX);
    c->X2 = reorder ? (float *)(a + oX2) : nullptr;
    c->keys = (uint64_t *)(a + oK);
    c->keys2 = reorder ? (uint64_t *)(a + oK2) : nullptr;
    c->locks = (int *)(a + oL);
    c->pcursor = c->locks + n;
    c->pchunk = c->locks + 2 * n;
    c->pool_next = c->pchunk + (size_t)n * kBucketChunks;
    c->pbucket = (uint64_t *)(a + oB);
    c->ppool = (uint64_t *)(a + oQ);
    c->ibuf = (int *)(a + oI);
    c->cand = (int *)(a + oC);
    if (reorder) {
        int32_t *p = (int32_t *)(a + oP);
        c->sigma = p;
        c->sigma_inv = p + n;
        c->total_perm = p + 2 * n;
        c->total_inv = p + 3 * n;
    }
    c->stats = (long long *)(a + oS);
    c->it_stats = (long long *)(a + oT);
    c->err = (int *)(a + oE);
    if (c->bf16 || c->fp8) {
        c->Xb = (uint16_t *)(a + oXb);
        c->xnorm = (float *)(a + oXn);
    }
    if (ring) {
        c->cset = (int *)(a + oCs);
        c->cmeta = (int *)(a + oCm);
    }
    if (prel) c->rscratch = a + oR;
    if (c->heap) {
        c->hoff = (int *)(a + oHo);
        c->hcursor = c->hoff + 2 * n;
        c->hcsr = (uint64_t *)(a + oHc);
    }
    KNNG_TRY(cudaMemsetAsync(c->locks, 0, sizeof(int) * nint, c->stream));
    // test hook: the locks of the first h lists start held, so a locked
    // insertion into one of them runs its bounded wait out and the call
    // reports KNNG_ERR_TIMEOUT
    if (const char *e = std::getenv("KNNG_TEST_HOLD_LOCKS")) {
        const int64_t h = std::min<int64_t>(n, std::max<int64_t>(1, std::atoll(e)));
        KNNG_TRY(cudaMemsetAsync(c->locks, 1, sizeof(int) * h, c->stream));
    }
    KNNG_TRY(cudaMemsetAsync(c->ibuf, 0, sizeof(int) * 6 * n, c->stream));
    KNNG_TRY(cudaMemsetAsync(c->stats, 0, sizeof(long long) * kStatCount, c->stream));
    KNNG_TRY(cudaMemsetAsync(c->it_stats, 0, sizeof(long long) * kItCount * kMaxLocalIters, c->stream));
    KNNG_TRY(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    return KNNG_OK;
}

// The low-precision copy of the staged rows the join reads, if any.
cudaError_t stage_low_precision(knng_ctx *c) {
    if (c->fp8) {
        c->launches++;
        return launch_stage_fp8(c->X, c->n, c->dp, c->d, reinterpret_cast<uint8_t *>(c->Xb), c->dpb, c->xnorm,
                                c->stream);
    }
    if (c->bf16) {
        c->launches++;
        return launch_stage_bf16(c->X, c->n, c->dp, c->d, c->Xb, c->dpb, c->xnorm, c->stream);
    }
    return cudaSuccess;
}

// Stage the caller's points (host or device) into the padded layout.
int ctx_stage(knng_ctx *c, const float *data) {
    const size_t bytes = sizeof(float) * c->n * c->d;
    const float *src = data;
    float *tmp = nullptr;
    cudaError_t e = cudaSuccess;
    if (!is_device_ptr(data)) {
        e = lib_malloc((void **)&tmp, bytes, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, data, bytes, cudaMemcpyHostToDevice, c->stream);
        src = tmp;
    }
    if (e == cudaSuccess) e = launch_stage(src, c->n, c->d, c->X, c->dp, c->stream);
    if (e == cudaSuccess) {
        c->launches++;
        e = stage_low_precision(c);
    }
    // the staging copy is freed on every path, a failed one included
    if (tmp) {
        const cudaError_t f = cudaFreeAsync(tmp, c->stream);
        if (e == cudaSuccess) e = f;
    }
    return cuda_code(e);
}

// data == nullptr: allocate only (the batched build stages its data sets)
int ctx_create(knng_ctx **out, const float *data, int64_t n, int d, int K, float rho, float delta, uint64_t seed,
               uint32_t flags, void *stream) {
    if (!out) return KNNG_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = check_args(n, d, K, rho, delta);
    if (rc) return rc;
    if (data && is_foreign_ptr(data)) return KNNG_ERR_INVALID_ARG;
    // lists of more than 32 keys: float32 keys with turbosampling only (the
    // low-precision forms resolve keys per id, and heap selection keeps its
    // lists one per lane)
    if (K > kLaneK && (flags & (KNNG_FLAG_BF16 | KNNG_FLAG_FP8 | KNNG_FLAG_HEAP_SAMPLING)))
        return KNNG_ERR_UNSUPPORTED;
    knng_ctx *c = new (std::nothrow) knng_ctx();
    if (!c) return KNNG_ERR_OOM;
    c->n = n;
    c->d = d;
    c->dp = (d + 3) & ~3;
    c->nv = c->dp / 4;
    c->K = K;
    c->s = sample_size(rho, K);
    c->R = rev_capacity(c->s);
    c->cap = K + c->R;
    // bucket pool: two 256-key runs per node on top of the inline run (the
    // first, dense iteration averages about (2s)^2 proposals per node), but at
    // most 16 GiB: past about 4M points an iteration takes more node-range
    // passes (join_passes) instead of more memory, so the buckets cost a
    // fixed 2 KiB inline run per node plus the pool
    constexpr int64_t kPoolMaxChunks = ((int64_t)16 << 30) / ((int64_t)kBucketRun * (int64_t)sizeof(uint64_t));
    c->pool_chunks = (int)std::min<int64_t>(2 * n + 4096, kPoolMaxChunks);
    // test hook: a smaller pool drives proposals through the poisoned-run and
    // locked-insertion paths
    if (const char *e = std::getenv("KNNG_TEST_BUCKET_POOL_CHUNKS")) c->pool_chunks = std::max(1, std::atoi(e));
    c->rho = rho;
    c->delta = delta;
    c->seed = seed;
    c->flags = flags;
    // bf16 tensor-core dots where the contraction is long enough to pay
    c->bf16 = (flags & KNNG_FLAG_BF16) && d >= 64;
    c->heap = (flags & KNNG_FLAG_HEAP_SAMPLING) != 0;
    // the reverse-offer segments are addressed with 32-bit offsets
    if (c->heap && (int64_t)n * K >= ((int64_t)1 << 31)) {
        delete c;
        return KNNG_ERR_UNSUPPORTED;
    }
    c->dpb = (d + 63) & ~63;
    // FP8 (e4m3) rows where the ring kernel holds them (it is their only join
    // kernel); otherwise the flag is not taken
    c->fp8 = (flags & KNNG_FLAG_FP8) && d >= 64 && ring_join_fits(2, c->nv, c->dpb, K);
    if (c->fp8) c->bf16 = false;
    // test hook: run another join kernel the context can use (parity of the
    // three kernels on the same inputs)
    int force = -1;
    if (const char *e = std::getenv("KNNG_TEST_JOIN_PATH")) {
        if (!std::strcmp(e, "warp")) force = kJoinWarp;
        else if (!std::strcmp(e, "tile")) force = kJoinTile;
        else if (!std::strcmp(e, "ring")) force = kJoinRing;
        else if (!std::strcmp(e, "pipe")) force = kJoinPipe;
        else if (!std::strcmp(e, "pipe8")) force = kJoinPipe8;
    }
    c->join_path = choose_join_path(c->kind(), c->nv, c->dpb, K, force);
    if ((flags & KNNG_FLAG_AUTOTUNE) && force < 0) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(tune_key(c));
        if (it != g_tune_cache.end()) c->join_path = it->second;
        else c->tune_pending = true;
    }
    c->stream = (cudaStream_t)stream;
    c->thr = (double)delta * (double)n * (double)K;
    rc = ctx_alloc(c);
    if (!rc && data) rc = ctx_stage(c, data);
    if (!rc && c->total_perm) {
        // the relabelling original -> spot starts as the identity
        rc = cuda_code(launch_iota(c->total_perm, c->n, c->stream));
        c->launches++;
    }
    if (rc) {
        knng_destroy(c);
        return rc;
    }
    *out = c;
    return KNNG_OK;
}

// Read the device error word and lock-timeout counter (synchronises the stream).
int ctx_check(knng_ctx *c) {
    int err = 0;
    long long st[kStatCount];
    KNNG_TRY(cudaMemcpyAsync(&err, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    KNNG_TRY(cudaMemcpyAsync(st, c->stats, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    KNNG_TRY(cudaStreamSynchronize(c->stream));
    KNNG_TRY(cudaGetLastError());
    if (err & 2) return KNNG_ERR_INVALID_ARG;
    if (err) return KNNG_ERR_INTERNAL;
    if (st[kStatLockTimeout]) return KNNG_ERR_TIMEOUT;
    if (st[kStatRevOverflow] || st[kStatSetOverflow]) return KNNG_WARN_OVERFLOW;
    return KNNG_OK;
}

int enqueue_reorder(knng_ctx *c) {
    if (!c->sigma) return KNNG_ERR_STATE;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (c->flags & KNNG_FLAG_TIMING) {
        for (auto &e : ev) KNNG_TRY(cudaEventCreate(&e));
        for (auto &e : ev) c->rev.push_back(e);
        KNNG_TRY(cudaEventRecord(ev[0], c->stream));
    }
    if (c->rscratch) {
        int nl = 0;
        KNNG_TRY(launch_parallel_relabel(c->X, c->keys, c->n, c->K, c->nv, c->sigma, c->rscratch, &nl, c->stream));
        c->launches += nl;
    } else {
        const int reading_b = (c->flags & KNNG_FLAG_REORDER_B) ? 1 : 0;
        KNNG_TRY(launch_greedy_reorder(c->keys, c->n, c->K, reading_b, c->sigma, c->sigma_inv, c->stream));
        c->launches++;
    }
    DevState st = c->dev(false);
    KNNG_TRY(launch_permute(st, c->X2, c->keys2, c->sigma, c->total_perm, c->stream));
    c->launches++;
    if (ev[1]) KNNG_TRY(cudaEventRecord(ev[1], c->stream));
    std::swap(c->X, c->X2);
    std::swap(c->keys, c->keys2);
    KNNG_TRY(stage_low_precision(c));
    c->reordered = true;
    return KNNG_OK;
}

// One iteration: count, sample, join (+ Algorithm 1 after the first one).
// Time every join kernel the context can run on its current (first)
// iteration, between the sampling and the real join.  Each trial's side
// effects are undone: bucket cursors, chunk tables and pool cursor zeroed,
// the lists (which a full bucket's locked insertion may touch), the global
// counters and the iteration's counters restored.  Synchronises the stream.
int autotune_join(knng_ctx *c, int li) {
    std::vector<int> paths;
    if (c->kind() < 2) paths.push_back(kJoinTile);
    if (c->kind() == 0) paths.push_back(kJoinWarp);
    if (ring_join_fits(c->kind(), c->nv, c->dpb, c->K) && c->cset) paths.push_back(kJoinRing);
    if (pipe_join_fits(c->kind(), c->nv) && c->cset) {
        paths.push_back(kJoinPipe);
        paths.push_back(kJoinPipe8);
    }
    const size_t kb = sizeof(uint64_t) * (size_t)c->n * c->K;
    unsigned char *tmp = nullptr;
    KNNG_TRY(lib_malloc((void **)&tmp, align256(kb) + sizeof(long long) * kStatCount, c->stream));
    uint64_t *keys0 = (uint64_t *)tmp;
    long long *stats0 = (long long *)(tmp + align256(kb));
    KNNG_TRY(cudaMemcpyAsync(keys0, c->keys, kb, cudaMemcpyDeviceToDevice, c->stream));
    KNNG_TRY(cudaMemcpyAsync(stats0, c->stats, sizeof(long long) * kStatCount, cudaMemcpyDeviceToDevice, c->stream));
    std::vector<cudaEvent_t> ev(2 * paths.size());
    for (auto &e : ev) KNNG_TRY(cudaEventCreate(&e));
    int rc = KNNG_OK;
    for (size_t i = 0; i < paths.size() && !rc; ++i) {
        const int keep = c->join_path;
        c->join_path = paths[i];
        DevState st = c->dev(false);
        c->join_path = keep;
        cudaError_t e = cudaEventRecord(ev[2 * i], c->stream);
        if (e == cudaSuccess) e = launch_join(st, li, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * i + 1], c->stream);
        c->launches += join_launches(paths[i]);
        // undo the trial
        if (e == cudaSuccess) e = cudaMemsetAsync(c->pcursor, 0, sizeof(int) * (size_t)c->n, c->stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(c->pchunk, 0, sizeof(int) * ((size_t)c->n * kBucketChunks + 1), c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->keys, keys0, kb, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->stats, stats0, sizeof(long long) * kStatCount, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(c->it_stats + (size_t)li * kItCount, 0, sizeof(long long) * kItCount, c->stream);
        if (e != cudaSuccess) rc = cuda_code(e);
    }
    if (!rc) rc = cuda_code(cudaStreamSynchronize(c->stream));
    int best = c->join_path;
    float best_ms = 0.f;
    for (size_t i = 0; i < paths.size() && !rc; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) != cudaSuccess) continue;
        if (i == 0 || ms < best_ms) {
            best = paths[i];
            best_ms = ms;
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    cudaFreeAsync(tmp, c->stream);
    if (rc) return rc;
    c->join_path = best;
    c->tune_pending = false;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[tune_key(c)] = best;
    return KNNG_OK;
}

// Node-range passes of iteration `it`'s join.  Proposal capacity per pass:
// one 256-key run per node plus the pool.  A node joins up to m = min(64, 2s)
// new candidates (s forward and about s reverse), whose pairs give up to
// m (m - 1) proposals; in the first iteration the lists are random and nearly
// all of them pass the worst-key filter, later ones about 70% at most
// (measured on the 1M x 128 mixture at s = 23).  Most workloads take one pass.
int join_passes(const knng_ctx *c, int it) {
    // test hook: a fixed number of passes (parity of the pass split)
    if (const char *e = std::getenv("KNNG_TEST_JOIN_PASSES")) return std::max(1, std::min(std::atoi(e), 64));
    const double m = std::min(kSetMax, 2 * c->s);
    const double want = (double)c->n * m * (m - 1.0) * (it <= 1 ? 1.0 : 0.7);
    const double cap = 0.85 * ((double)c->n + (double)c->pool_chunks) * kBucketRun;
    const int p = (int)std::ceil(want / cap);
    return std::max(1, std::min(p, 64));
}

int enqueue_iteration(knng_ctx *c, bool gate) {
    if (c->li >= kMaxLocalIters) return KNNG_ERR_STATE;
    const int li = c->li, it = c->it_done + 1;
    DevState st = c->dev(gate);
    const bool timing = (c->flags & KNNG_FLAG_TIMING) != 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (timing) {
        for (auto &e : ev) KNNG_TRY(cudaEventCreate(&e));
        for (auto &e : ev) c->ev.push_back(e);
        c->ev_li.push_back(li);
        KNNG_TRY(cudaEventRecord(ev[0], c->stream));
    }
    KNNG_TRY(launch_count(st, li, c->stream));
    KNNG_TRY(c->heap ? launch_heap_sample(st, li, it, c->seed, c->stream)
                     : launch_sample(st, li, it, c->seed, c->stream));
    if (timing) KNNG_TRY(cudaEventRecord(ev[1], c->stream));
    if (c->tune_pending) {
        int rc = autotune_join(c, li);
        if (rc) return rc;
        st = c->dev(gate);
    }
    // the join in node-range passes, each followed by a list merge, so that
    // one pass's proposals fit the buckets and the pool (the set kernel runs
    // with the first pass; later passes filter against the merged lists)
    const int passes = join_passes(c, it);
    for (int p = 0; p < passes; ++p) {
        st.u_lo = c->n * p / passes;
        st.u_hi = c->n * (p + 1) / passes;
        knng_ctx::PassEvents pe{li, nullptr, nullptr, nullptr};
        if (timing) {
            KNNG_TRY(cudaEventCreate(&pe.join0));
            KNNG_TRY(cudaEventCreate(&pe.join1));
            KNNG_TRY(cudaEventCreate(&pe.merge1));
            c->pev.push_back(pe);
            KNNG_TRY(cudaEventRecord(pe.join0, c->stream));
        }
        KNNG_TRY(launch_join(st, li, c->stream));
        if (timing) KNNG_TRY(cudaEventRecord(pe.join1, c->stream));
        KNNG_TRY(launch_merge(st, li, c->stream));
        if (timing) KNNG_TRY(cudaEventRecord(pe.merge1, c->stream));
        if (p + 1 < passes) KNNG_TRY(cudaMemsetAsync(c->pool_next, 0, sizeof(int), c->stream));
    }
    c->launches += (c->heap ? 4 : 2) + passes * (1 + join_launches(c->join_path)) - (passes - 1) *
                   (join_launches(c->join_path) - 1);
    c->li++;
    c->it_done++;
    if ((c->flags & KNNG_FLAG_REORDER) && !c->reordered && it == 1) {
        int rc = enqueue_reorder(c);
        if (rc) return rc;
    }
    return KNNG_OK;
}

}  // namespace

extern "C" {

const char *knng_strerror(int code) {
    switch (code) {
        case KNNG_OK: return "ok";
        case KNNG_WARN_OVERFLOW: return "warning: sampled candidates beyond capacity were skipped";
        case KNNG_ERR_INVALID_ARG: return "invalid argument";
        case KNNG_ERR_OOM: return "out of device memory";
        case KNNG_ERR_CUDA: return "CUDA error";
        case KNNG_ERR_TIMEOUT: return "a bounded device wait gave up";
        case KNNG_ERR_UNSUPPORTED: return "unsupported parameters (K > 64, or K > 32 with a low-precision or heap flag)";
        case KNNG_ERR_STATE: return "call not valid in the context's state";
        case KNNG_ERR_INTERNAL: return "internal error";
        default: return "unknown code";
    }
}

const char *knng_version(void) { return "knng-gb300 0.1 (sm_103a)"; }

int knng_init(knng_ctx **out, const float *data, int64_t n, int d, int K, float rho, float delta, uint64_t seed,
              uint32_t flags, void *stream) {
    if (!data) {
        if (out) *out = nullptr;
        return KNNG_ERR_INVALID_ARG;
    }
    int rc = ctx_create(out, data, n, d, K, rho, delta, seed, flags, stream);
    if (rc) return rc;
    knng_ctx *c = *out;
    DevState st = c->dev(false);
    cudaError_t e = launch_init_random(st, seed, c->err, c->stream);
    c->launches++;
    if (e != cudaSuccess) {
        knng_destroy(c);
        *out = nullptr;
        return cuda_code(e);
    }
    return KNNG_OK;
}

int knng_init_from_graph(knng_ctx **out, const float *data, int64_t n, int d, int K, float rho, float delta,
                         uint64_t seed, uint32_t flags, void *stream, const int32_t *ids, const uint8_t *is_new,
                         int iter) {
    if (out) *out = nullptr;
    if (!data || !ids || !is_new || iter < 0) return KNNG_ERR_INVALID_ARG;
    if (is_foreign_ptr(ids) || is_foreign_ptr(is_new)) return KNNG_ERR_INVALID_ARG;
    int rc = ctx_create(out, data, n, d, K, rho, delta, seed, flags, stream);
    if (rc) return rc;
    knng_ctx *c = *out;
    c->it_done = iter;
    int32_t *dids = nullptr;
    uint8_t *dnew = nullptr;
    const size_t nb = sizeof(int32_t) * n * K, fb = (size_t)n * K;
    cudaError_t e = cudaSuccess;
    const int32_t *ids_d = ids;
    const uint8_t *new_d = is_new;
    if (!is_device_ptr(ids)) {
        e = lib_malloc((void **)&dids, nb, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dids, ids, nb, cudaMemcpyHostToDevice, c->stream);
        ids_d = dids;
    }
    if (e == cudaSuccess && !is_device_ptr(is_new)) {
        e = lib_malloc((void **)&dnew, fb, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dnew, is_new, fb, cudaMemcpyHostToDevice, c->stream);
        new_d = dnew;
    }
    if (e == cudaSuccess) {
        e = launch_init_graph(c->dev(false), ids_d, new_d, c->err, c->stream);
        c->launches++;
    }
    if (dids) cudaFreeAsync(dids, c->stream);
    if (dnew) cudaFreeAsync(dnew, c->stream);
    if (e == cudaSuccess) {
        rc = ctx_check(c);
        if (rc == KNNG_ERR_INVALID_ARG || rc < 0) {
            knng_destroy(c);
            *out = nullptr;
            return rc;
        }
        return KNNG_OK;
    }
    knng_destroy(c);
    *out = nullptr;
    return cuda_code(e);
}

int knng_iterate(knng_ctx *c, int64_t *changes_out) {
    if (!c) return KNNG_ERR_INVALID_ARG;
    const int li = c->li;
    int rc = enqueue_iteration(c, false);
    if (rc) return rc;
    long long its[kItCount];
    KNNG_TRY(cudaMemcpyAsync(its, c->it_stats + (size_t)li * kItCount, sizeof(its), cudaMemcpyDeviceToHost,
                             c->stream));
    rc = ctx_check(c);
    if (rc < 0) return rc;
    if (changes_out) *changes_out = its[kItChanges];
    return (double)its[kItChanges] < c->thr ? 1 : 0;
}

int knng_run(knng_ctx *c, int max_iters) {
    if (!c || max_iters < 0 || max_iters > kMaxItersArg) return KNNG_ERR_INVALID_ARG;
    if (c->tune_pending && max_iters > 0) {
        // the tuning iteration synchronises: it runs before any capture
        int rc = enqueue_iteration(c, true);
        if (rc) return rc;
        --max_iters;
    }
    const bool graph = (c->flags & KNNG_FLAG_GRAPH) && max_iters > 0;
    if (!graph) {
        for (int t = 0; t < max_iters; ++t) {
            int rc = enqueue_iteration(c, true);
            if (rc) return rc;
        }
        return KNNG_OK;
    }
    // The whole loop (every kernel of every iteration, skipping itself on the
    // device after convergence) becomes one graph, captured on a private
    // stream (the caller's may be the legacy stream, which cannot be
    // captured) and launched on the caller's stream.
    if (!c->capture) KNNG_TRY(cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking));
    cudaStream_t user = c->stream;
    KNNG_TRY(cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal));
    c->stream = c->capture;
    int rc = KNNG_OK;
    for (int t = 0; t < max_iters && !rc; ++t) rc = enqueue_iteration(c, true);
    c->stream = user;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->capture, &g);
    if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc ? rc : cuda_code(e);
    }
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_code(e);
    c->graphs.push_back(ge);
    KNNG_TRY(cudaGraphLaunch(ge, c->stream));
    return KNNG_OK;
}

int knng_reorder(knng_ctx *c) {
    if (!c) return KNNG_ERR_INVALID_ARG;
    return enqueue_reorder(c);
}

int knng_get(knng_ctx *c, int32_t *ids, float *dists) {
    if (!c || !ids || !dists) return KNNG_ERR_INVALID_ARG;
    if (is_foreign_ptr(ids) || is_foreign_ptr(dists)) return KNNG_ERR_INVALID_ARG;
    // both on the device: written in place; otherwise through a device buffer
    // and copied out with the direction taken from each pointer
    const bool dev_out = is_device_ptr(ids) && is_device_ptr(dists);
    const size_t ib = sizeof(int32_t) * c->n * c->K, db = sizeof(float) * c->n * c->K;
    int32_t *oi = ids;
    float *od = dists;
    unsigned char *tmp = nullptr;
    if (!dev_out) {
        KNNG_TRY(lib_malloc((void **)&tmp, align256(ib) + db, c->stream));
        oi = (int32_t *)tmp;
        od = (float *)(tmp + align256(ib));
    }
    if (c->reordered) {
        KNNG_TRY(launch_invert(c->total_perm, c->n, c->total_inv, c->stream));
        c->launches++;
    }
    DevState st = c->dev(false);
    KNNG_TRY(launch_output(st, c->reordered ? c->total_perm : nullptr, c->reordered ? c->total_inv : nullptr, oi,
                           od, c->stream));
    c->launches++;
    if (!dev_out) {
        KNNG_TRY(cudaMemcpyAsync(ids, oi, ib, cudaMemcpyDefault, c->stream));
        KNNG_TRY(cudaMemcpyAsync(dists, od, db, cudaMemcpyDefault, c->stream));
        KNNG_TRY(cudaFreeAsync(tmp, c->stream));
        return ctx_check(c);
    }
    return KNNG_OK;
}

int knng_get_state(knng_ctx *c, int32_t *ids, float *dists, uint8_t *flags) {
    if (!c) return KNNG_ERR_INVALID_ARG;
    std::vector<uint64_t> k((size_t)c->n * c->K);
    KNNG_TRY(cudaMemcpyAsync(k.data(), c->keys, sizeof(uint64_t) * k.size(), cudaMemcpyDeviceToHost, c->stream));
    KNNG_TRY(cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < k.size(); ++i) {
        if (ids) ids[i] = (int32_t)key_id(k[i]);
        if (dists) {
            uint32_t b = (uint32_t)(k[i] >> 32);
            std::memcpy(&dists[i], &b, 4);
        }
        if (flags) flags[i] = (uint8_t)(key_flags(k[i]) & kFlagNew);
    }
    return KNNG_OK;
}

int knng_get_samples(knng_ctx *c, int cap, int32_t *new_ids, int32_t *new_cnt, int32_t *old_ids, int32_t *old_cnt) {
    if (!c || cap < 1 || !new_ids || !new_cnt || !old_ids || !old_cnt) return KNNG_ERR_INVALID_ARG;
    const int64_t n = c->n;
    std::vector<int> cand((size_t)2 * n * c->cap), ib((size_t)6 * n);
    KNNG_TRY(cudaMemcpyAsync(cand.data(), c->cand, sizeof(int) * cand.size(), cudaMemcpyDeviceToHost, c->stream));
    KNNG_TRY(cudaMemcpyAsync(ib.data(), c->ibuf, sizeof(int) * ib.size(), cudaMemcpyDeviceToHost, c->stream));
    KNNG_TRY(cudaStreamSynchronize(c->stream));
    const int *fill_new = ib.data() + 2 * n, *fill_old = ib.data() + 3 * n;
    const int *fwd_new = ib.data() + 4 * n, *fwd_old = ib.data() + 5 * n;
    for (int64_t u = 0; u < n; ++u) {
        for (int kind = 0; kind < 2; ++kind) {
            const int *src = cand.data() + (size_t)kind * n * c->cap + (size_t)u * c->cap;
            const int f = kind ? fwd_old[u] : fwd_new[u];
            const int r = std::min(kind ? fill_old[u] : fill_new[u], c->R);
            int32_t *dst = (kind ? old_ids : new_ids) + (size_t)u * cap;
            int m = 0;
            for (int i = 0; i < f && m < cap; ++i) dst[m++] = src[i];
            for (int i = 0; i < r && m < cap; ++i) dst[m++] = src[c->K + i];
            (kind ? old_cnt : new_cnt)[u] = m;
            for (int i = m; i < cap; ++i) dst[i] = -1;
        }
    }
    return KNNG_OK;
}

int knng_get_permutation(knng_ctx *c, int32_t *sigma) {
    if (!c || !sigma) return KNNG_ERR_INVALID_ARG;
    if (!c->reordered) {
        for (int64_t u = 0; u < c->n; ++u) sigma[u] = (int32_t)u;
        return KNNG_OK;
    }
    KNNG_TRY(cudaMemcpyAsync(sigma, c->total_perm, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost, c->stream));
    KNNG_TRY(cudaStreamSynchronize(c->stream));
    return KNNG_OK;
}

int knng_get_stats(knng_ctx *c, knng_stats *out) {
    if (!c || !out) return KNNG_ERR_INVALID_ARG;
    long long st[kStatCount];
    std::vector<long long> its((size_t)kItCount * std::max(1, c->li));
    KNNG_TRY(cudaMemcpyAsync(st, c->stats, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    KNNG_TRY(cudaMemcpyAsync(its.data(), c->it_stats, sizeof(long long) * its.size(), cudaMemcpyDeviceToHost,
                             c->stream));
    KNNG_TRY(cudaStreamSynchronize(c->stream));
    std::memset(out, 0, sizeof(*out));
    out->n = c->n;
    out->d = c->d;
    out->K = c->K;
    out->s = c->s;
    for (int i = 0; i < c->li; ++i) {
        const long long *r = its.data() + (size_t)i * kItCount;
        if (r[kItRan]) {
            out->iterations++;
            out->last_changes = r[kItChanges];
        }
    }
    out->dist_evals = st[kStatEvals];
    out->inserts = st[kStatInserts];
    out->merges = st[kStatMerges];
    out->gathered_rows = st[kStatGathered];
    out->rev_overflow = st[kStatRevOverflow];
    out->set_overflow = st[kStatSetOverflow];
    out->lock_timeouts = st[kStatLockTimeout];
    out->kernel_launches = c->launches;
    out->reordered = c->reordered ? 1 : 0;
    out->join_path = c->join_path;
    out->cand_ids = 0;
    out->proposals = 0;
    for (int i = 0; i < c->li; ++i) {
        out->cand_ids += its[(size_t)i * kItCount + kItCandIds];
        out->proposals += its[(size_t)i * kItCount + kItProposals];
    }
    out->join_ms = 0;
    out->join_ms_ran = 0;
    out->merge_ms_ran = 0;
    out->sample_ms_ran = 0;
    for (size_t i = 0; i + 1 < c->ev.size(); i += 2) {
        float ms0 = 0;
        const bool ran = its[(size_t)c->ev_li[i / 2] * kItCount + kItRan] != 0;
        if (cudaEventElapsedTime(&ms0, c->ev[i], c->ev[i + 1]) == cudaSuccess) {
            out->join_launches++;
            if (ran) {
                out->sample_ms_ran += ms0;
                out->join_ran++;
            }
        } else {
            cudaGetLastError();
        }
    }
    for (const auto &pe : c->pev) {
        float ms = 0, ms2 = 0;
        if (cudaEventElapsedTime(&ms, pe.join0, pe.join1) == cudaSuccess &&
            cudaEventElapsedTime(&ms2, pe.join1, pe.merge1) == cudaSuccess) {
            out->join_ms += ms;
            if (its[(size_t)pe.li * kItCount + kItRan]) {
                out->join_ms_ran += ms;
                out->merge_ms_ran += ms2;
            }
        } else {
            cudaGetLastError();
        }
    }
    out->bucket_overflow = st[kStatBucketOverflow];
    out->reorder_ms = 0;
    for (size_t i = 0; i + 1 < c->rev.size(); i += 2) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, c->rev[i], c->rev[i + 1]) == cudaSuccess) out->reorder_ms += ms;
        else cudaGetLastError();
    }
    return KNNG_OK;
}

int knng_destroy(knng_ctx *c) {
    if (!c) return KNNG_OK;
    if (!c->graphs.empty()) {
        cudaStreamSynchronize(c->stream);  // executable graphs may still run
        for (cudaGraphExec_t g : c->graphs) cudaGraphExecDestroy(g);
    }
    if (c->capture) cudaStreamDestroy(c->capture);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (const auto &pe : c->pev) {
        cudaEventDestroy(pe.join0);
        cudaEventDestroy(pe.join1);
        cudaEventDestroy(pe.merge1);
    }
    for (cudaEvent_t e : c->rev) cudaEventDestroy(e);
    if (c->arena) cudaFreeAsync(c->arena, c->stream);
    if (c->barena) cudaFreeAsync(c->barena, c->stream);
    delete c;
    return KNNG_OK;
}

int knng_build_ex(const float *data, int64_t n, int d, int K, float rho, float delta, int max_iters, uint64_t seed,
                  uint32_t flags, void *stream, int32_t *ids, float *dists, knng_stats *stats) {
    if (max_iters < 0 || max_iters > kMaxItersArg || !ids || !dists) return KNNG_ERR_INVALID_ARG;
    if (is_foreign_ptr(ids) || is_foreign_ptr(dists)) return KNNG_ERR_INVALID_ARG;
    knng_ctx *c = nullptr;
    int rc = knng_init(&c, data, n, d, K, rho, delta, seed, flags, stream);
    if (rc) return rc;
    rc = knng_run(c, max_iters);
    if (!rc) rc = knng_get(c, ids, dists);
    if (rc >= 0 && stats) {
        int r2 = knng_get_stats(c, stats);
        if (r2) rc = r2;
    }
    if (rc >= 0) {
        int r3 = ctx_check(c);
        if (r3) rc = r3;
    }
    knng_destroy(c);
    return rc;
}

int knng_build(const float *data, int64_t n, int d, int K, float rho, float delta, int max_iters, uint64_t seed,
               int32_t *ids, float *dists) {
    return knng_build_ex(data, n, d, K, rho, delta, max_iters, seed, 0u, nullptr, ids, dists, nullptr);
}

}  // extern "C"

namespace {

// One batched build over data sets of one row-width class (below) that share
// K, the sample size, max_iters and the seed; deltas (may be NULL: delta for
// all) gives each data set its own stopping count.
int build_batched_group(const knng_desc *descs, int count, int K, float rho, float delta, int max_iters,
                        uint64_t seed, uint32_t flags, void *stream, knng_stats *stats,
                        const float *deltas = nullptr) {
    int64_t ntot = 0;
    int dmax = 0;
    std::vector<long long> off(count + 1);
    std::vector<int> nn(count);
    std::vector<double> thr(count);
    for (int b = 0; b < count; ++b) {
        const knng_desc &e = descs[b];
        if (!e.data || !e.ids || !e.dists || e.n < 2 || e.d < 1 || K > e.n - 1) return KNNG_ERR_INVALID_ARG;
        off[b] = ntot;
        nn[b] = (int)e.n;
        thr[b] = (double)(deltas ? deltas[b] : delta) * (double)e.n * (double)K;
        ntot += e.n;
        dmax = std::max(dmax, e.d);
    }
    off[count] = ntot;
    knng_ctx *c = nullptr;
    int rc = ctx_create(&c, nullptr, ntot, dmax, K, rho, delta, seed, flags, stream);
    if (rc) return rc;
    c->thr = -1.0;  // convergence is decided per data set
    c->nds = count;
    cudaStream_t s = c->stream;
    cudaError_t e = cudaSuccess;
    // per-data-set arrays
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o += align256(bytes);
        return r;
    };
    const size_t oDs = take(sizeof(int) * ntot), oOff = take(sizeof(long long) * (count + 1)),
                 oN = take(sizeof(int) * count), oT = take(sizeof(double) * count),
                 oC = take(sizeof(long long) * (size_t)count * kMaxLocalIters);
    e = lib_malloc((void **)&c->barena, o, s);
    if (e == cudaSuccess) {
        c->ds = (int *)(c->barena + oDs);
        c->ds_off = (long long *)(c->barena + oOff);
        c->ds_n = (int *)(c->barena + oN);
        c->ds_thr = (double *)(c->barena + oT);
        c->ds_changes = (long long *)(c->barena + oC);
        e = cudaMemcpyAsync(c->ds_off, off.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ds_n, nn.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ds_thr, thr.data(), sizeof(double) * count, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->ds_changes, 0, sizeof(long long) * (size_t)count * kMaxLocalIters, s);
    if (e == cudaSuccess) e = launch_ds_map(c->ds_off, count, ntot, c->ds, s);
    // stage every data set into its node range (zero padding to the widest row
    // leaves every distance unchanged)
    for (int b = 0; e == cudaSuccess && b < count; ++b) {
        const knng_desc &d = descs[b];
        const float *src = d.data;
        float *tmp = nullptr;
        if (!is_device_ptr(d.data)) {
            e = lib_malloc((void **)&tmp, sizeof(float) * d.n * d.d, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, d.data, sizeof(float) * d.n * d.d, cudaMemcpyHostToDevice, s);
            src = tmp;
        }
        if (e == cudaSuccess) e = launch_stage(src, d.n, d.d, c->X + (size_t)off[b] * c->dp, c->dp, s);
        if (tmp) cudaFreeAsync(tmp, s);
    }
    if (e == cudaSuccess) e = stage_low_precision(c);
    if (e == cudaSuccess) e = launch_init_random(c->dev(false), seed, c->err, s);
    c->launches += count + 2;
    if (e != cudaSuccess) {
        knng_destroy(c);
        return cuda_code(e);
    }
    rc = knng_run(c, max_iters);
    // output into one concatenated buffer, then one copy per data set
    int32_t *oi = nullptr;
    float *od = nullptr;
    if (!rc) {
        e = lib_malloc((void **)&oi, sizeof(int32_t) * ntot * K, s);
        if (e == cudaSuccess) e = lib_malloc((void **)&od, sizeof(float) * ntot * K, s);
        if (e == cudaSuccess) e = launch_output(c->dev(false), nullptr, nullptr, oi, od, s);
        c->launches++;
        for (int b = 0; e == cudaSuccess && b < count; ++b) {
            e = cudaMemcpyAsync(descs[b].ids, oi + off[b] * K, sizeof(int32_t) * descs[b].n * K, cudaMemcpyDefault, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(descs[b].dists, od + off[b] * K, sizeof(float) * descs[b].n * K, cudaMemcpyDefault, s);
        }
        if (oi) cudaFreeAsync(oi, s);
        if (od) cudaFreeAsync(od, s);
        if (e != cudaSuccess) rc = cuda_code(e);
    }
    if (rc >= 0 && stats) {
        int r2 = knng_get_stats(c, stats);
        if (r2) rc = r2;
    }
    if (rc >= 0) {
        int r3 = ctx_check(c);
        if (r3) rc = r3;
    }
    knng_destroy(c);
    return rc;
}

// Row-width classes of the batched build: a data set is padded to the
// smallest class width >= d (at most 1.5x its row), so narrow data sets do
// not pay for the widest one and take the join kernel that suits their width.
int width_class(int d) {
    if (d > (1 << 24)) return d;
    int w = 32;
    while (w < d) w = (w % 3 == 0) ? w / 3 * 4 : w / 2 * 3;  // 32, 48, 64, 96, 128, 192, 256, ...
    return w;
}

void add_stats(knng_stats &a, const knng_stats &b) {
    a.n += b.n;
    a.d = std::max(a.d, b.d);
    a.K = b.K;
    a.s = b.s;
    a.iterations = std::max(a.iterations, b.iterations);
    a.dist_evals += b.dist_evals;
    a.last_changes += b.last_changes;
    a.inserts += b.inserts;
    a.merges += b.merges;
    a.gathered_rows += b.gathered_rows;
    a.rev_overflow += b.rev_overflow;
    a.set_overflow += b.set_overflow;
    a.lock_timeouts += b.lock_timeouts;
    a.kernel_launches += b.kernel_launches;
    a.cand_ids += b.cand_ids;
    a.proposals += b.proposals;
    a.bucket_overflow += b.bucket_overflow;
    a.join_launches += b.join_launches;
    a.join_ms += b.join_ms;
    a.join_ran += b.join_ran;
    a.join_path = b.join_path;
    a.join_ms_ran += b.join_ms_ran;
    a.merge_ms_ran += b.merge_ms_ran;
    a.sample_ms_ran += b.sample_ms_ran;
    a.reorder_ms += b.reorder_ms;
}

}  // namespace

extern "C" {

int knng_build_batched(const knng_desc *descs, int count, int K, float rho, float delta, int max_iters,
                       uint64_t seed, uint32_t flags, void *stream, knng_stats *stats) {
    if (!descs || count < 1 || max_iters < 0 || max_iters > kMaxItersArg) return KNNG_ERR_INVALID_ARG;
    if (flags & (KNNG_FLAG_REORDER | KNNG_FLAG_REORDER_B)) return KNNG_ERR_UNSUPPORTED;
    for (int b = 0; b < count; ++b) {
        const knng_desc &e = descs[b];
        if (e.d < 1 || is_foreign_ptr(e.data) || is_foreign_ptr(e.ids) || is_foreign_ptr(e.dists))
            return KNNG_ERR_INVALID_ARG;
    }
    // one batched build per row-width class, widest last
    std::vector<int> cls(count);
    for (int b = 0; b < count; ++b) cls[b] = width_class(descs[b].d);
    std::vector<int> widths(cls);
    std::sort(widths.begin(), widths.end());
    widths.erase(std::unique(widths.begin(), widths.end()), widths.end());
    knng_stats total;
    std::memset(&total, 0, sizeof(total));
    int rc = KNNG_OK;
    for (int w : widths) {
        std::vector<knng_desc> g;
        for (int b = 0; b < count; ++b)
            if (cls[b] == w) g.push_back(descs[b]);
        knng_stats gs;
        const int r = build_batched_group(g.data(), (int)g.size(), K, rho, delta, max_iters, seed, flags, stream,
                                          stats ? &gs : nullptr);
        if (r < 0) return r;
        if (r > 0) rc = r;
        if (stats) add_stats(total, gs);
    }
    if (stats) *stats = total;
    return rc;
}

int knng_build_batched_ex(const knng_desc_ex *descs, int count, uint32_t flags, void *stream, knng_stats *stats) {
    if (!descs || count < 1) return KNNG_ERR_INVALID_ARG;
    if (flags & (KNNG_FLAG_REORDER | KNNG_FLAG_REORDER_B)) return KNNG_ERR_UNSUPPORTED;
    for (int b = 0; b < count; ++b) {
        const knng_desc_ex &e = descs[b];
        if (!e.data || !e.ids || !e.dists || e.n < 2 || e.d < 1 || e.K < 1 || !(e.rho > 0.f && e.rho <= 1.f) ||
            !(e.delta >= 0.f) || e.max_iters < 0 || e.max_iters > kMaxItersArg)
            return KNNG_ERR_INVALID_ARG;
        if (is_foreign_ptr(e.data) || is_foreign_ptr(e.ids) || is_foreign_ptr(e.dists)) return KNNG_ERR_INVALID_ARG;
        if (e.K > kMaxK) return KNNG_ERR_UNSUPPORTED;
        if (e.K > kLaneK && (flags & (KNNG_FLAG_BF16 | KNNG_FLAG_FP8 | KNNG_FLAG_HEAP_SAMPLING)))
            return KNNG_ERR_UNSUPPORTED;
        if (e.K > e.n - 1) return KNNG_ERR_INVALID_ARG;
    }
    // one batched build per (row-width class, K, sample size, max_iters,
    // seed), in that order; delta stays per data set
    using GroupKey = std::tuple<int, int, int, int, uint64_t>;
    std::map<GroupKey, std::vector<int>> groups;
    for (int b = 0; b < count; ++b) {
        const knng_desc_ex &e = descs[b];
        groups[GroupKey(width_class(e.d), e.K, sample_size(e.rho, e.K), e.max_iters, e.seed)].push_back(b);
    }
    knng_stats total;
    std::memset(&total, 0, sizeof(total));
    int rc = KNNG_OK;
    for (const auto &kv : groups) {
        std::vector<knng_desc> g;
        std::vector<float> deltas;
        for (int b : kv.second) {
            const knng_desc_ex &e = descs[b];
            g.push_back(knng_desc{e.data, e.n, e.d, e.ids, e.dists});
            deltas.push_back(e.delta);
        }
        const knng_desc_ex &f = descs[kv.second[0]];
        knng_stats gs;
        const int r = build_batched_group(g.data(), (int)g.size(), f.K, f.rho, f.delta, f.max_iters, f.seed, flags,
                                          stream, stats ? &gs : nullptr, deltas.data());
        if (r < 0) return r;
        if (r > 0) rc = r;
        if (stats) add_stats(total, gs);
    }
    if (stats) *stats = total;
    return rc;
}

int knng_bruteforce_last_fallbacks(void) { return g_bf_fallbacks; }

float knng_bruteforce_last_prefilter_ms(void) { return g_bf_prefilter_ms; }

int knng_measure_l2_read(int64_t bytes, int passes, void *stream, double *gbs) {
    if (bytes < (1 << 20) || passes < 1 || !gbs) return KNNG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n4 = (size_t)bytes / 16;
    unsigned char *buf = nullptr;
    KNNG_TRY(lib_malloc((void **)&buf, n4 * 16 + 256, s));
    float *sink = reinterpret_cast<float *>(buf + n4 * 16);
    cudaEvent_t a = nullptr, b = nullptr;
    float ms = 0.f;
    cudaError_t e = cudaMemsetAsync(buf, 0, n4 * 16 + 256, s);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = launch_l2_read(buf, n4, 1, sink, s);  // brings the buffer into L2
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
    if (e == cudaSuccess) e = launch_l2_read(buf, n4, passes, sink, s);
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return cuda_code(e);
    *gbs = (double)n4 * 16.0 * passes / (ms / 1e3) / 1e9;
    return KNNG_OK;
}

int knng_bruteforce(const float *data, int64_t n, int d, int K, const int64_t *rows, int64_t nq, int32_t *ids,
                    float *dists, void *stream) {
    if (!data || !ids || !dists || n < 2 || d < 1 || K < 1 || K > n - 1) return KNNG_ERR_INVALID_ARG;
    if (K > kMaxK) return KNNG_ERR_UNSUPPORTED;
    if (!rows) nq = n;
    if (nq < 1) return KNNG_ERR_INVALID_ARG;
    if (is_foreign_ptr(data) || is_foreign_ptr(ids) || is_foreign_ptr(dists) || is_foreign_ptr(rows))
        return KNNG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int dp = (d + 3) & ~3;
    const size_t xb = align256(sizeof(float) * n * dp), rb = rows ? align256(sizeof(int64_t) * nq) : 0;
    const size_t ib = align256(sizeof(int32_t) * nq * K), db = align256(sizeof(float) * nq * K);
    const bool dev_out = is_device_ptr(ids) && is_device_ptr(dists);
    // slices of the point set when there are too few queries to fill the GPU
    // (their lists are merged one key per lane: K <= 32)
    const int S = K > kLaneK ? 1 : bruteforce_slices(n, nq);
    const size_t pb = S > 1 ? sizeof(uint64_t) * (size_t)nq * S * K : 0;
    unsigned char *tmp = nullptr;
    KNNG_TRY(lib_malloc((void **)&tmp, xb + rb + (dev_out ? 0 : ib + db) + pb, s));
    uint64_t *part = S > 1 ? (uint64_t *)(tmp + xb + rb + (dev_out ? 0 : ib + db)) : nullptr;
    float *X = (float *)tmp;
    int rc = KNNG_OK;
    const float *src = data;
    float *staged = nullptr;
    cudaError_t e = cudaSuccess;
    if (!is_device_ptr(data)) {
        e = lib_malloc((void **)&staged, sizeof(float) * n * d, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(staged, data, sizeof(float) * n * d, cudaMemcpyHostToDevice, s);
        src = staged;
    }
    if (e == cudaSuccess) e = launch_stage(src, n, d, X, dp, s);
    const int64_t *rows_d = rows;
    if (e == cudaSuccess && rows) {
        if (!is_device_ptr(rows)) {
            int64_t *r = (int64_t *)(tmp + xb);
            e = cudaMemcpyAsync(r, rows, sizeof(int64_t) * nq, cudaMemcpyHostToDevice, s);
            rows_d = r;
        }
    }
    int32_t *oi = ids;
    float *od = dists;
    if (!dev_out) {
        oi = (int32_t *)(tmp + xb + rb);
        od = (float *)(tmp + xb + rb + ib);
    }
    // tensor-core prefilter with exact re-rank where the rows allow it
    // (KNNG_TEST_BF_PATH=cuda|tensor forces a path in tests)
    const char *force = std::getenv("KNNG_TEST_BF_PATH");
    bool tc = bruteforce_tc_supported(dp) && n >= 4096 && K <= kLaneK;
    if (force && !std::strcmp(force, "cuda")) tc = false;
    if (force && !std::strcmp(force, "tensor")) tc = bruteforce_tc_supported(dp) && K <= kLaneK;
    g_bf_fallbacks = -1;
    g_bf_prefilter_ms = -1.f;
    if (e == cudaSuccess && tc) {
        int TS = 1, nredo = 0;
        float pf_ms = -1.f;
        unsigned char *tcs = nullptr;
        const size_t tb = bruteforce_tc_scratch(n, nq, dp, K, &TS);
        e = lib_malloc((void **)&tcs, tb, s);
        if (e == cudaSuccess) {
            e = launch_bruteforce_tc(X, n, dp, d, K, rows_d, nq, oi, od, s, tcs, TS, &nredo, &pf_ms);
            cudaFreeAsync(tcs, s);
        }
        if (e == cudaErrorNotSupported) {  // no tensor map encoder: the exact kernel
            cudaGetLastError();
            e = cudaSuccess;
            tc = false;
        } else if (e == cudaSuccess) {
            g_bf_fallbacks = nredo;
            g_bf_prefilter_ms = pf_ms;
        }
    }
    if (e == cudaSuccess && !tc) e = launch_bruteforce(X, n, dp, K, rows_d, nq, oi, od, s, part, S);
    if (e == cudaSuccess && !dev_out) {
        e = cudaMemcpyAsync(ids, oi, sizeof(int32_t) * nq * K, cudaMemcpyDefault, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dists, od, sizeof(float) * nq * K, cudaMemcpyDefault, s);
    }
    if (staged) cudaFreeAsync(staged, s);
    cudaFreeAsync(tmp, s);
    if (e == cudaSuccess && !dev_out) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_code(e);
    return rc;
}

}  // extern "C"
