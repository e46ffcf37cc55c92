// nnd_kernels.cu -- the NN-Descent steps around the local join: staging of
// the points, random initialisation, degree counting, one-pass sampling, the
// greedy relabelling (Algorithm 1) with its permutation, and the re-ranked
// output.  One warp owns one node's list wherever a list is touched: list
// entry k sits on lane k, and for K > 32 entry k + 32 on lane k too (the list
// kernels take KW = 1 or 2 keys per lane).
#include <map>
#include <mutex>
#include <utility>

#include "internal.h"

namespace knng {

namespace {
constexpr int kWarpsPerBlock = 8;
constexpr int kBlock = kWarpsPerBlock * 32;
constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ long long gwarp() { return ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }

// Rows gathered whole into shared memory before the distances of a list:
// blocks of four warps, each warp with 33 rows on a stride of (nv | 1)
// 16-byte units (consecutive rows on distinct banks); taken for rows of up to
// kStageMinNv to kStageMaxNv units.  A lane reading its own row 16 bytes at a time from
// global memory used half of each sector it fetched.
constexpr int kStageWarps = 4;
constexpr int kStageMinNv = 16;  // shorter rows are a sector or two: read directly
constexpr int kStageMaxNv = 90;
__host__ __device__ __forceinline__ size_t stage_smem_bytes(int nv) {
    return (size_t)kStageWarps * 33 * (size_t)(nv | 1) * 16;
}
__device__ __forceinline__ void cp_async16_n(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
// Lane k (< cnt) gets the canonical distance between row u and row v_k (v
// held by lane k); the rows are first copied whole into the warp's area sm
// with asynchronous 16-byte copies (one warp instruction per 512 bytes).
__device__ __forceinline__ float warp_staged_dist(const float4 *__restrict__ X4, int nv, long long u, uint32_t v,
                                                  int cnt, float4 *sm) {
    const unsigned lane = lane_id();
    const int rs = nv | 1;
    float4 *own = sm + 32 * rs;
    for (int k = 0; k < cnt; ++k) {
        const uint32_t vk = __shfl_sync(0xFFFFFFFFu, v, k);
        for (int c = lane; c < nv; c += 32) cp_async16_n(sm + k * rs + c, X4 + (size_t)vk * nv + c);
    }
    for (int c = lane; c < nv; c += 32) cp_async16_n(own + c, X4 + (size_t)u * nv + c);
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    const float dd = (int)lane < cnt ? l2sq_rows(own, sm + lane * rs, nv) : 0.f;
    __syncwarp();
    return dd;
}
__device__ __forceinline__ long long nwarps() { return ((long long)gridDim.x * blockDim.x) >> 5; }
}  // namespace

int grid_for(const void *kernel, int block_threads, size_t dyn_smem) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block_threads, dyn_smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return sms * per_sm;
}

// Id of the calling thread's current CUDA context, from the driver's
// cuCtxGetCurrent and cuCtxGetId (looked up once through the runtime, so the
// library needs no link against the driver).  A context made after a device
// reset gets a new id, so state cached per id never outlives its context.
cudaError_t current_context_id(unsigned long long *id) {
    typedef int (*GetCurrentFn)(void **);
    typedef int (*GetIdFn)(void *, unsigned long long *);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrentFn>(a);
            get_id = reinterpret_cast<GetIdFn>(b);
        } else {
            cudaGetLastError();
        }
    });
    if (!get_current || !get_id) return cudaErrorNotSupported;
    void *ctx = nullptr;
    if (get_current(&ctx) == 0 && !ctx) {
        // a thread that has not used the runtime yet: bind the current
        // device's primary context
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaSetDevice(dev);
        if (e != cudaSuccess) return e;
        ctx = nullptr;
        get_current(&ctx);
    }
    if (!ctx) return cudaErrorDeviceUninitialized;
    return get_id(ctx, id) == 0 ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Dynamic shared memory above the 48 KB default needs a per-function opt-in.
// The attribute belongs to the current context: record the largest size
// granted per (kernel, context) under a lock (a context made after a device
// reset starts without any grant).
cudaError_t smem_opt_in(const void *kernel, size_t bytes) {
    if (bytes == 0) return cudaSuccess;
    unsigned long long ctx = 0;
    cudaError_t e = current_context_id(&ctx);
    if (e != cudaSuccess) {
        // no context id: set the attribute every time
        cudaGetLastError();
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    }
    // without the attribute a launch may use 48 KB of shared memory, static
    // and dynamic together: the kernel's static size is read once per context
    struct Grant {
        long long stat = -1;  // static shared memory of the kernel
        size_t have = 0;      // dynamic bytes the kernel may use
    };
    static std::mutex mu;
    static std::map<std::pair<const void *, unsigned long long>, Grant> granted;
    std::lock_guard<std::mutex> g(mu);
    Grant &gr = granted[{kernel, ctx}];
    if (gr.have >= bytes) return cudaSuccess;
    if (gr.stat < 0) {
        cudaFuncAttributes a;
        e = cudaFuncGetAttributes(&a, kernel);
        if (e != cudaSuccess) return e;
        gr.stat = (long long)a.sharedSizeBytes;
    }
    if (bytes + (size_t)gr.stat <= 48 * 1024) {
        gr.have = bytes;
        return cudaSuccess;
    }
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) gr.have = bytes;
    return e;
}

// ------------------------------------------------------------------ stage ----
// Copy n x d rows into the padded n x dp layout (zeros in the padding), so a
// row is a whole number of 16-byte vectors.
__global__ void stage_kernel(const float *__restrict__ src, int64_t n, int d, float *__restrict__ X, int dp) {
    const int64_t total = n * (int64_t)dp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t u = e / dp;
        int t = (int)(e - u * dp);
        X[e] = t < d ? src[u * d + t] : 0.0f;
    }
}

cudaError_t launch_stage(const float *src, int64_t n, int d, float *X, int dp, cudaStream_t s) {
    int grid = grid_for((const void *)stage_kernel, 256, 0);
    stage_kernel<<<grid, 256, 0, s>>>(src, n, d, X, dp);
    return cudaGetLastError();
}

cudaError_t prepare_stage() {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, stage_kernel);
    if (e == cudaSuccess) grid_for((const void *)stage_kernel, 256, 0);
    return e;
}

// ------------------------------------------------------------ random init ----
// Section 2: K distinct neighbours != u, uniform over V.  Attempt a of node u
// proposes v = floor(hi32(h(seed, INIT, 0, u, a)) * n / 2^32); attempts are
// taken in order and a proposal is accepted unless it is u or already chosen.
// A warp evaluates 32 consecutive attempts at once and accepts, in lane order,
// exactly the proposals the sequential rule would accept.
template <bool kStaged, int KW>
__global__ void __launch_bounds__(kBlock) init_random_kernel(DevState st, uint64_t base, int *err) {
    __shared__ uint32_t chosen_s[kWarpsPerBlock][kMaxK];
    extern __shared__ __align__(16) float4 stage_sm[];
    uint32_t *chosen = chosen_s[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const int K = st.K;
    const uint64_t n = (uint64_t)st.n;
    const float4 *X4 = reinterpret_cast<const float4 *>(st.X);
    constexpr uint64_t kMaxAttempts = 1ull << 26;
    for (long long u = gwarp(); u < st.n; u += nwarps()) {
        // batched mode: sample within u's data set, keyed by local ids
        const long long off = st.ds ? st.ds_off[st.ds[u]] : 0;
        const uint64_t nb = st.ds ? (uint64_t)st.ds_n[st.ds[u]] : n;
        const uint64_t ul = (uint64_t)(u - off);
        int have = 0;
        uint64_t a = 0;
        while (have < K) {
            uint64_t h = hash_uj(base, ul, a + lane);
            uint32_t v = (uint32_t)(off + (long long)(((h >> 32) * nb) >> 32));
            bool ok = v != (uint32_t)u;
            for (int k = 0; k < have; ++k) ok = ok && (chosen[k] != v);
            unsigned same = __match_any_sync(kFull, v);
            bool acc = ok && ((unsigned)(__ffs(same) - 1) == lane);
            unsigned accm = __ballot_sync(kFull, acc);
            int rank = __popc(accm & lanemask_lt());
            __syncwarp();
            if (acc && have + rank < K) chosen[have + rank] = v;
            have = min(K, have + __popc(accm));
            __syncwarp();
            a += 32;
            if (a >= kMaxAttempts) {
                if (lane == 0) atomic_add_ll(&st.stats[kStatInitAttemptsExceeded], 1ll);
                if (lane == 0) atomicOr(err, 1);
                for (int k = have + (int)lane; k < K; k += 32)
                    chosen[k] = (uint32_t)(off + (long long)((ul + 1 + k) % nb));
                have = K;
                __syncwarp();
            }
        }
        // entries lane (and lane + 32): distances, keys, one sorted list
        uint64_t key[KW];
#pragma unroll
        for (int h = 0; h < KW; ++h) {
            const int k = (int)lane + 32 * h;
            const int cnt = K - 32 * h < 32 ? K - 32 * h : 32;
            const uint32_t v = k < K ? chosen[k] : (uint32_t)u;
            float dd;
            if (kStaged) dd = warp_staged_dist(X4, st.nv, u, v, cnt, stage_sm + (threadIdx.x >> 5) * 33 * (st.nv | 1));
            else dd = k < K ? l2sq_rows(X4 + (size_t)u * st.nv, X4 + (size_t)v * st.nv, st.nv) : 0.f;
            key[h] = k < K ? make_key(dd, v, kFlagNew) : kKeyEmpty;
        }
        if constexpr (KW == 2) warp_sort_u64x2(key[0], key[KW - 1]);
        else key[0] = warp_sort_u64(key[0]);
#pragma unroll
        for (int h = 0; h < KW; ++h)
            if ((int)lane + 32 * h < K) st.keys[(size_t)u * K + lane + 32 * h] = key[h];
        __syncwarp();
    }
}

template <int KW>
cudaError_t launch_init_random_t(const DevState &st, uint64_t base, int *err, cudaStream_t s) {
    if (st.nv >= kStageMinNv && st.nv <= kStageMaxNv) {
        const size_t dyn = stage_smem_bytes(st.nv);
        cudaError_t e = smem_opt_in((const void *)init_random_kernel<true, KW>, dyn);
        if (e != cudaSuccess) return e;
        const int grid = grid_for((const void *)init_random_kernel<true, KW>, kStageWarps * 32, dyn);
        init_random_kernel<true, KW><<<grid, kStageWarps * 32, dyn, s>>>(st, base, err);
        return cudaGetLastError();
    }
    int grid = grid_for((const void *)init_random_kernel<false, KW>, kBlock, 0);
    init_random_kernel<false, KW><<<grid, kBlock, 0, s>>>(st, base, err);
    return cudaGetLastError();
}

cudaError_t launch_init_random(const DevState &st, uint64_t seed, int *err, cudaStream_t s) {
    const uint64_t base = hash_base(seed, kStreamInit, 0);
    return st.K > kLaneK ? launch_init_random_t<2>(st, base, err, s) : launch_init_random_t<1>(st, base, err, s);
}

// Lists from a given graph: validate (in range, != u, distinct), compute
// distances, sort.  err |= 2 on an invalid row.
template <int KW>
__global__ void __launch_bounds__(kBlock) init_graph_kernel(DevState st, const int32_t *__restrict__ ids,
                                                            const uint8_t *__restrict__ is_new, int *err) {
    const unsigned lane = lane_id();
    const int K = st.K;
    const float4 *X4 = reinterpret_cast<const float4 *>(st.X);
    for (long long u = gwarp(); u < st.n; u += nwarps()) {
        int32_t v[KW];
        bool bad = false;
#pragma unroll
        for (int h = 0; h < KW; ++h) {
            const int k = (int)lane + 32 * h;
            const bool valid = k < K;
            v[h] = valid ? ids[(size_t)u * K + k] : -1 - k;  // distinct negatives off the list
            // every lane takes part in the warp-wide match (never under a
            // short-circuit: the collective needs the whole warp)
            const unsigned same = __match_any_sync(kFull, v[h]);
            bad = bad || (valid && (v[h] < 0 || v[h] >= st.n || v[h] == u || __popc(same) > 1));
        }
        if constexpr (KW == 2) {
            // repeats between the two halves
            for (int j = 0; j < 32; ++j) {
                const int32_t vj = __shfl_sync(kFull, v[0], j);
                bad = bad || ((int)lane + 32 < K && v[1] == vj);
            }
        }
        if (__any_sync(kFull, bad)) {
            if (lane == 0) atomicOr(err, 2);
#pragma unroll
            for (int h = 0; h < KW; ++h) v[h] = (int)lane + 32 * h < K ? (int32_t)((u + 1 + lane + 32 * h) % st.n) : 0;
        }
        uint64_t key[KW];
#pragma unroll
        for (int h = 0; h < KW; ++h) {
            const int k = (int)lane + 32 * h;
            key[h] = kKeyEmpty;
            if (k < K) {
                const float dd = l2sq_rows(X4 + (size_t)u * st.nv, X4 + (size_t)v[h] * st.nv, st.nv);
                key[h] = make_key(dd, (uint32_t)v[h], is_new[(size_t)u * K + k] ? kFlagNew : 0u);
            }
        }
        if constexpr (KW == 2) warp_sort_u64x2(key[0], key[KW - 1]);
        else key[0] = warp_sort_u64(key[0]);
#pragma unroll
        for (int h = 0; h < KW; ++h)
            if ((int)lane + 32 * h < K) st.keys[(size_t)u * K + lane + 32 * h] = key[h];
    }
}

cudaError_t launch_init_graph(const DevState &st, const int32_t *ids, const uint8_t *is_new, int *err,
                              cudaStream_t s) {
    if (st.K > kLaneK) {
        int grid = grid_for((const void *)init_graph_kernel<2>, kBlock, 0);
        init_graph_kernel<2><<<grid, kBlock, 0, s>>>(st, ids, is_new, err);
        return cudaGetLastError();
    }
    int grid = grid_for((const void *)init_graph_kernel<1>, kBlock, 0);
    init_graph_kernel<1><<<grid, kBlock, 0, s>>>(st, ids, is_new, err);
    return cudaGetLastError();
}

// ----------------------------------------------------------- degree count ----
// Section 3.1 keeps |N(u)| known during the pass; here the reverse degrees
// are counted per flag in one edge pass before sampling (forward degrees are
// counted by the sampling warp itself).
__global__ void count_kernel(DevState st, int li) {
    if (iteration_skipped(st, li)) return;
    const int64_t total = st.n * (int64_t)st.K;
    // the reverse candidate fill counters of the previous iteration are no
    // longer needed: restart them for this iteration's sampling
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < st.n; u += (int64_t)gridDim.x * blockDim.x) {
        st.fill_new[u] = 0;
        st.fill_old[u] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *st.pool_next = 0;                   // bucket pool restarts
        if (st.hcursor) *st.hcursor = 0;     // reverse-offer segments restart
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        if (st.ds && node_skipped(st, e / st.K, li)) continue;
        uint64_t key = st.keys[e];
        uint32_t v = key_id(key);
        atomicAdd((key & kFlagNew) ? &st.rev_new[v] : &st.rev_old[v], 1);
    }
}

cudaError_t launch_count(const DevState &st, int li, cudaStream_t s) {
    int grid = grid_for((const void *)count_kernel, 256, 0);
    count_kernel<<<grid, 256, 0, s>>>(st, li);
    return cudaGetLastError();
}

// --------------------------------------------------------------- sampling ----
// Section 3.1, one pass over the edges: edge (u, v) with flag f enters u's
// forward candidates of kind f with probability min(1, s / fwd_f(u)) and u
// enters v's reverse candidates of kind f with probability
// min(1, s / rev_f(v)), from two independent hash streams keyed by (u, j).
// Accepted forward new entries lose their "new" flag; every entry loses the
// "inserted this iteration" flag.  Forward candidates are written compacted
// by u's warp; reverse ones take an atomic slot in v's reverse part (capacity
// R, overflow counted).
template <int KW>
__global__ void __launch_bounds__(kBlock) sample_kernel(DevState st, int li, uint64_t fbase, uint64_t rbase) {
    if (iteration_skipped(st, li)) return;
    const unsigned lane = lane_id();
    const int K = st.K;
    const uint32_t s = (uint32_t)st.s;
    long long overflow = 0;
    for (long long u = gwarp(); u < st.n; u += nwarps()) {
        if (node_skipped(st, u, li)) continue;
        const uint64_t ul = (uint64_t)node_local(st, u);
        // entry lane + 32 h of u's list
        uint64_t key[KW];
        bool isnew[KW];
        uint32_t cnew = 0;
#pragma unroll
        for (int h = 0; h < KW; ++h) {
            const bool valid = (int)lane + 32 * h < K;
            key[h] = valid ? st.keys[(size_t)u * K + lane + 32 * h] : kKeyEmpty;
            isnew[h] = valid && (key[h] & kFlagNew);
            cnew += __popc(__ballot_sync(kFull, isnew[h]));
        }
        const uint32_t cold = (uint32_t)K - cnew;
        uint32_t nbase = 0, obase = 0;  // accepted new / old entries of the halves before
#pragma unroll
        for (int h = 0; h < KW; ++h) {
            const int k = (int)lane + 32 * h;
            const bool valid = k < K;
            const uint32_t v = key_id(key[h]);
            bool accf = false;
            if (valid) accf = accept(hash_uj(fbase, ul, (uint64_t)k), isnew[h] ? cnew : cold, s);
            const unsigned mn = __ballot_sync(kFull, accf && isnew[h]);
            const unsigned mo = __ballot_sync(kFull, accf && !isnew[h]);
            if (accf && isnew[h]) st.cand_new[(size_t)u * st.cap + nbase + __popc(mn & lanemask_lt())] = (int)v;
            if (accf && !isnew[h]) st.cand_old[(size_t)u * st.cap + obase + __popc(mo & lanemask_lt())] = (int)v;
            nbase += __popc(mn);
            obase += __popc(mo);
            if (valid) {
                const int rc = isnew[h] ? st.rev_new[v] : st.rev_old[v];
                if (accept(hash_uj(rbase, ul, (uint64_t)k), (uint32_t)rc, s)) {
                    int slot = atomicAdd(isnew[h] ? &st.fill_new[v] : &st.fill_old[v], 1);
                    if (slot < st.R)
                        (isnew[h] ? st.cand_new : st.cand_old)[(size_t)v * st.cap + K + slot] = (int)u;
                    else
                        ++overflow;
                }
                uint64_t nk = key[h] & ~(uint64_t)kFlagIns;
                if (accf && isnew[h]) nk &= ~(uint64_t)kFlagNew;
                if (nk != key[h]) st.keys[(size_t)u * K + k] = nk;
            }
        }
        if (lane == 0) {
            st.fwd_new[u] = (int)nbase;
            st.fwd_old[u] = (int)obase;
        }
    }
    overflow = warp_sum(overflow);
    if (lane == 0 && overflow) atomic_add_ll(&st.stats[kStatRevOverflow], overflow);
}

cudaError_t launch_sample(const DevState &st, int li, int it, uint64_t seed, cudaStream_t s) {
    const uint64_t fb = hash_base(seed, kStreamFwd, (uint32_t)it), rb = hash_base(seed, kStreamRev, (uint32_t)it);
    if (st.K > kLaneK) {
        int grid = grid_for((const void *)sample_kernel<2>, kBlock, 0);
        sample_kernel<2><<<grid, kBlock, 0, s>>>(st, li, fb, rb);
        return cudaGetLastError();
    }
    int grid = grid_for((const void *)sample_kernel<1>, kBlock, 0);
    sample_kernel<1><<<grid, kBlock, 0, s>>>(st, li, fb, rb);
    return cudaGetLastError();
}

// ------------------------------------------------ priority-heap sampling ----
// The candidate construction of PyNNDescent, the alternative to Section 3.1's
// turbosampling: edge (u, j) with v = list[u][j] draws one priority
// p = hi32(h(seed, HEAP, it, u, j)) and offers v to u and u to v, both of the
// edge's kind (new/old) and with priority p.  Each node keeps per kind the s
// smallest (priority, id) offers, one per id (its smallest priority).
//   heap_alloc_kernel   each node's segments for its reverse offers (sizes:
//                       the count kernel's reverse degrees), claimed from one
//                       cursor a warp at a time; the layout does not matter,
//                       the selection is order-independent;
//   heap_scatter_kernel every edge writes (p << 32 | u) into v's segment;
//   heap_select_kernel  one warp per node folds its forward entries and its
//                       reverse offers into two sorted lane lists of s keys,
//                       writes the kept ids as the forward part of its
//                       candidates (reverse part empty, old ones that are also
//                       new dropped) and clears the "new" flag of its forward
//                       entries kept as new candidates.
__global__ void __launch_bounds__(256) heap_alloc_kernel(DevState st, int li) {
    if (iteration_skipped(st, li)) return;
    const unsigned lane = lane_id();
    for (long long w = gwarp(); w * 32 < st.n; w += nwarps()) {
        const long long v = w * 32 + lane;
        const bool ok = v < st.n;  // nodes of finished data sets have no reverse degree
        const int cn = ok ? st.rev_new[v] : 0, co = ok ? st.rev_old[v] : 0;
        int incl = cn + co;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if ((int)lane >= o) incl += t;
        }
        int base = 0;
        if (lane == 31) base = atomicAdd(st.hcursor, incl);
        base = __shfl_sync(kFull, base, 31);
        const int start = base + incl - (cn + co);
        if (ok) {
            st.hoff[v] = start;
            st.hoff[st.n + v] = start + cn;
        }
    }
}

__global__ void __launch_bounds__(kBlock) heap_scatter_kernel(DevState st, int li, uint64_t hbase) {
    if (iteration_skipped(st, li)) return;
    const unsigned lane = lane_id();
    const int K = st.K;
    long long dropped = 0;
    for (long long u = gwarp(); u < st.n; u += nwarps()) {
        if (node_skipped(st, u, li) || (int)lane >= K) continue;
        const uint64_t key = st.keys[(size_t)u * K + lane];
        const uint32_t v = key_id(key);
        const bool isnew = (key & kFlagNew) != 0;
        const uint32_t p = (uint32_t)(hash_uj(hbase, (uint64_t)node_local(st, u), lane) >> 32);
        const int slot = atomicAdd(isnew ? &st.fill_new[v] : &st.fill_old[v], 1);
        if (slot < (isnew ? st.rev_new[v] : st.rev_old[v]))
            st.hcsr[(size_t)st.hoff[(isnew ? 0 : st.n) + v] + slot] = ((uint64_t)p << 32) | (uint64_t)(uint32_t)u;
        else
            ++dropped;  // the segment was sized by the count kernel: cannot happen
    }
    dropped = warp_sum(dropped);
    if (lane == 0 && dropped) atomic_add_ll(&st.stats[kStatRevOverflow], dropped);
}

// Offer the 32 lanes' keys c (kKeyEmpty = none) to the ascending list S held
// in lanes 0 .. s-1 (empty above): a key enters if it is among the s smallest;
// a second offer of an id already listed replaces it only when smaller.
__device__ __forceinline__ void heap_offer(uint64_t &S, uint64_t c, int s, unsigned lane) {
    unsigned m = __ballot_sync(kFull, c < __shfl_sync(kFull, S, s - 1));
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const uint64_t x = __shfl_sync(kFull, c, src);
        const unsigned hit = __ballot_sync(kFull, (int)lane < s && S != kKeyEmpty && (uint32_t)S == (uint32_t)x);
        if (hit) {
            const int h = __ffs(hit) - 1;
            if (x >= __shfl_sync(kFull, S, h)) continue;
            const uint64_t nxt = __shfl_down_sync(kFull, S, 1);
            if ((int)lane >= h && (int)lane < s) S = (int)lane == s - 1 ? kKeyEmpty : nxt;
        } else if (x >= __shfl_sync(kFull, S, s - 1)) {
            continue;
        }
        const int pos = __popc(__ballot_sync(kFull, (int)lane < s && S < x));
        const uint64_t prv = __shfl_up_sync(kFull, S, 1);
        if ((int)lane < s) {
            if ((int)lane == pos) S = x;
            else if ((int)lane > pos) S = prv;
        }
    }
}

__global__ void __launch_bounds__(kBlock) heap_select_kernel(DevState st, int li, uint64_t hbase) {
    if (iteration_skipped(st, li)) return;
    const unsigned lane = lane_id();
    const int K = st.K, s = st.s;
    for (long long x = gwarp(); x < st.n; x += nwarps()) {
        if (node_skipped(st, x, li)) continue;
        const bool valid = (int)lane < K;
        const uint64_t key = valid ? st.keys[(size_t)x * K + lane] : kKeyEmpty;
        const bool isnew = valid && (key & kFlagNew);
        const uint32_t p = valid ? (uint32_t)(hash_uj(hbase, (uint64_t)node_local(st, x), lane) >> 32) : 0u;
        const uint64_t fwd = ((uint64_t)p << 32) | (uint64_t)key_id(key);
        uint64_t Sn = kKeyEmpty, So = kKeyEmpty;
        heap_offer(Sn, isnew ? fwd : kKeyEmpty, s, lane);
        heap_offer(So, valid && !isnew ? fwd : kKeyEmpty, s, lane);
        for (int f = 0; f < 2; ++f) {
            const int cnt = min(f ? st.fill_old[x] : st.fill_new[x], f ? st.rev_old[x] : st.rev_new[x]);
            const size_t off = (size_t)st.hoff[(f ? st.n : 0) + x];
            for (int b = 0; b < cnt; b += 32) {
                const uint64_t c = b + (int)lane < cnt ? st.hcsr[off + b + lane] : kKeyEmpty;
                if (f) heap_offer(So, c, s, lane);
                else heap_offer(Sn, c, s, lane);
            }
        }
        const size_t cb = (size_t)x * st.cap;
        const int nn = __popc(__ballot_sync(kFull, Sn != kKeyEmpty));
        if (Sn != kKeyEmpty) st.cand_new[cb + lane] = (int)(uint32_t)Sn;
        bool keep_old = So != kKeyEmpty, kept = false;
        for (int k = 0; k < nn; ++k) {
            const uint32_t id = (uint32_t)__shfl_sync(kFull, Sn, k);
            keep_old = keep_old && (uint32_t)So != id;
            kept = kept || key_id(key) == id;
        }
        const unsigned mo = __ballot_sync(kFull, keep_old);
        if (keep_old) st.cand_old[cb + __popc(mo & lanemask_lt())] = (int)(uint32_t)So;
        __syncwarp();
        if (lane == 0) {
            st.fwd_new[x] = nn;
            st.fwd_old[x] = __popc(mo);
            st.fill_new[x] = 0;
            st.fill_old[x] = 0;
        }
        if (valid) {
            uint64_t nk = key & ~(uint64_t)kFlagIns;
            if (isnew && kept) nk &= ~(uint64_t)kFlagNew;
            if (nk != key) st.keys[(size_t)x * K + lane] = nk;
        }
    }
}

cudaError_t launch_heap_sample(const DevState &st, int li, int it, uint64_t seed, cudaStream_t s) {
    const uint64_t hb = hash_base(seed, kStreamHeap, (uint32_t)it);
    heap_alloc_kernel<<<grid_for((const void *)heap_alloc_kernel, 256, 0), 256, 0, s>>>(st, li);
    heap_scatter_kernel<<<grid_for((const void *)heap_scatter_kernel, kBlock, 0), kBlock, 0, s>>>(st, li, hb);
    heap_select_kernel<<<grid_for((const void *)heap_select_kernel, kBlock, 0), kBlock, 0, s>>>(st, li, hb);
    return cudaGetLastError();
}

// ----------------------------------------------------- greedy relabelling ----
// Section 3.2, Algorithm 1, exact and sequential: spot i = 0 .. n-2 looks at
// the list a_i of the node on spot i (reading_b: node i), ascending; the first
// entry x not yet placed before spot i+1 either already holds spot i+1 (stop)
// or is moved there, the previous holder y of spot i+1 taking x's old spot p
// (the value of sigma(x) before the first swap).  One warp runs the whole
// chain: lanes hold the K list entries and test their spots in parallel; the
// first qualifying lane is found with a ballot.
template <int KW>
__global__ void __launch_bounds__(32) greedy_reorder_kernel(const uint64_t *__restrict__ keys, int64_t n, int K,
                                                            int reading_b, int32_t *sigma, int32_t *sigma_inv) {
    const unsigned lane = lane_id();
    for (int64_t i = lane; i < n; i += 32) {
        sigma[i] = (int32_t)i;
        sigma_inv[i] = (int32_t)i;
    }
    __syncwarp();
    int32_t node = 0;  // node on spot i (reading A); kept in a register across steps
    for (int64_t i = 0; i + 1 < n; ++i) {
        const int64_t who = reading_b ? i : node;
        // the first entry (in list order) whose node sits on a later spot
        int32_t xs = -1;
        int64_t ps = -1;
        bool found = false;
#pragma unroll
        for (int h = 0; h < KW && !found; ++h) {
            const int k = (int)lane + 32 * h;
            int32_t x = -1;
            int64_t p = -1;
            if (k < K) {
                x = (int32_t)key_id(__ldg(keys + (size_t)who * K + k));
                p = ((volatile int32_t *)sigma)[x];
            }
            const unsigned later = __ballot_sync(kFull, k < K && p >= i + 1);
            if (later) {
                const int src = __ffs(later) - 1;
                xs = __shfl_sync(kFull, x, src);
                ps = __shfl_sync(kFull, p, src);
                found = true;
            }
        }
        int32_t next_node;
        const int32_t held = ((volatile int32_t *)sigma_inv)[i + 1];
        if (!found) {
            next_node = held;
        } else {
            if (ps == i + 1) {
                next_node = xs;
            } else {
                if (lane == 0) {
                    sigma[xs] = (int32_t)(i + 1);
                    sigma[held] = (int32_t)ps;
                    sigma_inv[i + 1] = xs;
                    sigma_inv[ps] = held;
                }
                next_node = xs;
            }
        }
        __syncwarp();
        node = next_node;
    }
}

cudaError_t launch_greedy_reorder(const uint64_t *keys, int64_t n, int K, int reading_b, int32_t *sigma,
                                  int32_t *sigma_inv, cudaStream_t s) {
    if (K > kLaneK) greedy_reorder_kernel<2><<<1, 32, 0, s>>>(keys, n, K, reading_b, sigma, sigma_inv);
    else greedy_reorder_kernel<1><<<1, 32, 0, s>>>(keys, n, K, reading_b, sigma, sigma_inv);
    return cudaGetLastError();
}

// Move node u to spot sigma(u) (Section 3.2, all at once): its padded row and
// its list, ids renamed through sigma and re-sorted by (dist, new id).  The
// total relabelling original -> spot is composed with sigma.
template <int KW>
__global__ void __launch_bounds__(kBlock) permute_kernel(DevState st, float *__restrict__ X_dst,
                                                         uint64_t *__restrict__ keys_dst,
                                                         const int32_t *__restrict__ sigma,
                                                         int32_t *__restrict__ total_perm) {
    const unsigned lane = lane_id();
    const int K = st.K;
    const float4 *X4 = reinterpret_cast<const float4 *>(st.X);
    float4 *D4 = reinterpret_cast<float4 *>(X_dst);
    for (long long u = gwarp(); u < st.n; u += nwarps()) {
        const int32_t p = sigma[u];
        for (int c = lane; c < st.nv; c += 32) D4[(size_t)p * st.nv + c] = X4[(size_t)u * st.nv + c];
        uint64_t key[KW];
#pragma unroll
        for (int h = 0; h < KW; ++h) {
            const int k = (int)lane + 32 * h;
            key[h] = kKeyEmpty;
            if (k < K) {
                const uint64_t k0 = st.keys[(size_t)u * K + k];
                key[h] = (k0 & 0xFFFFFFFF00000003ull) | ((uint64_t)(uint32_t)sigma[key_id(k0)] << 2);
            }
        }
        if constexpr (KW == 2) warp_sort_u64x2(key[0], key[KW - 1]);
        else key[0] = warp_sort_u64(key[0]);
#pragma unroll
        for (int h = 0; h < KW; ++h)
            if ((int)lane + 32 * h < K) keys_dst[(size_t)p * K + lane + 32 * h] = key[h];
        if (lane == 0) total_perm[u] = sigma[total_perm[u]];
    }
}

cudaError_t launch_permute(const DevState &src, float *X_dst, uint64_t *keys_dst, const int32_t *sigma,
                           int32_t *total_perm, cudaStream_t s) {
    if (src.K > kLaneK) {
        int grid = grid_for((const void *)permute_kernel<2>, kBlock, 0);
        permute_kernel<2><<<grid, kBlock, 0, s>>>(src, X_dst, keys_dst, sigma, total_perm);
        return cudaGetLastError();
    }
    int grid = grid_for((const void *)permute_kernel<1>, kBlock, 0);
    permute_kernel<1><<<grid, kBlock, 0, s>>>(src, X_dst, keys_dst, sigma, total_perm);
    return cudaGetLastError();
}

// node -> data set of a batched context (data sets are contiguous node ranges)
__global__ void ds_map_kernel(const long long *__restrict__ ds_off, int nds, int64_t n, int *__restrict__ ds) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nds - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (ds_off[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        ds[u] = lo;
    }
}

cudaError_t launch_ds_map(const long long *ds_off, int nds, int64_t n, int *ds, cudaStream_t s) {
    int grid = grid_for((const void *)ds_map_kernel, 256, 0);
    ds_map_kernel<<<grid, 256, 0, s>>>(ds_off, nds, n, ds);
    return cudaGetLastError();
}

__global__ void iota_kernel(int32_t *__restrict__ p, int64_t n) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        p[u] = (int32_t)u;
}

cudaError_t launch_iota(int32_t *p, int64_t n, cudaStream_t s) {
    int grid = grid_for((const void *)iota_kernel, 256, 0);
    iota_kernel<<<grid, 256, 0, s>>>(p, n);
    return cudaGetLastError();
}

__global__ void invert_kernel(const int32_t *__restrict__ perm, int64_t n, int32_t *__restrict__ inv) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        inv[perm[u]] = (int32_t)u;
}

cudaError_t launch_invert(const int32_t *perm, int64_t n, int32_t *inv, cudaStream_t s) {
    int grid = grid_for((const void *)invert_kernel, 256, 0);
    invert_kernel<<<grid, 256, 0, s>>>(perm, n, inv);
    return cudaGetLastError();
}

// ------------------------------------------------------ re-rank + output ----
// Final lists in the caller's labelling: original node u's list lives at spot
// total_perm[u]; ids are renamed back and the row is re-sorted by (dist,
// original id).  Float32 keys already hold the canonical float32 distance of
// their pair (init and every join compute it the same way, and both orders of
// a pair agree bit for bit), so they are taken as they are; the approximate
// keys of the bf16 and FP8 forms are re-ranked with the canonical distance.
template <bool kStaged, int KW>
__global__ void __launch_bounds__(kBlock) output_kernel(DevState st, const int32_t *__restrict__ total_perm,
                                                        const int32_t *__restrict__ total_inv,
                                                        int32_t *__restrict__ ids, float *__restrict__ dists) {
    extern __shared__ __align__(16) float4 stage_sm[];
    const unsigned lane = lane_id();
    const int K = st.K;
    const float4 *X4 = reinterpret_cast<const float4 *>(st.X);
    for (long long u = gwarp(); u < st.n; u += nwarps()) {
        const int64_t p = total_perm ? total_perm[u] : u;
        uint64_t key[KW];
#pragma unroll
        for (int h = 0; h < KW; ++h) {
            const int k = (int)lane + 32 * h;
            const int cnt = K - 32 * h < 32 ? K - 32 * h : 32;
            key[h] = kKeyEmpty;
            const uint64_t lk = k < K ? st.keys[(size_t)p * K + k] : kKeyEmpty;
            const uint32_t v = k < K ? key_id(lk) : (uint32_t)p;
            float dd;
            if (!st.bf16) dd = k < K ? key_dist(lk) : 0.f;
            else if (kStaged) dd = warp_staged_dist(X4, st.nv, p, v, cnt, stage_sm + (threadIdx.x >> 5) * 33 * (st.nv | 1));
            else dd = k < K ? l2sq_rows(X4 + (size_t)p * st.nv, X4 + (size_t)v * st.nv, st.nv) : 0.f;
            if (k < K) {
                uint32_t vo = total_inv ? (uint32_t)total_inv[v] : v;
                if (st.ds) vo -= (uint32_t)st.ds_off[st.ds[u]];  // batched: ids local to the data set
                key[h] = make_key(dd, vo, 0);
            }
        }
        if constexpr (KW == 2) warp_sort_u64x2(key[0], key[KW - 1]);
        else key[0] = warp_sort_u64(key[0]);
#pragma unroll
        for (int h = 0; h < KW; ++h) {
            const int k = (int)lane + 32 * h;
            if (k < K) {
                ids[(size_t)u * K + k] = (int32_t)key_id(key[h]);
                dists[(size_t)u * K + k] = key_dist(key[h]);
            }
        }
    }
}

cudaError_t launch_output(const DevState &st, const int32_t *total_perm, const int32_t *total_inv,
                          int32_t *ids, float *dists, cudaStream_t s) {
    if (st.K > kLaneK) {  // float32 keys only: no re-rank
        int grid = grid_for((const void *)output_kernel<false, 2>, kBlock, 0);
        output_kernel<false, 2><<<grid, kBlock, 0, s>>>(st, total_perm, total_inv, ids, dists);
        return cudaGetLastError();
    }
    if (st.bf16 && st.nv >= kStageMinNv && st.nv <= kStageMaxNv) {
        const size_t dyn = stage_smem_bytes(st.nv);
        cudaError_t e = smem_opt_in((const void *)output_kernel<true, 1>, dyn);
        if (e != cudaSuccess) return e;
        const int grid = grid_for((const void *)output_kernel<true, 1>, kStageWarps * 32, dyn);
        output_kernel<true, 1><<<grid, kStageWarps * 32, dyn, s>>>(st, total_perm, total_inv, ids, dists);
        return cudaGetLastError();
    }
    int grid = grid_for((const void *)output_kernel<false, 1>, kBlock, 0);
    output_kernel<false, 1><<<grid, kBlock, 0, s>>>(st, total_perm, total_inv, ids, dists);
    return cudaGetLastError();
}

}  // namespace knng
