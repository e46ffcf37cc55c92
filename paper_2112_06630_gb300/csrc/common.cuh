// common.cuh -- device-side building blocks shared by the NN-Descent kernels:
// packed list keys, the counter-based hash, the canonical float32 squared-l2
// distance, warp sorting, and the bounded per-list lock.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace knng {

// ---------------------------------------------------------------- keys ----
// A list entry is one 64-bit key: float bits of the squared distance (high
// word; distances are >= +0 so the bit pattern orders like the float), then
// the neighbour id (30 bits) and two flag bits.  Ordering keys as integers
// orders entries by (dist, id), the tie rule of the method; the flag bits sit
// below the id and never decide an order between different ids.
constexpr uint32_t kFlagNew = 1u;  // not yet sampled as a forward "new" candidate
constexpr uint32_t kFlagIns = 2u;  // inserted during the current iteration
constexpr uint64_t kKeyEmpty = ~0ull;
constexpr int kMaxK = 64;        // lists of up to 64 keys: one key per lane up to 32, two above
constexpr int kLaneK = 32;       // the largest K held one key per lane

__host__ __device__ __forceinline__ uint64_t make_key(float dist, uint32_t id, uint32_t flags) {
#ifdef __CUDA_ARCH__
    uint32_t bits = __float_as_uint(dist);
#else
    uint32_t bits;
    __builtin_memcpy(&bits, &dist, 4);
#endif
    return ((uint64_t)bits << 32) | ((uint64_t)id << 2) | (uint64_t)flags;
}
__host__ __device__ __forceinline__ uint32_t key_id(uint64_t k) { return (uint32_t)(k >> 2) & 0x3FFFFFFFu; }
__host__ __device__ __forceinline__ uint32_t key_flags(uint64_t k) { return (uint32_t)k & 3u; }
__device__ __forceinline__ float key_dist(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }
// same (dist, id), flags stripped
__host__ __device__ __forceinline__ uint64_t key_order(uint64_t k) { return k & ~3ull; }

// ---------------------------------------------------------------- hash ----
// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).  The random
// word for (seed, stream, iter, u, j) is mix(mix(mix(mix(seed) ^ (stream<<32 |
// iter)) ^ u) ^ j); the first two levels depend on the launch only and are
// computed on the host ("base").
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
enum Stream : uint32_t { kStreamInit = 1, kStreamFwd = 2, kStreamRev = 3, kStreamHeap = 4 };
__host__ __device__ __forceinline__ uint64_t hash_base(uint64_t seed, uint32_t stream, uint32_t iter) {
    return splitmix64(splitmix64(seed) ^ (((uint64_t)stream << 32) | (uint64_t)iter));
}
__host__ __device__ __forceinline__ uint64_t hash_uj(uint64_t base, uint64_t u, uint64_t j) {
    return splitmix64(splitmix64(base ^ u) ^ j);
}
// Bernoulli(s / cnt) in integers: hi32(h) * cnt < s * 2^32
__device__ __forceinline__ bool accept(uint64_t h, uint32_t cnt, uint32_t s) {
    return (h >> 32) * (uint64_t)cnt < ((uint64_t)s << 32);
}

// ----------------------------------------------------------- distance ----
// Canonical float32 squared l2 (difference form, no square root): rows are
// zero-padded to a multiple of 4 floats; two partial sums over t mod 2, each
// accumulated in ascending t with fused multiply-add, combined as s0 + s1.
// Every float32 distance in the library (init, join, brute force, re-rank)
// uses exactly this order, so one pair always gets one value and the two
// orders of a pair agree bit for bit.
// The partial sums run as one packed pair (s0, s1) on the paired float32
// instructions of sm_100+ (sub.rn.f32x2, fma.rn.f32x2): each lane of the pair
// is the IEEE round-to-nearest operation of the scalar form, so the values are
// those of two scalar chains, with half the instructions.  Two sums (not
// four) keep a pair's accumulator in one 64-bit register, which leaves the
// register-blocked join kernels room to load the next unit ahead.
__device__ __forceinline__ unsigned long long f32x2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f32x2_unpack(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
struct Acc2 {
    unsigned long long s;  // (s0, s1): the elements t even and t odd
    __device__ __forceinline__ Acc2() : s(0ull) {}
    __device__ __forceinline__ void add(float4 a, float4 b) {
        unsigned long long d01, d23;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d01) : "l"(f32x2_pack(a.x, a.y)), "l"(f32x2_pack(b.x, b.y)));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d23) : "l"(f32x2_pack(a.z, a.w)), "l"(f32x2_pack(b.z, b.w)));
        asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(s) : "l"(d01));
        asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(s) : "l"(d23));
    }
    __device__ __forceinline__ float sum() const {
        float s0, s1;
        f32x2_unpack(s, s0, s1);
        return s0 + s1;
    }
};

__device__ __forceinline__ float l2sq_rows(const float4 *__restrict__ a, const float4 *__restrict__ b, int nv) {
    Acc2 acc;
#pragma unroll 8
    for (int v = 0; v < nv; ++v) acc.add(a[v], b[v]);
    return acc.sum();
}

// --------------------------------------------------------------- warps ----
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int m) {
    return __shfl_xor_sync(0xFFFFFFFFu, v, m);
}

// Ascending bitonic sort of one 64-bit key per lane across the full warp.
__device__ __forceinline__ uint64_t warp_sort_u64(uint64_t v) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            uint64_t o = shfl_xor_u64(v, j);
            bool up = (lane & k) == 0;
            bool low = (lane & j) == 0;
            uint64_t mn = v < o ? v : o, mx = v < o ? o : v;
            v = (low == up) ? mn : mx;
        }
    }
    return v;
}

// Ascending bitonic sort of 64 keys held two per lane across the full warp:
// a is element lane, b element lane + 32.
__device__ __forceinline__ void warp_sort_u64x2(uint64_t &a, uint64_t &b) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j == 32) {
                // k == 64: element lane against element lane + 32, ascending
                const uint64_t mn = a < b ? a : b, mx = a < b ? b : a;
                a = mn;
                b = mx;
                continue;
            }
            const bool low = (lane & j) == 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint64_t &v = h ? b : a;
                const uint64_t o = shfl_xor_u64(v, j);
                const bool up = (((int)lane + 32 * h) & k) == 0;
                const uint64_t mn = v < o ? v : o, mx = v < o ? o : v;
                v = (low == up) ? mn : mx;
            }
        }
    }
}

// A list of K <= 64 ascending keys held by one warp: entry lane in lo, entry
// lane + 32 in hi (kKeyEmpty at and past K).  For K <= 32 hi stays empty and
// every operation is the one-key-per-lane form.
struct WList {
    uint64_t lo, hi;
};
__device__ __forceinline__ WList wlist_load(const uint64_t *row, int K) {
    const int lane = (int)lane_id();
    WList L;
    L.lo = lane < K ? __ldcg(row + lane) : kKeyEmpty;
    L.hi = lane + 32 < K ? __ldcg(row + 32 + lane) : kKeyEmpty;
    return L;
}
__device__ __forceinline__ void wlist_store(const WList &L, uint64_t *row, int K) {
    const int lane = (int)lane_id();
    if (lane < K) __stcg(row + lane, L.lo);
    if (lane + 32 < K) __stcg(row + 32 + lane, L.hi);
}
// entry idx (the same on every lane)
__device__ __forceinline__ uint64_t wlist_at(const WList &L, int idx) {
    const uint64_t a = __shfl_sync(0xFFFFFFFFu, L.lo, idx & 31), b = __shfl_sync(0xFFFFFFFFu, L.hi, idx & 31);
    return idx < 32 ? a : b;
}
// entries carrying all bits of `flag`
__device__ __forceinline__ int wlist_count(const WList &L, int K, uint64_t flag) {
    const int lane = (int)lane_id();
    return __popc(__ballot_sync(0xFFFFFFFFu, lane < K && (L.lo & flag) == flag)) +
           __popc(__ballot_sync(0xFFFFFFFFu, lane + 32 < K && (L.hi & flag) == flag));
}
// Insert x if it orders before the worst entry and its id is not listed; the
// worst entry leaves.  Warp-uniform result: true if inserted.
__device__ __forceinline__ bool wlist_insert(WList &L, uint64_t x, int K) {
    const int lane = (int)lane_id();
    const bool vl = lane < K, vh = lane + 32 < K;
    if (x >= wlist_at(L, K - 1)) return false;
    const uint32_t id = key_id(x);
    if (__any_sync(0xFFFFFFFFu, (vl && key_id(L.lo) == id) || (vh && key_id(L.hi) == id))) return false;
    const unsigned gl = __ballot_sync(0xFFFFFFFFu, vl && L.lo > x), gh = __ballot_sync(0xFFFFFFFFu, vh && L.hi > x);
    const int pos = gl ? __ffs(gl) - 1 : 32 + __ffs(gh) - 1;  // first entry ordered after x
    const uint64_t lo_up = __shfl_up_sync(0xFFFFFFFFu, L.lo, 1), hi_up = __shfl_up_sync(0xFFFFFFFFu, L.hi, 1);
    const uint64_t lo_last = __shfl_sync(0xFFFFFFFFu, L.lo, 31);
    if (vl && lane >= pos) L.lo = lane == pos ? x : lo_up;
    if (vh && lane + 32 >= pos) L.hi = lane + 32 == pos ? x : (lane == 0 ? lo_last : hi_up);
    return true;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
    return v;
}

// --------------------------------------------------------------- locks ----
// Per-list spin lock with a bounded wait: after kLockSpinLimit failed tries
// the caller gives up (the proposal is dropped and an error counter is
// raised, which the host turns into KNNG_ERR_TIMEOUT).  Never waits forever.
constexpr int kLockSpinLimit = 1 << 22;

__device__ __forceinline__ bool lock_acquire(int *lock) {
    int spins = 0;
    while (atomicCAS(lock, 0, 1) != 0) {
        if (++spins >= kLockSpinLimit) return false;
        __nanosleep(spins < 64 ? 20 : 200);
    }
    __threadfence();
    return true;
}
__device__ __forceinline__ void lock_release(int *lock) {
    __threadfence();
    atomicExch(lock, 0);
}

// ------------------------------------------------------------ counters ----
// two's-complement add on a signed 64-bit counter
__device__ __forceinline__ void atomic_add_ll(long long *p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}
// Global int64 counters (index into DevState::stats).
enum Stat : int {
    kStatEvals = 0,
    kStatInserts,
    kStatMerges,
    kStatGathered,
    kStatRevOverflow,
    kStatSetOverflow,
    kStatLockTimeout,
    kStatInitAttemptsExceeded,
    kStatBucketOverflow,
    kStatCount
};
// Per-iteration counters (index into it_stats[iter * kItCount]).
enum ItStat : int {
    kItRan = 0,      // set when the iteration's join ran
    kItChanges,      // entries inserted and still present at the end
    kItEvals,        // distance evaluations
    kItGathered,     // candidate rows gathered
    kItMerges,       // locked merges
    kItInserts,      // insertions (incl. evicted later)
    kItCandIds,      // raw candidate ids read
    kItProposals,    // proposal keys written to buckets (or inserted past a full one)
    kItCount = 8
};

struct DevState {
    const float *X;      // n x dp, zero padded
    const uint16_t *Xb;  // n x dpb bf16 bits (zero padded to a multiple of 64), bf16 mode only;
                         // in FP8 mode n x dpb e4m3 bytes
    const float *xnorm;  // n squared norms of the bf16 (or e4m3) rows, low-precision modes only
    uint64_t *keys;      // n x K, ascending
    int *locks;          // n, taken only when a proposal bucket is full
    int *pcursor;        // n, proposals reserved in each node's bucket this iteration
    uint64_t *pbucket;   // n x kBucketRun proposal keys (the first run of every bucket)
    int *pchunk;         // n x kBucketChunks: pool chunk + 1 of the bucket's further runs, 0 = none
    uint64_t *ppool;     // pool_chunks x kBucketRun keys
    int *pool_next;      // next free pool chunk (restarted every iteration)
    int pool_chunks;
    int *rev_new, *rev_old;    // reverse degrees by flag
    int *fill_new, *fill_old;  // reverse candidate fill counters
    int *fwd_new, *fwd_old;    // accepted forward counts
    int *cand_new, *cand_old;  // n x cap: [0, K) forward part, [K, K + R) reverse part
    // priority-heap sampling only (else null): each node's reverse offers of
    // each kind at hcsr[hoff[kind * n + v] ..), claimed from *hcursor
    int *hoff;                 // 2 x n
    uint64_t *hcsr;            // n x K keys (priority << 32 | source)
    int *hcursor;
    long long *stats;
    long long *it_stats;       // (max_iters + 2) x kItCount
    int64_t n;
    int d, dp, nv, K, s, R, cap, dpb;
    int bf16;                  // 1: high-d joins use low-precision tensor-core Gram blocks (bf16 or
                               // FP8): list keys are not the canonical float32 distances
    int fp8;                   // 1: the low-precision rows are e4m3 (FP8 mode)
    // batched mode (many independent data sets in one node space), else null:
    const int *ds;             // node -> data set
    const long long *ds_off;   // data set -> first node
    const int *ds_n;           // data set -> number of nodes
    const double *ds_thr;      // data set -> delta * n * K
    long long *ds_changes;     // data set x kMaxLocalIters change counts
    double thr;                // delta * n * K
    // ring and pipelined join paths only (else null): per-node candidate sets
    // written by the set kernel and read by the join kernel
    int *cset;                 // n x 64 candidate ids, new ones first
    int *cmeta;                // n: ns | m << 8 (0: no join pair)
    int join_path;             // JoinPath chosen for this context
    // nodes whose joins this launch runs, [u_lo, u_hi): the whole set, or one
    // pass of an iteration split into node ranges with a list merge after
    // each (the set kernel runs once, with the first pass)
    long long u_lo, u_hi;
};

// Which local-join kernel a context uses (fixed at creation).
// kJoinPipe: the pipelined kernel with four compute warps and one row slot per
// block; kJoinPipe8: the same kernel with eight warps and two slots
enum JoinPath : int { kJoinWarp = 0, kJoinTile = 1, kJoinRing = 2, kJoinPipe = 3, kJoinPipe8 = 4 };

// Proposal buckets: run 0 of node p is inline (pbucket), runs 1..15 are pool
// chunks claimed on demand with a CAS (a lane that loses the race uses the
// winner's chunk; its own stays unused until the pool restarts).  A run whose
// chunk cannot be claimed (pool spent) is poisoned for the iteration.
constexpr int kBucketRunBits = 8;
constexpr int kBucketRun = 1 << kBucketRunBits;
constexpr int kBucketChunks = 15;
constexpr int kBucketMax = kBucketRun * (kBucketChunks + 1);
constexpr int kChunkPoison = -1;

// Slot of proposal number `pos` of node p, or nullptr when the bucket or the
// pool is exhausted (the caller then inserts into the list under its lock).
__device__ __forceinline__ uint64_t *bucket_slot(const DevState &st, uint32_t p, int pos);

constexpr int kMaxLocalIters = 1024;  // iterations one context can run

// True when iteration `it` must not run because an earlier one converged.
__device__ __forceinline__ bool iteration_skipped(const DevState &st, int it) {
    if (it <= 1) return false;
    const volatile long long *prev = st.it_stats + (size_t)(it - 1) * kItCount;
    return (double)prev[kItChanges] < st.thr;
}

}  // namespace knng

namespace knng {
__device__ __forceinline__ uint64_t *bucket_slot(const DevState &st, uint32_t p, int pos) {
    const int k = pos >> kBucketRunBits, off = pos & (kBucketRun - 1);
    if (k == 0) return st.pbucket + ((size_t)p << kBucketRunBits) + off;
    if (k > kBucketChunks) return nullptr;
    int *ent = st.pchunk + (size_t)p * kBucketChunks + (k - 1);
    int c = *reinterpret_cast<volatile int *>(ent);
    if (c == 0) {
        // claim a chunk; with the pool spent, install the poison mark instead,
        // so that no warp can install a chunk for this run afterwards and all
        // of the run's proposals take the locked way (no unwritten slot is
        // ever read by the merge)
        const int fresh = atomicAdd(st.pool_next, 1);
        const int want = fresh < st.pool_chunks ? fresh + 1 : kChunkPoison;
        const int old = atomicCAS(ent, 0, want);
        c = old ? old : want;
    }
    if (c == kChunkPoison) return nullptr;
    return st.ppool + ((size_t)(c - 1) << kBucketRunBits) + off;
}
}  // namespace knng

namespace knng {
// Batched mode: node u's data set converged in an earlier iteration.
__device__ __forceinline__ bool node_skipped(const DevState &st, long long u, int li) {
    if (!st.ds || li < 1) return false;
    const int b = st.ds[u];
    const volatile long long *ch = st.ds_changes;
    return (double)ch[(size_t)b * kMaxLocalIters + li - 1] < st.ds_thr[b];
}
// node id local to its data set (the random streams are keyed by local ids, so
// a data set gets the same build alone or batched)
__device__ __forceinline__ long long node_local(const DevState &st, long long u) {
    return st.ds ? u - st.ds_off[st.ds[u]] : u;
}
}  // namespace knng
