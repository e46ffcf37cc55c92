// join.cu -- the local join and the list update (the paper's Calculation
// step, Section 2 and Section 3.3), float32 difference-form distances.
//
// Two kernels per iteration, no locks on the common path:
//
// join_kernel: one warp owns one node u at a time (persistent grid-stride):
//   1. read u's sampled candidates (forward part written by u's sampling warp,
//      reverse part filled by other warps), drop repeats keeping the first
//      occurrence (new before old), cap the set S at 64; a node without new
//      candidates has no join pair and is skipped;
//   2. gather the candidate rows into shared memory (padded row stride) and
//      snapshot each candidate's current worst key;
//   3. enumerate every join pair once -- {p, q} inside new(u) through a
//      circulant walk (pair (r, r+1+c mod m'), m' = m rounded up to odd, meets
//      every unordered pair exactly once) and new(u) x old(u) as a rectangle --
//      with all 32 lanes taking consecutive pairs.  A pair whose key beats the
//      snapshot worst of an endpoint sets the partner's bit in that endpoint's
//      proposal mask (two 32-bit words, shared-memory atomicOr);
//   4. lane per target with proposals: one atomicAdd reserves a range of the
//      target's proposal bucket and the lane writes the keys (recomputing each
//      pair with the same arithmetic, so the same bits).  A proposal whose run
//      has no slot (bucket full or pool spent) is marked and then inserted
//      into the list under the list's lock (bounded spin; rare).  A
//      bucket is a 256-key run per node plus up to 15 runs claimed from a pool
//      on demand, so hub nodes hold up to 4,096 proposals.
// merge_kernel: one warp per node with a non-empty bucket: lane k holds list
//   entry k; bucket keys arrive 32 at a time, those that order before the
//   worst and are not listed go in (a sort-merge for six or more, else one by
//   one with ballots).  The entries still flagged "inserted in this
//   iteration" at the end are the iteration's changes for that list.
// Since every float32 distance in the library uses the same arithmetic, a pair
// always yields the same key, and each list ends as the K smallest distinct
// keys of its start entries and all proposals it received, whatever the order.
#include "join_common.cuh"

namespace knng {

namespace {
__device__ __forceinline__ void cp_async16_w(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8_w(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
constexpr int kJoinWarps = 4;
constexpr int kMergeWarps = 8;
constexpr int kWarpMaxNv = 8;   // float32 rows of up to 32 floats take the warp kernel (measured crossover)
constexpr int kSortMergeMin = 10;  // candidates per 32-key batch from which a sort-merge beats insertions (measured: 4 slower, 8-12 flat)

struct JoinLayout {
    int raw_max;      // ints for raw candidate ids
    int row_stride;   // float4 per staged row
    size_t off_swk;   // byte offsets inside a warp's region
    size_t off_rows;
    size_t per_warp;  // bytes
};

// per-warp shared memory: sid[64] | (spare)[64] | swk[64] | mask[64] | scratch,
// where scratch holds the raw candidate ids and the hash set until repeats
// are removed, and the staged rows[64][rs] afterwards; swk becomes the
// per-target mask of proposals that found no bucket slot
__host__ __device__ inline JoinLayout join_layout(int cap, int nv, bool rows_smem) {
    JoinLayout L;
    L.raw_max = ((2 * cap + 31) / 32) * 32;
    L.row_stride = (nv % 2 == 0) ? nv + 1 : nv;
    L.off_swk = kSetMax * 4 * 2;
    L.off_rows = L.off_swk + kSetMax * 8 * 2;
    const size_t dedup = (size_t)L.raw_max * 4 + (4u << hash_bits(cap));
    const size_t rows = rows_smem ? (size_t)kSetMax * L.row_stride * 16 : 0;
    L.per_warp = L.off_rows + (dedup > rows ? dedup : rows);
    L.per_warp = (L.per_warp + 15) & ~(size_t)15;
    return L;
}

}  // namespace

template <bool kRowsSmem>
__global__ void __launch_bounds__(kJoinWarps * 32, 8) join_kernel(DevState st, int li) {
    if (iteration_skipped(st, li)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long bstat[kItCount];
    __shared__ long long bovf, btimeout;
    if (threadIdx.x < kItCount) bstat[threadIdx.x] = 0;
    if (threadIdx.x == 0) bovf = btimeout = 0;
    __syncthreads();

    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int K = st.K, cap = st.cap, nv = st.nv;
    const JoinLayout lay = join_layout(cap, nv, kRowsSmem);
    unsigned char *wbase = smem + (size_t)warp * lay.per_warp;
    int *sid = reinterpret_cast<int *>(wbase);
    uint64_t *swk = reinterpret_cast<uint64_t *>(wbase + lay.off_swk);
    unsigned long long *mask = reinterpret_cast<unsigned long long *>(swk + kSetMax);
    unsigned *mw = reinterpret_cast<unsigned *>(mask);  // the masks as 32-bit words (native shared atomics)
    float4 *rows = reinterpret_cast<float4 *>(wbase + lay.off_rows);
    int *hset = reinterpret_cast<int *>(wbase + lay.off_rows);  // aliases rows until they are staged
    int *raw = hset + (1 << hash_bits(st.cap));
    const int rs = lay.row_stride;
    const float4 *X4 = reinterpret_cast<const float4 *>(st.X);

    long long w_evals = 0, w_gathered = 0, w_candids = 0, w_setovf = 0, w_ovf = 0, w_ins = 0, w_to = 0;
    long long l_props = 0;  // per lane

    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = st.u_lo + gw; u < st.u_hi; u += nw) {
        if (node_skipped(st, u, li)) continue;  // batched: u's data set converged
        // ---- 1. candidates of u, repeats removed (new first, then old)
        int ns, m;
        w_candids += warp_gather_candidates(st, u, raw, hset, sid, ns, m, w_setovf);
        if (ns == 0) continue;  // no new candidate: no join pair
        const int o = ns - m;
        __syncwarp();
        // ---- 2. snapshot worst keys, clear masks, stage rows (asynchronous
        //         copies: one round trip for all of them)
        for (int i = lane; i < ns; i += 32) {
            cp_async8_w(swk + i, st.keys + (size_t)sid[i] * K + (K - 1));
            mask[i] = 0ull;
        }
        if (kRowsSmem) {
            for (int idx = lane; idx < ns * nv; idx += 32) {
                const int r = idx / nv, c = idx - r * nv;
                cp_async16_w(rows + r * rs + c, X4 + (size_t)sid[r] * nv + c);
            }
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        w_gathered += ns;
        // ---- 3. every join pair once, all lanes busy
        const int mo = m | 1, half = (mo - 1) >> 1;
        const uint32_t t1 = (uint32_t)mo * (uint32_t)half;  // circulant slots over new(u)
        const uint32_t t2 = (uint32_t)m * (uint32_t)o;       // new(u) x old(u)
        const uint32_t mg1 = div_magic((uint32_t)half), mg2 = div_magic((uint32_t)o);
        w_evals += (long long)m * (m - 1) / 2 + (long long)m * o;
        for (uint32_t k = lane; k < t1 + t2; k += 32) {
            int i, j;
            if (k < t1) {
                const uint32_t r = div_small(k, (uint32_t)half, mg1);
                const uint32_t c = k - r * (uint32_t)half;
                i = (int)r;
                j = (int)(r + 1 + c);
                if (j >= mo) j -= mo;
                if (i >= m || j >= m) continue;  // the padding slot of an even m
            } else {
                const uint32_t q = k - t1;
                const uint32_t r = div_small(q, (uint32_t)o, mg2);
                i = (int)r;
                j = m + (int)(q - r * (uint32_t)o);
            }
            const float4 *ri = kRowsSmem ? rows + i * rs : X4 + (size_t)sid[i] * nv;
            const float4 *rj = kRowsSmem ? rows + j * rs : X4 + (size_t)sid[j] * nv;
            const float dd = l2sq_rows(ri, rj, nv);
            if (make_key(dd, (uint32_t)sid[j], kFlagNew | kFlagIns) < swk[i])
                atomicOr(&mw[2 * i + (j >> 5)], 1u << (j & 31));
            if (make_key(dd, (uint32_t)sid[i], kFlagNew | kFlagIns) < swk[j])
                atomicOr(&mw[2 * j + (i >> 5)], 1u << (i & 31));
        }
        __syncwarp();
        // ---- 4. bucket runs, flattened over the warp: lane t reserves
        //         target t's range (one atomicAdd per target) and the pool
        //         chunks of the runs it spans (one claim per run); then lane k
        //         writes proposal k of the node -- its target found by a
        //         binary search over the targets' prefix counts, its partner
        //         as the r-th set bit of the target's mask -- so every lane
        //         has work however unevenly the proposals fall.  Each key is
        //         recomputed with the arithmetic of step 3 (bit-identical); a
        //         proposal whose run has no slot (bucket or pool spent) is
        //         marked for the locked insertion
        unsigned long long *fails = reinterpret_cast<unsigned long long *>(swk);  // swk is done
        int *rbase = sid + kSetMax;  // per target: reserved start minus its prefix count
        int inc0, inc1;              // inclusive prefix counts of targets lane and 32 + lane
        {
            const unsigned long long ma = (int)lane < ns ? mask[lane] : 0ull;
            const unsigned long long mb = (int)lane + 32 < ns ? mask[lane + 32] : 0ull;
            const int ca = __popcll(ma), cb = __popcll(mb);
            int ba = 0, bb = 0;
            if (ca) ba = atomicAdd(st.pcursor + sid[lane], ca);
            if (cb) bb = atomicAdd(st.pcursor + sid[lane + 32], cb);
            if (ca)
                for (int r = ba >> kBucketRunBits > 1 ? ba >> kBucketRunBits : 1; r <= (ba + ca - 1) >> kBucketRunBits;
                     ++r)
                    bucket_slot(st, (uint32_t)sid[lane], r << kBucketRunBits);
            if (cb)
                for (int r = bb >> kBucketRunBits > 1 ? bb >> kBucketRunBits : 1; r <= (bb + cb - 1) >> kBucketRunBits;
                     ++r)
                    bucket_slot(st, (uint32_t)sid[lane + 32], r << kBucketRunBits);
            l_props += ca + cb;
            inc0 = ca;
            inc1 = cb;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(kFull, inc0, o);
                if ((int)lane >= o) inc0 += v;
            }
            const int tot0 = __shfl_sync(kFull, inc0, 31);
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(kFull, inc1, o);
                if ((int)lane >= o) inc1 += v;
            }
            inc1 += tot0;
            if ((int)lane < ns) {
                rbase[lane] = ba - (inc0 - ca);
                fails[lane] = 0ull;
            }
            if ((int)lane + 32 < ns) {
                rbase[lane + 32] = bb - (inc1 - cb);
                fails[lane + 32] = 0ull;
            }
        }
        const int total = __shfl_sync(kFull, inc1, 31);
        __threadfence_block();
        __syncwarp();
        unsigned ovf_lo = 0, ovf_hi = 0;  // targets with marked proposals
        for (int k0 = 0; k0 < total; k0 += 32) {
            const int k = k0 + (int)lane;
            const bool act = k < total;
            const int kk = act ? k : total - 1;
            // target of proposal kk: the number of targets whose inclusive
            // prefix count is <= kk (prefixes of targets past ns equal total)
            int t = 0;
#pragma unroll
            for (int step = 32; step > 0; step >>= 1) {
                const int probe = t + step - 1;
                const int v0 = __shfl_sync(kFull, inc0, probe & 31), v1 = __shfl_sync(kFull, inc1, probe & 31);
                if ((probe < 32 ? v0 : v1) <= kk) t += step;
            }
            const int tp = t > 0 ? t - 1 : 0;
            const int e0 = __shfl_sync(kFull, inc0, tp & 31), e1 = __shfl_sync(kFull, inc1, tp & 31);
            const int excl = t == 0 ? 0 : (tp < 32 ? e0 : e1);
            if (!act) continue;
            const uint32_t p = (uint32_t)sid[t];
            const int j = nth_set_bit64(mask[t], k - excl);
            uint64_t *slot = bucket_slot(st, p, k + rbase[t]);
            if (slot) {
                const float4 *rt = kRowsSmem ? rows + t * rs : X4 + (size_t)p * nv;
                const float4 *rj = kRowsSmem ? rows + j * rs : X4 + (size_t)sid[j] * nv;
                *slot = make_key(l2sq_rows(rt, rj, nv), (uint32_t)sid[j], kFlagNew | kFlagIns);
            } else {
                atomicOr(&fails[t], 1ull << j);
                if (t < 32) ovf_lo |= 1u << t;
                else ovf_hi |= 1u << (t - 32);
            }
        }
        ovf_lo = __reduce_or_sync(kFull, ovf_lo);
        ovf_hi = __reduce_or_sync(kFull, ovf_hi);
        __syncwarp();
        // full buckets (rare): insert those proposals straight into the list, locked
        for (unsigned long long om = (unsigned long long)ovf_lo | ((unsigned long long)ovf_hi << 32); om;
             om &= om - 1) {
            const int t = __ffsll((long long)om) - 1;
            const uint32_t p = (uint32_t)sid[t];
            const unsigned long long rest = fails[t];
            w_ovf += __popcll(rest);
            const float4 *rt = kRowsSmem ? rows + t * rs : X4 + (size_t)p * nv;
            uint64_t xs[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = (int)lane + 32 * h;
                xs[h] = kKeyEmpty;
                if ((rest >> j) & 1ull) {
                    const float4 *rj = kRowsSmem ? rows + j * rs : X4 + (size_t)sid[j] * nv;
                    xs[h] = make_key(l2sq_rows(rt, rj, nv), (uint32_t)sid[j], kFlagNew | kFlagIns);
                }
            }
            const int ins = warp_locked_insert(st, p, rest, xs[0], xs[1], li);
            if (ins < 0) ++w_to;
            else w_ins += ins;
        }
        __syncwarp();
    }
    // ---- counters (w_* are warp-uniform): warp -> block -> global
    const long long w_props = warp_sum(l_props);
    if (lane == 0) {
        atomic_add_ll(&bstat[kItProposals], w_props);
        atomic_add_ll(&bstat[kItEvals], w_evals);
        atomic_add_ll(&bstat[kItGathered], w_gathered);
        atomic_add_ll(&bstat[kItCandIds], w_candids);
        atomic_add_ll(&bstat[kItInserts], w_ins);
        atomic_add_ll(&bovf, w_ovf);
        atomic_add_ll(&btimeout, w_to);
        if (w_setovf) atomic_add_ll(&st.stats[kStatSetOverflow], w_setovf);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long *its = st.it_stats + (size_t)li * kItCount;
        its[kItRan] = 1;
        atomic_add_ll(&its[kItEvals], bstat[kItEvals]);
        atomic_add_ll(&its[kItGathered], bstat[kItGathered]);
        atomic_add_ll(&its[kItCandIds], bstat[kItCandIds]);
        atomic_add_ll(&its[kItInserts], bstat[kItInserts]);
        atomic_add_ll(&its[kItProposals], bstat[kItProposals]);
        atomic_add_ll(&st.stats[kStatEvals], bstat[kItEvals]);
        atomic_add_ll(&st.stats[kStatInserts], bstat[kItInserts]);
        atomic_add_ll(&st.stats[kStatGathered], bstat[kItGathered]);
        if (bovf) atomic_add_ll(&st.stats[kStatBucketOverflow], bovf);
        if (btimeout) atomic_add_ll(&st.stats[kStatLockTimeout], btimeout);
    }
}

// Merge of up to 32 candidate keys (one per lane, kKeyEmpty = none; none is
// listed and all order before the worst entry) into the list held one entry
// per lane: bitonic sort of the candidates, repeats dropped (a pair has one
// key, so a repeated id is a repeated key, adjacent after sorting), then every
// element goes to rank "own rank + elements of the other sequence before it"
// (two binary searches over lanes), scattered through shared memory.  The K
// smallest of list and candidates stay.  Returns the number of candidates
// that entered.
__device__ __forceinline__ int warp_sort_merge(uint64_t &Lk, uint64_t x, int K, uint64_t *scratch) {
    const unsigned lane = lane_id();
    x = warp_sort_u64(x);
    const uint64_t prev = __shfl_up_sync(kFull, x, 1);
    const bool valid = x != kKeyEmpty && (lane == 0 || key_order(prev) != key_order(x));
    const unsigned vm = __ballot_sync(kFull, valid);
    // list entry k: candidates ordered before it (lower bound over all 32 lanes,
    // then the dropped repeats below that bound removed)
    int lo = 0, hi = 32;
#pragma unroll
    for (int step = 0; step < 6; ++step) {
        const int mid = (lo + hi) >> 1;
        const uint64_t cm = __shfl_sync(kFull, x, mid & 31);
        if (lo < hi) {
            if (cm < Lk) lo = mid + 1;
            else hi = mid;
        }
    }
    const int rank_l = (int)lane + __popc(vm & ((lo >= 32) ? 0xFFFFFFFFu : ((1u << lo) - 1u)));
    // candidate: list entries ordered before it
    int a = 0, b = K;
#pragma unroll
    for (int step = 0; step < 6; ++step) {
        const int mid = (a + b) >> 1;
        const uint64_t lm = __shfl_sync(kFull, Lk, mid < K ? mid : K - 1);
        if (a < b) {
            if (lm < x) a = mid + 1;
            else b = mid;
        }
    }
    const int rank_c = __popc(vm & lanemask_lt()) + a;
    __syncwarp();
    if ((int)lane < K && rank_l < K) scratch[rank_l] = Lk;
    if (valid && rank_c < K) scratch[rank_c] = x;
    __syncwarp();
    if ((int)lane < K) Lk = scratch[lane];
    __syncwarp();
    return __popc(__ballot_sync(kFull, valid && rank_c < K));
}

// bf16 mode: the two orientations of a pair may round to different keys, so
// an id can come with several.  The list keeps, per id, the smallest key seen
// (whatever the arrival order): of repeats in one batch only the smallest
// stays, and a smaller key for a listed id replaces the listed entry.
// Returns true when x is to be inserted as a new id; replacements are done
// here (rare).
__device__ __forceinline__ bool bf16_resolve_ids(uint64_t &Lk, uint64_t &x, int K, int &ins) {
    const unsigned lane = lane_id();
    const bool real = x != kKeyEmpty;
    const uint32_t xi = key_id(x);
    // repeats within the batch with different keys (equal keys are one key:
    // the insertions skip a listed id, the sort-merge drops equal neighbours)
    const unsigned peers = __match_any_sync(kFull, real ? xi : 0xFFFFFFFFu);
    const unsigned same = __match_any_sync(kFull, (unsigned long long)x);
    if (__any_sync(kFull, real && peers != same)) {
        bool keep = true;
        for (int l = 0; l < 32; ++l) {
            const uint64_t y = __shfl_sync(kFull, x, l);
            if (real && y != kKeyEmpty && key_id(y) == xi && (y < x || (y == x && l < (int)lane))) keep = false;
        }
        if (!keep) x = kKeyEmpty;
    }
    // the id in the list
    uint64_t listed_key = kKeyEmpty;
    for (int k = 0; k < K; ++k) {
        const uint64_t lk = __shfl_sync(kFull, Lk, k);
        if (x != kKeyEmpty && key_id(lk) == xi) listed_key = lk;
    }
    // smaller keys of listed ids replace their entries, one at a time
    unsigned rep = __ballot_sync(kFull, x != kKeyEmpty && listed_key != kKeyEmpty && x < listed_key);
    for (; rep; rep &= rep - 1) {
        const int l = __ffs(rep) - 1;
        const uint64_t y = __shfl_sync(kFull, x, l);
        const unsigned at = __ballot_sync(kFull, (int)lane < K && key_id(Lk) == key_id(y));
        if (!at) continue;            // (cannot happen: ids in one batch are distinct)
        const int p = __ffs(at) - 1;  // the listed entry: drop it, close the gap
        const uint64_t below = __shfl_down_sync(kFull, Lk, 1);
        if ((int)lane >= p && (int)lane < K) Lk = (int)lane == K - 1 ? kKeyEmpty : below;
        ins += warp_insert(Lk, y, K);
    }
    return x != kKeyEmpty && listed_key == kKeyEmpty;
}

// One batch of up to 32 bucket keys (one per lane, kKeyEmpty = none) into
// the list held one entry per lane.  Keys that cannot enter are dropped in
// parallel: not before the worst, or already listed (a pair has one key, so
// "listed" is "the same (dist, id) at its lower bound", a binary search over
// the lanes; bf16 mode resolves ids as above).  Returns the number of
// insertions.
__device__ __forceinline__ int merge_batch(uint64_t &Lk, uint64_t x, int K, bool bf16, uint64_t *scratch) {
    int ins = 0;
    bool listed;
    if (bf16) {
        listed = !bf16_resolve_ids(Lk, x, K, ins);
    } else {
        // lower bound of (dist, id) among the entries: xo has its flag bits
        // clear and a (dist, id) is listed at most once, so comparing whole
        // keys with xo decides as comparing them without their flags
        const uint64_t xo = key_order(x);
        int lo = 0, hi = K - 1;
#pragma unroll
        for (int step = 0; step < 5; ++step) {
            const int mid = (lo + hi) >> 1;
            const uint64_t lm = __shfl_sync(kFull, Lk, mid);
            if (lo < hi) {
                if (lm < xo) lo = mid + 1;
                else hi = mid;
            }
        }
        listed = key_order(__shfl_sync(kFull, Lk, lo)) == xo;
    }
    unsigned cand = __ballot_sync(kFull, x < __shfl_sync(kFull, Lk, K - 1) && !listed);
    if (__popc(cand) >= kSortMergeMin) {
        ins += warp_sort_merge(Lk, ((cand >> lane_id()) & 1u) ? x : kKeyEmpty, K, scratch);
    } else {
        for (; cand; cand &= cand - 1) ins += warp_insert(Lk, __shfl_sync(kFull, x, __ffs(cand) - 1), K);
    }
    return ins;
}

// Merge of up to 32 candidate keys (one per lane, kKeyEmpty = none) into a
// list of K > 32 float32 keys held two per lane (WList): a key search over
// the K entries drops the listed ones (a pair has one key), then the others
// that order before the worst entry go in one at a time.
__device__ __forceinline__ int merge_batch_wide(WList &L, uint64_t x, int K) {
    const uint64_t xo = key_order(x);
    int lo = 0, hi = K - 1;
#pragma unroll
    for (int step = 0; step < 6; ++step) {
        const int mid = (lo + hi) >> 1;
        const uint64_t a = __shfl_sync(kFull, L.lo, mid & 31), b = __shfl_sync(kFull, L.hi, mid & 31);
        if (lo < hi) {
            if ((mid < 32 ? a : b) < xo) lo = mid + 1;  // as in merge_batch: flags need no mask
            else hi = mid;
        }
    }
    const uint64_t a = __shfl_sync(kFull, L.lo, lo & 31), b = __shfl_sync(kFull, L.hi, lo & 31);
    const bool listed = key_order(lo < 32 ? a : b) == xo;
    unsigned cand = __ballot_sync(kFull, x < wlist_at(L, K - 1) && !listed);
    int ins = 0;
    for (; cand; cand &= cand - 1) ins += wlist_insert(L, __shfl_sync(kFull, x, __ffs(cand) - 1), K);
    return ins;
}

// One warp per node with proposals: merge its bucket into its list (KW keys
// per lane).  The bucket's inline run (up to 256 keys) is loaded two batches
// ahead of the merges; pool runs (hub nodes) stream batch by batch.
template <int KW>
__global__ void __launch_bounds__(kMergeWarps * 32, 4) merge_kernel(DevState st, int li) {
    if (iteration_skipped(st, li)) return;
    __shared__ uint64_t scratch_all[kMergeWarps][KW == 1 ? kLaneK : 1];  // the sort-merge of one-key-per-lane lists
    uint64_t *scratch = scratch_all[threadIdx.x >> 5];
    __shared__ long long bstat[3];
    if (threadIdx.x < 3) bstat[threadIdx.x] = 0;
    __syncthreads();
    const unsigned lane = lane_id();
    const int K = st.K;
    const bool valid = (int)lane < K;
    long long w_ins = 0, w_changes = 0, w_merges = 0;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    int cur_ds = -1;          // batched: changes are added up per data set
    long long cur_changes = 0;
    for (long long p = gw; p < st.n; p += nw) {
        const int cnt_all = st.pcursor[p];
        if (cnt_all == 0) continue;
        __syncwarp();
        if (lane == 0) st.pcursor[p] = 0;
        const int cnt = min(cnt_all, kBucketMax);
        uint64_t *row = st.keys + (size_t)p * K;
        int *chunks = st.pchunk + (size_t)p * kBucketChunks;
        uint64_t Lk = kKeyEmpty;
        WList L{kKeyEmpty, kKeyEmpty};
        if constexpr (KW == 1) Lk = valid ? row[lane] : kKeyEmpty;
        else L = wlist_load(row, K);
        // entries already inserted in this iteration (an earlier pass's merge
        // or a locked insertion, which counted them)
        const int ch0 = KW == 1 ? __popc(__ballot_sync(kFull, valid && (Lk & kFlagIns))) : wlist_count(L, K, kFlagIns);
        int ins = 0;
        const bool bf16 = st.bf16 != 0;
        auto merge = [&](uint64_t x) {
            if constexpr (KW == 1) return merge_batch(Lk, x, K, bf16, scratch);
            else return merge_batch_wide(L, x, K);
        };
        // the inline run, its loads two batches ahead of the merges
        const uint64_t *run = st.pbucket + ((size_t)p << kBucketRunBits);
        const int c_in = min(cnt, kBucketRun);
        uint64_t x0 = (int)lane < c_in ? __ldcs(run + lane) : kKeyEmpty;
        uint64_t x1 = 32 + (int)lane < c_in ? __ldcs(run + 32 + lane) : kKeyEmpty;
        for (int c0 = 0; c0 < c_in; c0 += 32) {
            const uint64_t x = x0;
            x0 = x1;
            x1 = c0 + 64 + (int)lane < c_in ? __ldcs(run + c0 + 64 + lane) : kKeyEmpty;
            ins += merge(x);
        }
        // pool runs (runs are multiples of 32 keys: a batch never straddles two)
        for (int c0 = kBucketRun; c0 < cnt; c0 += 32) {
            const int k = c0 >> kBucketRunBits;
            if ((c0 & (kBucketRun - 1)) == 0) {
                const int ch = chunks[k - 1];
                __syncwarp();
                if (lane == 0) chunks[k - 1] = 0;
                // no chunk (or poisoned): these proposals went the locked way
                run = ch > 0 ? st.ppool + ((size_t)(ch - 1) << kBucketRunBits) : nullptr;
            }
            if (!run) continue;
            const int off = c0 & (kBucketRun - 1);
            const uint64_t x = c0 + (int)lane < cnt ? __ldcs(run + off + lane) : kKeyEmpty;
            ins += merge(x);
        }
        // entries flagged "inserted in this iteration" that are still listed
        // (the sampling pass cleared that flag everywhere before the join),
        // less those already counted
        const int ch =
            (KW == 1 ? __popc(__ballot_sync(kFull, valid && (Lk & kFlagIns))) : wlist_count(L, K, kFlagIns)) - ch0;
        w_changes += ch;
        if (st.ds) {
            const int b = st.ds[p];
            if (b != cur_ds) {
                if (cur_ds >= 0 && cur_changes && lane == 0)
                    atomic_add_ll(st.ds_changes + (size_t)cur_ds * kMaxLocalIters + li, cur_changes);
                cur_ds = b;
                cur_changes = 0;
            }
            cur_changes += ch;
        }
        if constexpr (KW == 1) {
            if (ins && valid) row[lane] = Lk;
        } else {
            if (ins) wlist_store(L, row, K);
        }
        w_ins += ins;
        ++w_merges;
    }
    if (cur_ds >= 0 && cur_changes && lane == 0)
        atomic_add_ll(st.ds_changes + (size_t)cur_ds * kMaxLocalIters + li, cur_changes);
    if (lane == 0) {
        atomic_add_ll(&bstat[0], w_ins);
        atomic_add_ll(&bstat[1], w_changes);
        atomic_add_ll(&bstat[2], w_merges);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long *its = st.it_stats + (size_t)li * kItCount;
        atomic_add_ll(&its[kItInserts], bstat[0]);
        atomic_add_ll(&its[kItChanges], bstat[1]);
        atomic_add_ll(&its[kItMerges], bstat[2]);
        atomic_add_ll(&st.stats[kStatInserts], bstat[0]);
        atomic_add_ll(&st.stats[kStatMerges], bstat[2]);
    }
}

namespace {
template <bool S>
cudaError_t launch_join_t(const DevState &st, int li, cudaStream_t s) {
    const JoinLayout lay = join_layout(st.cap, st.nv, S);
    const size_t dyn = lay.per_warp * kJoinWarps;
    auto kern = join_kernel<S>;
    cudaError_t e = smem_opt_in((const void *)kern, dyn);
    if (e != cudaSuccess) return e;
    const int grid = grid_for((const void *)kern, kJoinWarps * 32, dyn);
    kern<<<grid, kJoinWarps * 32, dyn, s>>>(st, li);
    return cudaGetLastError();
}
}  // namespace

int choose_join_path(int bf16, int nv, int dpb, int K, int force) {
    // FP8 rows (kind 2) have only the ring kernel (the caller checks the fit)
    if (bf16 == 2) return kJoinRing;
    const bool ring = ring_join_fits(bf16, nv, dpb, K);
    const bool pipe = pipe_join_fits(bf16, nv);
    if (force == kJoinWarp && !bf16) return kJoinWarp;
    if (force == kJoinTile) return kJoinTile;
    if (force == kJoinRing && ring) return kJoinRing;
    if ((force == kJoinPipe || force == kJoinPipe8) && pipe) return force;
    if (!bf16 && nv <= kWarpMaxNv) return kJoinWarp;
    if (pipe) return kJoinPipe;
    return ring && ring_join_preferred(bf16, nv, dpb) ? kJoinRing : kJoinTile;
}

int join_launches(int path) { return path == kJoinRing || path == kJoinPipe || path == kJoinPipe8 ? 2 : 1; }

cudaError_t launch_join(const DevState &st, int li, cudaStream_t s) {
    if (st.join_path == kJoinRing) return launch_ring_join(st, li, s);
    if (st.join_path == kJoinPipe || st.join_path == kJoinPipe8) return launch_pipe_join(st, li, s);
    // high dimensions: block-per-node tiles (bf16 tensor cores when asked)
    if (st.join_path == kJoinTile) return launch_tile_join(st, li, st.bf16 != 0, s);
    const JoinLayout lay = join_layout(st.cap, st.nv, true);
    if (lay.per_warp * kJoinWarps <= 110 * 1024) return launch_join_t<true>(st, li, s);
    return launch_join_t<false>(st, li, s);
}

cudaError_t launch_merge(const DevState &st, int li, cudaStream_t s) {
    if (st.K > kLaneK) {
        const int grid = grid_for((const void *)merge_kernel<2>, kMergeWarps * 32, 0);
        merge_kernel<2><<<grid, kMergeWarps * 32, 0, s>>>(st, li);
        return cudaGetLastError();
    }
    const int grid = grid_for((const void *)merge_kernel<1>, kMergeWarps * 32, 0);
    merge_kernel<1><<<grid, kMergeWarps * 32, 0, s>>>(st, li);
    return cudaGetLastError();
}

}  // namespace knng
