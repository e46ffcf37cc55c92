// join.cu -- the local join (the paper's Calculation step, Section 2 and
// Section 3.3) with the list updates, float32 difference-form distances.
//
// One warp owns one node u at a time (persistent grid-stride loop):
//   1. read u's sampled candidates (forward part written by u's sampling warp,
//      reverse part filled by other warps), drop repeats keeping the first
//      occurrence (new before old), cap the set S at 64;
//   2. gather the candidate rows into shared memory (padded row stride so
//      lanes reading different rows hit different banks) and snapshot each
//      candidate's current worst key;
//   3. lane i takes target S_i and walks every partner S_j that forms a join
//      pair with it (both new, or one new and one old); partner rows are read
//      by all lanes at once (shared-memory broadcast).  A pair whose key
//      (dist, S_j) beats the snapshot worst of S_i sets bit j of a mask;
//   4. lanes with a non-empty mask lock S_i's list (bounded wait), load it
//      into registers, insert the masked partners in order (insertion only if
//      the key beats the current worst and the id is not listed), write the
//      list back and unlock.
// Each unordered pair is evaluated from both ends, so no pairwise matrix is
// stored and no lane writes another lane's target.  Since every float32
// distance in the library uses the same arithmetic, a pair always yields the
// same key and the final lists do not depend on the order in which warps take
// the locks: each list ends as the K smallest distinct keys of its start
// entries and all proposals it received.
#include "internal.h"

namespace knng {

namespace {
constexpr int kSetMax = 64;
constexpr int kJoinWarps = 4;
constexpr unsigned kFull = 0xFFFFFFFFu;

struct JoinLayout {
    int raw_max;     // ints for raw candidate ids
    int row_stride;  // float4 per staged row
    size_t per_warp; // bytes
};

__host__ __device__ inline JoinLayout join_layout(int cap, int nv, bool rows_smem) {
    JoinLayout L;
    L.raw_max = ((2 * cap + 31) / 32) * 32;
    L.row_stride = (nv % 2 == 0) ? nv + 1 : nv;
    size_t b = (size_t)L.raw_max * 4 + kSetMax * 4 + kSetMax * 8;
    b = (b + 15) & ~(size_t)15;
    if (rows_smem) b += (size_t)kSetMax * L.row_stride * 16;
    L.per_warp = b;
    return L;
}

}  // namespace

template <int KMAX, bool kRowsSmem>
__global__ void __launch_bounds__(kJoinWarps * 32) join_kernel(DevState st, int li) {
    if (iteration_skipped(st, li)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long bstat[kItCount];
    __shared__ long long btimeout;
    if (threadIdx.x < kItCount) bstat[threadIdx.x] = 0;
    if (threadIdx.x == 0) btimeout = 0;
    __syncthreads();

    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int K = st.K, R = st.R, cap = st.cap, nv = st.nv;
    const JoinLayout lay = join_layout(cap, nv, kRowsSmem);
    unsigned char *wbase = smem + (size_t)warp * lay.per_warp;
    int *raw = reinterpret_cast<int *>(wbase);
    int *sid = raw + lay.raw_max;
    uint64_t *swk = reinterpret_cast<uint64_t *>(sid + kSetMax);
    float4 *rows = reinterpret_cast<float4 *>(wbase + (((size_t)lay.raw_max * 4 + kSetMax * 12 + 15) & ~(size_t)15));
    const int rs = lay.row_stride;
    const float4 *X4 = reinterpret_cast<const float4 *>(st.X);

    long long w_evals = 0, w_gathered = 0, w_candids = 0, w_setovf = 0;
    long long l_ins = 0, l_evins = 0, l_merges = 0, l_timeouts = 0;

    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = gw; u < st.n; u += nw) {
        // ---- 1. candidates of u, repeats removed (new first, then old)
        const size_t cb = (size_t)u * cap;
        const int fn = st.fwd_new[u], fo = st.fwd_old[u];
        const int rn = min(st.fill_new[u], R), ro = min(st.fill_old[u], R);
        __syncwarp();
        if (lane == 0) {  // reverse degrees of the next iteration start from zero
            st.rev_new[u] = 0;
            st.rev_old[u] = 0;
        }
        const int nnew_raw = fn + rn;
        const int total = nnew_raw + fo + ro;
        for (int idx = lane; idx < total; idx += 32) {
            int v;
            if (idx < fn) v = st.cand_new[cb + idx];
            else if (idx < nnew_raw) v = st.cand_new[cb + K + (idx - fn)];
            else if (idx < nnew_raw + fo) v = st.cand_old[cb + (idx - nnew_raw)];
            else v = st.cand_old[cb + K + (idx - nnew_raw - fo)];
            raw[idx] = v;
        }
        __syncwarp();
        int ns = 0, m = 0;
        for (int base = 0; base < total; base += 32) {
            const int idx = base + lane;
            bool keep = false;
            int v = -1;
            if (idx < total) {
                v = raw[idx];
                keep = true;
                for (int k = 0; k < idx; ++k)
                    if (raw[k] == v) {
                        keep = false;
                        break;
                    }
            }
            const unsigned km = __ballot_sync(kFull, keep);
            const int pos = ns + __popc(km & lanemask_lt());
            if (keep && pos < kSetMax) sid[pos] = v;
            m += __popc(__ballot_sync(kFull, keep && idx < nnew_raw));
            ns += __popc(km);
        }
        if (ns > kSetMax) {
            w_setovf += ns - kSetMax;
            ns = kSetMax;
        }
        m = min(m, ns);
        __syncwarp();
        // ---- 2. snapshot worst keys, stage rows
        for (int i = lane; i < ns; i += 32) swk[i] = __ldcg(st.keys + (size_t)sid[i] * K + (K - 1));
        if (kRowsSmem) {
            for (int idx = lane; idx < ns * nv; idx += 32) {
                const int r = idx / nv, c = idx - r * nv;
                rows[r * rs + c] = __ldg(X4 + (size_t)sid[r] * nv + c);
            }
        }
        __syncwarp();
        w_evals += (long long)m * (m - 1) / 2 + (long long)m * (ns - m);
        w_gathered += ns;
        w_candids += total;
        // ---- 3./4. lane = target
        for (int base = 0; base < ns; base += 32) {
            const int i = base + lane;
            const bool act = i < ns;
            const int jend = act ? (i < m ? ns : m) : 0;
            const int jmax = __reduce_max_sync(kFull, jend);
            const float4 *own = kRowsSmem ? rows + (act ? i : 0) * rs : X4 + (size_t)sid[act ? i : 0] * nv;
            const uint64_t wk = act ? swk[i] : 0ull;
            uint64_t mask = 0;
            for (int j = 0; j < jmax; ++j) {
                const float4 *pr = kRowsSmem ? rows + j * rs : X4 + (size_t)sid[j] * nv;
                const uint32_t vj = (uint32_t)sid[j];
                if (j < jend && j != i) {
                    const float dd = l2sq_rows(own, pr, nv);
                    if (make_key(dd, vj, kFlagNew | kFlagIns) < wk) mask |= 1ull << j;
                }
            }
            if (mask) {
                const uint32_t p = (uint32_t)sid[i];
                int *lk = st.locks + p;
                if (lock_acquire(lk)) {
                    // right-aligned register list: slots [KMAX-K, KMAX) hold the
                    // list, slots below it hold 0, which orders before every
                    // proposal (proposal keys carry flag bits, so they are > 0);
                    // the worst entry is always L[KMAX-1].
                    const int off = KMAX - K;
                    uint64_t *row = st.keys + (size_t)p * K - off;
                    uint64_t L[KMAX];
#pragma unroll
                    for (int k = 0; k < KMAX; ++k) L[k] = k >= off ? __ldcg(row + k) : 0ull;
                    bool changed = false;
                    while (mask) {
                        const int j = __ffsll((long long)mask) - 1;
                        mask &= mask - 1;
                        const uint32_t vj = (uint32_t)sid[j];
                        const float4 *pr = kRowsSmem ? rows + j * rs : X4 + (size_t)vj * nv;
                        const uint64_t x = make_key(l2sq_rows(own, pr, nv), vj, kFlagNew | kFlagIns);
                        if (x >= L[KMAX - 1]) continue;
                        bool dup = false;
#pragma unroll
                        for (int k = 0; k < KMAX; ++k) dup |= (k >= off) && key_id(L[k]) == vj;
                        if (dup) continue;
                        if (L[KMAX - 1] & kFlagIns) ++l_evins;
                        ++l_ins;
#pragma unroll
                        for (int k = KMAX - 1; k >= 1; --k) {
                            const uint64_t lo = L[k] < x ? L[k] : x;
                            L[k] = lo > L[k - 1] ? lo : L[k - 1];
                        }
                        L[0] = L[0] < x ? L[0] : x;
                        changed = true;
                    }
                    if (changed) {
#pragma unroll
                        for (int k = 0; k < KMAX; ++k)
                            if (k >= off) __stcg(row + k, L[k]);
                    }
                    lock_release(lk);
                    ++l_merges;
                } else {
                    ++l_timeouts;
                }
            }
        }
        __syncwarp();
    }
    // ---- counters: warp -> block -> global
    l_ins = warp_sum(l_ins);
    l_evins = warp_sum(l_evins);
    l_merges = warp_sum(l_merges);
    l_timeouts = warp_sum(l_timeouts);
    if (lane == 0) {
        atomic_add_ll(&bstat[kItEvals], w_evals);
        atomic_add_ll(&bstat[kItGathered], w_gathered);
        atomic_add_ll(&bstat[kItCandIds], w_candids);
        atomic_add_ll(&bstat[kItMerges], l_merges);
        atomic_add_ll(&bstat[kItInserts], l_ins);
        atomic_add_ll(&bstat[kItChanges], l_ins - l_evins);
        atomic_add_ll(&btimeout, l_timeouts);
        if (w_setovf) atomic_add_ll(&st.stats[kStatSetOverflow], w_setovf);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long *its = st.it_stats + (size_t)li * kItCount;
        its[kItRan] = 1;
        atomic_add_ll(&its[kItChanges], bstat[kItChanges]);
        atomic_add_ll(&its[kItEvals], bstat[kItEvals]);
        atomic_add_ll(&its[kItGathered], bstat[kItGathered]);
        atomic_add_ll(&its[kItCandIds], bstat[kItCandIds]);
        atomic_add_ll(&its[kItMerges], bstat[kItMerges]);
        atomic_add_ll(&its[kItInserts], bstat[kItInserts]);
        atomic_add_ll(&st.stats[kStatEvals], bstat[kItEvals]);
        atomic_add_ll(&st.stats[kStatInserts], bstat[kItInserts]);
        atomic_add_ll(&st.stats[kStatMerges], bstat[kItMerges]);
        atomic_add_ll(&st.stats[kStatGathered], bstat[kItGathered]);
        if (btimeout) atomic_add_ll(&st.stats[kStatLockTimeout], btimeout);
    }
}

namespace {
template <int KMAX, bool S>
cudaError_t launch_join_t(const DevState &st, int li, cudaStream_t s) {
    const JoinLayout lay = join_layout(st.cap, st.nv, S);
    const size_t dyn = lay.per_warp * kJoinWarps;
    auto kern = join_kernel<KMAX, S>;
    static bool opted_in = false;  // allow up to the per-block maximum once
    if (!opted_in) {
        int dev = 0, mx = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaError_t e = cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             mx - 1024);
        if (e != cudaSuccess) return e;
        opted_in = true;
    }
    const int grid = grid_for((const void *)kern, kJoinWarps * 32, dyn);
    kern<<<grid, kJoinWarps * 32, dyn, s>>>(st, li);
    return cudaGetLastError();
}

template <int KMAX>
cudaError_t launch_join_k(const DevState &st, int li, cudaStream_t s) {
    const JoinLayout lay = join_layout(st.cap, st.nv, true);
    if (lay.per_warp * kJoinWarps <= 110 * 1024) return launch_join_t<KMAX, true>(st, li, s);
    return launch_join_t<KMAX, false>(st, li, s);
}
}  // namespace

cudaError_t launch_join(const DevState &st, int li, cudaStream_t s) {
    if (st.K <= 8) return launch_join_k<8>(st, li, s);
    if (st.K <= 16) return launch_join_k<16>(st, li, s);
    if (st.K <= 24) return launch_join_k<24>(st, li, s);
    return launch_join_k<32>(st, li, s);
}

}  // namespace knng
