// join_common.cuh -- pieces shared by the two local-join kernels (the
// warp-per-node kernel for low dimensions and the block-per-node tile kernel
// for high dimensions) and the list-merge kernel.
#pragma once

#include "internal.h"

namespace knng {

constexpr int kSetMax = 64;      // candidates per node and iteration after repeats are removed

// position of the r-th (from 0) set bit of x; r < popcount(x)
__device__ __forceinline__ int nth_set_bit64(unsigned long long x, int r) {
    const unsigned lo = (unsigned)x;
    const int pl = __popc(lo);
    unsigned w = r < pl ? lo : (unsigned)(x >> 32);
    int rr = r < pl ? r : r - pl, pos = r < pl ? 0 : 32;
#pragma unroll
    for (int sh = 16; sh >= 1; sh >>= 1) {
        const int c = __popc(w & ((1u << sh) - 1u));
        if (rr >= c) {
            rr -= c;
            w >>= sh;
            pos += sh;
        }
    }
    return pos;
}
// Hash set for repeat removal: 256 slots while a node's raw ids (at most
// 2 cap, cap = K + 2s + 8) fit it, 512 for the larger capacities of K > 32
// (at most 2 (64 + 136) = 400 ids).
constexpr int kHashBits = 8;
constexpr int kHashBitsMax = 9;
__host__ __device__ __forceinline__ int hash_bits(int cap) { return 2 * cap <= (1 << kHashBits) ? kHashBits : kHashBitsMax; }
constexpr int kLockSpins = 1 << 20;
constexpr unsigned kFull = 0xFFFFFFFFu;

// q / divisor for q < 2^12 and 2 <= divisor <= 64 given magic = ceil(2^32 /
// divisor): exact, the rounding error stays below 2^-20.  Divisor 1 (magic
// would need 33 bits) is passed through.
__device__ __forceinline__ uint32_t div_small(uint32_t q, uint32_t divisor, uint32_t magic) {
    return divisor == 1u ? q : __umulhi(q, magic);
}
__device__ __forceinline__ uint32_t div_magic(uint32_t divisor) {
    return divisor > 1u ? (uint32_t)((0x100000000ull + divisor - 1) / divisor) : 0u;
}

// Insert x into the list held one entry per lane (Lk, lane k = entry k of K,
// ascending): only if it orders before the worst entry and its id is not
// listed.  Warp-uniform result: true if inserted.
__device__ __forceinline__ bool warp_insert(uint64_t &Lk, uint64_t x, int K) {
    const unsigned lane = lane_id();
    const bool valid = (int)lane < K;
    const uint64_t worst = __shfl_sync(kFull, Lk, K - 1);
    if (x >= worst) return false;
    if (__ballot_sync(kFull, valid && key_id(Lk) == key_id(x))) return false;
    const unsigned gt = __ballot_sync(kFull, valid && Lk > x);
    const int pos = __ffs(gt) - 1;  // first entry ordered after x
    const uint64_t up = __shfl_up_sync(kFull, Lk, 1);
    if (valid && (int)lane >= pos) Lk = (int)lane == pos ? x : up;
    return true;
}

// Reverse part raw[b, b + cnt) (cnt <= 32 H; reverse capacities are at most
// 2 * 32 + 8 = 72 for K <= 32 and 2 * 64 + 8 = 136 above) put in a fixed
// order: ascending by (id - base) * 0x9E3779B1 mod 2^32, a bijection of the
// ids local to the data set (base: its first node),
// so the order is canonical, the same in a batched build, and not tied to id
// size.  The ids of one reverse part are distinct (a node lists an id once).
template <int H>
__device__ __forceinline__ void warp_order_part(int *raw, int b, int cnt, uint32_t base) {
    const unsigned lane = lane_id();
    int v[H], r[H];
    uint32_t k[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int i = (int)lane + 32 * h;
        v[h] = i < cnt ? raw[b + i] : 0;
        k[h] = ((uint32_t)v[h] - base) * 0x9E3779B1u;
        r[h] = 0;
    }
    for (int j = 0; j < cnt; ++j) {
        const uint32_t kj = ((uint32_t)raw[b + j] - base) * 0x9E3779B1u;
#pragma unroll
        for (int h = 0; h < H; ++h) r[h] += kj < k[h];
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < H; ++h)
        if ((int)lane + 32 * h < cnt) raw[b + r[h]] = v[h];
    __syncwarp();
}

// Node u's sampled candidates (one warp): the forward part written by u's
// sampling warp and the reverse part filled by other warps, repeats removed
// with a shared-memory hash set (new entries first, so an id that is both new
// and old stays new; of repeats the first in read order stays).  Writes
// sid[0 .. ns), new ones first (m of them), capped at kSetMax.  When the ids
// read exceed the cap, each reverse part is first put in the fixed order of
// warp_order_part: the forward parts are in list order already, so which ids
// the cap drops does not depend on the order in which other warps took the
// reverse slots, and the build stays deterministic.  raw must hold 2 * cap
// ints and hset 2^hash_bits(cap) ints.  Lane 0 also restarts u's reverse degrees
// for the next iteration.  Returns total raw ids read; ns = 0 when u has no
// new candidate (no join pair).  Results are warp-uniform.
// kWide: 0 = the form for reverse capacities up to 96 with a 256-slot hash
// set, 1 = the form for the larger ones of K > 32, -1 = either, chosen at run
// time (kernels that keep one instance for both).
template <int kWide = -1>
__device__ __forceinline__ int warp_gather_candidates(const DevState &st, long long u, int *raw, int *hset, int *sid,
                                                      int &ns_out, int &m_out, long long &setovf) {
    const unsigned lane = lane_id();
    const int K = st.K, R = st.R;
    const size_t cb = (size_t)u * st.cap;
    const int fn = st.fwd_new[u], fo = st.fwd_old[u];
    const int rn = min(st.fill_new[u], R), ro = min(st.fill_old[u], R);
    __syncwarp();
    if (lane == 0) {
        st.rev_new[u] = 0;
        st.rev_old[u] = 0;
    }
    const int nnew_raw = fn + rn;
    const int total = nnew_raw + fo + ro;
    ns_out = 0;
    m_out = 0;
    if (nnew_raw == 0) return total;
    for (int idx = lane; idx < total; idx += 32) {
        int v;
        if (idx < fn) v = st.cand_new[cb + idx];
        else if (idx < nnew_raw) v = st.cand_new[cb + K + (idx - fn)];
        else if (idx < nnew_raw + fo) v = st.cand_old[cb + (idx - nnew_raw)];
        else v = st.cand_old[cb + K + (idx - nnew_raw - fo)];
        raw[idx] = v;
    }
    const bool wide = kWide < 0 ? (R > 96 || hash_bits(st.cap) > kHashBits) : kWide == 1;
    const int hb = wide ? hash_bits(st.cap) : kHashBits;
    for (int i = lane; i < (1 << hb); i += 32) hset[i] = -1;
    __syncwarp();
    if (total > kSetMax) {
        const uint32_t base = (uint32_t)(u - node_local(st, u));
        if (!wide) {
            warp_order_part<3>(raw, fn, rn, base);
            warp_order_part<3>(raw, nnew_raw + fo, ro, base);
        } else {
            warp_order_part<5>(raw, fn, rn, base);
            warp_order_part<5>(raw, nnew_raw + fo, ro, base);
        }
    }
    int ns = 0, m = 0;
    for (int pass = 0; pass < 2; ++pass) {
        const int lo_i = pass ? nnew_raw : 0, hi_i = pass ? total : nnew_raw;
        for (int b0 = lo_i; b0 < hi_i; b0 += 32) {
            const int idx = b0 + lane;
            bool keep = false;
            const int v = idx < hi_i ? raw[idx] : -1;
            // of repeats within the batch only the lowest lane competes
            const unsigned grp = __match_any_sync(kFull, v);
            if (idx < hi_i && (grp & lanemask_lt()) == 0) {
                unsigned h = ((unsigned)v * 0x9E3779B1u) >> (32 - hb);
                for (int probe = 0; probe < (1 << hb); ++probe) {
                    const int prev = atomicCAS(hset + h, -1, v);
                    if (prev == -1) {
                        keep = true;
                        break;
                    }
                    if (prev == v) break;
                    h = (h + 1) & ((1u << hb) - 1);
                }
            }
            const unsigned km = __ballot_sync(kFull, keep);
            const int pos = ns + __popc(km & lanemask_lt());
            if (keep && pos < kSetMax) sid[pos] = v;
            if (!pass) m += __popc(km);
            ns += __popc(km);
        }
        __syncwarp();
    }
    if (ns > kSetMax) {
        setovf += ns - kSetMax;
        ns = kSetMax;
    }
    ns_out = ns;
    m_out = min(m, ns);
    return total;
}

// Locked insertion (one warp) of proposals into node p's list, used when a
// proposal bucket is full.  Lane j holds the key of partner j in x0 and of
// partner 32 + j in x1; `rest` selects the partners.  The lock wait is
// bounded; returns -1 when it gave up, else the number of insertions.  The
// list's entries inserted in this iteration (flag kFlagIns) before and after
// are counted, and the difference is added to iteration li's change count
// (and to its data set's in batched mode): list merges add theirs the same
// way, so the count is exact however the updates of a list interleave.
__device__ __forceinline__ int warp_locked_insert(const DevState &st, uint32_t p, unsigned long long rest,
                                                  uint64_t x0, uint64_t x1, int li) {
    const unsigned lane = lane_id();
    const int K = st.K;
    bool got = false;
    if (lane == 0) {
        for (int spin = 0; spin < kLockSpins; ++spin) {
            if (atomicCAS(st.locks + p, 0, 1) == 0) {
                got = true;
                break;
            }
            __nanosleep(spin < 64 ? 64 : 512);
        }
        if (got) __threadfence();
    }
    got = __shfl_sync(kFull, got, 0);
    if (!got) return -1;
    uint64_t *row = st.keys + (size_t)p * K;
    WList L = wlist_load(row, K);
    const int before = wlist_count(L, K, kFlagIns);
    int ins = 0;
    for (unsigned long long mm = rest; mm; mm &= mm - 1) {
        const int j = __ffsll((long long)mm) - 1;
        const uint64_t xa = __shfl_sync(kFull, x0, j & 31), xb = __shfl_sync(kFull, x1, j & 31);
        ins += wlist_insert(L, j < 32 ? xa : xb, K);
    }
    const int after = wlist_count(L, K, kFlagIns);
    if (lane == 0 && after != before) {
        atomic_add_ll(st.it_stats + (size_t)li * kItCount + kItChanges, after - before);
        if (st.ds) atomic_add_ll(st.ds_changes + (size_t)st.ds[p] * kMaxLocalIters + li, after - before);
    }
    wlist_store(L, row, K);
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicExch(st.locks + p, 0);
    return ins;
}

}  // namespace knng
