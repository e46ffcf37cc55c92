// pipe_join.cu -- the local join (the paper's Calculation step, Section 2;
// blocked mutual distances of a bounded neighbourhood, Section 3.3) for
// float32 rows of 33 to 256 floats, as a software pipeline over nodes in
// which all warps of a block work on one node at a time.
//
// The set kernel (ring_join.cu) has written each node's candidate set
// (repeats removed, new first, at most 64) to cset / cmeta.  Each block of
// pipe_join_kernel (persistent; up to four per SM) walks the nodes
// u = blockIdx.x, blockIdx.x + gridDim.x, ...:
//   producer warp: for every node with a join pair it takes a free row slot
//     (one per block: the other blocks of the SM cover the wait), writes the ids into it and issues asynchronous copies
//     of the candidate rows (one 16-byte cp.async per lane, a whole 512-byte
//     row per warp instruction, rows on an odd number of 16-byte units so
//     that consecutive rows start on different banks) and of each
//     candidate's worst-key snapshot; the copies arrive on the slot's
//     mbarrier, so the next node's rows land while the current one's
//     proposals go out;
//   compute warps (four, together on the current node):
//     1. the distances the node's joins need, each pair once (new x new in
//        2 x 2 register blocks over the upper triangle, new x old in 2 x 4
//        blocks), or for small nodes the whole block of new rows against all
//        rows in 1 x 4 items (more items to spread), whichever ends sooner on
//        the slowest thread; canonical float32 difference form (bit-identical
//        to every other float32 distance of the library) into D[i][j] for new
//        i and every j; then the row slot is released to the producer;
//     2. proposals, one warp per target: a new target takes partner j when
//        key(D[t][j], j) orders before its snapshot worst entry, an old target
//        takes new partner i when key(D[i][t], i) does -- every proposal of the
//        node's join pairs once -- two ballots giving the target's mask;
//     3. bucket runs: the lanes of a warp reserve its targets' ranges at once
//        (one atomicAdd each) and claim the pool chunks they span, then write
//        the warp's proposals flattened over its lanes (target by a search
//        over the lanes' prefix counts, partner as the r-th set bit of its
//        mask); a proposal whose run has no slot (bucket or pool spent) is
//        inserted into the list under the list's lock.
// Two block barriers per node: after the distance block, and at its end.
// The proposals are those of the other join kernels, so the lists after the
// merge are the same bit for bit.  Every wait is bounded by the global timer;
// a wait that gives up raises the timeout counter and the block winds down
// once the copies it issued have landed (again a bounded wait).
#include <cstdint>

#include "join_common.cuh"

namespace knng {

namespace {
// Block shapes (compute warps W, row slots S): four warps with one slot (four
// blocks per SM, the default) or eight warps with two slots (two per SM).
constexpr int kPipeMaxSlots = 2;
template <int W, int S>
struct PipeShape {
    static constexpr int kThreads = 32 * (W + 1);
    static constexpr int kMinBlocks = W == 8 ? 2 : 4;
};
constexpr int kPipeMaxUnits = 64;                   // 16-byte units per row: rows of up to 256 floats
constexpr uint32_t kPipeHdrBytes = 1024;            // slot header: ns, m | ids[64] | worst keys[64]
constexpr int kPipeDStride = kSetMax + 1;
constexpr unsigned long long kPipeWaitNs = 2000000000ull;  // 2 s

// Row layout in a slot: column block cb (32 units = 128 floats) holds every
// row's units [32 cb, 32 cb + 32) on a stride of (units | 1) 16-byte units.
struct PipeGeo {
    int nv;                 // 16-byte units per row
    int nblk;               // column blocks
    uint32_t stride[2];     // bytes per row in each block
    uint32_t off[2];        // byte offset of each block in the slot's row area
    uint32_t rows_bytes;    // the row area
    uint32_t slot_bytes;    // header + row area
};
__host__ __device__ __forceinline__ PipeGeo pipe_geo(int nv) {
    PipeGeo g;
    g.nv = nv;
    g.nblk = (nv + 31) / 32;
    uint32_t off = 0;
    for (int cb = 0; cb < 2; ++cb) {
        const int units = cb < g.nblk ? (nv - 32 * cb < 32 ? nv - 32 * cb : 32) : 0;
        g.stride[cb] = (uint32_t)(units | 1) * 16u;
        g.off[cb] = off;
        if (cb < g.nblk) off += (uint32_t)kSetMax * g.stride[cb];
    }
    g.rows_bytes = off;
    g.slot_bytes = kPipeHdrBytes + ((off + 127u) & ~127u);
    return g;
}

// Per-node scratch of the compute warps.
struct PipeCur {
    int sid[kSetMax];
    uint64_t swk[kSetMax];
    unsigned long long fails[kSetMax];  // per target: proposals that found no bucket slot
    float D[kSetMax * kPipeDStride];
};

struct PipeShared {
    uint64_t full[kPipeMaxSlots];
    uint64_t empty[kPipeMaxSlots];
    int abort_flag;
    long long stat[8];
};

__host__ __device__ __forceinline__ size_t pipe_smem_bytes(int nv, int slots) {
    const PipeGeo g = pipe_geo(nv);
    return 128 + (size_t)slots * g.slot_bytes + ((sizeof(PipeCur) + 127) & ~(size_t)127);
}

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t *b) {
    asm volatile("{\n\t.reg .b64 s;\n\tmbarrier.arrive.shared::cta.b64 s, [%0];\n\t}" ::"r"(su32(b)) : "memory");
}
// arrives on the barrier once all of this thread's earlier cp.async copies
// have landed (counted in the barrier's expected arrivals)
__device__ __forceinline__ void bar_arrive_copies(uint64_t *b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase of the given parity; false when it gave up or
// the block is aborting
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t parity, volatile int *abort_flag) {
    const unsigned long long t0 = gtimer();
    while (!bar_try(b, parity)) {
        if (*abort_flag) return false;
        if (gtimer() - t0 > kPipeWaitNs) return false;
    }
    return true;
}
__device__ __forceinline__ void cpa16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
// named barrier of the compute warps only
template <int NT>
__device__ __forceinline__ void compute_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); }

// Canonical distances of the given rows (RB) against the given columns (CB)
// of a slot, accumulated over every 16-byte unit in ascending order.
template <int RB, int CB>
__device__ __forceinline__ void pipe_block(const unsigned char *rows, const PipeGeo &g, const int (&ri)[RB],
                                           const int (&cj)[CB], Acc2 (&acc)[RB][CB]) {
    for (int cb = 0; cb < g.nblk; ++cb) {
        const unsigned char *base = rows + g.off[cb];
        const uint32_t st = g.stride[cb];
        const int units = g.nv - 32 * cb < 32 ? g.nv - 32 * cb : 32;
        const float4 *pr[RB], *pc[CB];
#pragma unroll
        for (int r = 0; r < RB; ++r) pr[r] = reinterpret_cast<const float4 *>(base + (uint32_t)ri[r] * st);
#pragma unroll
        for (int q = 0; q < CB; ++q) pc[q] = reinterpret_cast<const float4 *>(base + (uint32_t)cj[q] * st);
        // unrolled by eight (measured on the 1M x 128 build: 150.1 -> 149.0 ms;
        // by four no change, by sixteen or more slower)
#pragma unroll 8
        for (int v = 0; v < units; ++v) {
            float4 x[RB], y[CB];
#pragma unroll
            for (int r = 0; r < RB; ++r) x[r] = pr[r][v];
#pragma unroll
            for (int q = 0; q < CB; ++q) y[q] = pc[q][v];
#pragma unroll
            for (int r = 0; r < RB; ++r)
#pragma unroll
                for (int q = 0; q < CB; ++q) acc[r][q].add(x[r], y[q]);
        }
    }
}

// The whole block of the new rows against all rows, one row x 4 columns per
// item (rows i, columns b + q NB): more, smaller items than pipe_dist_pairs,
// which small nodes need to spread over the block.
template <int NT>
__device__ __forceinline__ void pipe_dist_rows(const unsigned char *rows, const PipeGeo &g, float *D, int ns, int m,
                                               int tid) {
    const int NB = (ns + 3) >> 2, items = m * NB;
    const uint32_t nbm = div_magic((uint32_t)NB);
    for (int e = tid; e < items; e += NT) {
        const int i = (int)div_small((uint32_t)e, (uint32_t)NB, nbm), b = e - i * NB;
        int ri[1] = {i}, cj[4];
        bool vc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            cj[q] = b + q * NB;
            vc[q] = cj[q] < ns;
            if (!vc[q]) cj[q] = b;
        }
        Acc2 acc[1][4];
        pipe_block<1, 4>(rows, g, ri, cj, acc);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (vc[q]) D[i * kPipeDStride + cj[q]] = acc[0][q].sum();
    }
}

// The distance block a node's joins need, each pair once: the new x new
// pairs and the new x old pairs.  New x new: rows a, a + M against columns
// b, b + M (M = ceil(m / 2)) for a <= b only, so every unordered pair of new
// rows is computed once (the a == b items also give the diagonal, unused, and
// both orders of one pair, equal bit for bit); each distance is written to
// D[x][y] and D[y][x].  New x old: rows a, a + M against old columns
// m + b + q NBo.  Consecutive threads take consecutive b (consecutive rows,
// distinct banks); a warp shares the rows a, a + M (broadcast).
template <int NT>
__device__ __forceinline__ void pipe_dist_pairs(const unsigned char *rows, const PipeGeo &g, float *D, int ns,
                                                int m, int tid) {
    const int M = (m + 1) >> 1, o = ns - m;
    const int n1 = M * (M + 1) / 2;
    const int NBo = (o + 3) >> 2, n2 = M * NBo;
    const uint32_t nbm = div_magic((uint32_t)(NBo > 0 ? NBo : 1));
    for (int e = tid; e < n1 + n2; e += NT) {
        if (e < n1) {
            // row a of the upper triangle starts at a (2M - a + 1) / 2
            int a = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int c = a + step;
                if (c < M && c * (2 * M - c + 1) / 2 <= e) a = c;
            }
            const int b = a + (e - a * (2 * M - a + 1) / 2);
            int ri[2] = {a, a + M}, cj[2] = {b, b + M};
            const bool vr1 = ri[1] < m, vc1 = cj[1] < m;
            if (!vr1) ri[1] = a;
            if (!vc1) cj[1] = b;
            Acc2 acc[2][2];
            pipe_block<2, 2>(rows, g, ri, cj, acc);
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    if ((r && !vr1) || (q && !vc1)) continue;
                    const float dd = acc[r][q].sum();
                    D[ri[r] * kPipeDStride + cj[q]] = dd;
                    D[cj[q] * kPipeDStride + ri[r]] = dd;
                }
        } else {
            const int e2 = e - n1;
            const int a = (int)div_small((uint32_t)e2, (uint32_t)NBo, nbm), b = e2 - a * NBo;
            int ri[2] = {a, a + M}, cj[4];
            bool vc[4];
            const bool vr1 = ri[1] < m;
            if (!vr1) ri[1] = a;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                cj[q] = m + b + q * NBo;
                vc[q] = cj[q] < ns;
                if (!vc[q]) cj[q] = m + b;
            }
            Acc2 acc[2][4];
            pipe_block<2, 4>(rows, g, ri, cj, acc);
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if ((r == 0 || vr1) && vc[q]) D[ri[r] * kPipeDStride + cj[q]] = acc[r][q].sum();
        }
    }
}
}  // namespace

template <int W, int S>
__global__ void __launch_bounds__(PipeShape<W, S>::kThreads, PipeShape<W, S>::kMinBlocks)
    pipe_join_kernel(DevState st, int li) {
    constexpr int kPipeWarps = W, kPipeCompute = 32 * W, kPipeSlots = S;
    if (iteration_skipped(st, li)) return;
    extern __shared__ __align__(128) unsigned char smem[];
    PipeShared *sh = reinterpret_cast<PipeShared *>(smem);
    const PipeGeo geo = pipe_geo(st.nv);
    unsigned char *slots = smem + 128;
    PipeCur *cur = reinterpret_cast<PipeCur *>(slots + (size_t)kPipeSlots * geo.slot_bytes);
    volatile int *abort_flag = &sh->abort_flag;
    const int tid = threadIdx.x;
    const unsigned lane = lane_id();
    const int warp = tid >> 5;
    const int K = st.K;
    if (tid == 0) {
        for (int s = 0; s < kPipeSlots; ++s) {
            bar_init(&sh->full[s], 33);  // 32 copy arrivals of the producer lanes + its release arrive
            bar_init(&sh->empty[s], 1);  // the compute warps, once the rows are read
        }
        sh->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 8) sh->stat[tid] = 0;
    __syncthreads();

    long long w_to = 0;
    if (warp == kPipeWarps) {
        // ------------------------------------------------------- producer --
        int k = 0;  // nodes handed out
        bool ok = true;
        // the next node of this block with a join pair (ids in registers)
        long long u = st.u_lo + blockIdx.x;
        auto next_node = [&](long long from, int &meta, int &id0, int &id1) -> long long {
            for (long long v = from; v < st.u_hi; v += gridDim.x) {
                meta = __ldg(st.cmeta + v);
                if (meta & 0xFF) {
                    const int ns = meta & 0xFF;
                    id0 = (int)lane < ns ? __ldg(st.cset + (size_t)v * kSetMax + lane) : 0;
                    id1 = (int)lane + 32 < ns ? __ldg(st.cset + (size_t)v * kSetMax + 32 + lane) : 0;
                    return v;
                }
            }
            return st.u_hi;
        };
        int meta = 0, id0 = 0, id1 = 0;
        u = next_node(u, meta, id0, id1);
        const unsigned char *X = reinterpret_cast<const unsigned char *>(st.X);
        const size_t row_bytes = (size_t)st.nv * 16;
        for (;;) {
            const int slot = k % kPipeSlots;
            unsigned char *sb = slots + (size_t)slot * geo.slot_bytes;
            if (k >= kPipeSlots && !bar_wait(&sh->empty[slot], (k / kPipeSlots - 1) & 1, abort_flag)) {
                ok = false;
                break;
            }
            int *hdr = reinterpret_cast<int *>(sb);
            int *sid = hdr + 4;
            uint64_t *swk = reinterpret_cast<uint64_t *>(sb + 16 + 4 * kSetMax);
            if (u >= st.u_hi) {
                // end mark: no rows; the copy arrivals complete at once
                if (lane == 0) hdr[0] = 0;
                __syncwarp();
                bar_arrive_copies(&sh->full[slot]);
                if (lane == 0) bar_arrive(&sh->full[slot]);
                ++k;
                break;
            }
            const int ns = meta & 0xFF, m = (meta >> 8) & 0xFF;
            if (lane == 0) {
                hdr[0] = ns;
                hdr[1] = m;
            }
            if ((int)lane < ns) sid[lane] = id0;
            if ((int)lane + 32 < ns) sid[lane + 32] = id1;
            // rows: lane l copies units l, l + 32 of every row
            const uint32_t rows_s = su32(sb + kPipeHdrBytes);
            for (int r = 0; r < ns; ++r) {
                const int id = __shfl_sync(kFull, r < 32 ? id0 : id1, r & 31);
                const unsigned char *src = X + (size_t)id * row_bytes;
#pragma unroll
                for (int cb = 0; cb < 2; ++cb) {
                    const int v = 32 * cb + (int)lane;
                    if (cb < geo.nblk && v < st.nv)
                        cpa16(rows_s + geo.off[cb] + (uint32_t)r * geo.stride[cb] + lane * 16u, src + (size_t)v * 16);
                }
            }
            // worst-key snapshots
            if ((int)lane < ns) cpa8(su32(swk + lane), st.keys + (size_t)id0 * K + (K - 1));
            if ((int)lane + 32 < ns) cpa8(su32(swk + lane + 32), st.keys + (size_t)id1 * K + (K - 1));
            __syncwarp();
            bar_arrive_copies(&sh->full[slot]);
            if (lane == 0) bar_arrive(&sh->full[slot]);
            ++k;
            u = next_node(u + gridDim.x, meta, id0, id1);
        }
        if (!ok && lane == 0 && !*abort_flag) {
            sh->abort_flag = 1;
            ++w_to;
        }
        // every copy issued lands before the block can exit
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else {
        // ---------------------------------------------------------- compute --
        long long l_evals = 0, l_gath = 0, l_props = 0, l_ovf = 0, l_ins = 0;
        for (int k = 0;; ++k) {
            const int slot = k % kPipeSlots;
            const unsigned char *sb = slots + (size_t)slot * geo.slot_bytes;
            if (!bar_wait(&sh->full[slot], (k / kPipeSlots) & 1, abort_flag)) {
                if (tid == 0 && !*abort_flag) {
                    sh->abort_flag = 1;
                    ++w_to;
                }
                break;
            }
            const int *hdr = reinterpret_cast<const int *>(sb);
            const int ns = hdr[0], m = hdr[1], o = ns - m;
            if (ns == 0) break;
            const int *ssid = hdr + 4;
            const uint64_t *sswk = reinterpret_cast<const uint64_t *>(sb + 16 + 4 * kSetMax);
            if (tid < ns) {
                cur->sid[tid] = ssid[tid];
                cur->swk[tid] = sswk[tid];
                cur->fails[tid] = 0ull;
            }
            // ---- 1. distance block (RB so that the items fill the block)
            const unsigned char *rows = sb + kPipeHdrBytes;
            // each pair once in larger items, unless they would keep fewer than
            // half the threads busy: then the whole block in 1 x 4 items, which
            // spread a small node over more threads (measured on the 1M x 128
            // mixture against pairs only: rho 0.3 join 12.1 -> 10.3 ms per
            // iteration; rho 0.7, where most nodes are large, 17.9 -> 17.1 ms)
            {
                const int M = (m + 1) >> 1, items_p = M * (M + 1) / 2 + M * ((ns - m + 3) >> 2);
                if (2 * items_p >= kPipeCompute) pipe_dist_pairs<kPipeCompute>(rows, geo, cur->D, ns, m, tid);
                else pipe_dist_rows<kPipeCompute>(rows, geo, cur->D, ns, m, tid);
            }
            compute_sync<kPipeCompute>();
            if (tid == 0) bar_arrive(&sh->empty[slot]);  // the rows are no longer read
            if (tid == 0) {
                l_evals += (long long)m * (m - 1) / 2 + (long long)m * o;
                l_gath += ns;
            }
            // ---- 2. proposals, one warp per target (targets warp, warp + 8,
            //         ...): a new target t takes partner j (j != t) when
            //         key(D[t][j], j) orders before t's snapshot worst, an old
            //         target t takes new partner i when key(D[i][t], i) does --
            //         every proposal of the node's join pairs once.  Two
            //         ballots give a target's 64-bit mask; lane q keeps the
            //         mask of the warp's target q.
            const int nt = warp < ns ? (ns - warp + kPipeWarps - 1) / kPipeWarps : 0;
            unsigned long long my_mask = 0ull;
            for (int q = 0; q < nt; ++q) {
                const int t = warp + kPipeWarps * q;
                const uint64_t wt = cur->swk[t];
                unsigned b0, b1;
                if (t < m) {
                    const int j0 = (int)lane, j1 = (int)lane + 32;
                    b0 = __ballot_sync(kFull, j0 < ns && j0 != t &&
                                                  make_key(cur->D[t * kPipeDStride + j0], (uint32_t)cur->sid[j0],
                                                           kFlagNew | kFlagIns) < wt);
                    b1 = __ballot_sync(kFull, j1 < ns && j1 != t &&
                                                  make_key(cur->D[t * kPipeDStride + j1], (uint32_t)cur->sid[j1],
                                                           kFlagNew | kFlagIns) < wt);
                } else {
                    const int i0 = (int)lane, i1 = (int)lane + 32;
                    b0 = __ballot_sync(kFull, i0 < m &&
                                                  make_key(cur->D[i0 * kPipeDStride + t], (uint32_t)cur->sid[i0],
                                                           kFlagNew | kFlagIns) < wt);
                    b1 = __ballot_sync(kFull, i1 < m &&
                                                  make_key(cur->D[i1 * kPipeDStride + t], (uint32_t)cur->sid[i1],
                                                           kFlagNew | kFlagIns) < wt);
                }
                if ((int)lane == q) my_mask = (unsigned long long)b0 | ((unsigned long long)b1 << 32);
            }
            // ---- 3. bucket runs of the warp's targets: lanes q < nt reserve
            //         their target's range at once (one atomicAdd each) and
            //         claim the pool chunks it spans; then lane k writes
            //         proposal k of the warp's targets (target by a search over
            //         the lanes' prefix counts, partner as the r-th set bit)
            {
                const int cnt = (int)lane < nt ? __popcll(my_mask) : 0;
                const int t_me = warp + kPipeWarps * (int)lane;
                int base = 0;
                if (cnt) {
                    const uint32_t p = (uint32_t)cur->sid[t_me];
                    base = atomicAdd(st.pcursor + p, cnt);
                    for (int r = base >> kBucketRunBits > 1 ? base >> kBucketRunBits : 1;
                         r <= (base + cnt - 1) >> kBucketRunBits; ++r)
                        bucket_slot(st, p, r << kBucketRunBits);
                }
                int inc = cnt;
#pragma unroll
                for (int o2 = 1; o2 < 32; o2 <<= 1) {
                    const int v = __shfl_up_sync(kFull, inc, o2);
                    if ((int)lane >= o2) inc += v;
                }
                const int total_w = __shfl_sync(kFull, inc, 31);
                const int rb = base - (inc - cnt);
                l_props += (lane == 0) ? total_w : 0;
                __threadfence_block();
                unsigned fail_q = 0;  // lane q: the target q had a proposal without a slot
                for (int k0 = 0; k0 < total_w; k0 += 32) {
                    const int kk = k0 + (int)lane;
                    const bool act = kk < total_w;
                    const int kc = act ? kk : total_w - 1;
                    int q = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int v = __shfl_sync(kFull, inc, q + step - 1);
                        if (v <= kc) q += step;
                    }
                    const int qe = q > 0 ? q - 1 : 0;
                    const int ev = __shfl_sync(kFull, inc, qe);
                    const unsigned long long mq = __shfl_sync(kFull, my_mask, q);
                    const int rbq = __shfl_sync(kFull, rb, q);
                    const int excl = q == 0 ? 0 : ev;
                    unsigned failed_here = 0;
                    if (act) {
                        const int t = warp + kPipeWarps * q;
                        const int j = nth_set_bit64(mq, kk - excl);
                        uint64_t *dst = bucket_slot(st, (uint32_t)cur->sid[t], kk + rbq);
                        const float dd = t < m ? cur->D[t * kPipeDStride + j] : cur->D[j * kPipeDStride + t];
                        if (dst) {
                            *dst = make_key(dd, (uint32_t)cur->sid[j], kFlagNew | kFlagIns);
                        } else {
                            atomicOr(&cur->fails[t], 1ull << j);
                            failed_here = 1u << q;
                        }
                    }
                    fail_q |= __reduce_or_sync(kFull, failed_here);
                }
                __syncwarp();
                // full buckets (rare): this warp's targets, locked insertion
                for (unsigned fm = fail_q; fm; fm &= fm - 1) {
                    const int q = __ffs(fm) - 1;
                    const int t = warp + kPipeWarps * q;
                    const unsigned long long rest = cur->fails[t];
                    if (lane == 0) l_ovf += __popcll(rest);
                    uint64_t xs[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = (int)lane + 32 * h;
                        xs[h] = kKeyEmpty;
                        if ((rest >> j) & 1ull) {
                            const float dd = t < m ? cur->D[t * kPipeDStride + j] : cur->D[j * kPipeDStride + t];
                            xs[h] = make_key(dd, (uint32_t)cur->sid[j], kFlagNew | kFlagIns);
                        }
                    }
                    const int ins = warp_locked_insert(st, (uint32_t)cur->sid[t], rest, xs[0], xs[1], li);
                    if (lane == 0) {
                        if (ins < 0) ++w_to;
                        else l_ins += ins;
                    }
                }
            }
            compute_sync<kPipeCompute>();  // cur is reused by the next node
        }
        const long long w_props = warp_sum(l_props);
        if (lane == 0 && w_props) atomic_add_ll(&sh->stat[2], w_props);
        if (tid == 0) {
            atomic_add_ll(&sh->stat[0], l_evals);
            atomic_add_ll(&sh->stat[1], l_gath);
        }
        if (l_ins) atomic_add_ll(&sh->stat[3], l_ins);
        if (l_ovf) atomic_add_ll(&sh->stat[4], l_ovf);
    }
    if (w_to) atomic_add_ll(&sh->stat[5], w_to);
    __syncthreads();
    if (tid == 0) {
        long long *its = st.it_stats + (size_t)li * kItCount;
        its[kItRan] = 1;
        atomic_add_ll(&its[kItEvals], sh->stat[0]);
        atomic_add_ll(&its[kItGathered], sh->stat[1]);
        atomic_add_ll(&its[kItProposals], sh->stat[2]);
        atomic_add_ll(&its[kItInserts], sh->stat[3]);
        atomic_add_ll(&st.stats[kStatEvals], sh->stat[0]);
        atomic_add_ll(&st.stats[kStatGathered], sh->stat[1]);
        atomic_add_ll(&st.stats[kStatInserts], sh->stat[3]);
        if (sh->stat[4]) atomic_add_ll(&st.stats[kStatBucketOverflow], sh->stat[4]);
        if (sh->stat[5]) atomic_add_ll(&st.stats[kStatLockTimeout], sh->stat[5]);
    }
}

bool pipe_join_fits(int bf16, int nv) { return !bf16 && nv > 8 && nv <= kPipeMaxUnits; }

namespace {
template <int W, int S>
cudaError_t launch_pipe_shape(const DevState &st, int li, cudaStream_t s) {
    const size_t dyn = pipe_smem_bytes(st.nv, S);
    auto kern = pipe_join_kernel<W, S>;
    cudaError_t e = smem_opt_in((const void *)kern, dyn);
    if (e != cudaSuccess) return e;
    const int grid = grid_for((const void *)kern, PipeShape<W, S>::kThreads, dyn);
    kern<<<grid, PipeShape<W, S>::kThreads, dyn, s>>>(st, li);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_pipe_join(const DevState &st, int li, cudaStream_t s) {
    cudaError_t e = st.u_lo == 0 ? launch_set_kernel(st, li, s) : cudaSuccess;
    if (e != cudaSuccess) return e;
    // four compute warps and one row slot per block, four blocks per SM (the
    // default): measured against eight warps with two slots (two blocks per
    // SM) on the 1M x 128 mixture, join per launch 14.4 -> 10.2 ms at rho 0.3
    // and 29.4 -> 23.4 ms at rho 0.7, and 1.28 -> 0.71 ms on the 54k x 192
    // audio shape (more nodes in flight per SM beat deeper prefetch per
    // block); the autotuner tries both
    if (st.join_path == kJoinPipe8) return launch_pipe_shape<8, 2>(st, li, s);
    return launch_pipe_shape<4, 1>(st, li, s);
}

}  // namespace knng
