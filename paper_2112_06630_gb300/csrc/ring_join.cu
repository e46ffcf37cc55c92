// ring_join.cu -- the local join (the paper's Calculation step, Section 2;
// blocked mutual distances of a bounded neighbourhood, Section 3.3) for
// high-dimensional points, with the candidate rows staged in shared memory
// by asynchronous copies.
//
// Two kernels per iteration:
//
// set_kernel (one warp per node): node u's sampled candidates with repeats
//   removed (new first, at most 64) are written to cset[u][0 .. ns) and
//   (ns, m) to cmeta[u]; 0 when u has no new candidate.
//
// ring_join_kernel (persistent, one 512-thread block per SM, two circular
// byte rings in shared memory):
//   warp 0 (producer) walks this block's nodes eight at a time (groups
//     blockIdx.x, blockIdx.x + gridDim.x, ...; the next group's sets are
//     loaded while the current one is placed).  For every node with a join
//     pair it places a slot in ring A (the candidate rows) and one in ring B
//     (ids, worst keys, masks, norms, the distance block), writes the ids and
//     arrives on the node's mbarrier.  It issues no copies: one warp cannot
//     issue them fast enough for fifteen (single-row cp.async.bulk copies
//     were measured at about 80 issuing cycles each).
//   warps 1..15 (consumers) take nodes in order from a shared counter.  A
//     consumer issues the copies of its next node (warp-wide 16-byte cp.async
//     per row, the worst keys, bf16 norms) as soon as the current node's rows
//     are released, so they land while the current node's proposals go out;
//     it never waits for a placement while it holds a node.  The join of a
//     node:
//       1. the distance block D[i][j] of new rows i against all rows j:
//          float32: the canonical difference form (bit-identical to every
//            other float32 distance in the library), register-blocked two
//            rows by four columns per lane (six row reads per eight pairs);
//          bf16: the Gram block on the tensor cores (mma.sync m16n8k16,
//            float32 accumulate), |x_i|^2 + |x_j|^2 - 2 x_i . x_j clamped at 0;
//          then ring A is released;
//       2. the proposal masks: element (i, j) of the block carries the
//          proposal of j to i (j != i) and, for an old j, of i to j -- each
//          proposal of the node's join pairs once -- kept when its key orders
//          before the target's worst entry (32-bit shared atomics);
//       3. one bucket run per target (one atomicAdd), full buckets take the
//          locked insertion; then ring B is released.
//   Proposals of ids already listed are dropped by the list merge.  Slots
//   are released out of order; the producer reuses ring bytes in allocation
//   order once the oldest slots are released.  A node's join is the same set
//   of pairs and keys as in the other join kernels, so the lists after the
//   merge are the same.
// Every wait (mbarrier phases, ring space, list locks) is bounded by the
// global timer; a wait that gives up raises the timeout counter, sets the
// block's abort flag, and the block winds down once its copies have landed.
#include <cuda_bf16.h>

#include <cstdint>

#include "join_common.cuh"

namespace knng {

namespace {
constexpr int kRingConsumers = 15;
constexpr int kRingThreads = 32 * (kRingConsumers + 1);
constexpr int kRingDesc = 32;                          // nodes in flight per block
constexpr int kGroup = 8;                              // nodes per producer group
constexpr uint32_t kRingBytes = 221u * 1024u;          // both rings (with the static part: <= 227 KB)
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s: a bounded wait gives up after this
constexpr int kSetWarps = 8;

__host__ __device__ __forceinline__ uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) & ~(a - 1); }

// Row bytes in global memory and the shared-memory row stride (an odd number
// of 16-byte units: conflict-free float4 reads and ldmatrix phases).
struct Geometry {
    uint32_t gbytes, stride;
};
// kind: 0 float32 rows (nv 16-byte units), 1 bf16 rows of dpb elements, 2
// e4m3 rows of dpb elements (one byte each)
__host__ __device__ __forceinline__ Geometry geometry(int kind, int nv, int dpb) {
    Geometry g;
    const uint32_t units = kind == 2 ? (uint32_t)dpb / 16u : kind == 1 ? (uint32_t)dpb / 8u : (uint32_t)nv;
    g.gbytes = units * 16u;
    g.stride = (units | 1u) * 16u;
    return g;
}
// ring A: the candidate rows
__host__ __device__ __forceinline__ uint32_t slot_a_bytes(int ns, const Geometry &g) {
    return align_up((uint32_t)ns * g.stride, 128);
}
// ring B: ids | worst keys | masks | norms | failed-proposal masks | distance block
// (m rows of stride ns | 1 floats)
struct SlotB {
    uint32_t o_swk, o_mask, o_nrm, o_ovf, o_D, size;
};
__host__ __device__ __forceinline__ SlotB slot_b(int ns, int m) {
    SlotB L;
    L.o_swk = align_up(4u * ns, 16);
    L.o_mask = align_up(L.o_swk + 8u * ns, 16);
    L.o_nrm = align_up(L.o_mask + 8u * ns, 16);
    L.o_ovf = align_up(L.o_nrm + 4u * ns, 16);
    L.o_D = align_up(L.o_ovf + 8u * ns, 16);
    L.size = align_up(L.o_D + 4u * (uint32_t)m * (uint32_t)(ns | 1), 128);
    return L;
}

// Split of the ring bytes: ring B gets the share a node of 24 candidates (12
// new) needs next to its rows, at least one worst-case node; ring A the rest.
__host__ __device__ __forceinline__ uint32_t ring_b_bytes(const Geometry &g) {
    const double a = (double)slot_a_bytes(24, g), b = (double)slot_b(24, 12).size;
    uint32_t rb = (uint32_t)((double)kRingBytes * b / (a + b)) & ~127u;
    const uint32_t lo = slot_b(kSetMax, kSetMax).size;
    return rb < lo ? lo : rb;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase with the given parity; false when the wait gave up or
// the block is aborting.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    const unsigned long long t0 = global_ns();
    while (!mbar_try(bar, parity)) {
        if (*abort_flag) return false;
        if (global_ns() - t0 > kWaitNs) return false;
    }
    return true;
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

struct RingDesc {
    uint32_t off_a, off_b;
    int nsm;  // ns | m << 8; 0 = no further node
};

struct RingShared {
    RingDesc desc[kRingDesc];
    uint64_t full[kRingDesc];
    uint64_t empty_a[kRingDesc];
    uint64_t empty_b[kRingDesc];
    int psid[2][kGroup][kSetMax];  // producer: ids of the current and the next group
    int next_k;
    int abort_flag;
    long long stat[8];
};

// One circular byte ring of the producer: slots are handed out in order and
// retired in order once released.
struct ByteRing {
    uint32_t head, tail, cap;  // next free byte, start of the oldest slot in use
    int k_tail;                // oldest node whose slot is not known to be released
    // place `bytes` (k_head nodes handed out so far); false when they do not fit
    __device__ __forceinline__ bool fit(uint32_t bytes, int k_head, uint32_t &off) const {
        if (k_tail == k_head) {
            off = 0;
            return bytes <= cap;
        }
        if (head > tail) {
            if (head + bytes <= cap) { off = head; return true; }
            if (bytes <= tail) { off = 0; return true; }
            return false;
        }
        if (head < tail && head + bytes <= tail) { off = head; return true; }
        return false;
    }
};

// D[i][j] (stride ds) of new rows i < m against all rows j < ns, float32
// canonical difference form.  Work item = rows (a, a + MA) x columns (b,
// b + NB, b + 2 NB, b + 3 NB): six row reads per eight pairs; consecutive
// lanes take consecutive columns, distinct rows on an odd 16-byte stride.
__device__ __forceinline__ void warp_dist_f32(const float4 *rows, uint32_t rs, int nv, float *D, int ds, int ns,
                                              int m) {
    const unsigned lane = lane_id();
    const int MA = (m + 1) >> 1, NB = (ns + 3) >> 2, items = MA * NB;
    for (int e = lane; e < items; e += 32) {
        const int a = e / NB, b = e - a * NB;
        const int i0 = a, i1 = a + MA;
        const bool v1 = i1 < m;
        const float4 *r0 = rows + (size_t)i0 * rs, *r1 = rows + (size_t)(v1 ? i1 : i0) * rs;
        const float4 *c[4];
        bool vc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = b + q * NB;
            vc[q] = j < ns;
            c[q] = rows + (size_t)(vc[q] ? j : b) * rs;
        }
        Acc2 acc0[4], acc1[4];
        for (int v = 0; v < nv; ++v) {
            const float4 x0 = r0[v], x1 = r1[v];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 y = c[q][v];
                acc0[q].add(x0, y);
                acc1[q].add(x1, y);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!vc[q]) continue;
            const int j = b + q * NB;
            D[i0 * ds + j] = acc0[q].sum();
            if (v1) D[i1 * ds + j] = acc1[q].sum();
        }
    }
}

// Gram block of the new rows (i < m) against all rows (j < ns) on the tensor
// cores, one warp: D[i][j] = max(0, |x_i|^2 + |x_j|^2 - 2 x_i . x_j).
__device__ __forceinline__ void warp_gram_bf16(const unsigned char *rows, uint32_t stride, const float *nrm,
                                               float *D, int ds, int ns, int m, int dpb) {
    const unsigned lane = lane_id();
    const int nk = dpb / 16, ntiles = (ns + 7) >> 3;
    const int gid = lane >> 2, tig = lane & 3;
    for (int r0 = 0; r0 < m; r0 += 16) {
        float acc[8][4];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
        // rows past the set are clamped to its last row: their results are
        // discarded, their addresses stay inside the slot
        const int ar = min(r0 + (int)(lane & 15), ns - 1), ac = 8 * (int)(lane >> 4);
        const uint32_t abase = smem_u32(rows + (size_t)ar * stride) + ac * 2;
        uint32_t bbase[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int br = min(q * 8 + (int)(lane & 7), ns - 1), bc = 8 * (int)((lane >> 3) & 1);
            bbase[q] = smem_u32(rows + (size_t)br * stride) + bc * 2;
        }
        for (int kk = 0; kk < nk; ++kk) {
            uint32_t a0, a1, a2, a3;
            asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                         : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3)
                         : "r"(abase + kk * 32));
            // all B fragments of the k-step first, then the MMAs: the loads
            // overlap instead of each MMA waiting on its own load
            uint32_t b0[8], b1[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q < ntiles)
                    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                                 : "=r"(b0[q]), "=r"(b1[q])
                                 : "r"(bbase[q] + kk * 32));
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q < ntiles)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                        "{%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[q][0]), "+f"(acc[q][1]), "+f"(acc[q][2]), "+f"(acc[q][3])
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0[q]), "r"(b1[q]));
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int i = r0 + gid + 8 * (h >> 1), j = q * 8 + tig * 2 + (h & 1);
                if (q < ntiles && i < m && j < ns) D[i * ds + j] = fmaxf(0.f, nrm[i] + nrm[j] - 2.f * acc[q][h]);
            }
    }
}
// The same Gram block from e4m3 rows (FP8, one byte per element): 32
// elements per k-step, mma.sync m16n8k32 e4m3 with float32 accumulate.  The
// fragments of a 32-byte k-step have the layout of a bf16 m16n8k16 step (four
// consecutive bytes where bf16 has two elements), so the ldmatrix addressing
// is the bf16 one.
__device__ __forceinline__ void warp_gram_fp8(const unsigned char *rows, uint32_t stride, const float *nrm,
                                              float *D, int ds, int ns, int m, int dpb) {
    const unsigned lane = lane_id();
    const int nk = dpb / 32, ntiles = (ns + 7) >> 3;
    const int gid = lane >> 2, tig = lane & 3;
    for (int r0 = 0; r0 < m; r0 += 16) {
        float acc[8][4];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
        const int ar = min(r0 + (int)(lane & 15), ns - 1), ac = 16 * (int)(lane >> 4);
        const uint32_t abase = smem_u32(rows + (size_t)ar * stride) + ac;
        uint32_t bbase[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int br = min(q * 8 + (int)(lane & 7), ns - 1), bc = 16 * (int)((lane >> 3) & 1);
            bbase[q] = smem_u32(rows + (size_t)br * stride) + bc;
        }
        for (int kk = 0; kk < nk; ++kk) {
            uint32_t a0, a1, a2, a3;
            asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                         : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3)
                         : "r"(abase + kk * 32));
            // all B fragments of the k-step first, then the MMAs (as in bf16)
            uint32_t b0[8], b1[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q < ntiles)
                    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                                 : "=r"(b0[q]), "=r"(b1[q])
                                 : "r"(bbase[q] + kk * 32));
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q < ntiles)
                    asm volatile(
                        "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                        "{%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[q][0]), "+f"(acc[q][1]), "+f"(acc[q][2]), "+f"(acc[q][3])
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0[q]), "r"(b1[q]));
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int i = r0 + gid + 8 * (h >> 1), j = q * 8 + tig * 2 + (h & 1);
                if (q < ntiles && i < m && j < ns) D[i * ds + j] = fmaxf(0.f, nrm[i] + nrm[j] - 2.f * acc[q][h]);
            }
    }
}
}  // namespace

// ------------------------------------------------------------ set_kernel --
template <int kWide>
__global__ void __launch_bounds__(kSetWarps * 32) set_kernel(DevState st, int li) {
    if (iteration_skipped(st, li)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long bstat[2];
    if (threadIdx.x < 2) bstat[threadIdx.x] = 0;
    __syncthreads();
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int raw_max = ((2 * st.cap + 31) / 32) * 32;
    int *wbase = reinterpret_cast<int *>(smem) + (size_t)warp * (raw_max + (1 << hash_bits(st.cap)) + kSetMax);
    int *hset = wbase;
    int *raw = hset + (1 << hash_bits(st.cap));
    int *sid = raw + raw_max;
    long long w_candids = 0, w_setovf = 0;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = gw; u < st.n; u += nw) {
        int ns = 0, m = 0;
        if (!node_skipped(st, u, li))
            w_candids += warp_gather_candidates<kWide>(st, u, raw, hset, sid, ns, m, w_setovf);
        for (int i = lane; i < ns; i += 32) st.cset[(size_t)u * kSetMax + i] = sid[i];
        if (lane == 0) st.cmeta[u] = ns | (m << 8);
        __syncwarp();
    }
    if (lane == 0) {
        atomic_add_ll(&bstat[0], w_candids);
        atomic_add_ll(&bstat[1], w_setovf);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomic_add_ll(&st.it_stats[(size_t)li * kItCount + kItCandIds], bstat[0]);
        if (bstat[1]) atomic_add_ll(&st.stats[kStatSetOverflow], bstat[1]);
    }
}

// ------------------------------------------------------ ring_join_kernel --
namespace {
// Copies of a node's candidate rows, worst keys (and bf16 norms) into its
// slots, issued by the consumer warp that runs the node, as one cp.async
// group per lane.
template <int kKind>
__device__ __forceinline__ void issue_copies(const DevState &st, const Geometry &geo, const unsigned char *src,
                                             unsigned char *sa, unsigned char *sb, const SlotB &LB, int ns) {
    const unsigned lane = lane_id();
    const int K = st.K;
    const int *sid = reinterpret_cast<const int *>(sb);
    // rows: lane l copies 16-byte chunks l, l + 32, ... of each row
    for (int i = 0; i < ns; ++i) {
        const size_t v = (size_t)sid[i];
        const unsigned char *g = src + v * geo.gbytes;
        unsigned char *d = sa + (size_t)i * geo.stride;
        for (uint32_t c = lane * 16u; c < geo.gbytes; c += 512u) cp_async16(d + c, g + c);
    }
    for (int i = lane; i < ns; i += 32) {
        cp_async8(sb + LB.o_swk + 8 * i, st.keys + (size_t)sid[i] * K + (K - 1));
        if (kKind != 0) cp_async4(sb + LB.o_nrm + 4 * i, st.xnorm + sid[i]);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
}  // namespace

template <int kKind>
__global__ void __launch_bounds__(kRingThreads, 1) ring_join_kernel(DevState st, int li) {
    constexpr bool kBF16 = kKind != 0;  // low-precision rows: Gram blocks with norms
    if (iteration_skipped(st, li)) return;
    __shared__ RingShared sh;
    extern __shared__ __align__(128) unsigned char ring[];
    const Geometry geo = geometry(kKind, st.nv, st.dpb);
    const uint32_t ring_b_cap = ring_b_bytes(geo), ring_a_cap = kRingBytes - ring_b_cap;
    unsigned char *ring_a = ring, *ring_b = ring + ring_a_cap;
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    volatile int *abort_flag = &sh.abort_flag;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kRingDesc; ++s) {
            mbar_init(&sh.full[s], 1);     // the producer: slots placed, ids written
            mbar_init(&sh.empty_a[s], 1);  // the consumer, after the distance block
            mbar_init(&sh.empty_b[s], 1);  // the consumer, at the end
        }
        sh.next_k = 0;
        sh.abort_flag = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < 8) sh.stat[threadIdx.x] = 0;
    __syncthreads();

    long long w_to = 0;

    if (warp == 0) {
        // ------------------------------------------------------ producer --
        const long long ngroups = (st.u_hi - st.u_lo + kGroup - 1) / kGroup;
        int k_head = 0;  // nodes handed out
        ByteRing ra{0u, 0u, ring_a_cap, 0}, rb{0u, 0u, ring_b_cap, 0};
        bool ok = true;
        // retire released slots of both rings in order (end marks are never released)
        auto retire = [&]() {
            while (ra.k_tail < k_head && mbar_test(&sh.empty_a[ra.k_tail % kRingDesc], (ra.k_tail / kRingDesc) & 1)) {
                ++ra.k_tail;
                if (ra.k_tail == k_head) ra.head = ra.tail = 0;
                else ra.tail = sh.desc[ra.k_tail % kRingDesc].off_a;
            }
            while (rb.k_tail < k_head && mbar_test(&sh.empty_b[rb.k_tail % kRingDesc], (rb.k_tail / kRingDesc) & 1)) {
                ++rb.k_tail;
                if (rb.k_tail == k_head) rb.head = rb.tail = 0;
                else rb.tail = sh.desc[rb.k_tail % kRingDesc].off_b;
            }
        };
        // a free descriptor (both of its slots released) and room in both rings
        auto alloc = [&](uint32_t bytes_a, uint32_t bytes_b, uint32_t &off_a, uint32_t &off_b) -> bool {
            const unsigned long long t0 = global_ns();
            for (;;) {
                retire();
                if (k_head - rb.k_tail < kRingDesc && ra.fit(bytes_a, k_head, off_a) && rb.fit(bytes_b, k_head, off_b))
                    return true;
                if (*abort_flag || global_ns() - t0 > kWaitNs) return false;
                __nanosleep(32);
            }
        };
        // sets of group g into registers (next) and shared memory (current)
        int nmeta = 0, nids[kGroup][2];
        auto load_group = [&](long long g) {
            nmeta = 0;
            if (g >= ngroups) return;
            const long long u0 = st.u_lo + g * kGroup;
            if ((int)lane < kGroup && u0 + lane < st.u_hi) nmeta = __ldg(st.cmeta + u0 + lane);
#pragma unroll
            for (int j = 0; j < kGroup; ++j) {
                nids[j][0] = nids[j][1] = 0;
                if (u0 + j < st.u_hi) {
                    nids[j][0] = __ldg(st.cset + (size_t)(u0 + j) * kSetMax + lane);
                    nids[j][1] = __ldg(st.cset + (size_t)(u0 + j) * kSetMax + 32 + lane);
                }
            }
        };
        int buf = 0;
        long long g = blockIdx.x;
        load_group(g);
        while (ok && g < ngroups) {
            const int cmeta = nmeta;
#pragma unroll
            for (int j = 0; j < kGroup; ++j) {
                sh.psid[buf][j][lane] = nids[j][0];
                sh.psid[buf][j][lane + 32] = nids[j][1];
            }
            __syncwarp();
            g += gridDim.x;
            load_group(g);  // in flight while this group is placed
            for (int j = 0; j < kGroup && ok; ++j) {
                const int nsm = __shfl_sync(kFull, cmeta, j);
                const int ns = nsm & 0xFF, m = (nsm >> 8) & 0xFF;
                if (ns == 0) continue;
                const uint32_t bytes_a = slot_a_bytes(ns, geo);
                const SlotB LB = slot_b(ns, m);
                uint32_t off_a = 0, off_b = 0;
                if (!alloc(bytes_a, LB.size, off_a, off_b)) {
                    ok = false;
                    break;
                }
                const int s = k_head % kRingDesc;
                int *sid = reinterpret_cast<int *>(ring_b + off_b);
                const int *ids = sh.psid[buf][j];
                for (int i = lane; i < ns; i += 32) sid[i] = ids[i];
                if (lane == 0) {
                    sh.desc[s].off_a = off_a;
                    sh.desc[s].off_b = off_b;
                    sh.desc[s].nsm = nsm;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh.full[s]);
                ra.head = off_a + bytes_a;
                rb.head = off_b + LB.size;
                ++k_head;
            }
            buf ^= 1;
        }
        // one end mark per consumer: a descriptor, no ring bytes
        for (int c = 0; c < kRingConsumers && ok; ++c) {
            const unsigned long long t0 = global_ns();
            for (;;) {
                retire();
                if (k_head - rb.k_tail < kRingDesc) break;
                if (*abort_flag || global_ns() - t0 > kWaitNs) {
                    ok = false;
                    break;
                }
                __nanosleep(32);
            }
            if (!ok) break;
            const int s = k_head % kRingDesc;
            if (lane == 0) {
                sh.desc[s].nsm = 0;
                mbar_arrive(&sh.full[s]);
            }
            __syncwarp();
            ++k_head;
        }
        if (!ok && lane == 0 && !*abort_flag) {
            sh.abort_flag = 1;
            ++w_to;
        }
    } else {
        // ----------------------------------------------------- consumers --
        const unsigned char *src = kBF16 ? reinterpret_cast<const unsigned char *>(st.Xb)
                                         : reinterpret_cast<const unsigned char *>(st.X);
        long long w_evals = 0, l_props = 0, w_ins = 0, w_ovf = 0, w_gathered = 0;
        auto claim = [&]() -> int {
            int k = 0;
            if (lane == 0) k = atomicAdd(&sh.next_k, 1);
            return __shfl_sync(kFull, k, 0);
        };
        // node k's slots placed: its descriptor (0 = end mark)
        auto wait_placed = [&](int k, int &nsm) -> bool {
            if (!mbar_wait(&sh.full[k % kRingDesc], (k / kRingDesc) & 1, abort_flag)) return false;
            nsm = sh.desc[k % kRingDesc].nsm;
            return true;
        };
        auto start = [&](int k, int nsm) {
            const int s = k % kRingDesc, ns = nsm & 0xFF, m = (nsm >> 8) & 0xFF;
            issue_copies<kKind>(st, geo, src, ring_a + sh.desc[s].off_a, ring_b + sh.desc[s].off_b, slot_b(ns, m),
                                ns);
        };
        bool ok = true;
        int k_cur = claim(), nsm_cur = 0;
        ok = wait_placed(k_cur, nsm_cur);
        if (ok && nsm_cur) start(k_cur, nsm_cur);
        while (ok && nsm_cur) {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncwarp();

            const int s = k_cur % kRingDesc;
            const int ns = nsm_cur & 0xFF, m = (nsm_cur >> 8) & 0xFF, o = ns - m;
            const SlotB LB = slot_b(ns, m);
            const unsigned char *rows = ring_a + sh.desc[s].off_a;
            unsigned char *sb = ring_b + sh.desc[s].off_b;
            const int *sid = reinterpret_cast<const int *>(sb);
            const uint64_t *swk = reinterpret_cast<const uint64_t *>(sb + LB.o_swk);
            unsigned *mw = reinterpret_cast<unsigned *>(sb + LB.o_mask);  // two 32-bit words per target
            unsigned long long *mask = reinterpret_cast<unsigned long long *>(sb + LB.o_mask);
            const float *nrm = reinterpret_cast<const float *>(sb + LB.o_nrm);
            unsigned long long *fails = reinterpret_cast<unsigned long long *>(sb + LB.o_ovf);
            float *D = reinterpret_cast<float *>(sb + LB.o_D);
            const int ds = ns | 1;
            for (int i = lane; i < 2 * ns; i += 32) mw[i] = 0u;
            // ---- 1. distance block
            if (kKind == 2) warp_gram_fp8(rows, geo.stride, nrm, D, ds, ns, m, st.dpb);
            else if (kKind == 1) warp_gram_bf16(rows, geo.stride, nrm, D, ds, ns, m, st.dpb);
            else warp_dist_f32(reinterpret_cast<const float4 *>(rows), geo.stride >> 4, st.nv, D, ds, ns, m);
            w_evals += (long long)m * (m - 1) / 2 + (long long)m * o;
            w_gathered += ns;
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.empty_a[s]);  // the rows are no longer needed
            // claim the next node and start its copies if it is already placed:
            // they land while this node's proposals go out (a consumer never
            // waits for a placement while it holds a node)
            const int k_nxt = claim();
            int nsm_nxt = 0;
            const bool placed = mbar_test(&sh.full[k_nxt % kRingDesc], (k_nxt / kRingDesc) & 1);
            if (placed) {
                nsm_nxt = sh.desc[k_nxt % kRingDesc].nsm;
                if (nsm_nxt) start(k_nxt, nsm_nxt);
            }
            // ---- 2. proposals that order before the target's worst entry:
            //         element (i, j) of the block (i new) carries "j to i"
            //         (j != i) and, for an old j, "i to j" -- every proposal of
            //         the node's join pairs exactly once
            for (int i = 0; i < m; ++i) {
                const uint64_t wi = swk[i];
                const uint32_t qi = (uint32_t)sid[i];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = (int)lane + 32 * h;
                    if (j < ns) {
                        const float dd = D[i * ds + j];
                        if (j != i && make_key(dd, (uint32_t)sid[j], kFlagNew | kFlagIns) < wi)
                            atomicOr(&mw[2 * i + (j >> 5)], 1u << (j & 31));
                        if (j >= m && make_key(dd, qi, kFlagNew | kFlagIns) < swk[j])
                            atomicOr(&mw[2 * j + (i >> 5)], 1u << (i & 31));
                    }
                }
            }
            __syncwarp();
            // ---- 3. bucket runs.  Keys and slots are the same either way;
            //         bf16 nodes (cheap distance blocks) write flattened over
            //         the lanes, float32 nodes one run per lane, whichever
            //         measured faster (1M x 128: bf16 join 7.57 -> 6.89 ms
            //         flattened, float32 11.87 -> 12.07 ms)
            unsigned ovf_lo = 0, ovf_hi = 0;
            if constexpr (kBF16) {
                // ---- 3. bucket runs, flattened over the warp: lane t reserves
                //         target t's range (one atomicAdd) and the pool chunks
                //         of the runs it spans (one claim per run); lane k then
                //         writes proposal k of the node, its target found by a
                //         binary search over the targets' prefix counts and its
                //         partner as the r-th set bit of the target's mask.  A
                //         proposal whose run has no slot (bucket or pool spent) is
                //         marked for the locked insertion
                int inc0, inc1, ra, rb;  // per target lane / 32 + lane: inclusive prefix, base - exclusive prefix
                {
                    const unsigned long long ma = (int)lane < ns ? mask[lane] : 0ull;
                    const unsigned long long mb = (int)lane + 32 < ns ? mask[lane + 32] : 0ull;
                    const int ca = __popcll(ma), cb = __popcll(mb);
                    int ba = 0, bb = 0;
                    if (ca) ba = atomicAdd(st.pcursor + sid[lane], ca);
                    if (cb) bb = atomicAdd(st.pcursor + sid[lane + 32], cb);
                    if (ca)
                        for (int r = ba >> kBucketRunBits > 1 ? ba >> kBucketRunBits : 1;
                             r <= (ba + ca - 1) >> kBucketRunBits; ++r)
                            bucket_slot(st, (uint32_t)sid[lane], r << kBucketRunBits);
                    if (cb)
                        for (int r = bb >> kBucketRunBits > 1 ? bb >> kBucketRunBits : 1;
                             r <= (bb + cb - 1) >> kBucketRunBits; ++r)
                            bucket_slot(st, (uint32_t)sid[lane + 32], r << kBucketRunBits);
                    l_props += ca + cb;
                    inc0 = ca;
                    inc1 = cb;
                    for (int o2 = 1; o2 < 32; o2 <<= 1) {
                        const int v = __shfl_up_sync(kFull, inc0, o2);
                        if ((int)lane >= o2) inc0 += v;
                    }
                    const int tot0 = __shfl_sync(kFull, inc0, 31);
                    for (int o2 = 1; o2 < 32; o2 <<= 1) {
                        const int v = __shfl_up_sync(kFull, inc1, o2);
                        if ((int)lane >= o2) inc1 += v;
                    }
                    inc1 += tot0;
                    ra = ba - (inc0 - ca);
                    rb = bb - (inc1 - cb);
                    if ((int)lane < ns) fails[lane] = 0ull;
                    if ((int)lane + 32 < ns) fails[lane + 32] = 0ull;
                }
                const int total = __shfl_sync(kFull, inc1, 31);
                __threadfence_block();
                __syncwarp();
                for (int k0 = 0; k0 < total; k0 += 32) {
                    const int k = k0 + (int)lane;
                    const bool act = k < total;
                    const int kk = act ? k : total - 1;
                    int t = 0;
    #pragma unroll
                    for (int step = 32; step > 0; step >>= 1) {
                        const int probe = t + step - 1;
                        const int v0 = __shfl_sync(kFull, inc0, probe & 31), v1 = __shfl_sync(kFull, inc1, probe & 31);
                        if ((probe < 32 ? v0 : v1) <= kk) t += step;
                    }
                    const int tp = t > 0 ? t - 1 : 0;
                    const int e0 = __shfl_sync(kFull, inc0, tp & 31), e1 = __shfl_sync(kFull, inc1, tp & 31);
                    const int r0 = __shfl_sync(kFull, ra, t & 31), r1 = __shfl_sync(kFull, rb, t & 31);
                    if (!act) continue;
                    const int excl = t == 0 ? 0 : (tp < 32 ? e0 : e1);
                    const int j = nth_set_bit64(mask[t], k - excl);
                    uint64_t *dst = bucket_slot(st, (uint32_t)sid[t], k + (t < 32 ? r0 : r1));
                    if (dst) {
                        const float dd = t < m ? D[t * ds + j] : D[j * ds + t];
                        *dst = make_key(dd, (uint32_t)sid[j], kFlagNew | kFlagIns);
                    } else {
                        atomicOr(&fails[t], 1ull << j);
                        if (t < 32) ovf_lo |= 1u << t;
                        else ovf_hi |= 1u << (t - 32);
                    }
                }
            } else {
                // ---- 3. one bucket run per target
                for (int t = lane; t < ns; t += 32) {
                    const unsigned long long mt = mask[t];
                    const int c = __popcll(mt);
                    if (!c) continue;
                    l_props += c;
                    const uint32_t p = (uint32_t)sid[t];
                    const int b = atomicAdd(st.pcursor + p, c);
                    // a proposal whose run has no slot (bucket or pool spent) is
                    // marked for the locked insertion; the others are written
                    unsigned long long mm = mt, failed = 0ull;
                    uint64_t *dst = nullptr;
                    for (int r = 0; r < c; ++r, mm &= mm - 1) {
                        const int pos = b + r;
                        if (r == 0 || (pos & (kBucketRun - 1)) == 0) dst = bucket_slot(st, p, pos);
                        else if (dst) ++dst;
                        const int j = __ffsll((long long)mm) - 1;
                        const float dd = t < m ? D[t * ds + j] : D[j * ds + t];
                        if (dst) *dst = make_key(dd, (uint32_t)sid[j], kFlagNew | kFlagIns);
                        else failed |= 1ull << j;
                    }
                    fails[t] = failed;
                    if (failed) {
                        if (t < 32) ovf_lo |= 1u << t;
                        else ovf_hi |= 1u << (t - 32);
                    }
                }
            }
            ovf_lo = __reduce_or_sync(kFull, ovf_lo);
            ovf_hi = __reduce_or_sync(kFull, ovf_hi);
            __syncwarp();
            // ---- full buckets (rare): locked insertion of the rest
            for (unsigned long long om = (unsigned long long)ovf_lo | ((unsigned long long)ovf_hi << 32); om;
                 om &= om - 1) {
                const int t = __ffsll((long long)om) - 1;
                const unsigned long long rest = fails[t];
                w_ovf += __popcll(rest);
                uint64_t xs[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = (int)lane + 32 * h;
                    xs[h] = kKeyEmpty;
                    if ((rest >> j) & 1ull) {
                        const float dd = t < m ? D[t * ds + j] : D[j * ds + t];
                        xs[h] = make_key(dd, (uint32_t)sid[j], kFlagNew | kFlagIns);
                    }
                }
                const int ins = warp_locked_insert(st, (uint32_t)sid[t], rest, xs[0], xs[1], li);
                if (ins < 0) ++w_to;
                else w_ins += ins;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.empty_b[s]);

            // ---- next node (wait for its placement only now)
            if (!placed) {
                ok = wait_placed(k_nxt, nsm_nxt);
                if (ok && nsm_nxt) start(k_nxt, nsm_nxt);
            }
            k_cur = k_nxt;
            nsm_cur = nsm_nxt;
        }
        if (!ok && lane == 0 && !*abort_flag) {
            sh.abort_flag = 1;
            ++w_to;
        }
        // copies still in flight land before the block can exit
        asm volatile("cp.async.wait_all;" ::: "memory");
        const long long w_props = warp_sum(l_props);
        if (lane == 0) {
            atomic_add_ll(&sh.stat[0], w_evals);
            atomic_add_ll(&sh.stat[1], w_gathered);
            atomic_add_ll(&sh.stat[2], w_props);
            atomic_add_ll(&sh.stat[3], w_ins);
            atomic_add_ll(&sh.stat[4], w_ovf);
        }
    }
    if (lane == 0 && w_to) atomic_add_ll(&sh.stat[5], w_to);
    __syncthreads();
    if (threadIdx.x == 0) {
        long long *its = st.it_stats + (size_t)li * kItCount;
        its[kItRan] = 1;
        atomic_add_ll(&its[kItEvals], sh.stat[0]);
        atomic_add_ll(&its[kItGathered], sh.stat[1]);
        atomic_add_ll(&its[kItProposals], sh.stat[2]);
        atomic_add_ll(&its[kItInserts], sh.stat[3]);
        atomic_add_ll(&st.stats[kStatEvals], sh.stat[0]);
        atomic_add_ll(&st.stats[kStatGathered], sh.stat[1]);
        atomic_add_ll(&st.stats[kStatInserts], sh.stat[3]);
        if (sh.stat[4]) atomic_add_ll(&st.stats[kStatBucketOverflow], sh.stat[4]);
        if (sh.stat[5]) atomic_add_ll(&st.stats[kStatLockTimeout], sh.stat[5]);
    }
}

bool ring_join_fits(int bf16, int nv, int dpb, int K) {
    (void)K;
    const Geometry g = geometry(bf16, nv, dpb);
    return slot_a_bytes(kSetMax, g) <= kRingBytes - ring_b_bytes(g);
}

bool ring_join_preferred(int bf16, int nv, int dpb) {
    // enough ring for four nodes of 24 candidates: below that the rows of a
    // few nodes fill the ring and the block-per-node tile kernel does better
    const Geometry g = geometry(bf16, nv, dpb);
    return 4u * slot_a_bytes(24, g) <= kRingBytes - ring_b_bytes(g);
}

size_t set_kernel_smem(int cap) {
    const int raw_max = ((2 * cap + 31) / 32) * 32;
    return sizeof(int) * (size_t)kSetWarps * (raw_max + (1 << hash_bits(cap)) + kSetMax);
}

namespace {
template <int kKind>
cudaError_t launch_ring_t(const DevState &st, int li, cudaStream_t s) {
    auto kern = ring_join_kernel<kKind>;
    constexpr uint32_t dyn = kRingBytes;
    cudaError_t e = smem_opt_in((const void *)kern, dyn);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    kern<<<sms, kRingThreads, dyn, s>>>(st, li);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_set_kernel(const DevState &st, int li, cudaStream_t s) {
    const size_t dyn = set_kernel_smem(st.cap);
    // the narrow form (reverse capacity <= 96, 256-slot hash set) keeps the
    // registers of the usual K <= 32 builds
    if (st.R > 96 || hash_bits(st.cap) > kHashBits) {
        const int grid = grid_for((const void *)set_kernel<1>, kSetWarps * 32, dyn);
        set_kernel<1><<<grid, kSetWarps * 32, dyn, s>>>(st, li);
        return cudaGetLastError();
    }
    const int grid = grid_for((const void *)set_kernel<0>, kSetWarps * 32, dyn);
    set_kernel<0><<<grid, kSetWarps * 32, dyn, s>>>(st, li);
    return cudaGetLastError();
}

cudaError_t launch_ring_join(const DevState &st, int li, cudaStream_t s) {
    cudaError_t e = st.u_lo == 0 ? launch_set_kernel(st, li, s) : cudaSuccess;
    if (e != cudaSuccess) return e;
    if (st.fp8) return launch_ring_t<2>(st, li, s);
    return st.bf16 ? launch_ring_t<1>(st, li, s) : launch_ring_t<0>(st, li, s);
}

}  // namespace knng
