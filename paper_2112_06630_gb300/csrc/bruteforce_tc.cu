// bruteforce_tc.cu -- exact K-NNG rows (Section 2) with the distance block on
// the tensor cores: a bf16 Gram prefilter in TMEM, then an exact float32
// re-rank with a proven error bound, falling back to the CUDA-core kernel for
// any query the bound cannot certify.
//
// Prefilter (bf_tc_kernel, one CTA per 128 queries and one slice of the
// points): the points are centred on a sampled mean (distances do not change,
// the error bound shrinks) and every point x and query q is split into two
// bf16 terms (x = xh + xl + r, |r| <= 2^-16 |x| per element); q.x is taken as
// qh.xh + qh.xl + ql.xh on the tensor cores (tcgen05.mma, M=128 queries x
// N=128 points, K=16, float32 accumulate in tensor memory).  Operand tiles
// arrive by TMA (cp.async.bulk.tensor): rows of more than 32 floats as 2-d
// boxes of whole 128-byte rows with the 128-byte swizzle (SWIZZLE_128B
// descriptors, 1 KB between 8-row groups, +32 B per k-step inside a 64-column
// block); narrower rows in the no-swizzle K-major core-matrix layout (8 rows
// x 16 bytes per core matrix, K-direction stride 128 B, 8-row-group stride
// dpb * 16 B).  Warp 0 issues the loads, warp 1 the MMAs into two
// alternating TMEM accumulators, warps 4..11 (two per TMEM subpartition, 64
// columns each) turn a finished tile into approximate distances
// D' = |q|^2 + |x|^2 - 2 q.x and keep the 32 smallest per query in registers,
// testing a whole tile at once through the minimum of its 64 values.
// Re-rank (bf_rerank_kernel, one warp per query): the kept lists are merged
// to their 64 smallest D', which get the canonical float32 difference-form
// distance; the K smallest by (dist, id) are the answer if every point
// outside those 64 provably has a larger distance: D'(y) >= T (the smallest
// "worst kept" value of the full lists, or the 64th merged one), and
// |D' - D| <= E(q), so D(y) >= T - E(q) must exceed the K-th distance.
// Otherwise the query is listed for the exact kernel.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"
#include "join_common.cuh"

namespace knng {

namespace {
constexpr int kTcRows = 128;                  // queries per CTA, points per tile
constexpr int kTcStages = 2;                  // point-tile stages
constexpr int kTcThreads = 384;               // 12 warps: loader, MMA, 2 idle, 8 epilogue
constexpr unsigned long long kTcWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t c) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(c) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t *b) {
    asm volatile("{\n\t.reg .b64 s;\n\tmbarrier.arrive.shared::cta.b64 s, [%0];\n\t}" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t *b, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 s;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 s, [%0], %1;\n\t}" ::"r"(su32(b)),
                 "r"(bytes)
                 : "memory");
}
// bounded wait for the phase of the given parity; false when it gave up
__device__ __forceinline__ bool bar_try(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t parity, volatile int *abort_flag) {
    if (bar_try(b, parity)) return true;
    const unsigned long long t0 = gns();
    for (;;) {
        if (bar_try(b, parity)) return true;
        if (*abort_flag || gns() - t0 > kTcWaitNs) return false;
    }
}
// 4-d tile load (coordinates kk, r, c, g) into shared memory, completion in bytes
__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *map, int g, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(0), "r"(0), "r"(g), "r"(su32(bar))
        : "memory");
}
// 2-d tile load (coordinates x = column, y = row) into shared memory
__device__ __forceinline__ void tma_load2(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}
// shared-memory matrix descriptor, 128-byte swizzle, K-major: rows of 128 B,
// 8-row groups 1,024 B apart (LBO unused); a k-step inside the 64-element
// swizzle atom advances the start address by 32 B
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}
// shared-memory matrix descriptor: no swizzle, K-direction core stride lbo,
// 8-row-group stride sbo
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// instruction descriptor: bf16 x bf16 -> f32, both K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, bool acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc ? 1 : 0)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
// 32 consecutive columns of this warp's 32 lanes; tmem_wait() before use
__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(addr));
}
// three-input minimum (sm_100 and later)
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

struct TcShared {
    uint64_t a_full, b_full[kTcStages], b_empty[kTcStages], t_full[2], t_empty[2];
    uint32_t tmem;
    int abort_flag;
};
}  // namespace

// Centre mu: the mean of up to 4096 evenly spaced rows, zero past column d.
// Distances do not change under a translation, but the error bound on the
// Gram prefilter scales with the norms, which centring shrinks for data with
// a common offset (non-negative features, for instance).  Block b sums the
// sample rows b, b + 32, ... of column threadIdx.x (float64) into
// psum[b][col]; bf_mean_final adds the 32 partial sums in a fixed order.
constexpr int kTcMeanBlocks = 32;
__global__ void bf_mean_kernel(const float *__restrict__ X, int dp, int d, int64_t n, double *__restrict__ psum) {
    const int t = threadIdx.x;
    const int64_t m = n < 4096 ? n : 4096;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (t < d) {
        int64_t i = blockIdx.x;
        for (; i + 3 * kTcMeanBlocks < m; i += 4 * kTcMeanBlocks) {
            a0 += (double)X[(size_t)(i * n / m) * dp + t];
            a1 += (double)X[(size_t)((i + kTcMeanBlocks) * n / m) * dp + t];
            a2 += (double)X[(size_t)((i + 2 * kTcMeanBlocks) * n / m) * dp + t];
            a3 += (double)X[(size_t)((i + 3 * kTcMeanBlocks) * n / m) * dp + t];
        }
        for (; i < m; i += kTcMeanBlocks) a0 += (double)X[(size_t)(i * n / m) * dp + t];
    }
    psum[blockIdx.x * 128 + t] = (a0 + a1) + (a2 + a3);
}
__global__ void bf_mean_final(const double *__restrict__ psum, int d, int64_t n, float *__restrict__ mu) {
    const int t = threadIdx.x;
    const int64_t m = n < 4096 ? n : 4096;
    double acc = 0.0;
    for (int b = 0; b < kTcMeanBlocks; ++b) acc += psum[b * 128 + t];
    mu[t] = t < d ? (float)(acc / (double)m) : 0.f;
}

// Split of n rows (padded to rows_pad with zeros) of X - mu (dp floats per
// row, rows selected by `rows` when not null) into bf16 hi/lo terms in dpb
// columns, and the float32 squared norms of the centred rows (float64
// accumulation); the largest norm goes to *nmax (float bits, non-negative,
// so integer max orders them).
__global__ void bf_split_kernel(const float *__restrict__ X, int dp, int d, const int64_t *__restrict__ rows,
                                const float *__restrict__ mu, int64_t n, int64_t rows_pad, int dpb,
                                uint16_t *__restrict__ hi, uint16_t *__restrict__ lo, float *__restrict__ nrm,
                                unsigned *__restrict__ nmax) {
    const unsigned lane = lane_id();
    for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows_pad;
         r += ((long long)gridDim.x * blockDim.x) >> 5) {
        const bool live = r < n;
        const int64_t src = live ? (rows ? rows[r] : r) : 0;
        double acc = 0.0;
        for (int t = lane; t < dpb; t += 32) {
            const float v = live && t < d ? X[(size_t)src * dp + t] - mu[t] : 0.f;
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
            hi[(size_t)r * dpb + t] = __bfloat16_as_ushort(h);
            lo[(size_t)r * dpb + t] = __bfloat16_as_ushort(l);
            acc += (double)v * (double)v;
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            const float f = (float)acc;
            if (live) nrm[r] = f;
            if (live && nmax) atomicMax(nmax, __float_as_uint(f));
        }
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
    bf_tc_kernel(const __grid_constant__ CUtensorMap mqh, const __grid_constant__ CUtensorMap mql,
                 const __grid_constant__ CUtensorMap mxh, const __grid_constant__ CUtensorMap mxl,
                 const float *__restrict__ qn, const float *__restrict__ xn, const int64_t *__restrict__ qrow,
                 int64_t nq, int64_t n, int dpb, int sw, int64_t tiles_per_slice, uint64_t *__restrict__ part,
                 int *__restrict__ err) {
    __shared__ TcShared sh;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-aligned operand region: Qh | Ql | stages x (Xh | Xl)
    unsigned char *base = smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023);
    const uint32_t tile_bytes = (uint32_t)kTcRows * dpb * 2;
    unsigned char *sqh = base, *sql = base + tile_bytes;
    auto sxh = [&](int s) { return base + (2 + 2 * s) * tile_bytes; };
    auto sxl = [&](int s) { return base + (3 + 2 * s) * tile_bytes; };
    const int warp = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    volatile int *abort_flag = &sh.abort_flag;
    const int64_t ntiles = (n + kTcRows - 1) / kTcRows;
    const int64_t t0 = (int64_t)blockIdx.y * tiles_per_slice;
    const int64_t t1 = t0 + tiles_per_slice < ntiles ? t0 + tiles_per_slice : ntiles;
    const int64_t q0 = (int64_t)blockIdx.x * kTcRows;
    if (threadIdx.x == 0) {
        bar_init(&sh.a_full, 1);
        for (int s = 0; s < kTcStages; ++s) {
            bar_init(&sh.b_full[s], 1);
            bar_init(&sh.b_empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            bar_init(&sh.t_full[a], 1);
            bar_init(&sh.t_empty[a], 8);
        }
        sh.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(su32(&sh.tmem)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sh.tmem;
    const uint32_t lbo = 128, sbo = (uint32_t)dpb * 16;

    if (warp == 0) {
        // ---- loader
        if (lane == 0) {
            // an operand tile: one 4-d core-matrix box, or (128-byte swizzle)
            // one 128-row x 64-column box per 16 KB block
            auto load_tile = [&](unsigned char *dst, const CUtensorMap *m, int64_t row0, uint64_t *bar) {
                if (sw) {
                    for (int b = 0; b < dpb / 64; ++b) tma_load2(dst + b * 16384, m, b * 64, (int)row0, bar);
                } else {
                    tma_load(dst, m, (int)(row0 / 8), bar);
                }
            };
            bar_expect(&sh.a_full, 2 * tile_bytes);
            load_tile(sqh, &mqh, q0, &sh.a_full);
            load_tile(sql, &mql, q0, &sh.a_full);
            int64_t issued = 0;
            for (int64_t t = t0; t < t1; ++t) {
                const int64_t it = t - t0;
                const int s = (int)(it % kTcStages);
                if (!bar_wait(&sh.b_empty[s], (uint32_t)(((it / kTcStages) & 1) ^ 1), abort_flag)) {
                    sh.abort_flag = 1;
                    break;
                }
                bar_expect(&sh.b_full[s], 2 * tile_bytes);
                load_tile(sxh(s), &mxh, t * kTcRows, &sh.b_full[s]);
                load_tile(sxl(s), &mxl, t * kTcRows, &sh.b_full[s]);
                ++issued;
            }
            // the copies this warp issued land before the block can exit
            volatile int never = 0;
            bar_wait(&sh.a_full, 0, &never);
            for (int64_t it = issued - kTcStages < 0 ? 0 : issued - kTcStages; it < issued; ++it)
                bar_wait(&sh.b_full[it % kTcStages], (uint32_t)((it / kTcStages) & 1), &never);
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            bool ok = bar_wait(&sh.a_full, 0, abort_flag);
            int64_t done = 0;
            for (int64_t t = t0; t < t1 && ok; ++t) {
                const int64_t it = t - t0;
                const int s = (int)(it % kTcStages), a = (int)(it & 1);
                ok = bar_wait(&sh.b_full[s], (uint32_t)((it / kTcStages) & 1), abort_flag) &&
                     bar_wait(&sh.t_empty[a], (uint32_t)(((it >> 1) & 1) ^ 1), abort_flag);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)a * 128;
                const uint32_t qh = su32(sqh), ql = su32(sql), xh = su32(sxh(s)), xl = su32(sxl(s));
                for (int k = 0; k < dpb / 16; ++k) {
                    if (sw) {
                        // 64-column block k / 4, k-step k % 4 inside its swizzle atom
                        const uint32_t off = (uint32_t)(k >> 2) * 16384 + (uint32_t)(k & 3) * 32;
                        mma(d, smem_desc_sw128(qh + off), smem_desc_sw128(xh + off), k > 0);
                        mma(d, smem_desc_sw128(qh + off), smem_desc_sw128(xl + off), true);
                        mma(d, smem_desc_sw128(ql + off), smem_desc_sw128(xh + off), true);
                    } else {
                        const uint32_t off = (uint32_t)k * 256;  // two K-direction core matrices
                        mma(d, smem_desc(qh + off, lbo, sbo), smem_desc(xh + off, lbo, sbo), k > 0);
                        mma(d, smem_desc(qh + off, lbo, sbo), smem_desc(xl + off, lbo, sbo), true);
                        mma(d, smem_desc(ql + off, lbo, sbo), smem_desc(xh + off, lbo, sbo), true);
                    }
                }
                mma_commit(&sh.b_empty[s]);
                mma_commit(&sh.t_full[a]);
                ++done;
            }
            if (!ok) sh.abort_flag = 1;
            // the last tile's MMAs finish before the tensor memory is freed
            if (done) {
                volatile int never = 0;
                bar_wait(&sh.t_full[(done - 1) & 1], (uint32_t)(((done - 1) >> 1) & 1), &never);
            }
        }
    } else if (warp >= 4) {
        // ---- epilogue: rows 32 * (warp % 4) .. + 32, columns 64 * h .. + 64
        const int sub = warp & 3, h = (warp - 4) >> 2;
        const int64_t q = q0 + sub * 32 + (int)lane;
        const bool live = q < nq;
        const int64_t self = live ? (qrow ? qrow[q] : q) : -1;
        const float qnorm = live ? qn[q] : 0.f;
        uint64_t L[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) L[k] = kKeyEmpty;
        float thr = INFINITY;  // distance of L[31]: every candidate passes until the list is full
        bool ok = true;
        // the 64 columns' squared norms, one per lane and half, loaded a tile ahead
        auto norms = [&](int64_t t, float &xa, float &xb) {
            const int64_t c = t * kTcRows + h * 64 + lane;
            xa = t < t1 && c < n ? __ldg(xn + c) : 0.f;
            xb = t < t1 && c + 32 < n ? __ldg(xn + c + 32) : 0.f;
        };
        float na, nb;
        norms(t0, na, nb);
        for (int64_t t = t0; t < t1; ++t) {
            const int64_t it = t - t0;
            const int a = (int)(it & 1);
            ok = __all_sync(kFull, bar_wait(&sh.t_full[a], (uint32_t)((it >> 1) & 1), abort_flag));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t v0[32], v1[32];
            const uint32_t addr = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)a * 128 + (uint32_t)h * 64;
            tmem_ld32(addr, v0);
            tmem_ld32(addr + 32, v1);
            tmem_wait();
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) bar_arrive(&sh.t_empty[a]);
            const int64_t c0 = t * kTcRows + h * 64;
            const float xa = na, xb = nb;
            norms(t + 1, na, nb);
            // pass 1 (straight-line): the unclamped D' of all 64 columns and
            // their minimum.  Rounding is monotone and thr >= 0, so some
            // column has max(0, D') <= thr exactly when the minimum does; only
            // then is the tile scanned again column by column, with one copy
            // of the insertion network
            float lo = INFINITY;
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
                const float e0 = qnorm + __shfl_sync(kFull, xa, j) - 2.f * __uint_as_float(v0[j]);
                const float e1 = qnorm + __shfl_sync(kFull, xa, j + 1) - 2.f * __uint_as_float(v0[j + 1]);
                v0[j] = __float_as_uint(e0);
                v0[j + 1] = __float_as_uint(e1);
                lo = fmin3(lo, e0, e1);
            }
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
                const float e0 = qnorm + __shfl_sync(kFull, xb, j) - 2.f * __uint_as_float(v1[j]);
                const float e1 = qnorm + __shfl_sync(kFull, xb, j + 1) - 2.f * __uint_as_float(v1[j + 1]);
                v1[j] = __float_as_uint(e0);
                v1[j + 1] = __float_as_uint(e1);
                lo = fmin3(lo, e0, e1);
            }
            if (lo <= thr) {
                // existing columns other than the query itself
                const int64_t nval = n - c0;
                uint64_t m = nval >= 64 ? ~0ull : (nval <= 0 ? 0ull : (1ull << nval) - 1);
                if (self >= c0 && self < c0 + 64) m &= ~(1ull << (self - c0));
                uint32_t m0 = 0, m1 = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    v0[j] = __float_as_uint(fmaxf(0.f, __uint_as_float(v0[j])));
                    v1[j] = __float_as_uint(fmaxf(0.f, __uint_as_float(v1[j])));
                    m0 |= (__uint_as_float(v0[j]) <= thr ? 1u : 0u) << j;
                    m1 |= (__uint_as_float(v1[j]) <= thr ? 1u : 0u) << j;
                }
                m &= (uint64_t)m1 << 32 | m0;
                uint32_t buf[64];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    buf[j] = v0[j];
                    buf[32 + j] = v1[j];
                }
                for (; m; m &= m - 1) {
                    const int j = __ffsll((long long)m) - 1;
                    const uint64_t x = make_key(__uint_as_float(buf[j]), (uint32_t)(c0 + j), 1u);
                    if (x < L[31]) {
#pragma unroll
                        for (int k = 31; k >= 1; --k) {
                            const uint64_t mn = L[k] < x ? L[k] : x;
                            L[k] = mn > L[k - 1] ? mn : L[k - 1];
                        }
                        L[0] = L[0] < x ? L[0] : x;
                    }
                }
                if (L[31] != kKeyEmpty) thr = key_dist(L[31]);
            }
        }
        if (!ok) sh.abort_flag = 1;
        if (live) {
            uint64_t *dst = part + (((size_t)q * gridDim.y + blockIdx.y) * 2 + h) * 32;
#pragma unroll
            for (int k = 0; k < 32; ++k) dst[k] = L[k];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
    if (threadIdx.x == 0 && sh.abort_flag) atomicAdd(err, 1);
}

// Compare-exchange of a key with the one in lane ^ j: ascending runs keep
// the smaller key in the lower lane.
__device__ __forceinline__ uint64_t bf_cx(uint64_t v, int j, bool up, unsigned lane) {
    const uint64_t o = __shfl_xor_sync(kFull, v, j);
    const bool low = !(lane & j);
    return (low == up) ? (v < o ? v : o) : (v < o ? o : v);
}
// Ascending order of a bitonic 64-key sequence held as a (entries lane) and
// b (entries 32 + lane).
__device__ __forceinline__ void bf_merge64(uint64_t &a, uint64_t &b, unsigned lane) {
    const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        a = bf_cx(a, j, true, lane);
        b = bf_cx(b, j, true, lane);
    }
}
// Ascending bitonic sort of 64 keys (a: entries lane, b: entries 32 + lane).
__device__ __forceinline__ void bf_sort64(uint64_t &a, uint64_t &b, unsigned lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            a = bf_cx(a, j, !(lane & k), lane);
            b = bf_cx(b, j, k == 32 ? false : !(lane & k), lane);
        }
    bf_merge64(a, b, lane);
}

// One warp per query: the 64 smallest approximate keys of all kept lists
// (bitonic merges), their exact canonical distances, the K smallest by
// (dist, id), and the completeness check; queries that fail it are appended
// to `redo`.
__global__ void __launch_bounds__(256) bf_rerank_kernel(const float4 *__restrict__ X4, int nv, int d,
                                                        const int64_t *__restrict__ qrow, int64_t nq, int K,
                                                        int lists, const uint64_t *__restrict__ part,
                                                        const float *__restrict__ qn, const unsigned *nmax,
                                                        int32_t *__restrict__ ids, float *__restrict__ dists,
                                                        int64_t *__restrict__ redo, int *__restrict__ nredo) {
    const unsigned lane = lane_id();
    const float xmax = sqrtf(__uint_as_float(*nmax));
    // squared norms this large could overflow D' to +inf: nothing is certified
    const bool huge = __uint_as_float(*nmax) >= 1.2676506e30f;  // 2^100
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq;
         q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t self = qrow ? qrow[q] : q;
        const float4 *own = X4 + (size_t)self * nv;
        uint64_t A = kKeyEmpty, B = kKeyEmpty;  // 64 smallest approximate keys so far, ascending
        float tau = INFINITY;                   // no point outside the kept lists has D' below this
        for (int l = 0; l < lists; ++l) {
            const uint64_t x = part[((size_t)q * lists + l) * 32 + lane];
            const uint64_t worst = __shfl_sync(kFull, x, 31);
            if (worst != kKeyEmpty) tau = fminf(tau, key_dist(worst));
            if (__shfl_sync(kFull, x, 0) >= __shfl_sync(kFull, B, 31)) continue;
            // the 64 smallest of (A, B) and the sorted list x: A, then the
            // element-wise minimum of B and x reversed (a bitonic sequence)
            const uint64_t xr = __shfl_sync(kFull, x, 31 - lane);
            B = B < xr ? B : xr;
            bf_merge64(A, B, lane);
        }
        // every point outside the merged 64 has D' >= T
        const uint64_t last = __shfl_sync(kFull, B, 31);
        const float T = last == kKeyEmpty ? tau : fminf(tau, key_dist(last));
        uint64_t ea = kKeyEmpty, eb = kKeyEmpty;
        if (A != kKeyEmpty) ea = make_key(l2sq_rows(own, X4 + (size_t)key_id(A) * nv, nv), key_id(A), 0u);
        if (B != kKeyEmpty) eb = make_key(l2sq_rows(own, X4 + (size_t)key_id(B) * nv, nv), key_id(B), 0u);
        bf_sort64(ea, eb, lane);
        // |D' - D| <= E, with |q|, |x| the centred norms: the split residuals
        // and dropped lo.lo term (3.1 x 2^-16) and the float32 accumulation of
        // 3d products (3d x 2^-24), both on 2 q.x; the float32 evaluation of
        // D' (2^-22 (|q|+|x|)^2) and the rounding of the centring subtraction
        // (2^-23 (|q|+|x|)^2), taken together as 2^-21 (|q|+|x|)^2; doubled
        // for safety
        const float qa = sqrtf(qn[q]);
        const float dot_rel = 3.1f * 1.52587890625e-5f + 3.0f * (float)d * 5.9604645e-8f;
        const float E = 2.f * (2.f * dot_rel * qa * xmax + 4.768371582e-7f * (qa + xmax) * (qa + xmax));
        const float dk = key_dist(__shfl_sync(kFull, ea, K - 1));
        const bool ok = !huge && (T - E) * (1.f - 4.f * (float)d * 5.9604645e-8f) > dk;
        if ((int)lane < K) {
            ids[(size_t)q * K + lane] = (int32_t)key_id(ea);
            dists[(size_t)q * K + lane] = key_dist(ea);
        }
        if (!ok && lane == 0) redo[atomicAdd(nredo, 1)] = q;
    }
}

// Results of the exact kernel for the listed queries back into place.
__global__ void bf_scatter_kernel(const int64_t *__restrict__ redo, int nredo, int K, const int32_t *__restrict__ ri,
                                  const float *__restrict__ rd, int32_t *__restrict__ ids,
                                  float *__restrict__ dists) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nredo * K;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / K, k = e - r * K;
        ids[(size_t)redo[r] * K + k] = ri[e];
        dists[(size_t)redo[r] * K + k] = rd[e];
    }
}

// ------------------------------------------------------------------ host --
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}
// rows x dpb bf16 (rows a multiple of 128) as the 4-d tensor (kk 8, r 8, c dpb/8,
// g rows/8) with byte strides (r: dpb*2, c: 16, g: 8*dpb*2): a box of
// (8, 8, dpb/8, 16) lands as [g][c][r][kk], the canonical core-matrix order
bool encode_map(CUtensorMap *m, const void *base, int64_t rows, int dpb, bool sw) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    if (sw) {
        // rows x dpb bf16 as a 2-d tensor; a 64 x 128 box lands as 128 rows of
        // 128 B with the 128-byte swizzle (16-byte chunk c of row r at c ^ (r % 8))
        const cuuint64_t dims2[2] = {(cuuint64_t)dpb, (cuuint64_t)rows};
        const cuuint64_t strides2[1] = {(cuuint64_t)dpb * 2};
        const cuuint32_t box2[2] = {64, kTcRows};
        const cuuint32_t es2[2] = {1, 1};
        return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims2, strides2, box2, es2,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    const cuuint64_t dims[4] = {8, 8, (cuuint64_t)dpb / 8, (cuuint64_t)rows / 8};
    const cuuint64_t strides[3] = {(cuuint64_t)dpb * 2, 16, (cuuint64_t)dpb * 16};
    const cuuint32_t box[4] = {8, 8, (cuuint32_t)dpb / 8, kTcRows / 8};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// operand width: rows of more than 32 floats take the 128-byte-swizzle layout
// (whole 64-column blocks), narrower rows the core-matrix layout (16 columns)
bool tc_swizzled(int dp) { return dp > 32; }
int tc_dpb(int dp) { return tc_swizzled(dp) ? (dp + 63) & ~63 : (dp + 15) & ~15; }
}  // namespace

size_t bruteforce_tc_scratch(int64_t n, int64_t nq, int dp, int K, int *slices_out) {
    const int dpb = tc_dpb(dp);
    const int64_t npad = (n + kTcRows - 1) / kTcRows * kTcRows, qpad = (nq + kTcRows - 1) / kTcRows * kTcRows;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t qtiles = qpad / kTcRows, ntiles = npad / kTcRows;
    // point slices per query tile: the fewest that fill 90% of the last wave
    // of one-CTA-per-SM launches (else the best fill), at most 64 and at
    // least 4 tiles a slice
    int64_t S = 1, smax = ntiles / 4 < 64 ? ntiles / 4 : 64;
    double best = -1.0;
    for (int64_t c = 1; c <= (smax > 1 ? smax : 1); ++c) {
        const int64_t ctas = qtiles * c, waves = (ctas + sms - 1) / sms;
        const double fill = (double)ctas / (double)(waves * sms);
        if (fill > best + 1e-9) {
            best = fill;
            S = c;
        }
        if (fill >= 0.9) break;
    }
    *slices_out = (int)S;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return al(2 * (size_t)npad * dpb * 2) + al(2 * (size_t)qpad * dpb * 2) + al((size_t)npad * 4) +
           al((size_t)qpad * 4) + al((size_t)nq * S * 2 * 32 * 8) + al((size_t)nq * 8) + al(16) + al(128 * 4) +
           al(kTcMeanBlocks * 128 * 8) +
           al((size_t)nq * K * 8);
}

bool bruteforce_tc_supported(int dp) { return tc_dpb(dp) <= 128 && encode_fn() != nullptr; }

namespace {
// CUDA events around the prefilter launch, per thread, made on first use on
// each device (the call waits for its stream anyway, so reading them is free)
struct PrefilterEvents {
    int dev = -1;
    cudaEvent_t a = nullptr, b = nullptr;
};
thread_local PrefilterEvents g_pf_events;
}  // namespace

// nredo_host: the number of queries the exact kernel redid; prefilter_ms:
// the prefilter kernel's CUDA-event time (statistics)
cudaError_t launch_bruteforce_tc(const float *X, int64_t n, int dp, int d, int K, const int64_t *rows, int64_t nq,
                                 int32_t *ids, float *dists, cudaStream_t s, unsigned char *scratch, int S,
                                 int *nredo_host, float *prefilter_ms) {
    const int dpb = tc_dpb(dp);
    const bool sw = tc_swizzled(dp);
    const int64_t npad = (n + kTcRows - 1) / kTcRows * kTcRows, qpad = (nq + kTcRows - 1) / kTcRows * kTcRows;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    unsigned char *p = scratch;
    uint16_t *xh = (uint16_t *)p, *xl = xh + (size_t)npad * dpb;
    p += al(2 * (size_t)npad * dpb * 2);
    uint16_t *qh = (uint16_t *)p, *ql = qh + (size_t)qpad * dpb;
    p += al(2 * (size_t)qpad * dpb * 2);
    float *xn = (float *)p;
    p += al((size_t)npad * 4);
    float *qn = (float *)p;
    p += al((size_t)qpad * 4);
    uint64_t *part = (uint64_t *)p;
    p += al((size_t)nq * S * 2 * 32 * 8);
    int64_t *redo = (int64_t *)p;
    p += al((size_t)nq * 8);
    int *counters = (int *)p;  // [0] redo count, [1] kernel give-ups, [2] norm max bits
    p += al(16);
    float *mu = (float *)p;
    p += al(128 * 4);
    double *psum = (double *)p;
    p += al(kTcMeanBlocks * 128 * 8);
    int32_t *ri = (int32_t *)p;
    float *rd = (float *)(ri + (size_t)nq * K);

    cudaError_t e = cudaMemsetAsync(counters, 0, 16, s);
    if (e != cudaSuccess) return e;
    const int gs = grid_for((const void *)bf_split_kernel, 256, 0);
    bf_mean_kernel<<<kTcMeanBlocks, 128, 0, s>>>(X, dp, d, n, psum);
    bf_mean_final<<<1, 128, 0, s>>>(psum, d, n, mu);
    bf_split_kernel<<<gs, 256, 0, s>>>(X, dp, d, nullptr, mu, n, npad, dpb, xh, xl, xn,
                                       (unsigned *)(counters + 2));
    bf_split_kernel<<<gs, 256, 0, s>>>(X, dp, d, rows, mu, nq, qpad, dpb, qh, ql, qn, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    CUtensorMap mqh, mql, mxh, mxl;
    if (!encode_map(&mqh, qh, qpad, dpb, sw) || !encode_map(&mql, ql, qpad, dpb, sw) ||
        !encode_map(&mxh, xh, npad, dpb, sw) || !encode_map(&mxl, xl, npad, dpb, sw))
        return cudaErrorNotSupported;
    const size_t dyn = 1024 + (size_t)(2 + 2 * kTcStages) * kTcRows * dpb * 2;
    if ((e = smem_opt_in((const void *)bf_tc_kernel, dyn)) != cudaSuccess) return e;
    const int64_t ntiles = npad / kTcRows, per = (ntiles + S - 1) / S;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    PrefilterEvents &ev = g_pf_events;
    if (ev.dev != dev) {
        if ((e = cudaEventCreate(&ev.a)) != cudaSuccess || (e = cudaEventCreate(&ev.b)) != cudaSuccess) return e;
        ev.dev = dev;
    }
    if ((e = cudaEventRecord(ev.a, s)) != cudaSuccess) return e;
    bf_tc_kernel<<<dim3((unsigned)(qpad / kTcRows), (unsigned)S), kTcThreads, dyn, s>>>(
        mqh, mql, mxh, mxl, qn, xn, rows, nq, n, dpb, sw ? 1 : 0, per, part, counters + 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ev.b, s)) != cudaSuccess) return e;
    const int gr = grid_for((const void *)bf_rerank_kernel, 256, 0);
    bf_rerank_kernel<<<gr, 256, 0, s>>>(reinterpret_cast<const float4 *>(X), dp / 4, d, rows, nq, K, 2 * S, part, qn,
                                       (const unsigned *)(counters + 2), ids, dists, redo, counters);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int hc[2] = {0, 0};
    if ((e = cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (prefilter_ms && cudaEventElapsedTime(prefilter_ms, ev.a, ev.b) != cudaSuccess) *prefilter_ms = -1.f;
    if (hc[1]) return cudaErrorLaunchTimeout;  // a bounded wait gave up
    if (nredo_host) *nredo_host = hc[0];
    if (hc[0] == 0) return cudaSuccess;
    // the exact kernel for the queries the bound could not certify
    std::vector<int64_t> redo_h(hc[0]);
    std::vector<int64_t> rows_h(hc[0]);
    if ((e = cudaMemcpyAsync(redo_h.data(), redo, sizeof(int64_t) * hc[0], cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    std::vector<int64_t> src(rows ? hc[0] : 0);
    if (rows) {
        // query q's point id
        std::vector<int64_t> allrows(nq);
        if ((e = cudaMemcpyAsync(allrows.data(), rows, sizeof(int64_t) * nq, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        for (int i = 0; i < hc[0]; ++i) rows_h[i] = allrows[redo_h[i]];
    } else {
        rows_h = redo_h;
    }
    int64_t *rows_d = redo;  // reuse: the listed queries' point ids, then the listed query indices
    int64_t *qidx_d = (int64_t *)part;
    if ((e = cudaMemcpyAsync(qidx_d, redo_h.data(), sizeof(int64_t) * hc[0], cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(rows_d, rows_h.data(), sizeof(int64_t) * hc[0], cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return e;
    // point slices for the exact kernel, their partial lists in the (now
    // unused) bf16 split of the points
    const size_t avail = al(2 * (size_t)npad * dpb * 2);
    int bs = bruteforce_slices(n, hc[0]);
    while (bs > 1 && (size_t)hc[0] * bs * K * sizeof(uint64_t) > avail) --bs;
    if ((e = launch_bruteforce(X, n, dp, K, rows_d, hc[0], ri, rd, s, bs > 1 ? (uint64_t *)xh : nullptr, bs)) !=
        cudaSuccess)
        return e;
    bf_scatter_kernel<<<grid_for((const void *)bf_scatter_kernel, 256, 0), 256, 0, s>>>(qidx_d, hc[0], K, ri, rd,
                                                                                      ids, dists);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace knng
