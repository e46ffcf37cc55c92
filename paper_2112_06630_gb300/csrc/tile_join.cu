// tile_join.cu -- the local join for high-dimensional points (the paper's
// Calculation step, Section 2 and Section 3.3), one 128-thread block per node.
//
// The distance block of a node's candidate set S (|S| <= 64, new ones first)
// is computed into shared memory as D[i][j] for every new row i and every
// column j.  Candidate rows stream through shared memory in chunks (32
// floats, or 64 bf16), double-buffered with cp.async.
//   - float32: one item = one new row and four columns, spread evenly over
//     the block (only the pairs the node needs), accumulating the canonical
//     difference form (two partial sums over t mod 2, ascending t, fused
//     multiply-add), so every value is bit-identical to the warp kernel and to
//     the rest of the library.  Rows are read by broadcast (i) and by 8-thread
//     phases on an odd float4 stride (j): no bank conflicts.
//   - bf16: the Gram block x_i . x_j on the tensor cores (mma.sync
//     m16n8k16, bf16 in, float32 accumulate; ldmatrix on a 144-byte row
//     stride), then d = |x_i|^2 + |x_j|^2 - 2 x_i . x_j with the norms of the
//     bf16 values, clamped at 0.  Lists built this way are re-ranked with the
//     float32 difference form at output.
// Then: every join pair once sets proposal-mask bits against the snapshot
// worst keys; each target's list is snapshotted in shared memory and the
// proposals it cannot take (not before its worst, or already listed) are
// dropped; one thread per target reserves a bucket run and writes its keys
// from D; full buckets take the locked way.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstdint>

#include "join_common.cuh"

namespace knng {

namespace {
constexpr int kTileThreads = 128;
constexpr int kChunkV = 8;                   // float4 per row chunk (32 floats)
constexpr int kStrideV = kChunkV + 1;        // odd float4 stride
constexpr int kItemsPerThread = 2;           // (new row, 4 columns) items per thread and pass
constexpr int kChunkB = 64;                  // bf16 per row chunk
constexpr int kStrideB = kChunkB + 8;        // 144-byte rows for ldmatrix
constexpr int kDStride = kSetMax + 1;
constexpr int kRawMax = 416;                 // >= 2 * (K + R) for K <= 64, s <= 64

struct TileSmem {
    int sid[kSetMax];
    int raw[kRawMax];
    int hset[1 << kHashBitsMax];
    uint64_t swk[kSetMax];
    unsigned long long mask[kSetMax];
    float nrm[kSetMax];
    float D[kSetMax * kDStride];
    unsigned long long ovf;
    unsigned long long fails[kSetMax];  // proposals that found no bucket slot, per target
    int ns, m;
    long long stat[8];
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// rows of S, chunk c of the padded float32 layout (16 float4), into buf
__device__ __forceinline__ void stage_f32(float4 *buf, const float4 *X4, const int *sid, int ns, int nv, int c) {
    const int v0 = c * kChunkV, vc = min(kChunkV, nv - v0);
    for (int e = threadIdx.x; e < ns * vc; e += kTileThreads) {
        const int r = e / vc, v = e - r * vc;
        cp_async16(buf + r * kStrideV + v, X4 + (size_t)sid[r] * nv + v0 + v);
    }
    cp_async_commit();
}

// rows of S, chunk c of the bf16 layout (64 bf16 = 8 x 16 bytes), into buf
__device__ __forceinline__ void stage_b16(uint16_t *buf, const uint16_t *Xb, const int *sid, int ns, int dpb, int c) {
    for (int e = threadIdx.x; e < ns * 8; e += kTileThreads) {
        const int r = e >> 3, q = e & 7;
        cp_async16(buf + r * kStrideB + q * 8, Xb + (size_t)sid[r] * dpb + (size_t)c * kChunkB + q * 8);
    }
    cp_async_commit();
}

// D[i][j] for every new row i < m and column j < ns, canonical float32 form.
// Work item = one row i and the four columns jq, jq + JQ, jq + 2 JQ, jq + 3 JQ
// (JQ = ceil(ns / 4)); items are spread over the block, up to two per thread
// per pass.  Consecutive threads take consecutive columns, which are distinct
// rows on an odd float4 stride: conflict-free 8-thread phases; row i is read
// by broadcast.
__device__ void tile_dist_f32(TileSmem &sm, float4 *stage, const float4 *X4, int nv, int ns, int m) {
    const int tid = threadIdx.x;
    const int JQ = (ns + 3) >> 2, items = m * JQ;
    const int nchunks = (nv + kChunkV - 1) / kChunkV;
    float4 *buf[2] = {stage, stage + kSetMax * kStrideV};
    for (int it0 = 0; it0 < items; it0 += kTileThreads * kItemsPerThread) {
        Acc2 acc[kItemsPerThread][4];
        int ii[kItemsPerThread], jj[kItemsPerThread];
#pragma unroll
        for (int w = 0; w < kItemsPerThread; ++w) {
            const int item = it0 + w * kTileThreads + tid;
            ii[w] = item < items ? item / JQ : -1;
            jj[w] = item < items ? item - ii[w] * JQ : 0;
        }
        stage_f32(buf[0], X4, sm.sid, ns, nv, 0);
        for (int c = 0; c < nchunks; ++c) {
            if (c + 1 < nchunks) {
                stage_f32(buf[(c + 1) & 1], X4, sm.sid, ns, nv, c + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const float4 *b = buf[c & 1];
            const int vc = min(kChunkV, nv - c * kChunkV);
#pragma unroll
            for (int w = 0; w < kItemsPerThread; ++w) {
                if (ii[w] < 0) continue;
                const float4 *ri = b + ii[w] * kStrideV;
                const float4 *rj = b + jj[w] * kStrideV;
                // unrolled (a chunk is at most 8 units): MNIST-shaped float32
                // build 35.5 -> 32.9 ms
#pragma unroll 8
                for (int v = 0; v < vc; ++v) {
                    const float4 a = ri[v];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[w][q].add(a, rj[q * JQ * kStrideV + v]);
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int w = 0; w < kItemsPerThread; ++w) {
            if (ii[w] < 0) continue;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = jj[w] + q * JQ;
                if (j < ns) sm.D[ii[w] * kDStride + j] = acc[w][q].sum();
            }
        }
    }
}

// D[i][j] for i in [r0, min(r0 + 32, m)), j < ns: bf16 tensor-core Gram block
__device__ void tile_dist_b16(TileSmem &sm, uint16_t *stage, const uint16_t *Xb, int dpb, int ns, int m, int r0) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = warp & 1, nt0 = (warp >> 1) * 4;  // 16-row tile, four 8-column tiles
    float acc[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    const int nchunks = dpb / kChunkB;
    uint16_t *buf[2] = {stage, stage + kSetMax * kStrideB};
    stage_b16(buf[0], Xb, sm.sid, ns, dpb, 0);
    const int arow = r0 + mt * 16 + (lane & 7) + 8 * ((lane >> 3) & 1), acol = 8 * (lane >> 4);
    const int brow = lane & 7, bcol = 8 * ((lane >> 3) & 1);
    for (int c = 0; c < nchunks; ++c) {
        if (c + 1 < nchunks) {
            stage_b16(buf[(c + 1) & 1], Xb, sm.sid, ns, dpb, c + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const uint16_t *b = buf[c & 1];
        const bool rows_live = r0 + mt * 16 < m;
#pragma unroll
        for (int ks = 0; ks < kChunkB / 16; ++ks) {
            if (!rows_live) break;  // warp-uniform: this warp's 16 rows are all past m
            uint32_t a0, a1, a2, a3;
            asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                         : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3)
                         : "r"(smem_u32(b + arow * kStrideB + ks * 16 + acol)));
            // the B fragments first, then the MMAs (the loads overlap); column
            // tiles past the set are skipped (warp-uniform)
            uint32_t b0[4], b1[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if ((nt0 + q) * 8 < ns)
                    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                                 : "=r"(b0[q]), "=r"(b1[q])
                                 : "r"(smem_u32(b + ((nt0 + q) * 8 + brow) * kStrideB + ks * 16 + bcol)));
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if ((nt0 + q) * 8 < ns)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                        "{%0,%1,%2,%3};\n"
                        : "+f"(acc[q][0]), "+f"(acc[q][1]), "+f"(acc[q][2]), "+f"(acc[q][3])
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0[q]), "r"(b1[q]));
        }
        __syncthreads();
    }
    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int i = r0 + mt * 16 + gid + 8 * (h >> 1), j = (nt0 + q) * 8 + tig * 2 + (h & 1);
            if (i < m && j < ns) sm.D[i * kDStride + j] = fmaxf(0.f, sm.nrm[i] + sm.nrm[j] - 2.f * acc[q][h]);
        }
}
}  // namespace

template <bool kBF16>
__global__ void __launch_bounds__(kTileThreads) tile_join_kernel(DevState st, int li) {
    if (iteration_skipped(st, li)) return;
    __shared__ TileSmem sm;
    extern __shared__ __align__(16) unsigned char stage_mem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = st.K, nv = st.nv;
    const float4 *X4 = reinterpret_cast<const float4 *>(st.X);
    if (tid < 8) sm.stat[tid] = 0;
    long long t_evals = 0, t_gathered = 0, t_candids = 0, t_setovf = 0, t_props = 0, t_ovf = 0, t_ins = 0,
              t_to = 0;
    __syncthreads();
    for (long long u = st.u_lo + blockIdx.x; u < st.u_hi; u += gridDim.x) {
        if (node_skipped(st, u, li)) continue;  // batched: u's data set converged (uniform in the block)
        // ---- 1. candidates (warp 0)
        if (warp == 0) {
            int ns, m;
            t_candids += warp_gather_candidates(st, u, sm.raw, sm.hset, sm.sid, ns, m, t_setovf);
            if (lane == 0) {
                sm.ns = ns;
                sm.m = m;
                sm.ovf = 0ull;
            }
        }
        __syncthreads();
        const int ns = sm.ns, m = sm.m, o = ns - m;
        if (ns > 0) {
            // ---- 2. snapshot worst keys, clear masks, norms
            for (int i = tid; i < ns; i += kTileThreads) {
                sm.swk[i] = __ldcg(st.keys + (size_t)sm.sid[i] * K + (K - 1));
                sm.mask[i] = 0ull;
                if (kBF16) sm.nrm[i] = st.xnorm[sm.sid[i]];
            }
            __syncthreads();
            // ---- 3. distance block
            if (kBF16) {
                for (int r0 = 0; r0 < m; r0 += 32)
                    tile_dist_b16(sm, reinterpret_cast<uint16_t *>(stage_mem), st.Xb, st.dpb, ns, m, r0);
            } else {
                tile_dist_f32(sm, reinterpret_cast<float4 *>(stage_mem), X4, nv, ns, m);
            }
            __syncthreads();
            if (tid == 0) {
                t_evals += (long long)m * (m - 1) / 2 + (long long)m * o;
                t_gathered += ns;
            }
            // ---- 4. every join pair once: proposal masks
            const int mo = m | 1, half = (mo - 1) >> 1;
            const uint32_t t1 = (uint32_t)mo * (uint32_t)half, t2 = (uint32_t)m * (uint32_t)o;
            const uint32_t mg1 = div_magic((uint32_t)half), mg2 = div_magic((uint32_t)o);
            for (uint32_t k = tid; k < t1 + t2; k += kTileThreads) {
                int i, j;
                if (k < t1) {
                    const uint32_t r = div_small(k, (uint32_t)half, mg1);
                    i = (int)r;
                    j = (int)(r + 1 + (k - r * (uint32_t)half));
                    if (j >= mo) j -= mo;
                    if (i >= m || j >= m) continue;
                } else {
                    const uint32_t q = k - t1;
                    const uint32_t r = div_small(q, (uint32_t)o, mg2);
                    i = (int)r;
                    j = m + (int)(q - r * (uint32_t)o);
                }
                const float dd = sm.D[i * kDStride + j];
                if (make_key(dd, (uint32_t)sm.sid[j], kFlagNew | kFlagIns) < sm.swk[i]) atomicOr(&sm.mask[i], 1ull << j);
                if (make_key(dd, (uint32_t)sm.sid[i], kFlagNew | kFlagIns) < sm.swk[j]) atomicOr(&sm.mask[j], 1ull << i);
            }
            __syncthreads();
            // ---- 5. snapshot the lists of targets with proposals and drop the
            //         proposals they cannot take: not before the worst entry
            //         (which only decreases) or already listed (an id listed at
            //         any time in the iteration is still listed or was pushed
            //         out by K better keys).  float32: a pair has one key, so
            //         "listed" is "the same (dist, id) at its lower bound";
            //         bf16: the id is searched.
            uint64_t *Lsnap = reinterpret_cast<uint64_t *>(stage_mem);  // the row stage is free now
            for (int e = tid; e < ns * K; e += kTileThreads) {
                const int t = e / K, k = e - t * K;
                if (sm.mask[t]) Lsnap[t * (K + 1) + k] = __ldcg(st.keys + (size_t)sm.sid[t] * K + k);
            }
            __syncthreads();
            for (int t = tid; t < ns; t += kTileThreads) {
                unsigned long long mt = sm.mask[t];
                if (!mt) continue;
                const uint64_t *Lt = Lsnap + t * (K + 1);
                const uint64_t worst = Lt[K - 1];
                for (unsigned long long mm = mt; mm; mm &= mm - 1) {
                    const int j = __ffsll((long long)mm) - 1;
                    const float dd = t < m ? sm.D[t * kDStride + j] : sm.D[j * kDStride + t];
                    const uint32_t q = (uint32_t)sm.sid[j];
                    const uint64_t x = make_key(dd, q, kFlagNew | kFlagIns);
                    bool drop = x >= worst;
                    if (!drop && !kBF16) {
                        const uint64_t xo = key_order(x);
                        int lo = 0, hi = K - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (key_order(Lt[mid]) < xo) lo = mid + 1;
                            else hi = mid;
                        }
                        drop = key_order(Lt[lo]) == xo;
                    } else if (!drop) {
                        // bf16: a listed id is kept only with its smaller key
                        // (the merge keeps each id's smallest key)
                        for (int k = 0; k < K; ++k)
                            if (key_id(Lt[k]) == q) {
                                drop = key_order(Lt[k]) <= key_order(x);
                                break;
                            }
                    }
                    if (drop) mt &= ~(1ull << j);
                }
                sm.mask[t] = mt;
            }
            __syncthreads();
            // ---- 6. bucket runs, one thread per target
            for (int t = tid; t < ns; t += kTileThreads) {
                const unsigned long long mt = sm.mask[t];
                const int c = __popcll(mt);
                if (!c) continue;
                t_props += c;
                const uint32_t p = (uint32_t)sm.sid[t];
                const int b = atomicAdd(st.pcursor + p, c);
                // a proposal whose run has no slot (bucket or pool spent) is
                // marked for the locked insertion; the others are written
                unsigned long long mm = mt, failed = 0ull;
                uint64_t *slot = nullptr;
                for (int r = 0; r < c; ++r, mm &= mm - 1) {
                    const int pos = b + r;
                    if (r == 0 || (pos & (kBucketRun - 1)) == 0) slot = bucket_slot(st, p, pos);
                    else if (slot) ++slot;
                    const int j = __ffsll((long long)mm) - 1;
                    const float dd = t < m ? sm.D[t * kDStride + j] : sm.D[j * kDStride + t];
                    if (slot) *slot = make_key(dd, (uint32_t)sm.sid[j], kFlagNew | kFlagIns);
                    else failed |= 1ull << j;
                }
                sm.fails[t] = failed;
                if (failed) atomicOr(&sm.ovf, 1ull << t);
            }
            __syncthreads();
            // ---- 7. full buckets (rare): locked insertion, warp 0
            if (warp == 0) {
                for (unsigned long long om = sm.ovf; om; om &= om - 1) {
                    const int t = __ffsll((long long)om) - 1;
                    const unsigned long long rest = sm.fails[t];
                    if (lane == 0) t_ovf += __popcll(rest);
                    uint64_t xs[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = lane + 32 * h;
                        xs[h] = kKeyEmpty;
                        if ((rest >> j) & 1ull) {
                            const float dd = t < m ? sm.D[t * kDStride + j] : sm.D[j * kDStride + t];
                            xs[h] = make_key(dd, (uint32_t)sm.sid[j], kFlagNew | kFlagIns);
                        }
                    }
                    const int ins = warp_locked_insert(st, (uint32_t)sm.sid[t], rest, xs[0], xs[1], li);
                    if (lane == 0) {
                        if (ins < 0) ++t_to;
                        else t_ins += ins;
                    }
                }
            }
        }
        __syncthreads();
    }
    // ---- counters: thread -> block -> global (warp-level values are counted
    // by one lane only)
    if (warp != 0 || lane != 0) t_candids = t_setovf = 0;
    atomic_add_ll(&sm.stat[0], t_evals);
    atomic_add_ll(&sm.stat[1], t_gathered);
    atomic_add_ll(&sm.stat[2], t_candids);
    atomic_add_ll(&sm.stat[3], t_props);
    atomic_add_ll(&sm.stat[4], t_ins);
    atomic_add_ll(&sm.stat[5], t_ovf);
    atomic_add_ll(&sm.stat[6], t_to);
    atomic_add_ll(&sm.stat[7], t_setovf);
    __syncthreads();
    if (tid == 0) {
        long long *its = st.it_stats + (size_t)li * kItCount;
        its[kItRan] = 1;
        atomic_add_ll(&its[kItEvals], sm.stat[0]);
        atomic_add_ll(&its[kItGathered], sm.stat[1]);
        atomic_add_ll(&its[kItCandIds], sm.stat[2]);
        atomic_add_ll(&its[kItProposals], sm.stat[3]);
        atomic_add_ll(&its[kItInserts], sm.stat[4]);
        atomic_add_ll(&st.stats[kStatEvals], sm.stat[0]);
        atomic_add_ll(&st.stats[kStatGathered], sm.stat[1]);
        atomic_add_ll(&st.stats[kStatInserts], sm.stat[4]);
        if (sm.stat[5]) atomic_add_ll(&st.stats[kStatBucketOverflow], sm.stat[5]);
        if (sm.stat[6]) atomic_add_ll(&st.stats[kStatLockTimeout], sm.stat[6]);
        if (sm.stat[7]) atomic_add_ll(&st.stats[kStatSetOverflow], sm.stat[7]);
    }
}

namespace {
template <bool kBF16>
cudaError_t launch_tile_t(const DevState &st, int li, cudaStream_t s) {
    // two row-chunk buffers, later reused for the targets' list snapshots
    size_t dyn = kBF16 ? 2ull * kSetMax * kStrideB * sizeof(uint16_t) : 2ull * kSetMax * kStrideV * 16;
    dyn = std::max(dyn, (size_t)kSetMax * (st.K + 1) * sizeof(uint64_t));
    auto kern = tile_join_kernel<kBF16>;
    cudaError_t e = smem_opt_in((const void *)kern, dyn);
    if (e != cudaSuccess) return e;
    const int grid = grid_for((const void *)kern, kTileThreads, dyn);
    kern<<<grid, kTileThreads, dyn, s>>>(st, li);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_tile_join(const DevState &st, int li, bool bf16, cudaStream_t s) {
    return bf16 ? launch_tile_t<true>(st, li, s) : launch_tile_t<false>(st, li, s);
}

// bf16 copy of the points (zero-padded to a multiple of 64) and the float32
// squared norms of the bf16 values, one warp per point
__global__ void stage_bf16_kernel(const float *__restrict__ X, int64_t n, int dp, int d, uint16_t *__restrict__ Xb,
                                  int dpb, float *__restrict__ nrm) {
    const unsigned lane = lane_id();
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n;
         u += ((long long)gridDim.x * blockDim.x) >> 5) {
        float acc = 0.f;
        for (int t = lane; t < dpb; t += 32) {
            const float v = t < d ? X[(size_t)u * dp + t] : 0.f;
            const __nv_bfloat16 b = __float2bfloat16_rn(v);
            Xb[(size_t)u * dpb + t] = __bfloat16_as_ushort(b);
            const float f = __bfloat162float(b);
            acc = fmaf(f, f, acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) nrm[u] = acc;
    }
}

__global__ void stage_fp8_kernel(const float *__restrict__ X, int64_t n, int dp, int d, uint8_t *__restrict__ X8,
                                 int dpb, float *__restrict__ nrm) {
    const unsigned lane = lane_id();
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n;
         u += ((long long)gridDim.x * blockDim.x) >> 5) {
        float acc = 0.f;
        for (int t = lane; t < dpb; t += 32) {
            const float v = t < d ? X[(size_t)u * dp + t] : 0.f;
            const __nv_fp8_e4m3 b(v);  // round to nearest even, saturating
            X8[(size_t)u * dpb + t] = b.__x;
            const float f = (float)b;
            acc = fmaf(f, f, acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) nrm[u] = acc;
    }
}

cudaError_t launch_stage_fp8(const float *X, int64_t n, int dp, int d, uint8_t *X8, int dpb, float *nrm,
                             cudaStream_t s) {
    const int grid = grid_for((const void *)stage_fp8_kernel, 256, 0);
    stage_fp8_kernel<<<grid, 256, 0, s>>>(X, n, dp, d, X8, dpb, nrm);
    return cudaGetLastError();
}

cudaError_t launch_stage_bf16(const float *X, int64_t n, int dp, int d, uint16_t *Xb, int dpb, float *nrm,
                              cudaStream_t s) {
    const int grid = grid_for((const void *)stage_bf16_kernel, 256, 0);
    stage_bf16_kernel<<<grid, 256, 0, s>>>(X, n, dp, d, Xb, dpb, nrm);
    return cudaGetLastError();
}

}  // namespace knng
