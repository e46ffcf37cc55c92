// bruteforce.cu -- exact K-NNG (Section 2: every distance, the K smallest per
// point), the ground truth that recall is measured against.
//
// A block of 128 threads takes 128 query points and one slice of the points;
// the slice streams through shared memory in tiles that every thread reads by
// broadcast.  Each thread keeps its query's best K keys (dist, id) sorted in
// registers and inserts a candidate only when it beats the current K-th key.
// With few queries the points are cut into S slices (a second grid
// dimension) so that every SM has work; each slice's sorted list goes to
// scratch and one warp per query merges the S lists (bitonic merges of 32
// keys).  Distances use the library's canonical float32 difference form, so
// ground truth and NN-Descent agree on the value of every pair.
#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>

#include "../../include/knng.h"
#include "internal.h"

namespace knng {

namespace {
constexpr int kBfThreads = 128;
constexpr int kBfSmem = 64 * 1024;

// own row in registers (NVR float4) when nv <= NVR; same operation order as l2sq_rows
template <int NVR>
__device__ __forceinline__ float l2sq_reg(const float4 (&a)[NVR], const float4 *__restrict__ b) {
    Acc2 acc;
#pragma unroll
    for (int v = 0; v < NVR; ++v) acc.add(a[v], b[v]);
    return acc.sum();
}
}  // namespace

template <int KMAX, int NVR>
__global__ void __launch_bounds__(kBfThreads) bruteforce_kernel(const float4 *__restrict__ X4, int64_t n, int nv,
                                                                int K, const int64_t *__restrict__ rows,
                                                                int64_t nq, int32_t *__restrict__ ids,
                                                                float *__restrict__ dists, int tile,
                                                                uint64_t *__restrict__ part, int64_t chunk) {
    extern __shared__ __align__(16) float4 tile_s[];
    const int64_t q = (int64_t)blockIdx.x * kBfThreads + threadIdx.x;
    const bool live = q < nq;
    const int64_t qc = live ? q : nq - 1;
    const int64_t qrow = rows ? rows[qc] : qc;
    const float4 *own = X4 + (size_t)qrow * nv;
    float4 ownr[NVR > 0 ? NVR : 1];
    if (NVR > 0) {
#pragma unroll
        for (int v = 0; v < (NVR > 0 ? NVR : 1); ++v) ownr[v] = own[v];
    }
    // right-aligned sorted list: slots [KMAX-K, KMAX) hold the best keys so
    // far (empty = all ones), slots below hold 0 and never leave the front,
    // so the K-th best is always L[KMAX-1]
    const int off = KMAX - K;
    uint64_t L[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) L[k] = k >= off ? kKeyEmpty : 0ull;
    const int64_t p0 = (int64_t)blockIdx.y * chunk, p1 = min(n, p0 + chunk);
    for (int64_t t0 = p0; t0 < p1; t0 += tile) {
        const int cnt = (int)min((int64_t)tile, p1 - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt * nv; e += kBfThreads) tile_s[e] = X4[(size_t)t0 * nv + e];
        __syncthreads();
        for (int c = 0; c < cnt; ++c) {
            const int64_t j = t0 + c;
            float dd;
            if (NVR > 0) dd = l2sq_reg<(NVR > 0 ? NVR : 1)>(ownr, tile_s + (size_t)c * nv);
            else dd = l2sq_rows(own, tile_s + (size_t)c * nv, nv);
            // flag bit 1 keeps every candidate key above the 0 sentinels
            const uint64_t x = make_key(dd, (uint32_t)j, 1u);
            if (x < L[KMAX - 1] && j != qrow) {
#pragma unroll
                for (int k = KMAX - 1; k >= 1; --k) {
                    const uint64_t lo = L[k] < x ? L[k] : x;
                    L[k] = lo > L[k - 1] ? lo : L[k - 1];
                }
                L[0] = L[0] < x ? L[0] : x;
            }
        }
    }
    if (live && part) {
        // this slice's sorted list (empty slots stay all ones)
        uint64_t *dst = part + ((size_t)q * gridDim.y + blockIdx.y) * K;
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k >= off) dst[k - off] = L[k];
    } else if (live) {
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k >= off) {
                ids[(size_t)q * K + k - off] = (int32_t)key_id(L[k]);
                dists[(size_t)q * K + k - off] = key_dist(L[k]);
            }
        }
    }
}

// One warp per query merges its S sorted slice lists of K keys: the running
// list A (ascending, lane k = entry k) and the next list B read in reverse
// give min(A[l], B[31 - l]), a bitonic sequence holding the 32 smallest keys
// of both, which five compare-exchange stages sort ascending.  A point lies in
// one slice only, so no key repeats.
__global__ void __launch_bounds__(256) bruteforce_merge_kernel(const uint64_t *__restrict__ part, int S, int K,
                                                               int64_t nq, int32_t *__restrict__ ids,
                                                               float *__restrict__ dists) {
    const unsigned lane = lane_id();
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq;
         q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const uint64_t *P = part + (size_t)q * S * K;
        uint64_t A = (int)lane < K ? P[lane] : kKeyEmpty;
        for (int y = 1; y < S; ++y) {
            const int r = 31 - (int)lane;
            const uint64_t B = r < K ? P[(size_t)y * K + r] : kKeyEmpty;
            uint64_t C = A < B ? A : B;
#pragma unroll
            for (int j = 16; j > 0; j >>= 1) {
                const uint64_t o = shfl_xor_u64(C, j);
                C = (lane & j) ? (C > o ? C : o) : (C < o ? C : o);
            }
            A = C;
        }
        if ((int)lane < K) {
            ids[(size_t)q * K + lane] = (int32_t)key_id(A);
            dists[(size_t)q * K + lane] = key_dist(A);
        }
    }
}

namespace {
template <int KMAX, int NVR>
cudaError_t launch_bf_t(const float *X, int64_t n, int nv, int K, const int64_t *rows, int64_t nq, int32_t *ids,
                        float *dists, cudaStream_t s, uint64_t *part, int S) {
    int tile = (int)(kBfSmem / ((size_t)nv * 16));
    if (tile > 256) tile = 256;
    if (tile < 1) tile = 1;
    const size_t dyn = (size_t)tile * nv * 16;
    auto kern = bruteforce_kernel<KMAX, NVR>;
    cudaError_t e = smem_opt_in((const void *)kern, dyn);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (nq + kBfThreads - 1) / kBfThreads;
    const int64_t chunk = (n + S - 1) / S;
    kern<<<dim3((unsigned)blocks, (unsigned)S), kBfThreads, dyn, s>>>(reinterpret_cast<const float4 *>(X), n, nv, K,
                                                                     rows, nq, ids, dists, tile,
                                                                     S > 1 ? part : nullptr, chunk);
    e = cudaGetLastError();
    if (e != cudaSuccess || S == 1) return e;
    const int mgrid = grid_for((const void *)bruteforce_merge_kernel, 256, 0);
    bruteforce_merge_kernel<<<mgrid, 256, 0, s>>>(part, S, K, nq, ids, dists);
    return cudaGetLastError();
}

template <int KMAX>
cudaError_t launch_bf_k(const float *X, int64_t n, int nv, int K, const int64_t *rows, int64_t nq, int32_t *ids,
                        float *dists, cudaStream_t s, uint64_t *part, int S) {
    if (nv == 2) return launch_bf_t<KMAX, 2>(X, n, nv, K, rows, nq, ids, dists, s, part, S);
    if (nv == 4) return launch_bf_t<KMAX, 4>(X, n, nv, K, rows, nq, ids, dists, s, part, S);
    if (nv == 8) return launch_bf_t<KMAX, 8>(X, n, nv, K, rows, nq, ids, dists, s, part, S);
    return launch_bf_t<KMAX, 0>(X, n, nv, K, rows, nq, ids, dists, s, part, S);
}
}  // namespace

int bruteforce_slices(int64_t n, int64_t nq) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t qblocks = (nq + kBfThreads - 1) / kBfThreads, want = 4LL * sms;
    int64_t S = (want + qblocks - 1) / qblocks;
    S = std::min<int64_t>(S, std::max<int64_t>(1, n / 4096));
    return (int)std::max<int64_t>(1, std::min<int64_t>(S, 256));
}

cudaError_t launch_bruteforce(const float *X, int64_t n, int dp, int K, const int64_t *rows, int64_t nq,
                              int32_t *ids, float *dists, cudaStream_t s, uint64_t *part, int S) {
    const int nv = dp / 4;
    if (!part) S = 1;
    if (K <= 8) return launch_bf_k<8>(X, n, nv, K, rows, nq, ids, dists, s, part, S);
    if (K <= 16) return launch_bf_k<16>(X, n, nv, K, rows, nq, ids, dists, s, part, S);
    if (K <= 24) return launch_bf_k<24>(X, n, nv, K, rows, nq, ids, dists, s, part, S);
    if (K <= 32) return launch_bf_k<32>(X, n, nv, K, rows, nq, ids, dists, s, part, S);
    return launch_bf_k<64>(X, n, nv, K, rows, nq, ids, dists, s, nullptr, 1);  // one slice: no list merge
}

namespace {
template <int KMAX, int NVR>
cudaError_t prepare_bf_t() {
    cudaFuncAttributes a;
    auto kern = bruteforce_kernel<KMAX, NVR>;
    cudaError_t e = cudaFuncGetAttributes(&a, kern);
    if (e == cudaSuccess) e = smem_opt_in((const void *)kern, kBfSmem);
    return e;
}
template <int KMAX>
cudaError_t prepare_bf_k() {
    cudaError_t e = prepare_bf_t<KMAX, 2>();
    if (e == cudaSuccess) e = prepare_bf_t<KMAX, 4>();
    if (e == cudaSuccess) e = prepare_bf_t<KMAX, 8>();
    if (e == cudaSuccess) e = prepare_bf_t<KMAX, 0>();
    return e;
}
}  // namespace

cudaError_t prepare_bruteforce_one_slice() {
    cudaError_t e = prepare_stage();
    if (e == cudaSuccess) e = prepare_bf_k<8>();
    if (e == cudaSuccess) e = prepare_bf_k<16>();
    if (e == cudaSuccess) e = prepare_bf_k<24>();
    if (e == cudaSuccess) e = prepare_bf_k<32>();
    return e;
}

}  // namespace knng

// ---------------------------------------------------------------------------
// knng_bruteforce_noalloc: the brute-force K-NNG for callers that cannot
// allocate device memory.  Its only scratch -- the zero-padded copy of the
// points that the kernel reads -- lives in the file-scope device array below,
// which is created with the module and stays resident on every GPU that loads
// this library until the process exits.
// ---------------------------------------------------------------------------
static __device__ __align__(256) float knng_noalloc_points[KNNG_NOALLOC_SCRATCH_BYTES / sizeof(float)];

namespace {
std::mutex g_noalloc_mu;
std::map<unsigned long long, float *> g_noalloc_addr;  // device address of the array, per context

// Set-up, once per context (the first call on a device, and the first after
// a device reset): the array's device address -- host code cannot use its
// name as one -- and every kernel of the path loaded and opted in to the
// shared memory it may use, so that later calls, captured ones included, do
// neither.
cudaError_t noalloc_scratch(float **out) {
    unsigned long long ctx = 0;
    cudaError_t e = knng::current_context_id(&ctx);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    auto it = g_noalloc_addr.find(ctx);
    if (it == g_noalloc_addr.end()) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, knng_noalloc_points);
        if (e != cudaSuccess) return e;
        e = knng::prepare_bruteforce_one_slice();
        if (e != cudaSuccess) return e;
        it = g_noalloc_addr.emplace(ctx, static_cast<float *>(p)).first;
    }
    *out = it->second;
    return cudaSuccess;
}

// True when the kernels of device `dev` may dereference p: device memory of
// that device, or managed memory it can reach (its own, or any when it
// accesses managed memory concurrently).  Host memory and other devices'
// memory are refused before anything is launched.
bool noalloc_pointer_ok(const void *p, int dev, int concurrent_managed) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice) return a.device == dev;
    if (a.type == cudaMemoryTypeManaged) return a.device == dev || concurrent_managed != 0;
    return false;
}
}  // namespace

extern "C" int knng_bruteforce_noalloc(const float *data, int64_t n, int d, int K, const int64_t *rows, int64_t nq,
                                       int32_t *ids, float *dists, void *stream) {
    if (!data || !ids || !dists || n < 2 || d < 1 || K < 1 || K > n - 1) return KNNG_ERR_INVALID_ARG;
    if (K > knng::kLaneK) return KNNG_ERR_UNSUPPORTED;
    const int dp = (d + 3) & ~3;
    if ((uint64_t)n * (uint64_t)dp * sizeof(float) > (uint64_t)KNNG_NOALLOC_SCRATCH_BYTES)
        return KNNG_ERR_INVALID_ARG;
    if (!rows) nq = n;
    if (nq < 1) return KNNG_ERR_INVALID_ARG;
    int dev = 0, cma = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return KNNG_ERR_CUDA;
    }
    if (cudaDeviceGetAttribute(&cma, cudaDevAttrConcurrentManagedAccess, dev) != cudaSuccess) {
        cudaGetLastError();
        cma = 0;
    }
    // test hook: check the pointers as if another device were current (every
    // device pointer then belongs to a foreign device), with nothing launched
    if (std::getenv("KNNG_TEST_NOALLOC_FOREIGN_DEVICE")) {
        dev += 1;
        cma = 0;
    }
    if (!noalloc_pointer_ok(data, dev, cma) || !noalloc_pointer_ok(ids, dev, cma) ||
        !noalloc_pointer_ok(dists, dev, cma) || (rows && !noalloc_pointer_ok(rows, dev, cma)))
        return KNNG_ERR_INVALID_ARG;
    float *X = nullptr;
    cudaError_t e = noalloc_scratch(&X);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return KNNG_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // staging writes every element of the n x dp region it uses (padding
    // included), so nothing left by an earlier call is read
    e = knng::launch_stage(data, n, d, X, dp, s);
    if (e == cudaSuccess) e = knng::launch_bruteforce(X, n, dp, K, rows, nq, ids, dists, s, nullptr, 1);
    return e == cudaSuccess ? KNNG_OK : KNNG_ERR_CUDA;
}
