// bruteforce.cu -- exact K-NNG (Section 2: every distance, the K smallest per
// point), the ground truth that recall is measured against.
//
// A block of 128 threads takes 128 query points; all points stream through
// shared memory in tiles that every thread reads by broadcast.  Each thread
// keeps its query's best K keys (dist, id) sorted in registers and inserts a
// candidate only when it beats the current K-th key.  Distances use the
// library's canonical float32 difference form, so ground truth and NN-Descent
// agree on the value of every pair.
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
    Acc4 acc;
#pragma unroll
    for (int v = 0; v < NVR; ++v) acc.add(a[v], b[v]);
    return acc.sum();
}
}  // namespace

template <int KMAX, int NVR>
__global__ void __launch_bounds__(kBfThreads) bruteforce_kernel(const float4 *__restrict__ X4, int64_t n, int nv,
                                                                int K, const int64_t *__restrict__ rows,
                                                                int64_t nq, int32_t *__restrict__ ids,
                                                                float *__restrict__ dists, int tile) {
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
    for (int64_t t0 = 0; t0 < n; t0 += tile) {
        const int cnt = (int)min((int64_t)tile, n - t0);
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
    if (live) {
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k >= off) {
                ids[(size_t)q * K + k - off] = (int32_t)key_id(L[k]);
                dists[(size_t)q * K + k - off] = key_dist(L[k]);
            }
        }
    }
}

namespace {
template <int KMAX, int NVR>
cudaError_t launch_bf_t(const float *X, int64_t n, int nv, int K, const int64_t *rows, int64_t nq, int32_t *ids,
                        float *dists, cudaStream_t s) {
    int tile = (int)(kBfSmem / ((size_t)nv * 16));
    if (tile > 256) tile = 256;
    if (tile < 1) tile = 1;
    const size_t dyn = (size_t)tile * nv * 16;
    auto kern = bruteforce_kernel<KMAX, NVR>;
    cudaError_t e = cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (nq + kBfThreads - 1) / kBfThreads;
    kern<<<(unsigned)blocks, kBfThreads, dyn, s>>>(reinterpret_cast<const float4 *>(X), n, nv, K, rows, nq, ids,
                                                  dists, tile);
    return cudaGetLastError();
}

template <int KMAX>
cudaError_t launch_bf_k(const float *X, int64_t n, int nv, int K, const int64_t *rows, int64_t nq, int32_t *ids,
                        float *dists, cudaStream_t s) {
    if (nv == 2) return launch_bf_t<KMAX, 2>(X, n, nv, K, rows, nq, ids, dists, s);
    if (nv == 4) return launch_bf_t<KMAX, 4>(X, n, nv, K, rows, nq, ids, dists, s);
    if (nv == 8) return launch_bf_t<KMAX, 8>(X, n, nv, K, rows, nq, ids, dists, s);
    return launch_bf_t<KMAX, 0>(X, n, nv, K, rows, nq, ids, dists, s);
}
}  // namespace

cudaError_t launch_bruteforce(const float *X, int64_t n, int dp, int K, const int64_t *rows, int64_t nq,
                              int32_t *ids, float *dists, cudaStream_t s) {
    const int nv = dp / 4;
    if (K <= 8) return launch_bf_k<8>(X, n, nv, K, rows, nq, ids, dists, s);
    if (K <= 16) return launch_bf_k<16>(X, n, nv, K, rows, nq, ids, dists, s);
    if (K <= 24) return launch_bf_k<24>(X, n, nv, K, rows, nq, ids, dists, s);
    return launch_bf_k<32>(X, n, nv, K, rows, nq, ids, dists, s);
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
constexpr int kNoAllocMaxDevices = 256;
float *g_noalloc_addr[kNoAllocMaxDevices];  // device address of the array, per device
std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device.  Looked up once
// per device (host code cannot use the array's name as a device address).
cudaError_t noalloc_scratch(float **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, knng_noalloc_points);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = static_cast<float *>(p);
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

bool noalloc_on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

extern "C" int knng_bruteforce_noalloc(const float *data, int64_t n, int d, int K, const int64_t *rows, int64_t nq,
                                       int32_t *ids, float *dists, void *stream) {
    if (!data || !ids || !dists || n < 2 || d < 1 || K < 1 || K > n - 1) return KNNG_ERR_INVALID_ARG;
    if (K > knng::kMaxK) return KNNG_ERR_UNSUPPORTED;
    const int dp = (d + 3) & ~3;
    if ((uint64_t)n * (uint64_t)dp * sizeof(float) > (uint64_t)KNNG_NOALLOC_SCRATCH_BYTES)
        return KNNG_ERR_INVALID_ARG;
    if (!rows) nq = n;
    if (nq < 1) return KNNG_ERR_INVALID_ARG;
    if (!noalloc_on_device(data) || !noalloc_on_device(ids) || !noalloc_on_device(dists) ||
        (rows && !noalloc_on_device(rows)))
        return KNNG_ERR_INVALID_ARG;
    float *X = nullptr;
    cudaError_t e = noalloc_scratch(&X);
    if (e != cudaSuccess) return KNNG_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // staging writes every element of the n x dp region it uses (padding
    // included), so nothing left by an earlier call is read
    e = knng::launch_stage(data, n, d, X, dp, s);
    if (e == cudaSuccess) e = knng::launch_bruteforce(X, n, dp, K, rows, nq, ids, dists, s);
    return e == cudaSuccess ? KNNG_OK : KNNG_ERR_CUDA;
}
