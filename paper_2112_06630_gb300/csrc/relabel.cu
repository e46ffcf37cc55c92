// relabel.cu -- parallel locality relabelling (a GB300 variant of the greedy
// clustering heuristic of Section 3.2 / Algorithm 1).
//
// Algorithm 1 walks the spots one after another; each step depends on the
// permutation built so far, so on this GPU it costs ~0.8 us per node (one
// warp, dependent memory round trips).  This variant reaches the same goal --
// points that are close in data space get nearby spots, clusters contiguous
// -- with rounds of data-parallel work: single-linkage agglomeration
// (Boruvka) on the graph of the current K-lists, laid out so that every
// component of every round occupies one contiguous range of spots.
//
// Edges are the list entries (u, v), undirected, ordered by (canonical
// float32 distance, min(u, v), max(u, v)), a strict total order.  Each round
// every component hooks onto the component across its smallest outgoing
// edge; with a strict order the hooks form trees plus 2-cycles (both ends
// chose the same edge), broken at the smaller representative, which becomes
// the root.  Cross-cluster edges are the longest, so clusters merge last.
//
// Layout: every point keeps its offset inside its current component.  When a
// component joins a root it claims a range inside the root's range with one
// atomicAdd of its size, and its points add that base to their offset.  The
// order of the children of a root depends on the atomics, not the hierarchy:
// any order keeps every component contiguous.  At the end the top-level
// components claim ranges of [0, n) the same way: sigma(u) = base(root) +
// offset(u).
#include "common.cuh"
#include "internal.h"

namespace knng {

namespace {
constexpr long long kRootSteps = 1LL << 26;  // bound on a root walk (a forest path is shorter)

__device__ __forceinline__ long long rl_warp() { return ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ long long rl_warps() { return ((long long)gridDim.x * blockDim.x) >> 5; }

struct RelabelState {
    const float *X;
    const uint64_t *keys;
    int64_t n;
    int K, nv;
    uint32_t *dist;         // n x K canonical distance bits of the list entries
    int32_t *comp;          // point -> representative of its component
    int32_t *parent;        // representative -> representative it hooks onto
    int32_t *root;          // representative -> root after this round
    int32_t *size;          // representative -> points in its component
    int32_t *acc;           // root -> size claimed so far this round
    int32_t *off;           // representative -> base inside its root's range
    int32_t *pos;           // point -> offset inside its component
    uint64_t *best1;        // representative -> min (dist << 32 | min endpoint) of its outgoing edges
    uint32_t *best2;        // representative -> min max endpoint among edges with that key
    int *ctl;               // [0] hooks this round, [1] done, [2] walk overflow, [3] top-level cursor
};

__device__ __forceinline__ bool relabel_done(const RelabelState &r) {
    return *(volatile const int *)(r.ctl + 1) != 0;
}

// canonical distances of every list entry, once
__global__ void __launch_bounds__(256) relabel_dist_kernel(RelabelState r) {
    const unsigned lane = lane_id();
    const float4 *X4 = reinterpret_cast<const float4 *>(r.X);
    for (long long u = rl_warp(); u < r.n; u += rl_warps()) {
        for (int k = (int)lane; k < r.K; k += 32) {
            const uint32_t v = key_id(r.keys[(size_t)u * r.K + k]);
            const float d = l2sq_rows(X4 + (size_t)u * r.nv, X4 + (size_t)v * r.nv, r.nv);
            r.dist[(size_t)u * r.K + k] = __float_as_uint(d);
        }
    }
}

__global__ void relabel_init_kernel(RelabelState r) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < r.n; u += (int64_t)gridDim.x * blockDim.x) {
        r.comp[u] = (int32_t)u;
        r.size[u] = 1;
        r.pos[u] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        r.ctl[0] = 0;
        r.ctl[1] = 0;
        r.ctl[2] = 0;
        r.ctl[3] = 0;
    }
}

// round start: a round without hooks ends the agglomeration; clear the
// per-representative scratch
__global__ void relabel_clear_kernel(RelabelState r, int round) {
    if (round > 0 && *(volatile int *)(r.ctl + 0) == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) r.ctl[1] = 1;
        return;
    }
    if (relabel_done(r)) return;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < r.n; c += (int64_t)gridDim.x * blockDim.x) {
        r.best1[c] = ~0ull;
        r.best2[c] = 0xFFFFFFFFu;
        r.acc[c] = 0;
    }
}

// the hook counter restarts only after every block of the clear kernel has
// read it
__global__ void relabel_reset_kernel(RelabelState r) {
    if (relabel_done(r)) return;
    r.ctl[0] = 0;
}

// pass 1: each component's smallest (dist, min endpoint) over the list edges
// that leave it (an edge leaves both of its end components)
__global__ void __launch_bounds__(256) relabel_best1_kernel(RelabelState r) {
    if (relabel_done(r)) return;
    const size_t total = (size_t)r.n * r.K;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const uint32_t u = (uint32_t)(e / r.K), v = key_id(r.keys[e]);
        const int32_t cu = r.comp[u], cv = r.comp[v];
        if (cu == cv) continue;
        const uint64_t k1 = ((uint64_t)r.dist[e] << 32) | (uint64_t)(u < v ? u : v);
        atomicMin((unsigned long long *)&r.best1[cu], (unsigned long long)k1);
        atomicMin((unsigned long long *)&r.best1[cv], (unsigned long long)k1);
    }
}

// pass 2: among the edges with that key, the smallest max endpoint
__global__ void __launch_bounds__(256) relabel_best2_kernel(RelabelState r) {
    if (relabel_done(r)) return;
    const size_t total = (size_t)r.n * r.K;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const uint32_t u = (uint32_t)(e / r.K), v = key_id(r.keys[e]);
        const int32_t cu = r.comp[u], cv = r.comp[v];
        if (cu == cv) continue;
        const uint64_t k1 = ((uint64_t)r.dist[e] << 32) | (uint64_t)(u < v ? u : v);
        const uint32_t mx = u < v ? v : u;
        if (r.best1[cu] == k1) atomicMin(&r.best2[cu], mx);
        if (r.best1[cv] == k1) atomicMin(&r.best2[cv], mx);
    }
}

// hook every representative onto the component across its chosen edge
__global__ void relabel_hook_kernel(RelabelState r) {
    if (relabel_done(r)) return;
    int hooks = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < r.n; c += (int64_t)gridDim.x * blockDim.x) {
        if (r.comp[c] != (int32_t)c) continue;
        const uint64_t b1 = r.best1[c];
        if (b1 == ~0ull) {
            r.parent[c] = (int32_t)c;
            continue;
        }
        const uint32_t a = (uint32_t)b1, b = r.best2[c];
        const uint32_t other = r.comp[a] == (int32_t)c ? b : a;
        r.parent[c] = r.comp[other];
        ++hooks;
    }
    if (hooks) atomicAdd(r.ctl + 0, hooks);
}

// a 2-cycle (both ends chose the same edge) keeps the smaller representative
// as the root
__global__ void relabel_break_kernel(RelabelState r) {
    if (relabel_done(r)) return;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < r.n; c += (int64_t)gridDim.x * blockDim.x) {
        if (r.comp[c] != (int32_t)c) continue;
        const int32_t p = r.parent[c];
        if (p != (int32_t)c && r.parent[p] == (int32_t)c && (int32_t)c < p) r.parent[c] = (int32_t)c;
    }
}

// roots by path halving (the hooks now form a forest); then every
// representative claims its range inside its root's range
__global__ void relabel_root_kernel(RelabelState r) {
    if (relabel_done(r)) return;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < r.n; c += (int64_t)gridDim.x * blockDim.x) {
        if (r.comp[c] != (int32_t)c) continue;
        int32_t x = (int32_t)c;
        long long steps = 0;
        for (;;) {
            const int32_t p = r.parent[x];
            if (p == x) break;
            const int32_t gp = r.parent[p];
            if (gp != p) r.parent[x] = gp;
            x = gp;
            if (++steps > kRootSteps) {
                atomicOr(r.ctl + 2, 1);
                break;
            }
        }
        r.root[c] = x;
    }
}

__global__ void relabel_claim_kernel(RelabelState r) {
    if (relabel_done(r)) return;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < r.n; c += (int64_t)gridDim.x * blockDim.x) {
        if (r.comp[c] != (int32_t)c) continue;
        r.off[c] = atomicAdd(r.acc + r.root[c], r.size[c]);
    }
}

// points move into their root's range; roots take their new sizes
__global__ void relabel_move_kernel(RelabelState r) {
    if (relabel_done(r)) return;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < r.n; u += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = r.comp[u];
        r.pos[u] += r.off[c];
        const int32_t rt = r.root[c];
        r.comp[u] = rt;
        if (rt == (int32_t)u) r.size[u] = r.acc[u];
    }
}

// top-level components claim ranges of [0, n); sigma(u) = base + offset
__global__ void relabel_top_kernel(RelabelState r) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < r.n; c += (int64_t)gridDim.x * blockDim.x)
        if (r.comp[c] == (int32_t)c) r.off[c] = atomicAdd(r.ctl + 3, r.size[c]);
}

__global__ void relabel_sigma_kernel(RelabelState r, int32_t *__restrict__ sigma) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < r.n; u += (int64_t)gridDim.x * blockDim.x)
        sigma[u] = r.off[r.comp[u]] + r.pos[u];
}
}  // namespace

size_t parallel_relabel_scratch(int64_t n, int K) {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return al(sizeof(uint32_t) * (size_t)n * K) + 7 * al(sizeof(int32_t) * (size_t)n) +
           al(sizeof(uint64_t) * (size_t)n) + al(sizeof(uint32_t) * (size_t)n) + al(4 * sizeof(int));
}

int parallel_relabel_rounds(int64_t n) {
    int r = 2;
    while (((int64_t)1 << (r - 2)) < n) ++r;  // components at least halve while any hooks
    return r;
}

cudaError_t launch_parallel_relabel(const float *X, const uint64_t *keys, int64_t n, int K, int nv, int32_t *sigma,
                                    unsigned char *scratch, int *launches, cudaStream_t s) {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    RelabelState r;
    unsigned char *p = scratch;
    r.X = X;
    r.keys = keys;
    r.n = n;
    r.K = K;
    r.nv = nv;
    r.dist = (uint32_t *)p;
    p += al(sizeof(uint32_t) * (size_t)n * K);
    int32_t **arr[7] = {&r.comp, &r.parent, &r.root, &r.size, &r.acc, &r.off, &r.pos};
    for (auto a : arr) {
        *a = (int32_t *)p;
        p += al(sizeof(int32_t) * (size_t)n);
    }
    r.best1 = (uint64_t *)p;
    p += al(sizeof(uint64_t) * (size_t)n);
    r.best2 = (uint32_t *)p;
    p += al(sizeof(uint32_t) * (size_t)n);
    r.ctl = (int *)p;
    const int gw = grid_for((const void *)relabel_dist_kernel, 256, 0);
    const int g = grid_for((const void *)relabel_best1_kernel, 256, 0);
    relabel_dist_kernel<<<gw, 256, 0, s>>>(r);
    relabel_init_kernel<<<g, 256, 0, s>>>(r);
    int nl = 2;
    const int rounds = parallel_relabel_rounds(n);
    for (int round = 0; round < rounds; ++round) {
        relabel_clear_kernel<<<g, 256, 0, s>>>(r, round);
        relabel_reset_kernel<<<1, 1, 0, s>>>(r);
        relabel_best1_kernel<<<g, 256, 0, s>>>(r);
        relabel_best2_kernel<<<g, 256, 0, s>>>(r);
        relabel_hook_kernel<<<g, 256, 0, s>>>(r);
        relabel_break_kernel<<<g, 256, 0, s>>>(r);
        relabel_root_kernel<<<g, 256, 0, s>>>(r);
        relabel_claim_kernel<<<g, 256, 0, s>>>(r);
        relabel_move_kernel<<<g, 256, 0, s>>>(r);
        nl += 9;
    }
    relabel_top_kernel<<<g, 256, 0, s>>>(r);
    relabel_sigma_kernel<<<g, 256, 0, s>>>(r, sigma);
    nl += 2;
    if (launches) *launches += nl;
    return cudaGetLastError();
}

}  // namespace knng
