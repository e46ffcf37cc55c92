/*
 * knng_oracle.c -- plain, slow, obviously-correct CPU reference ("oracle") for
 * K-nearest-neighbour graph construction with NN-Descent under the squared l2
 * metric, following "Fast single-core K-Nearest Neighbor Graph computation"
 * (Kluser, Bokstaller, Rutz, Buner).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA implementation; the only input both
 * sides share are the seeded arrays drawn by the `workloads` module.
 *
 * Precision.  The paper works in single precision (Section 4).  Distances are
 * accumulated here in double precision from the float32 inputs and rounded to
 * float32 once; every comparison that decides a neighbour is taken on those
 * float32 values together with the id, in the order (dist, id).
 *
 * Passages followed (paper sections):
 *   - K-NNG definition and brute force ............ Section 2 (simple directed
 *     graph, K nearest by the metric, all n(n-1)/2 distances)
 *   - random initialisation ....................... Section 2 (K neighbours
 *     uniformly from V), Section 3.2
 *   - one-pass probability sampling ("turbosampling") Section 3.1
 *   - local join (Calculation step), squared l2 ... Section 2, Section 3.3
 *   - termination on the number of changes ......... Section 2
 *   - greedy clustering heuristic .................. Section 3.2, Algorithm 1
 *
 * Readings where the paper is silent (the same list is kept in the design
 * notes): sample size s = ceil(rho*K) accepted with probability min(1, s/cnt)
 * where cnt counts forward/reverse x new/old separately; only accepted forward
 * new entries lose their "new" flag; ties ordered by (dist, id); a change is a
 * list entry present after the iteration that was not present before it
 * (batched count) or a successful sequential insertion (in-place count);
 * Algorithm 1 looks at the list of the node occupying spot i (reading A) or
 * of node i (reading B) and swaps with the pre-swap value of sigma(a_i[j]).
 *
 * Random numbers: one counter-based generator built from the SplitMix64 output
 * function (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), h(seed, stream, iter, u, j), implemented here
 * from that definition.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_NEW 1u   /* entry not yet sampled as a "new" forward candidate */
#define ORC_INS 2u   /* entry inserted during the current iteration        */

enum { ORC_STREAM_INIT = 1, ORC_STREAM_FWD = 2, ORC_STREAM_REV = 3, ORC_STREAM_HEAP = 4 };

/* ---------------------------------------------------------------- RNG ---- */

/* SplitMix64 output for the state x (state advanced by the golden gamma). */
uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* h(seed, stream, iter, u, j): chain of SplitMix64 outputs over the counter. */
uint64_t orc_hash(uint64_t seed, uint32_t stream, uint32_t iter, uint64_t u, uint64_t j)
{
    uint64_t h = orc_splitmix64(seed);
    h = orc_splitmix64(h ^ (((uint64_t)stream << 32) | (uint64_t)iter));
    h = orc_splitmix64(h ^ u);
    h = orc_splitmix64(h ^ j);
    return h;
}

/* Bernoulli(s / cnt) decided in integers: accept iff hi32(h) * cnt < s * 2^32. */
static int orc_accept(uint64_t h, uint64_t cnt, uint64_t s)
{
    return (h >> 32) * cnt < (s << 32);
}

/* ----------------------------------------------------------- distances ---- */

/* Squared l2 distance (no square root, Section 3.3), accumulated in double. */
double orc_dist64(const float *x, const float *y, int d)
{
    double acc = 0.0;
    for (int t = 0; t < d; ++t) {
        double diff = (double)x[t] - (double)y[t];
        acc += diff * diff;
    }
    return acc;
}

static float orc_dist32(const float *data, int d, int64_t a, int64_t b)
{
    return (float)orc_dist64(data + a * d, data + b * d, d);
}

/* ------------------------------------------------------- list entries ---- */

typedef struct {
    float dist;
    int32_t id;
    uint32_t flags;
} orc_entry;

static int orc_less(const orc_entry *a, const orc_entry *b)
{
    if (a->dist != b->dist) return a->dist < b->dist;
    return a->id < b->id;
}

static int orc_cmp_entry(const void *pa, const void *pb)
{
    const orc_entry *a = (const orc_entry *)pa, *b = (const orc_entry *)pb;
    if (orc_less(a, b)) return -1;
    if (orc_less(b, a)) return 1;
    return 0;
}

/* ------------------------------------------------------- brute force ---- */

typedef struct {
    double dist;
    int32_t id;
} orc_cand;

static int orc_cmp_cand(const void *pa, const void *pb)
{
    const orc_cand *a = (const orc_cand *)pa, *b = (const orc_cand *)pb;
    if (a->dist < b->dist) return -1;
    if (a->dist > b->dist) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

/*
 * Exact K-NNG rows (Section 2): for each query row q, every distance to j != q
 * in double precision; the K smallest by (distance, j) are kept in a sorted
 * array by plain insertion.  Rows are the given query ids; dists are rounded
 * to float32.  Returns 0, or -1 on bad input.
 */
int orc_bruteforce_rows(const float *data, int64_t n, int d, int K,
                        const int64_t *rows, int64_t nq, int32_t *ids, float *dists)
{
    if (n < 2 || K < 1 || K > n - 1 || d < 1) return -1;
    orc_cand *best = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)K);
    if (!best) return -2;
    for (int64_t r = 0; r < nq; ++r) {
        int64_t q = rows[r];
        int have = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == q) continue;
            orc_cand c = {orc_dist64(data + q * d, data + j * d, d), (int32_t)j};
            if (have == K && orc_cmp_cand(&c, &best[K - 1]) >= 0) continue;
            int pos = have < K ? have++ : K - 1;
            while (pos > 0 && orc_cmp_cand(&c, &best[pos - 1]) < 0) {
                best[pos] = best[pos - 1];
                --pos;
            }
            best[pos] = c;
        }
        for (int k = 0; k < K; ++k) {
            ids[r * K + k] = best[k].id;
            dists[r * K + k] = (float)best[k].dist;
        }
    }
    free(best);
    return 0;
}

int orc_bruteforce(const float *data, int64_t n, int d, int K, int32_t *ids, float *dists)
{
    int64_t *rows = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!rows) return -2;
    for (int64_t i = 0; i < n; ++i) rows[i] = i;
    int rc = orc_bruteforce_rows(data, n, d, K, rows, n, ids, dists);
    free(rows);
    return rc;
}

/* ---------------------------------------------------- NN-Descent state ---- */

typedef struct {
    int64_t n;
    int d, K, s;
    uint64_t seed;
    int iter;               /* iterations completed */
    float *data;            /* n x d, current labelling (owned copy) */
    orc_entry *lists;       /* n x K, ascending (dist, id) */
    int32_t *sigma;         /* new position of original node u; identity until reordered */
    int reordered;
    int sampler;            /* 0: turbosampling (Section 3.1), 1: priority heaps */
    /* per-iteration scratch */
    int32_t **new_c, **old_c;
    int32_t *new_n, *old_n;
    int32_t *cap_new, *cap_old;
} orc_state;

/* s = ceil(rho K); the tolerance absorbs the float32 rounding of rho (0.3f x
 * 10 = 3.0000001 must give 3). */
static int orc_ceil_rho_k(float rho, int K)
{
    double v = (double)rho * (double)K;
    int s = (int)ceil(v - 1e-5);
    if (s < 1) s = 1;
    if (s > K) s = K;
    return s;
}

static void orc_sort_list(orc_entry *l, int K)
{
    qsort(l, (size_t)K, sizeof(orc_entry), orc_cmp_entry);
}

static int orc_push(int32_t **arr, int32_t *len, int32_t *cap, int32_t v)
{
    if (*len == *cap) {
        int32_t nc = *cap ? *cap * 2 : 8;
        int32_t *na = (int32_t *)realloc(*arr, sizeof(int32_t) * (size_t)nc);
        if (!na) return -1;
        *arr = na;
        *cap = nc;
    }
    (*arr)[(*len)++] = v;
    return 0;
}

void orc_free(orc_state *st);

/*
 * Random initialisation (Section 2: each vertex gets K neighbours sampled
 * uniformly from V; no self-loops, no repeated ids).  Candidate number a of
 * node u is floor(hi32(h(seed, INIT, 0, u, a)) * n / 2^32); self and repeats
 * are rejected and the next a is tried.
 */
orc_state *orc_create(const float *data, int64_t n, int d, int K, float rho, uint64_t seed)
{
    if (n < 2 || K < 1 || K > n - 1 || d < 1 || !(rho > 0.0f && rho <= 1.0f)) return NULL;
    orc_state *st = (orc_state *)calloc(1, sizeof(orc_state));
    if (!st) return NULL;
    st->n = n; st->d = d; st->K = K; st->s = orc_ceil_rho_k(rho, K); st->seed = seed;
    st->data = (float *)malloc(sizeof(float) * (size_t)n * (size_t)d);
    st->lists = (orc_entry *)malloc(sizeof(orc_entry) * (size_t)n * (size_t)K);
    st->sigma = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    st->new_c = (int32_t **)calloc((size_t)n, sizeof(int32_t *));
    st->old_c = (int32_t **)calloc((size_t)n, sizeof(int32_t *));
    st->new_n = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    st->old_n = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    st->cap_new = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    st->cap_old = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    if (!st->data || !st->lists || !st->sigma || !st->new_c || !st->old_c || !st->new_n ||
        !st->old_n || !st->cap_new || !st->cap_old) {
        orc_free(st);
        return NULL;
    }
    memcpy(st->data, data, sizeof(float) * (size_t)n * (size_t)d);
    for (int64_t u = 0; u < n; ++u) st->sigma[u] = (int32_t)u;
    return st;
}

int orc_init_random(orc_state *st)
{
    int64_t n = st->n;
    int K = st->K;
    for (int64_t u = 0; u < n; ++u) {
        orc_entry *l = st->lists + u * K;
        int have = 0;
        for (uint64_t a = 0; have < K; ++a) {
            uint64_t h = orc_hash(st->seed, ORC_STREAM_INIT, 0, (uint64_t)u, a);
            int64_t v = (int64_t)(((h >> 32) * (uint64_t)n) >> 32);
            if (v == u) continue;
            int dup = 0;
            for (int k = 0; k < have; ++k)
                if (l[k].id == v) { dup = 1; break; }
            if (dup) continue;
            l[have].id = (int32_t)v;
            l[have].dist = orc_dist32(st->data, st->d, u, v);
            l[have].flags = ORC_NEW;
            ++have;
        }
        orc_sort_list(l, K);
    }
    st->iter = 0;
    return 0;
}

/* Start from a given graph (ids, new flags); distances computed here. */
int orc_init_graph(orc_state *st, const int32_t *ids, const uint8_t *is_new, int iter)
{
    int64_t n = st->n;
    int K = st->K;
    for (int64_t u = 0; u < n; ++u) {
        orc_entry *l = st->lists + u * K;
        for (int k = 0; k < K; ++k) {
            int32_t v = ids[u * K + k];
            if (v < 0 || v >= n || v == u) return -1;
            for (int k2 = 0; k2 < k; ++k2)
                if (ids[u * K + k2] == v) return -1;
            l[k].id = v;
            l[k].dist = orc_dist32(st->data, st->d, u, v);
            l[k].flags = is_new[u * K + k] ? ORC_NEW : 0u;
        }
        orc_sort_list(l, K);
    }
    st->iter = iter;
    return 0;
}

/*
 * Selection step (Section 3.1, one pass over the edges with neighbourhood
 * sizes known).  For edge e = (u, v) with flag f, v enters u's forward
 * candidates of kind f with probability min(1, s / fwd_cnt_f(u)), and u enters
 * v's reverse candidates of kind f with probability min(1, s / rev_cnt_f(v)),
 * from independent hash streams.  Accepted forward "new" entries are marked
 * not-new.  new[u] = forward-new then reverse-new, repeats removed; old[u] =
 * forward-old then reverse-old, repeats and members of new[u] removed.
 *
 * stats: [0] max reverse-new fill, [1] max reverse-old fill, [2] max |new|+|old|.
 */
int orc_sample(orc_state *st, int iter, int64_t *stats)
{
    int64_t n = st->n;
    int K = st->K;
    uint64_t s = (uint64_t)st->s;
    int32_t *fwd_new = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int32_t *rev_new = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int32_t *rev_old = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int32_t **fn = (int32_t **)calloc((size_t)n, sizeof(int32_t *));
    int32_t **fo = (int32_t **)calloc((size_t)n, sizeof(int32_t *));
    int32_t **rn = (int32_t **)calloc((size_t)n, sizeof(int32_t *));
    int32_t **ro = (int32_t **)calloc((size_t)n, sizeof(int32_t *));
    int32_t *len = (int32_t *)calloc((size_t)n * 4, sizeof(int32_t));
    int32_t *cap = (int32_t *)calloc((size_t)n * 4, sizeof(int32_t));
    uint8_t *clear = (uint8_t *)calloc((size_t)n * (size_t)K, 1);
    int rc = 0;
    if (!fwd_new || !rev_new || !rev_old || !fn || !fo || !rn || !ro || !len || !cap || !clear) {
        rc = -2;
        goto out;
    }
    /* neighbourhood sizes |N(u)|, split forward/reverse and new/old */
    for (int64_t u = 0; u < n; ++u)
        for (int k = 0; k < K; ++k) {
            const orc_entry *e = st->lists + u * K + k;
            if (e->flags & ORC_NEW) {
                fwd_new[u]++;
                rev_new[e->id]++;
            } else {
                rev_old[e->id]++;
            }
        }
    for (int64_t u = 0; u < n; ++u)
        for (int k = 0; k < K; ++k) {
            const orc_entry *e = st->lists + u * K + k;
            int64_t v = e->id;
            int isnew = (e->flags & ORC_NEW) != 0;
            uint64_t fc = isnew ? (uint64_t)fwd_new[u] : (uint64_t)(K - fwd_new[u]);
            uint64_t hf = orc_hash(st->seed, ORC_STREAM_FWD, (uint32_t)iter, (uint64_t)u, (uint64_t)k);
            if (orc_accept(hf, fc, s)) {
                if (isnew) {
                    if (orc_push(&fn[u], &len[4 * u + 0], &cap[4 * u + 0], (int32_t)v)) { rc = -2; goto out; }
                    clear[u * K + k] = 1;
                } else {
                    if (orc_push(&fo[u], &len[4 * u + 1], &cap[4 * u + 1], (int32_t)v)) { rc = -2; goto out; }
                }
            }
            uint64_t rcnt = isnew ? (uint64_t)rev_new[v] : (uint64_t)rev_old[v];
            uint64_t hr = orc_hash(st->seed, ORC_STREAM_REV, (uint32_t)iter, (uint64_t)u, (uint64_t)k);
            if (orc_accept(hr, rcnt, s)) {
                if (isnew) {
                    if (orc_push(&rn[v], &len[4 * v + 2], &cap[4 * v + 2], (int32_t)u)) { rc = -2; goto out; }
                } else {
                    if (orc_push(&ro[v], &len[4 * v + 3], &cap[4 * v + 3], (int32_t)u)) { rc = -2; goto out; }
                }
            }
        }
    for (int64_t u = 0; u < n; ++u)
        for (int k = 0; k < K; ++k)
            if (clear[u * K + k]) st->lists[u * K + k].flags &= ~ORC_NEW;
    /* union with repeats removed */
    int64_t mx_rn = 0, mx_ro = 0, mx_s = 0;
    for (int64_t u = 0; u < n; ++u) {
        st->new_n[u] = 0;
        st->old_n[u] = 0;
        for (int part = 0; part < 2; ++part) {
            int32_t *src = part ? rn[u] : fn[u];
            int32_t m = len[4 * u + (part ? 2 : 0)];
            for (int32_t i = 0; i < m; ++i) {
                int dup = 0;
                for (int32_t k = 0; k < st->new_n[u]; ++k)
                    if (st->new_c[u][k] == src[i]) { dup = 1; break; }
                if (!dup && orc_push(&st->new_c[u], &st->new_n[u], &st->cap_new[u], src[i])) { rc = -2; goto out; }
            }
        }
        for (int part = 0; part < 2; ++part) {
            int32_t *src = part ? ro[u] : fo[u];
            int32_t m = len[4 * u + (part ? 3 : 1)];
            for (int32_t i = 0; i < m; ++i) {
                int dup = 0;
                for (int32_t k = 0; k < st->new_n[u] && !dup; ++k)
                    if (st->new_c[u][k] == src[i]) dup = 1;
                for (int32_t k = 0; k < st->old_n[u] && !dup; ++k)
                    if (st->old_c[u][k] == src[i]) dup = 1;
                if (!dup && orc_push(&st->old_c[u], &st->old_n[u], &st->cap_old[u], src[i])) { rc = -2; goto out; }
            }
        }
        if (len[4 * u + 2] > mx_rn) mx_rn = len[4 * u + 2];
        if (len[4 * u + 3] > mx_ro) mx_ro = len[4 * u + 3];
        if (st->new_n[u] + st->old_n[u] > mx_s) mx_s = st->new_n[u] + st->old_n[u];
    }
    if (stats) { stats[0] = mx_rn; stats[1] = mx_ro; stats[2] = mx_s; }
out:
    if (fn) for (int64_t u = 0; u < n; ++u) { free(fn[u]); free(fo[u]); free(rn[u]); free(ro[u]); }
    free(fwd_new); free(rev_new); free(rev_old); free(fn); free(fo); free(rn); free(ro);
    free(len); free(cap); free(clear);
    return rc;
}

/*
 * Update of one list (Section 2, "update G if closer vertices were found"):
 * q enters p's list iff (dist, q) orders before the worst entry and q is not
 * already listed; the worst entry leaves.  Returns 1 on insertion.
 */
/*
 * Selection step, priority-heap variant: the candidate construction of
 * PyNNDescent, which Section 3.1 sets turbosampling against.  Edge e = (u, j)
 * with v = lists[u][j] and flag f draws one priority p_e = hi32(h(seed, HEAP,
 * iter, u, j)) and offers v to u's candidates of kind f and u to v's
 * candidates of kind f, both with priority p_e.  For each node x and kind f
 * the offers are reduced to one per id (its smallest priority) and the s
 * smallest by (priority, id) are kept: a uniform sample of s distinct
 * candidates without replacement.  A forward "new" entry of x loses its flag
 * when its id is kept among x's new candidates.  new[x] = the kept new ids,
 * old[x] = the kept old ids not in new[x], both ascending by (priority, id).
 *
 * stats: [0] max reverse-new offers, [1] max reverse-old offers, [2] max |new|+|old|.
 */
typedef struct {
    uint32_t p;
    int32_t id;
} orc_offer;

static int orc_cmp_offer_id(const void *pa, const void *pb)
{
    const orc_offer *a = (const orc_offer *)pa, *b = (const orc_offer *)pb;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    if (a->p != b->p) return a->p < b->p ? -1 : 1;
    return 0;
}

static int orc_cmp_offer_p(const void *pa, const void *pb)
{
    const orc_offer *a = (const orc_offer *)pa, *b = (const orc_offer *)pb;
    if (a->p != b->p) return a->p < b->p ? -1 : 1;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    return 0;
}

int orc_sample_heap(orc_state *st, int iter, int64_t *stats)
{
    int64_t n = st->n;
    int K = st->K, s = st->s;
    int64_t *start = (int64_t *)calloc((size_t)(2 * n + 1), sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)(2 * n), sizeof(int64_t));
    orc_offer *rev = (orc_offer *)malloc(sizeof(orc_offer) * (size_t)(n * K + 1));
    uint8_t *clear = (uint8_t *)calloc((size_t)n * (size_t)K, 1);
    int rc = 0;
    if (!start || !fill || !rev || !clear) {
        rc = -2;
        goto out;
    }
    /* reverse offers of node v and kind f (0 new, 1 old) at rev[start[2v+f] ..) */
    for (int64_t u = 0; u < n; ++u)
        for (int k = 0; k < K; ++k) {
            const orc_entry *e = st->lists + u * K + k;
            start[2 * (int64_t)e->id + ((e->flags & ORC_NEW) ? 0 : 1) + 1]++;
        }
    for (int64_t i = 0; i < 2 * n; ++i) start[i + 1] += start[i];
    for (int64_t u = 0; u < n; ++u)
        for (int k = 0; k < K; ++k) {
            const orc_entry *e = st->lists + u * K + k;
            int64_t slot = 2 * (int64_t)e->id + ((e->flags & ORC_NEW) ? 0 : 1);
            orc_offer *o = rev + start[slot] + fill[slot]++;
            o->p = (uint32_t)(orc_hash(st->seed, ORC_STREAM_HEAP, (uint32_t)iter, (uint64_t)u, (uint64_t)k) >> 32);
            o->id = (int32_t)u;
        }
    int64_t mx_rn = 0, mx_ro = 0, mx_s = 0;
    for (int64_t x = 0; x < n; ++x) {
        int32_t kept[2][64];
        int nkept[2] = {0, 0};
        for (int f = 0; f < 2; ++f) {
            int64_t nrev = start[2 * x + f + 1] - start[2 * x + f];
            if (f == 0 && nrev > mx_rn) mx_rn = nrev;
            if (f == 1 && nrev > mx_ro) mx_ro = nrev;
            orc_offer *buf = (orc_offer *)malloc(sizeof(orc_offer) * (size_t)(K + nrev + 1));
            if (!buf) { rc = -2; goto out; }
            int64_t m = 0;
            for (int k = 0; k < K; ++k) {
                const orc_entry *e = st->lists + x * K + k;
                if (((e->flags & ORC_NEW) ? 0 : 1) != f) continue;
                buf[m].p = (uint32_t)(orc_hash(st->seed, ORC_STREAM_HEAP, (uint32_t)iter, (uint64_t)x, (uint64_t)k) >> 32);
                buf[m].id = e->id;
                ++m;
            }
            for (int64_t i = 0; i < nrev; ++i) buf[m++] = rev[start[2 * x + f] + i];
            /* one offer per id: its smallest priority */
            qsort(buf, (size_t)m, sizeof(orc_offer), orc_cmp_offer_id);
            int64_t w = 0;
            for (int64_t i = 0; i < m; ++i)
                if (w == 0 || buf[w - 1].id != buf[i].id) buf[w++] = buf[i];
            qsort(buf, (size_t)w, sizeof(orc_offer), orc_cmp_offer_p);
            for (int64_t i = 0; i < w && i < s; ++i) kept[f][nkept[f]++] = buf[i].id;
            free(buf);
        }
        st->new_n[x] = 0;
        st->old_n[x] = 0;
        for (int i = 0; i < nkept[0]; ++i)
            if (orc_push(&st->new_c[x], &st->new_n[x], &st->cap_new[x], kept[0][i])) { rc = -2; goto out; }
        for (int i = 0; i < nkept[1]; ++i) {
            int dup = 0;
            for (int t = 0; t < nkept[0]; ++t)
                if (kept[0][t] == kept[1][i]) dup = 1;
            if (!dup && orc_push(&st->old_c[x], &st->old_n[x], &st->cap_old[x], kept[1][i])) { rc = -2; goto out; }
        }
        for (int k = 0; k < K; ++k) {
            const orc_entry *e = st->lists + x * K + k;
            if (!(e->flags & ORC_NEW)) continue;
            for (int t = 0; t < nkept[0]; ++t)
                if (kept[0][t] == e->id) clear[x * K + k] = 1;
        }
        if (st->new_n[x] + st->old_n[x] > mx_s) mx_s = st->new_n[x] + st->old_n[x];
    }
    for (int64_t u = 0; u < n; ++u)
        for (int k = 0; k < K; ++k)
            if (clear[u * K + k]) st->lists[u * K + k].flags &= ~ORC_NEW;
    if (stats) {
        stats[0] = mx_rn;
        stats[1] = mx_ro;
        stats[2] = mx_s;
    }
out:
    free(start); free(fill); free(rev); free(clear);
    return rc;
}

/* Which selection step orc_iterate runs: 0 turbosampling, 1 priority heaps. */
int orc_set_sampler(orc_state *st, int sampler)
{
    if (sampler != 0 && sampler != 1) return -1;
    st->sampler = sampler;
    return 0;
}

static int orc_update(orc_state *st, int32_t p, int32_t q, float dist)
{
    int K = st->K;
    orc_entry *l = st->lists + (int64_t)p * K;
    orc_entry e = {dist, q, ORC_NEW | ORC_INS};
    if (!orc_less(&e, &l[K - 1])) return 0;
    for (int k = 0; k < K; ++k)
        if (l[k].id == q) return 0;
    int pos = K - 1;
    while (pos > 0 && orc_less(&e, &l[pos - 1])) {
        l[pos] = l[pos - 1];
        --pos;
    }
    l[pos] = e;
    return 1;
}

/*
 * Calculation step (Section 2 and Section 3.3): for every node u, all pairs
 * {p, q} inside new[u] and all pairs (p in new[u], q in old[u]) get their
 * squared l2 distance, and each endpoint's list is updated with the other.
 * Nodes are visited in id order and updates take effect at once.
 *
 * out[0] = distance evaluations, out[1] = successful insertions (in-place
 * count), out[2] = entries present after the step that were not present before
 * it (batched count).
 */
/* The calculation step of nodes u0 <= u < u1 only (out[0] evaluations,
 * out[1] insertions; the change count is left to a whole step).  For timing
 * a bounded share of an iteration. */
int orc_join_range(orc_state *st, int64_t u0, int64_t u1, int64_t *out)
{
    int64_t evals = 0, ins = 0;
    if (u0 < 0) u0 = 0;
    if (u1 > st->n) u1 = st->n;
    for (int64_t u = u0; u < u1; ++u) {
        const int32_t *nw = st->new_c[u];
        const int32_t *od = st->old_c[u];
        int32_t m = st->new_n[u], o = st->old_n[u];
        for (int32_t i = 0; i < m; ++i) {
            for (int32_t j = i + 1; j < m; ++j) {
                float dd = orc_dist32(st->data, st->d, nw[i], nw[j]);
                ++evals;
                ins += orc_update(st, nw[i], nw[j], dd);
                ins += orc_update(st, nw[j], nw[i], dd);
            }
            for (int32_t j = 0; j < o; ++j) {
                float dd = orc_dist32(st->data, st->d, nw[i], od[j]);
                ++evals;
                ins += orc_update(st, nw[i], od[j], dd);
                ins += orc_update(st, od[j], nw[i], dd);
            }
        }
    }
    out[0] = evals;
    out[1] = ins;
    return 0;
}

int orc_join(orc_state *st, int64_t *out)
{
    int64_t n = st->n;
    int K = st->K;
    int64_t evals = 0, ins = 0;
    for (int64_t u = 0; u < n; ++u) {
        const int32_t *nw = st->new_c[u];
        const int32_t *od = st->old_c[u];
        int32_t m = st->new_n[u], o = st->old_n[u];
        for (int32_t i = 0; i < m; ++i) {
            for (int32_t j = i + 1; j < m; ++j) {
                float dd = orc_dist32(st->data, st->d, nw[i], nw[j]);
                ++evals;
                ins += orc_update(st, nw[i], nw[j], dd);
                ins += orc_update(st, nw[j], nw[i], dd);
            }
            for (int32_t j = 0; j < o; ++j) {
                float dd = orc_dist32(st->data, st->d, nw[i], od[j]);
                ++evals;
                ins += orc_update(st, nw[i], od[j], dd);
                ins += orc_update(st, od[j], nw[i], dd);
            }
        }
    }
    int64_t surv = 0;
    for (int64_t i = 0; i < n * K; ++i) {
        if (st->lists[i].flags & ORC_INS) {
            ++surv;
            st->lists[i].flags &= ~ORC_INS;
        }
    }
    out[0] = evals;
    out[1] = ins;
    out[2] = surv;
    return 0;
}

/* Read the candidate sets produced by the last orc_sample. */
int orc_get_samples(const orc_state *st, int cap, int32_t *new_ids, int32_t *new_cnt,
                    int32_t *old_ids, int32_t *old_cnt)
{
    for (int64_t u = 0; u < st->n; ++u) {
        new_cnt[u] = st->new_n[u];
        old_cnt[u] = st->old_n[u];
        for (int32_t i = 0; i < cap; ++i) {
            new_ids[u * cap + i] = i < st->new_n[u] ? st->new_c[u][i] : -1;
            old_ids[u * cap + i] = i < st->old_n[u] ? st->old_c[u][i] : -1;
        }
    }
    return 0;
}

/* Replace the candidate sets (for join tests with hand-made sets). */
int orc_set_samples(orc_state *st, int cap, const int32_t *new_ids, const int32_t *new_cnt,
                    const int32_t *old_ids, const int32_t *old_cnt)
{
    for (int64_t u = 0; u < st->n; ++u) {
        st->new_n[u] = 0;
        st->old_n[u] = 0;
        for (int32_t i = 0; i < new_cnt[u] && i < cap; ++i)
            if (orc_push(&st->new_c[u], &st->new_n[u], &st->cap_new[u], new_ids[u * cap + i])) return -2;
        for (int32_t i = 0; i < old_cnt[u] && i < cap; ++i)
            if (orc_push(&st->old_c[u], &st->old_n[u], &st->cap_old[u], old_ids[u * cap + i])) return -2;
    }
    return 0;
}

/*
 * Greedy clustering heuristic (Section 3.2, Algorithm 1).  sigma maps a node to
 * its new spot, sigma_inv a spot to its node, both start as the identity.  For
 * spot i = 0 .. n-2 the list a_i (ascending by distance) is scanned: entries
 * already on a spot before i+1 are skipped; an entry already on spot i+1 ends
 * the scan; an entry x on a later spot p is moved to spot i+1 and the node y
 * that held spot i+1 moves to spot p.  The second swap of the algorithm uses
 * the value sigma(x) = p held before the first swap.  reading_b = 0 scans the
 * list of the node on spot i (sigma_inv(i)); reading_b = 1 scans the list of
 * node i.  lists: n x K ids, each row ascending by distance.
 */
int orc_greedy_reorder(const int32_t *lists, int64_t n, int K, int reading_b,
                       int32_t *sigma, int32_t *sigma_inv)
{
    for (int64_t i = 0; i < n; ++i) {
        sigma[i] = (int32_t)i;
        sigma_inv[i] = (int32_t)i;
    }
    for (int64_t i = 0; i + 1 < n; ++i) {
        int64_t node = reading_b ? i : sigma_inv[i];
        const int32_t *a = lists + node * K;
        for (int j = 0; j < K; ++j) {
            int32_t x = a[j];
            int64_t p = sigma[x];
            if (p < i + 1) continue;
            if (p == i + 1) break;
            int32_t y = sigma_inv[i + 1];
            sigma[x] = (int32_t)(i + 1);
            sigma[y] = (int32_t)p;
            sigma_inv[i + 1] = x;
            sigma_inv[p] = y;
            break;
        }
    }
    return 0;
}

/*
 * Move every node u to spot sigma(u) at once (Section 3.2): its point, its
 * list (ids renamed through sigma, re-sorted by (dist, new id)).
 */
/*
 * Parallel relabelling variant (a data-parallel alternative to Algorithm 1,
 * Section 3.2): single-linkage agglomeration by Boruvka rounds on the graph of
 * the lists.  Edges are the list entries {u, v}, undirected, ordered by
 * (float32 distance, min(u, v), max(u, v)).  Each round every component picks
 * its smallest outgoing edge and hooks onto the component at its other end;
 * where two components picked the same edge the one with the smaller
 * representative stays the root; every component then takes the
 * representative at the end of its hooks.  Rounds stop when no component has
 * an outgoing edge (or after rmax).
 *
 * levels[r * n + u] = representative of u's component after round r, for
 * r < *rounds.  weight = total distance of the hooked edges (each counted
 * once): a minimum spanning forest of the list graph.  sigma[u] = spot of u
 * in the layout that sorts points by (levels[R-1], ..., levels[0], u): every
 * component of every round is one contiguous range.
 */
static const int32_t *orc_lv;
static int64_t orc_lv_n;
static int orc_lv_r;

static int orc_cmp_levels(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    for (int r = orc_lv_r - 1; r >= 0; --r) {
        int32_t x = orc_lv[(int64_t)r * orc_lv_n + a], y = orc_lv[(int64_t)r * orc_lv_n + b];
        if (x != y) return x < y ? -1 : 1;
    }
    return a < b ? -1 : (a > b ? 1 : 0);
}

int orc_parallel_relabel(const float *data, int64_t n, int d, int K, const int32_t *ids, int rmax,
                         int32_t *levels, int *rounds, double *weight, int32_t *sigma)
{
    int32_t *comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *broke = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint64_t *best1 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    uint32_t *best2 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    float *dist = (float *)malloc(sizeof(float) * (size_t)n * (size_t)K);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!comp || !parent || !broke || !best1 || !best2 || !dist || !order) {
        free(comp); free(parent); free(broke); free(best1); free(best2); free(dist); free(order);
        return -2;
    }
    for (int64_t u = 0; u < n; ++u) {
        comp[u] = (int32_t)u;
        for (int k = 0; k < K; ++k) dist[u * K + k] = orc_dist32(data, d, u, ids[u * K + k]);
    }
    double w = 0.0;
    int r = 0;
    for (; r < rmax; ++r) {
        for (int64_t c = 0; c < n; ++c) {
            best1[c] = UINT64_MAX;
            best2[c] = UINT32_MAX;
        }
        for (int pass = 0; pass < 2; ++pass)
            for (int64_t u = 0; u < n; ++u)
                for (int k = 0; k < K; ++k) {
                    uint32_t v = (uint32_t)ids[u * K + k], uu = (uint32_t)u;
                    int32_t cu = comp[u], cv = comp[v];
                    if (cu == cv) continue;
                    uint32_t bits;
                    memcpy(&bits, &dist[u * K + k], sizeof(bits));
                    uint64_t k1 = ((uint64_t)bits << 32) | (uint64_t)(uu < v ? uu : v);
                    uint32_t mx = uu < v ? v : uu;
                    if (pass == 0) {
                        if (k1 < best1[cu]) best1[cu] = k1;
                        if (k1 < best1[cv]) best1[cv] = k1;
                    } else {
                        if (best1[cu] == k1 && mx < best2[cu]) best2[cu] = mx;
                        if (best1[cv] == k1 && mx < best2[cv]) best2[cv] = mx;
                    }
                }
        int64_t hooks = 0;
        for (int64_t c = 0; c < n; ++c) {
            if (comp[c] != (int32_t)c) continue;
            if (best1[c] == UINT64_MAX) {
                parent[c] = (int32_t)c;
                continue;
            }
            uint32_t a = (uint32_t)best1[c], b = best2[c];
            uint32_t other = comp[a] == (int32_t)c ? b : a;
            parent[c] = comp[other];
            ++hooks;
        }
        if (hooks == 0) break;
        /* 2-cycles: the smaller representative stays the root */
        for (int64_t c = 0; c < n; ++c) broke[c] = 0;
        for (int64_t c = 0; c < n; ++c) {
            if (comp[c] != (int32_t)c) continue;
            int32_t p = parent[c];
            if (p != (int32_t)c && parent[p] == (int32_t)c && (int32_t)c < p) broke[c] = 1;
        }
        for (int64_t c = 0; c < n; ++c) {
            if (comp[c] != (int32_t)c) continue;
            if (broke[c]) parent[c] = (int32_t)c;
            if (parent[c] != (int32_t)c) {
                float f;
                uint32_t bits = (uint32_t)(best1[c] >> 32);
                memcpy(&f, &bits, sizeof(f));
                w += (double)f;
            }
        }
        for (int64_t u = 0; u < n; ++u) {
            int32_t x = comp[u];
            while (parent[x] != x) x = parent[x];
            order[u] = x;
        }
        for (int64_t u = 0; u < n; ++u) {
            comp[u] = order[u];
            levels[(int64_t)r * n + u] = comp[u];
        }
    }
    *rounds = r;
    if (weight) *weight = w;
    for (int64_t u = 0; u < n; ++u) order[u] = (int32_t)u;
    orc_lv = levels;
    orc_lv_n = n;
    orc_lv_r = r;
    qsort(order, (size_t)n, sizeof(int32_t), orc_cmp_levels);
    for (int64_t i = 0; i < n; ++i) sigma[order[i]] = (int32_t)i;
    free(comp); free(parent); free(broke); free(best1); free(best2); free(dist); free(order);
    return 0;
}

static int orc_apply_permutation(orc_state *st, const int32_t *sigma)
{
    int64_t n = st->n;
    int K = st->K, d = st->d;
    float *nd = (float *)malloc(sizeof(float) * (size_t)n * (size_t)d);
    orc_entry *nl = (orc_entry *)malloc(sizeof(orc_entry) * (size_t)n * (size_t)K);
    if (!nd || !nl) { free(nd); free(nl); return -2; }
    for (int64_t u = 0; u < n; ++u) {
        int64_t p = sigma[u];
        memcpy(nd + p * d, st->data + u * d, sizeof(float) * (size_t)d);
        for (int k = 0; k < K; ++k) {
            orc_entry e = st->lists[u * K + k];
            e.id = sigma[e.id];
            nl[p * K + k] = e;
        }
        orc_sort_list(nl + p * K, K);
    }
    free(st->data);
    free(st->lists);
    st->data = nd;
    st->lists = nl;
    /* compose: original node -> spot */
    for (int64_t u = 0; u < n; ++u) st->sigma[u] = sigma[st->sigma[u]];
    st->reordered = 1;
    return 0;
}

int orc_reorder(orc_state *st, int reading_b)
{
    int64_t n = st->n;
    int K = st->K;
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)K);
    int32_t *sg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *si = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int rc = -2;
    if (ids && sg && si) {
        for (int64_t i = 0; i < n * K; ++i) ids[i] = st->lists[i].id;
        orc_greedy_reorder(ids, n, K, reading_b, sg, si);
        rc = orc_apply_permutation(st, sg);
    }
    free(ids); free(sg); free(si);
    return rc;
}

/* One iteration: selection then calculation.  out as in orc_join plus
 * out[3..5] = the sampling stats. */
int orc_iterate(orc_state *st, int64_t *out)
{
    int it = st->iter + 1;
    int rc = st->sampler ? orc_sample_heap(st, it, out + 3) : orc_sample(st, it, out + 3);
    if (rc) return rc;
    rc = orc_join(st, out);
    if (rc) return rc;
    st->iter = it;
    return 0;
}

/* Current state in the current labelling: ids, dists, flags (n x K). */
int orc_get_state(const orc_state *st, int32_t *ids, float *dists, uint8_t *flags)
{
    for (int64_t i = 0; i < st->n * st->K; ++i) {
        if (ids) ids[i] = st->lists[i].id;
        if (dists) dists[i] = st->lists[i].dist;
        if (flags) flags[i] = (uint8_t)(st->lists[i].flags & ORC_NEW);
    }
    return 0;
}

/* Final graph in the original labelling, rows ascending by (dist, id). */
int orc_get_graph(const orc_state *st, int32_t *ids, float *dists)
{
    int64_t n = st->n;
    int K = st->K;
    int32_t *inv = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    orc_entry *tmp = (orc_entry *)malloc(sizeof(orc_entry) * (size_t)K);
    if (!inv || !tmp) { free(inv); free(tmp); return -2; }
    for (int64_t u = 0; u < n; ++u) inv[st->sigma[u]] = (int32_t)u;
    for (int64_t u = 0; u < n; ++u) {
        int64_t p = st->sigma[u];
        for (int k = 0; k < K; ++k) {
            tmp[k] = st->lists[p * K + k];
            tmp[k].id = inv[tmp[k].id];
        }
        orc_sort_list(tmp, K);
        for (int k = 0; k < K; ++k) {
            ids[u * K + k] = tmp[k].id;
            dists[u * K + k] = tmp[k].dist;
        }
    }
    free(inv);
    free(tmp);
    return 0;
}

int orc_get_sigma(const orc_state *st, int32_t *sigma)
{
    memcpy(sigma, st->sigma, sizeof(int32_t) * (size_t)st->n);
    return 0;
}

void orc_free(orc_state *st)
{
    if (!st) return;
    if (st->new_c) for (int64_t u = 0; u < st->n; ++u) free(st->new_c[u]);
    if (st->old_c) for (int64_t u = 0; u < st->n; ++u) free(st->old_c[u]);
    free(st->new_c); free(st->old_c); free(st->new_n); free(st->old_n);
    free(st->cap_new); free(st->cap_old);
    free(st->data); free(st->lists); free(st->sigma);
    free(st);
}

/*
 * Whole NN-Descent (Section 2): random initialisation, then iterations of
 * selection + calculation until the number of changes falls below
 * delta * n * K or max_iters iterations have run.  count_mode 0 = batched
 * count (entries new to a list after the iteration), 1 = in-place count
 * (successful sequential insertions).  reorder: 0 none, 1 Algorithm 1 reading
 * A after the first iteration, 2 reading B.  sampler: 0 turbosampling, 1
 * priority heaps.  stats (may be NULL), int64 x 4: iterations run, total
 * distance evaluations, last change count, reordered.
 */
int orc_build(const float *data, int64_t n, int d, int K, float rho, float delta,
              int max_iters, uint64_t seed, int count_mode, int reorder, int sampler,
              int32_t *ids, float *dists, int64_t *stats)
{
    if (delta < 0.0f || max_iters < 0) return -1;
    orc_state *st = orc_create(data, n, d, K, rho, seed);
    if (!st) return -1;
    if (orc_set_sampler(st, sampler)) {
        orc_free(st);
        return -1;
    }
    int rc = orc_init_random(st);
    int64_t evals = 0, last = 0;
    double thr = (double)delta * (double)n * (double)K;
    for (int it = 0; rc == 0 && it < max_iters; ++it) {
        int64_t out[6];
        rc = orc_iterate(st, out);
        if (rc) break;
        evals += out[0];
        last = count_mode ? out[1] : out[2];
        if (it == 0 && reorder) rc = orc_reorder(st, reorder == 2);
        if ((double)last < thr) break;
    }
    if (rc == 0) rc = orc_get_graph(st, ids, dists);
    if (stats) {
        stats[0] = st->iter; stats[1] = evals; stats[2] = last; stats[3] = st->reordered;
    }
    orc_free(st);
    return rc;
}

/* ------------------------------------------------ batched, multi-thread ---- */

/*
 * The same NN-Descent in batched mode on several threads.  Reading 6 of the
 * paper's Section 2 loop: within one iteration the candidate sets are fixed,
 * so every pair of the calculation step has the same distance whatever the
 * order, and a list that takes each of its proposals by the update rule of
 * orc_update ends as the K smallest distinct (dist, id) keys among its entries
 * and those proposals, in any order.  So this build visits the nodes in blocks
 * (each block split over the threads by u): the join of a block computes its
 * pairs and keeps a proposal (p, q, dist) only when (dist, q) orders before
 * p's current worst entry (one that does not can never enter, since a list's
 * worst entry only falls); then every thread applies the block's proposals to
 * the lists of its own range of targets with orc_update.  Selection is
 * orc_sample (serial) and the change count is the batched one (entries present
 * after the iteration that were not before), so the result equals orc_build
 * with count_mode 0, for any number of threads.
 */
typedef struct {
    int32_t p, q;
    float dist;
} orc_prop;

typedef struct {
    orc_prop *a;
    int64_t len, cap;
} orc_pvec;

typedef struct {
    orc_state *st;
    int threads;
    int64_t u0, u1;          /* the block */
    int64_t *next;           /* next node of the block to join (shared) */
    orc_pvec *buf;           /* threads x threads: [worker][target range] */
    int64_t evals;           /* this worker's distance evaluations */
    int64_t ins;             /* this worker's insertions */
    int worker, fail;
} orc_work;

static int orc_pvec_push(orc_pvec *v, int32_t p, int32_t q, float dist)
{
    if (v->len == v->cap) {
        int64_t nc = v->cap ? v->cap * 2 : 1024;
        orc_prop *na = (orc_prop *)realloc(v->a, sizeof(orc_prop) * (size_t)nc);
        if (!na) return -1;
        v->a = na;
        v->cap = nc;
    }
    v->a[v->len].p = p;
    v->a[v->len].q = q;
    v->a[v->len].dist = dist;
    v->len++;
    return 0;
}

/* target range of node p: [p * threads / n] */
static int orc_range_of(int64_t p, int64_t n, int threads)
{
    return (int)((p * (int64_t)threads) / n);
}

/* propose q to p when (dist, q) orders before p's worst entry */
static int orc_propose(orc_work *w, int32_t p, int32_t q, float dist)
{
    orc_state *st = w->st;
    const orc_entry *worst = st->lists + (int64_t)p * st->K + (st->K - 1);
    orc_entry e = {dist, q, 0u};
    if (!orc_less(&e, worst)) return 0;
    return orc_pvec_push(&w->buf[(int64_t)w->worker * w->threads + orc_range_of(p, st->n, w->threads)], p, q, dist);
}

static void *orc_join_worker(void *arg)
{
    orc_work *w = (orc_work *)arg;
    orc_state *st = w->st;
    for (;;) {
        int64_t u = __atomic_fetch_add(w->next, 1, __ATOMIC_RELAXED);
        if (u >= w->u1) break;
        const int32_t *nw = st->new_c[u], *od = st->old_c[u];
        int32_t m = st->new_n[u], o = st->old_n[u];
        for (int32_t i = 0; i < m; ++i) {
            for (int32_t j = i + 1; j < m; ++j) {
                float dd = orc_dist32(st->data, st->d, nw[i], nw[j]);
                ++w->evals;
                if (orc_propose(w, nw[i], nw[j], dd) || orc_propose(w, nw[j], nw[i], dd)) { w->fail = 1; return NULL; }
            }
            for (int32_t j = 0; j < o; ++j) {
                float dd = orc_dist32(st->data, st->d, nw[i], od[j]);
                ++w->evals;
                if (orc_propose(w, nw[i], od[j], dd) || orc_propose(w, od[j], nw[i], dd)) { w->fail = 1; return NULL; }
            }
        }
    }
    return NULL;
}

static void *orc_apply_worker(void *arg)
{
    orc_work *w = (orc_work *)arg;
    for (int src = 0; src < w->threads; ++src) {
        orc_pvec *v = &w->buf[(int64_t)src * w->threads + w->worker];
        for (int64_t i = 0; i < v->len; ++i) w->ins += orc_update(w->st, v->a[i].p, v->a[i].q, v->a[i].dist);
        v->len = 0;
    }
    return NULL;
}

/* pairs per block of orc_join_mt (tests make it small to cross blocks) */
static int64_t orc_mt_block_pairs = (int64_t)1 << 25;

int orc_set_mt_block_pairs(int64_t pairs)
{
    if (pairs < 1) return -1;
    orc_mt_block_pairs = pairs;
    return 0;
}

static int orc_run_workers(orc_work *w, int threads, void *(*fn)(void *))
{
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    if (!tid) return -2;
    int started = 0, rc = 0;
    for (int t = 1; t < threads; ++t) {
        if (pthread_create(&tid[t], NULL, fn, &w[t]) != 0) { rc = -2; break; }
        ++started;
    }
    fn(&w[0]);
    for (int t = 1; t <= started; ++t) pthread_join(tid[t], NULL);
    free(tid);
    return rc;
}

/* One calculation step in batched mode: out as in orc_join. */
static int orc_join_mt(orc_state *st, int threads, int64_t *out)
{
    int64_t n = st->n;
    orc_work *w = (orc_work *)calloc((size_t)threads, sizeof(orc_work));
    orc_pvec *buf = (orc_pvec *)calloc((size_t)threads * (size_t)threads, sizeof(orc_pvec));
    int rc = 0;
    if (!w || !buf) { free(w); free(buf); return -2; }
    int64_t next = 0;
    for (int t = 0; t < threads; ++t) {
        w[t].st = st;
        w[t].threads = threads;
        w[t].buf = buf;
        w[t].worker = t;
        w[t].next = &next;
    }
    /* blocks of about orc_mt_block_pairs pairs (2^25 by default), so the
     * kept proposals stay within a few hundred MB */
    int64_t u0 = 0;
    while (u0 < n && rc == 0) {
        int64_t pairs = 0, u1 = u0;
        while (u1 < n && (u1 == u0 || pairs < orc_mt_block_pairs)) {
            int64_t m = st->new_n[u1], o = st->old_n[u1];
            pairs += m * (m - 1) / 2 + m * o;
            ++u1;
        }
        next = u0;
        for (int t = 0; t < threads; ++t) { w[t].u0 = u0; w[t].u1 = u1; }
        rc = orc_run_workers(w, threads, orc_join_worker);
        for (int t = 0; t < threads; ++t) if (w[t].fail) rc = -2;
        if (rc == 0) rc = orc_run_workers(w, threads, orc_apply_worker);
        u0 = u1;
    }
    int64_t evals = 0, ins = 0;
    for (int t = 0; t < threads; ++t) { evals += w[t].evals; ins += w[t].ins; }
    for (int64_t i = 0; i < (int64_t)threads * threads; ++i) free(buf[i].a);
    free(w);
    free(buf);
    if (rc) return rc;
    int64_t surv = 0;
    for (int64_t i = 0; i < n * st->K; ++i) {
        if (st->lists[i].flags & ORC_INS) {
            ++surv;
            st->lists[i].flags &= ~ORC_INS;
        }
    }
    out[0] = evals;
    out[1] = ins;
    out[2] = surv;
    return 0;
}

/* Threads the multi-thread build uses for threads <= 0: the online cores. */
int orc_default_threads(void)
{
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c < 1 ? 1 : (c > 256 ? 256 : (int)c);
}

/*
 * Whole NN-Descent, batched mode, on `threads` threads (<= 0: every online
 * core): the loop of orc_build with count_mode 0 and the calculation step of
 * orc_join_mt.  Turbosampling, no reordering.  stats as in orc_build, plus
 * stats[4] = the threads used.
 */
int orc_build_mt(const float *data, int64_t n, int d, int K, float rho, float delta,
                 int max_iters, uint64_t seed, int threads, int32_t *ids, float *dists, int64_t *stats)
{
    if (delta < 0.0f || max_iters < 0) return -1;
    if (threads <= 0) threads = orc_default_threads();
    if (threads > 256) threads = 256;
    orc_state *st = orc_create(data, n, d, K, rho, seed);
    if (!st) return -1;
    int rc = orc_init_random(st);
    int64_t evals = 0, last = 0;
    double thr = (double)delta * (double)n * (double)K;
    for (int it = 0; rc == 0 && it < max_iters; ++it) {
        int64_t out[3], sst[3];
        rc = orc_sample(st, st->iter + 1, sst);
        if (rc) break;
        rc = orc_join_mt(st, threads, out);
        if (rc) break;
        st->iter++;
        evals += out[0];
        last = out[2];
        if ((double)last < thr) break;
    }
    if (rc == 0) rc = orc_get_graph(st, ids, dists);
    if (stats) {
        stats[0] = st->iter; stats[1] = evals; stats[2] = last; stats[3] = 0; stats[4] = threads;
    }
    orc_free(st);
    return rc;
}
