/*
 * knng.h -- C ABI of the GB300 (sm_103a) NN-Descent K-nearest-neighbour graph
 * library for the squared l2 metric.
 *
 * The method is NN-Descent as optimised in "Fast single-core K-Nearest
 * Neighbor Graph computation" (Kluser, Bokstaller, Rutz, Buner): random
 * initialisation (Section 2), one-pass probability sampling of forward and
 * reverse neighbours (Section 3.1), the local join that evaluates squared l2
 * distances between candidate pairs and updates both endpoints' lists
 * (Section 2, Section 3.3), termination on the number of changes (Section 2)
 * and the greedy clustering relabelling (Section 3.2, Algorithm 1).  Every
 * step runs in CUDA kernels; this header is the only boundary.
 *
 * Conventions shared by every call
 *   - Points: `data` is n x d float32, row-major, contiguous (row stride d).
 *     It may be a host pointer or a device pointer of the current device (or
 *     managed memory it can reach); the library tells them apart with
 *     cudaPointerGetAttributes.  Host inputs are copied to the device; host
 *     outputs are filled by a device-to-host copy; each buffer may be host or
 *     device independently of the others.  Another device's memory, in any
 *     argument, is refused with KNNG_ERR_INVALID_ARG before anything runs.
 *   - Output graph: ids[u*K + j] (int32) and dists[u*K + j] (float32 squared
 *     l2) hold u's j-th nearest neighbour found; each row is ascending by
 *     (dist, id), holds no self-loop and no repeated id.
 *   - Ownership: the caller owns data, ids, dists and every other pointer it
 *     passes; the library never frees them.  A knng_ctx owns all device
 *     memory it allocates and frees it in knng_destroy.
 *   - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 *     All work is enqueued on it.  Calls that return device-computed numbers
 *     to the host (knng_iterate's change count, host outputs) synchronise that
 *     stream only, never the whole device.
 *   - Errors: every call returns KNNG_OK (0), a negative KNNG_ERR_* code, or
 *     the positive warning KNNG_WARN_OVERFLOW (result valid, but some sampled
 *     candidates did not fit their fixed capacity and were skipped).  No C++
 *     exception crosses this boundary.  knng_strerror names a code.
 *   - Limits: 2 <= n < 2^30 - 1, 1 <= d, 1 <= K <= min(64, n - 1),
 *     0 < rho <= 1, delta >= 0, 0 <= max_iters <= 1000.  K up to 32 holds a
 *     list one key per lane of a warp, K of 33 to 64 two keys per lane; the
 *     latter builds float32 keys with turbosampling only (KNNG_FLAG_BF16,
 *     KNNG_FLAG_FP8 and KNNG_FLAG_HEAP_SAMPLING with K > 32 return
 *     KNNG_ERR_UNSUPPORTED, as does K > 64).
 */
#ifndef KNNG_H_
#define KNNG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KNNG_OK 0
#define KNNG_WARN_OVERFLOW 1
#define KNNG_ERR_INVALID_ARG (-1)
#define KNNG_ERR_OOM (-2)
#define KNNG_ERR_CUDA (-3)
#define KNNG_ERR_TIMEOUT (-4)
#define KNNG_ERR_UNSUPPORTED (-5)
#define KNNG_ERR_STATE (-6)
#define KNNG_ERR_INTERNAL (-7)

/* flags for knng_init / knng_build_ex */
#define KNNG_FLAG_REORDER 0x1u   /* Algorithm 1 (list of the node on spot i) + relabel after iteration 1 */
#define KNNG_FLAG_REORDER_B 0x2u /* with REORDER: the literal reading (list of node i) */
#define KNNG_FLAG_TIMING 0x4u    /* record CUDA events around every local-join and list-merge launch */
#define KNNG_FLAG_GRAPH 0x8u     /* knng_run: capture the iteration loop as one CUDA graph and launch it */
#define KNNG_FLAG_BF16 0x10u     /* d >= 64: local-join dots in bf16 on the tensor cores (float32
                                    accumulate, |x|^2+|y|^2-2x.y); output re-ranked in float32 */
#define KNNG_FLAG_AUTOTUNE 0x20u /* time every join kernel the geometry allows on the first iteration of the
                                    first context with this geometry (d, K, precision) in the process, and
                                    use the fastest from then on; that iteration synchronises */
#define KNNG_FLAG_HEAP_SAMPLING 0x40u /* candidate selection by priority heaps (PyNNDescent's construction)
                                        instead of Section 3.1's turbosampling: edge (u, j) draws one
                                        priority hi32(h(seed, 4, it, u, j)) for both of its offers (v to
                                        u, u to v, of the edge's new/old kind); each node keeps per kind
                                        the s smallest (priority, id) offers, one per id; forward new
                                        entries kept as new candidates lose their flag; requires
                                        n * K < 2^31 (else KNNG_ERR_UNSUPPORTED) */
#define KNNG_FLAG_FP8 0x100u /* d >= 64, rows that fit the ring join kernel: local-join dots in FP8 (e4m3 rows,
                                rounded to nearest and saturated at +-448, float32 accumulate on the tensor
                                cores, |x|^2+|y|^2-2x.y with the norms of the e4m3 values); output re-ranked
                                in float32.  Lossy beyond 4 significant bits (integers up to 16 are exact,
                                larger ones round); takes precedence over KNNG_FLAG_BF16 */
#define KNNG_FLAG_REORDER_PARALLEL 0x80u /* with REORDER: relabel by the data-parallel variant instead of
                                           Algorithm 1 -- single-linkage (Boruvka) rounds on the list graph,
                                           edges ordered by (float32 distance, min id, max id), every
                                           component of every round laid out in one contiguous range of
                                           spots; the order of siblings inside a parent's range comes from
                                           atomics, so it is not reproducible run to run */

typedef struct knng_ctx knng_ctx;

/* Counters read back by knng_get_stats.  Work counters add up over all
 * iterations run so far. */
typedef struct knng_stats {
    int64_t n;
    int32_t d, K, s;           /* s = ceil(rho * K), the sample size per kind */
    int32_t iterations;        /* iterations that ran (converged ones skip) */
    int64_t dist_evals;        /* local-join distance evaluations */
    int64_t last_changes;      /* list entries new after the last iteration run */
    int64_t inserts;           /* successful list insertions (incl. later evicted) */
    int64_t merges;            /* locked list merges */
    int64_t gathered_rows;     /* candidate rows read by the local join */
    int64_t rev_overflow;      /* reverse candidates skipped (capacity R per kind) */
    int64_t set_overflow;      /* candidates skipped beyond 64 per node and iteration */
    int64_t lock_timeouts;     /* bounded lock waits that gave up (then KNNG_ERR_TIMEOUT) */
    int64_t kernel_launches;   /* kernels this context launched */
    int64_t cand_ids;          /* sampled candidate ids read by the local join */
    int64_t proposals;         /* proposal keys the local join handed to the list merge */
    int64_t bucket_overflow;   /* proposals past a full bucket (inserted under a lock) */
    int32_t reordered;         /* 1 once Algorithm 1 relabelled the points */
    int32_t join_launches;     /* iterations whose local join was timed (KNNG_FLAG_TIMING) */
    double join_ms;            /* their summed CUDA-event time: every join pass of an iteration
                                  (an iteration with many candidates runs its join over node
                                  ranges, a list merge after each), merges excluded */
    int32_t join_ran;          /* timed iterations that ran (not skipped) */
    int32_t join_path;         /* local-join kernel: 0 warp per node (float32 rows of up to 32
                                  floats), 1 block-per-node tiles, 2 ring of nodes in flight
                                  (bf16 and FP8 rows), 3 pipelined block per node (float32 rows
                                  of 33 to 256 floats; four warps, one row slot), 4 the same
                                  with eight warps and two row slots */
    double join_ms_ran;        /* summed join-kernel time of those iterations (all passes) */
    double merge_ms_ran;       /* summed list-merge-kernel time of those iterations (all passes) */
    double sample_ms_ran;      /* summed selection-step time (degree count + sampling kernels) of
                                  those iterations (KNNG_FLAG_TIMING) */
    double reorder_ms;         /* summed relabelling time, permutation of rows and lists included
                                  (KNNG_FLAG_TIMING) */
} knng_stats;

/*
 * One-shot K-NNG build (Section 2): random init, then up to max_iters
 * iterations of selection + calculation, stopping after the first iteration
 * whose change count is below delta * n * K; the final lists carry float32
 * difference-form distances (float32 keys hold them already; the bf16 and
 * FP8 forms re-rank with them).  rho sets the sample size s = ceil(rho * K)
 * (Section 3.1).  seed drives every random choice through a counter-based
 * SplitMix64 hash, and the candidate cap drops a canonical tail, so a build
 * is reproducible bit for bit.  Uses the legacy
 * default stream and no flags; returns when ids/dists are written.
 */
int knng_build(const float *data, int64_t n, int d, int K, float rho, float delta,
               int max_iters, uint64_t seed, int32_t *ids, float *dists);

/* knng_build with flags (KNNG_FLAG_*), a stream and optional statistics
 * (stats may be NULL).  With device outputs the call does not wait for the
 * results beyond what reading stats needs. */
int knng_build_ex(const float *data, int64_t n, int d, int K, float rho, float delta,
                  int max_iters, uint64_t seed, uint32_t flags, void *stream,
                  int32_t *ids, float *dists, knng_stats *stats);

/*
 * Create a context and run the random initialisation (Section 2: K distinct
 * neighbours != u per point, uniform over V).  Allocates all device memory
 * the build needs: the padded points, lists, candidate arrays and proposal
 * buckets take about 2.5 KiB + 4 (d rounded up to 4) + 16 K + 16 s bytes per
 * point (s = ceil(rho K)), plus a bucket pool of 4 KiB per point up to
 * 16 GiB (at d = 128, K = 32, rho 0.7: 7.8 KiB per point up to 4M points,
 * then 3.8 KiB per point plus 16 GiB; past 4M points an iteration runs in
 * more node-range passes instead).  *out is NULL on error.
 */
int knng_init(knng_ctx **out, const float *data, int64_t n, int d, int K, float rho,
              float delta, uint64_t seed, uint32_t flags, void *stream);

/*
 * Create a context whose starting graph is given: ids (n x K, each row K
 * distinct ids != u) and is_new (n x K bytes, nonzero = "new" flag).  Lists
 * are sorted and their distances computed on the device.  `iter` is the
 * number of iterations already done (the next knng_iterate runs iter + 1, which
 * selects the random stream).  For resuming a build and for step-level tests.
 */
int knng_init_from_graph(knng_ctx **out, const float *data, int64_t n, int d, int K,
                         float rho, float delta, uint64_t seed, uint32_t flags, void *stream,
                         const int32_t *ids, const uint8_t *is_new, int iter);

/*
 * One NN-Descent iteration (Section 2): degree counting and one-pass sampling
 * (Section 3.1), then the local join with list updates (Sections 2, 3.3).
 * With KNNG_FLAG_REORDER, the first iteration is followed by Algorithm 1 and
 * the relabelling (Section 3.2).  Synchronises the stream and writes the
 * iteration's change count to *changes_out (may be NULL).  Returns 1 when the
 * count is below delta * n * K (converged), 0 otherwise, or an error.
 */
int knng_iterate(knng_ctx *ctx, int64_t *changes_out);

/*
 * Enqueue up to max_iters iterations without host round trips: each iteration's
 * kernels skip themselves on the device once a previous iteration's change count
 * fell below delta * n * K.  With KNNG_FLAG_GRAPH the loop is captured (stream
 * capture, thread-local mode) and launched as one CUDA graph.  Does not
 * synchronise.
 */
int knng_run(knng_ctx *ctx, int max_iters);

/* Algorithm 1 on the current lists (the node on spot i, or node i with
 * KNNG_FLAG_REORDER_B) and the relabelling of points and lists (Section 3.2).
 * Normally run by knng_iterate after the first iteration. */
int knng_reorder(knng_ctx *ctx);

/*
 * Final graph in the caller's labelling: every entry's distance recomputed in
 * float32 difference form, rows sorted by (dist, original id).  ids/dists are
 * n x K, host or device.
 */
int knng_get(knng_ctx *ctx, int32_t *ids, float *dists);

/*
 * Raw current state in the current (possibly relabelled) labelling: ids, list
 * distances, flags (bit 0 = new).  Any pointer may be NULL.  Host pointers.
 */
int knng_get_state(knng_ctx *ctx, int32_t *ids, float *dists, uint8_t *flags);

/*
 * Candidate sets of the last iteration's selection step, after repeats were
 * removed, in the current labelling: new_ids / old_ids are n x cap (host),
 * unused slots -1, counts in new_cnt / old_cnt.  Order within a set is not
 * specified.  Sets are kept until the next iteration.  For tests.
 */
int knng_get_samples(knng_ctx *ctx, int cap, int32_t *new_ids, int32_t *new_cnt,
                     int32_t *old_ids, int32_t *old_cnt);

/* sigma (n, host): the spot of each original point; identity until reordered. */
int knng_get_permutation(knng_ctx *ctx, int32_t *sigma);

/* Counters; synchronises the stream. */
int knng_get_stats(knng_ctx *ctx, knng_stats *stats);

/* Free a context and its device memory (stream-ordered).  NULL is fine. */
int knng_destroy(knng_ctx *ctx);

/* One data set of a batched build: n x d float32 points (host or device),
 * outputs n x K (host or device), ids local to the data set. */
typedef struct knng_desc {
    const float *data;
    int64_t n;
    int32_t d;
    int32_t *ids;
    float *dists;
} knng_desc;

/*
 * K-NNGs of many independent data sets in one run (each as knng_build with
 * the same K, rho, delta, max_iters, seed and flags).  The data sets are
 * grouped by row-width class (d up to 32, 48, 64, 96, 128, 192, 256, ...,
 * each class 4/3 or 3/2 of the one before); the data sets of a class share
 * one node space, so every step of every iteration is one kernel launch for
 * all of them, and their rows are zero-padded to the class width (this leaves
 * every distance unchanged).  Each data set stops on its own change count
 * (delta * n_b * K), and the random streams are keyed by ids local to the data
 * set, so each result equals what knng_build_ex gives for that data set alone.
 * stats (may be NULL) sums the counters of all classes.
 * Requires 2 <= n_b, K <= n_b - 1 for every data set and a total below 2^30
 * nodes; KNNG_FLAG_REORDER is not supported here (KNNG_ERR_UNSUPPORTED).
 * Returns when all outputs are written.
 */
int knng_build_batched(const knng_desc *descs, int count, int K, float rho, float delta, int max_iters,
                       uint64_t seed, uint32_t flags, void *stream, knng_stats *stats);

/* One data set of a batched build with its own parameters
 * (knng_build_batched_ex); each field as the argument of knng_build_ex. */
typedef struct knng_desc_ex {
    const float *data;   /* n x d float32 points (host or device) */
    int64_t n;
    int32_t d;
    int32_t K;           /* 1 <= K <= min(64, n - 1) */
    float rho;           /* sample rate, (0, 1] */
    float delta;         /* stopping threshold, >= 0 */
    int32_t max_iters;   /* 0 .. 1000 */
    uint64_t seed;
    int32_t *ids;        /* n x K outputs (host or device), ids local to the data set */
    float *dists;
} knng_desc_ex;

/*
 * knng_build_batched with the parameters per data set (Section 2's method on
 * many independent data sets; the batched call of the form descs, count,
 * flags, stream).  Data sets with the same row-width class, K, sample size
 * s = ceil(rho K), max_iters and seed share one batched run, in which each
 * keeps its own delta (its own stopping count delta * n_b * K); the runs go
 * one after the other on `stream`, ordered by width class.  Each result
 * equals knng_build_ex of that data set with its own parameters and the
 * shared flags.  Errors: KNNG_ERR_INVALID_ARG for a parameter out of range
 * (checked for every descriptor before any work), KNNG_ERR_UNSUPPORTED for
 * K > 64 (or K > 32 with a low-precision or heap flag) or the relabelling
 * flags; otherwise as knng_build_batched.  stats (may be NULL) sums the
 * counters of all runs.  Returns when all outputs are written.
 */
int knng_build_batched_ex(const knng_desc_ex *descs, int count, uint32_t flags, void *stream, knng_stats *stats);

/*
 * Exact K-NNG by brute force (Section 2: every distance, the K smallest per
 * point by (dist, id), float32 difference-form distances).  rows (host or
 * device int64, may be NULL = all n rows) selects nq query points; outputs
 * are nq x K.  Ground truth for recall.  For rows of at most 128 floats,
 * n >= 4096 and K <= 32 the call waits for the stream before it returns (the
 * tensor-core prefilter: it reads how many queries the exact kernel must
 * redo; see knng_bruteforce_last_fallbacks); otherwise (the exact kernel; for
 * K > 32 one thread per query over all points) it only enqueues work when ids
 * and dists are device pointers.
 */
int knng_bruteforce(const float *data, int64_t n, int d, int K, const int64_t *rows,
                    int64_t nq, int32_t *ids, float *dists, void *stream);

/*
 * Diagnostic of the calling thread's last knng_bruteforce: for rows of at most
 * 128 floats (and n >= 4096) the distance block runs on the tensor cores as a
 * bf16 split Gram prefilter whose kept candidates are re-ranked with exact
 * float32 distances; a query whose result the error bound cannot certify is
 * recomputed by the exact kernel.  Returns how many queries were recomputed,
 * or -1 when the last call did not take the tensor-core path.  The results
 * are the same either way.
 */
int knng_bruteforce_last_fallbacks(void);

/*
 * Diagnostic of the calling thread's last knng_bruteforce: the CUDA-event
 * time in milliseconds of its tensor-core prefilter kernel (the dense part of
 * the call; split, re-rank and exact recomputation excluded), or -1 when the
 * last call did not take the tensor-core path.
 */
float knng_bruteforce_last_prefilter_ms(void);

/*
 * Measurement helper (not in the paper): the rate at which this GPU reads a
 * buffer that stays in its L2, the denominator of the roofline of kernels
 * whose working set fits there.  Allocates `bytes` (at least 1 MiB; choose
 * well below the L2 size) on the current device, reads it once, then times one
 * launch that reads it `passes` times with 16-byte loads cached in L2 only.
 * *gbs = bytes * passes / time, in GB/s.  Synchronises `stream` (NULL = the
 * legacy default stream).  Errors: KNNG_ERR_INVALID_ARG, KNNG_ERR_OOM,
 * KNNG_ERR_CUDA.
 */
int knng_measure_l2_read(int64_t bytes, int passes, void *stream, double *gbs);

/*
 * Brute-force K-NNG that allocates nothing, for callers that cannot allocate
 * device memory: code that runs while a stream is being captured into a CUDA
 * graph in global capture mode (where cudaMalloc is refused), programs whose
 * device memory is owned entirely by their own pool allocator, and real-time
 * callers that must not allocate after start-up.  The paper has no
 * counterpart; it is the same computation as knng_bruteforce.
 *
 * data, ids, dists (and rows, when not NULL) must be device memory of the
 * current device (or managed memory it can reach), with the layouts of
 * knng_bruteforce; the caller owns them.  Host pointers and memory of another
 * device are refused with KNNG_ERR_INVALID_ARG before anything is launched.
 * The only scratch, the zero-padded copy of the points, is a static device
 * array of KNNG_NOALLOC_SCRATCH_BYTES that every GPU loading the library
 * holds until the process exits.  Returns KNNG_ERR_INVALID_ARG when
 * n * round_up(d, 4) * 4 exceeds KNNG_NOALLOC_SCRATCH_BYTES, and
 * KNNG_ERR_UNSUPPORTED for K > 32.
 *
 * The first call in a CUDA context (the first on a device, and the first
 * after a device reset, which makes a new context) does a set-up that
 * allocates nothing: it looks up the array's device address (one
 * cudaGetSymbolAddress), loads every kernel the call can use and opts them in
 * to their shared memory.  Make that first call before any stream capture;
 * later calls only enqueue kernels (rows of more than 16,384 floats may still
 * set a kernel's shared-memory attribute on their first call).  All calls
 * share the one array and it keeps the last call's contents; each call overwrites the whole region it
 * reads before reading it.  Calls whose work overlaps on the GPU (other
 * streams, other threads) race on the array: serialise them.  Enqueues on
 * `stream`, does not synchronise.
 */
#define KNNG_NOALLOC_SCRATCH_BYTES (8u << 20)
int knng_bruteforce_noalloc(const float *data, int64_t n, int d, int K, const int64_t *rows,
                            int64_t nq, int32_t *ids, float *dists, void *stream);

/* Name of a return code. */
const char *knng_strerror(int code);

/* Library version string. */
const char *knng_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KNNG_H_ */
