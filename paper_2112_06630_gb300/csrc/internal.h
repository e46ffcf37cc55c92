// internal.h -- host-side launchers shared between the library's translation
// units (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace knng {

// persistent grid size for a warp-per-item kernel: a multiple of the SM count
int grid_for(const void *kernel, int block_threads, size_t dyn_smem);
// opt `kernel` in to `bytes` of dynamic shared memory in the current context
// (once per kernel, context and size; thread-safe)
cudaError_t smem_opt_in(const void *kernel, size_t bytes);
// id of the calling thread's current CUDA context (new after a device reset)
cudaError_t current_context_id(unsigned long long *id);

cudaError_t launch_stage(const float *src, int64_t n, int d, float *X, int dp, cudaStream_t s);
// load stage_kernel in the current context
cudaError_t prepare_stage();
cudaError_t launch_init_random(const DevState &st, uint64_t seed, int *err, cudaStream_t s);
cudaError_t launch_init_graph(const DevState &st, const int32_t *ids, const uint8_t *is_new, int *err,
                              cudaStream_t s);
cudaError_t launch_count(const DevState &st, int li, cudaStream_t s);
// parallel locality relabelling (relabel.cu): scratch bytes, and the launch
// that writes sigma (new spot of every node) from the current lists
size_t parallel_relabel_scratch(int64_t n, int K);
cudaError_t launch_parallel_relabel(const float *X, const uint64_t *keys, int64_t n, int K, int nv, int32_t *sigma,
                                    unsigned char *scratch, int *launches, cudaStream_t s);
// l2probe.cu: `passes` reads of an n4 x 16-byte buffer in one launch
cudaError_t launch_l2_read(const void *buf, size_t n4, int passes, float *sink, cudaStream_t s);
cudaError_t launch_heap_sample(const DevState &st, int li, int it, uint64_t seed, cudaStream_t s);
cudaError_t launch_sample(const DevState &st, int li, int it, uint64_t seed, cudaStream_t s);
cudaError_t launch_join(const DevState &st, int li, cudaStream_t s);
cudaError_t launch_merge(const DevState &st, int li, cudaStream_t s);
cudaError_t launch_tile_join(const DevState &st, int li, bool bf16, cudaStream_t s);
cudaError_t launch_ring_join(const DevState &st, int li, cudaStream_t s);
// the set kernel alone: every node's candidate set (repeats removed, new
// first) into cset / cmeta, for the ring and pipelined join kernels
cudaError_t launch_set_kernel(const DevState &st, int li, cudaStream_t s);
// pipelined block join (float32 rows of 33 to 256 floats): set kernel + join
cudaError_t launch_pipe_join(const DevState &st, int li, cudaStream_t s);
bool pipe_join_fits(int bf16, int nv);
// true when a node with 64 candidates fits the ring of the ring join kernel
bool ring_join_fits(int bf16, int nv, int dpb, int K);
// true when the ring holds several typical nodes (the default choice)
bool ring_join_preferred(int bf16, int nv, int dpb);
// the join kernel for a context: the warp kernel for float32 rows of up to
// 64 floats, else the ring kernel where a 64-candidate node fits its ring,
// else the block-per-node tile kernel; `force` (>= 0) picks one a context can
// run instead (test hook), -1 = default
int choose_join_path(int bf16, int nv, int dpb, int K, int force);
// kernel launches of one local join on the given path
int join_launches(int path);
cudaError_t launch_stage_bf16(const float *X, int64_t n, int dp, int d, uint16_t *Xb, int dpb, float *nrm,
                              cudaStream_t s);
// e4m3 copy of the rows (round to nearest, saturating at +-448) and the
// squared norms of the e4m3 values
cudaError_t launch_stage_fp8(const float *X, int64_t n, int dp, int d, uint8_t *X8, int dpb, float *nrm,
                             cudaStream_t s);
cudaError_t launch_greedy_reorder(const uint64_t *keys, int64_t n, int K, int reading_b, int32_t *sigma,
                                  int32_t *sigma_inv, cudaStream_t s);
cudaError_t launch_permute(const DevState &src, float *X_dst, uint64_t *keys_dst, const int32_t *sigma,
                           int32_t *total_perm, cudaStream_t s);
cudaError_t launch_output(const DevState &st, const int32_t *total_perm, const int32_t *total_inv,
                          int32_t *ids, float *dists, cudaStream_t s);
cudaError_t launch_iota(int32_t *p, int64_t n, cudaStream_t s);
cudaError_t launch_ds_map(const long long *ds_off, int nds, int64_t n, int *ds, cudaStream_t s);
cudaError_t launch_invert(const int32_t *perm, int64_t n, int32_t *inv, cudaStream_t s);
// part: scratch for S slice lists of K keys per query (nq * S * K uint64), or
// null for one slice (no scratch)
cudaError_t launch_bruteforce(const float *X, int64_t n, int dp, int K, const int64_t *rows, int64_t nq,
                              int32_t *ids, float *dists, cudaStream_t s, uint64_t *part, int S);
// load every kernel launch_stage and a one-slice launch_bruteforce can use and
// opt them in to the shared memory they may ask for, in the current context,
// so that later launches neither load code nor set attributes
cudaError_t prepare_bruteforce_one_slice();
// slices that give every SM work for nq queries over n points
int bruteforce_slices(int64_t n, int64_t nq);
// tensor-core brute force (bf16 split Gram prefilter, exact re-rank, exact
// fallback per uncertified query): rows of at most 128 floats, and a driver
// that encodes tensor maps
bool bruteforce_tc_supported(int dp);
size_t bruteforce_tc_scratch(int64_t n, int64_t nq, int dp, int K, int *slices_out);
cudaError_t launch_bruteforce_tc(const float *X, int64_t n, int dp, int d, int K, const int64_t *rows, int64_t nq,
                                 int32_t *ids, float *dists, cudaStream_t s, unsigned char *scratch, int S,
                                 int *nredo_host, float *prefilter_ms);

}  // namespace knng
