// Host launchers of the walk and query kernels (wost_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "wost_internal.h"

namespace wost {

cudaError_t launch_walk_plain(const SceneView &sc, const SolveParams &sp, const Accumulators &acc, int block,
                              cudaStream_t s);
cudaError_t launch_walk_count(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                              unsigned long long *stats, int block, cudaStream_t s);
cudaError_t persistent_grid(int dim, int block, int depth, int *blocks_out, int lanes = 1);
cudaError_t batch_grid(int dim, int block, int depth, int *blocks_out);
cudaError_t launch_request_stats(const StatJob *jobs, int n_jobs, int64_t max_points, unsigned int *max_var_bits,
                                 unsigned long long *min_walks, unsigned long long *steps_sum,
                                 unsigned long long *walks_sum, cudaStream_t s);
cudaError_t launch_walk_batch(int dim, const BatchHeader *hdr, const BatchJob *jobs, unsigned long long *counter,
                              unsigned int *guard, int depth, const int *cancel, int block, int blocks,
                              cudaStream_t s, unsigned long long *steps_out = nullptr, bool screened = true);
// lanes: lanes per walk, 1 (binary trees) or 8 (8-lane teams over the 8-wide
// trees; Poisson solves)
cudaError_t launch_walk_persistent(const SceneView &sc, const SolveParams &sp, const Accumulators &acc, int block,
                                   int blocks, cudaStream_t s, int lanes = 1);
// resumable solves: grid of the fixed launch, its walk slots, one launch
cudaError_t resume_grid(int dim, int block, int depth, int *blocks_out, int lanes = 1);
int64_t resume_slots(int block, int blocks, int lanes = 1);
cudaError_t launch_walk_resume(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                               const ResumeState &rs, int iters, int block, int blocks, cudaStream_t s,
                               int lanes = 1);
cudaError_t launch_screened_kernels(int dim, int64_t n, const float *rho, const float *R, float sigma, float *G,
                                    float *Q, cudaStream_t s);
cudaError_t launch_query_closest(const SceneView &sc, int64_t n, const float *pts, float *dist, float *closest,
                                 int32_t *prim, int depth, unsigned int *guard, cudaStream_t s);
cudaError_t launch_query_silhouette(const SceneView &sc, int64_t n, const float *pts, const float *rmax, float *dist,
                                    int depth, unsigned int *guard, cudaStream_t s);
cudaError_t launch_query_ray(const SceneView &sc, int64_t n, const float *o, const float *v, const float *tmax,
                             const int32_t *skip, const int32_t *rec_of_id, int64_t n_ids, int32_t *hit, float *t,
                             int32_t *prim, int depth, unsigned int *guard, cudaStream_t s);
cudaError_t launch_query_sample(const SceneView &sc, int64_t n, const float *pts, const float *r, uint32_t k0,
                                uint32_t k1, uint32_t c1, uint32_t c2, float *z, float *pdf, int32_t *prim,
                                cudaStream_t s);

}  // namespace wost
