// The 8-lane team form of the persistent and resumable walk kernels
// (Poisson instantiations): 8 lanes carry one walk over the 8-wide trees
// (wost_group.cuh).  In a translation unit of its own so that it compiles
// in parallel with the one-lane forms and adds nothing to their module.
#include <cuda_runtime.h>

#include "wost_walk.cuh"

namespace wost {

cudaError_t persistent_grid_team(int dim, int block, int depth, int *blocks_out) {
    return resident_grid(dim == 2 ? (const void *)k_walk_persistent<2, false, WOST_WIDE>
                                  : (const void *)k_walk_persistent<3, false, WOST_WIDE>,
                         block, depth, blocks_out, WOST_WIDE);
}

cudaError_t launch_walk_persistent_team(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                                        int block, int blocks, cudaStream_t s) {
    return walk_persistent_launch<false, WOST_WIDE>(sc, sp, acc, block, blocks, s);
}

cudaError_t launch_walk_resume_team(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                                    const ResumeState &rs, int iters, int block, int blocks, cudaStream_t s) {
    return walk_resume_launch<false, WOST_WIDE>(sc, sp, acc, rs, iters, block, blocks, s);
}

}  // namespace wost
