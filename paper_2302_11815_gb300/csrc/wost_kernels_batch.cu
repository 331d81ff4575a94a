// The batched persistent kernel over many solves (wost_solve_batch and the
// serving engine's rounds) in its screened and Poisson-only forms, and their
// launchers (sm_103a).  The Poisson-only form runs when no job of a batch is
// screened: the screened terms enlarge the walk loop's code, and instruction
// supply is what stalls these kernels most.
#include <cuda_runtime.h>

#include <algorithm>

#include "wost_batch.cuh"
#include "wost_screened.cuh"

namespace wost {

namespace {

template <int D, bool SCR>
cudaError_t occupancy(int block, size_t sm, int *per_sm) {
    cudaError_t e = cudaSuccess;
    if (sm > 48 * 1024) e = cudaFuncSetAttribute(k_walk_batch<D, SCR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_walk_batch<D, SCR>, block, sm);
    return e;
}

}  // namespace

cudaError_t batch_grid(int dim, int block, int depth, int *blocks_out) {
    int dev = 0, sms = 0, per_sm = 0, per_sm_p = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t sm = smem_bytes(depth, block);
    // both forms get the grid of the one with fewer resident blocks (the
    // shared memory size is set for both)
    if (e == cudaSuccess) e = dim == 2 ? occupancy<2, true>(block, sm, &per_sm) : occupancy<3, true>(block, sm, &per_sm);
    if (e == cudaSuccess)
        e = dim == 2 ? occupancy<2, false>(block, sm, &per_sm_p) : occupancy<3, false>(block, sm, &per_sm_p);
    if (e != cudaSuccess) return e;
    per_sm = std::min(per_sm, per_sm_p);
    *blocks_out = sms * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

cudaError_t launch_walk_batch(int dim, const BatchHeader *hdr, const BatchJob *jobs, unsigned long long *counter,
                              unsigned int *guard, int depth, const int *cancel, int block, int blocks,
                              cudaStream_t s, unsigned long long *steps_out, bool screened) {
    const size_t sm = smem_bytes(depth, block);
    if (dim == 2) {
        if (screened)
            k_walk_batch<2, true><<<blocks, block, sm, s>>>(hdr, jobs, counter, guard, depth, cancel, steps_out);
        else
            k_walk_batch<2, false><<<blocks, block, sm, s>>>(hdr, jobs, counter, guard, depth, cancel, steps_out);
    } else {
        if (screened)
            k_walk_batch<3, true><<<blocks, block, sm, s>>>(hdr, jobs, counter, guard, depth, cancel, steps_out);
        else
            k_walk_batch<3, false><<<blocks, block, sm, s>>>(hdr, jobs, counter, guard, depth, cancel, steps_out);
    }
    return cudaGetLastError();
}

}  // namespace wost
