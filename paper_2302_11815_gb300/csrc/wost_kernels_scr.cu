// Screened walk kernels (the SCR = true instantiations of wost_walk.cuh:
// -Lap u + sigma u = f, App. A.2), the evaluation kernel of the screened
// Green's function and step weight, and their launchers (sm_103a).
#include <cuda_runtime.h>

#include "wost_screened.cuh"
#include "wost_walk.cuh"

namespace wost {

// Eqs. GreensFnsScreenedPoissonBall and ScreenedPoissonKernelsSphere at n
// (rho, R) pairs: the functions the screened walks evaluate (App. A.2)
template <int D>
__global__ void k_screened_kernels(int64_t n, const float *rho, const float *R, float sqs, float *G, float *Q) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float r = rho[i], RR = R[i];
    if (G) G[i] = screened_green<D>(r, RR, sqs);
    if (Q) Q[i] = screened_q<D>(r, RR, sqs);
}

cudaError_t launch_screened_kernels(int dim, int64_t n, const float *rho, const float *R, float sigma, float *G,
                                    float *Q, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int block = 256;
    unsigned grid = (unsigned)((n + block - 1) / block);
    float sqs = sqrtf(sigma);
    if (dim == 2)
        k_screened_kernels<2><<<grid, block, 0, s>>>(n, rho, R, sqs, G, Q);
    else
        k_screened_kernels<3><<<grid, block, 0, s>>>(n, rho, R, sqs, G, Q);
    return cudaGetLastError();
}

cudaError_t launch_walk_plain_scr(const SceneView &sc, const SolveParams &sp, const Accumulators &acc, int block,
                                  cudaStream_t s) {
    return walk_plain_launch<true>(sc, sp, acc, block, s);
}
cudaError_t launch_walk_count_scr(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                                  unsigned long long *stats, int block, cudaStream_t s) {
    return walk_count_launch<true>(sc, sp, acc, stats, block, s);
}
cudaError_t launch_walk_persistent_scr(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                                       int block, int blocks, cudaStream_t s) {
    return walk_persistent_launch<true, 1>(sc, sp, acc, block, blocks, s);
}
cudaError_t launch_walk_resume_scr(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                                   const ResumeState &rs, int iters, int block, int blocks, cudaStream_t s) {
    return walk_resume_launch<true, 1>(sc, sp, acc, rs, iters, block, blocks, s);
}

}  // namespace wost
