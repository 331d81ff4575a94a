// wost_solve_static: a solve that allocates no memory.
//
// wost_solve allocates its per-point accumulators with cudaMalloc for every
// solve.  Some callers cannot do that: a real-time loop in which the
// implicit device synchronisation of cudaMalloc/cudaFree would stall other
// streams, or a process whose device memory is already committed under a
// fixed budget (resident scenes, another framework's caching allocator).
// This entry point runs the same walks as wost_solve with the persistent
// kernel, but its FP64 accumulators and work counters live in one fixed
// device array of this library, g_static_scratch, sized for
// WOST_STATIC_MAX_POINTS points; every device that loads the library holds
// that array (about 2 MiB) until the process exits.
#include <cuda_runtime.h>

#include <cmath>

#include "capi_internal.h"

namespace wost {

// Layout of the scratch array (bytes):
//   [0, 8)    capped-walk count (u64)
//   [8, 16)   next-walk counter of the persistent kernel (u64)
//   [16, 20)  guard flags (u32)
//   [20, 24)  cancel flag (i32, never set by this entry point)
//   [256, ..) per point: walk-sum, sum of squares (f64), walk count, step
//             count (u64), four arrays of WOST_STATIC_MAX_POINTS entries
constexpr size_t kHeader = 256;
constexpr size_t kArray = 8 * (size_t)WOST_STATIC_MAX_POINTS;
constexpr size_t kScratchBytes = kHeader + 4 * kArray;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// mean and standard error per point; NaN for every point if a device guard
// fired (traversal stack overflow or visit limit)
__global__ void k_static_finish(const unsigned char *scratch, int64_t n, float *mean, float *se) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *sum = (const double *)(scratch + kHeader);
    const double *sumsq = (const double *)(scratch + kHeader + kArray);
    const unsigned long long *walks = (const unsigned long long *)(scratch + kHeader + 2 * kArray);
    const unsigned int guard = *(const unsigned int *)(scratch + 16);
    double c = (double)walks[i];
    double m = c > 0 ? sum[i] / c : 0.0;
    double v = c > 1 ? fmax(0.0, (sumsq[i] - c * m * m) / (c - 1.0)) : 0.0;
    const float nan = __int_as_float(0x7fc00000);
    mean[i] = guard ? nan : (float)m;
    if (se) se[i] = guard ? nan : (float)(c > 0 ? sqrt(v / c) : 0.0);
}

// Device address of the scratch array on the current device, looked up on
// every call: a cached address would outlive a device reset or a recreated
// primary context, after which it points at freed memory.  The lookup is a
// host-side table read once the module is loaded; the first one on a device
// can load the module, which a stream capture does not allow, so the first
// call on a device must come before any capture.
static cudaError_t scratch_address(unsigned char **out) {
    unsigned char *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace wost

using namespace wost;

extern "C" wost_status wost_solve_static(wost_scene *scene, int64_t n_points, const float *points,
                                         int32_t walks_per_point, float epsilon, float r_min, int32_t max_steps,
                                         uint64_t seed, uint32_t first_walk, float *mean_out, float *stderr_out,
                                         void *stream_arg) {
    if (!scene || !points || !mean_out) return fail(WOST_ERR_INVALID_ARG, "null argument");
    if (n_points < 1) return fail(WOST_ERR_INVALID_ARG, "n_points must be >= 1");
    if (n_points > WOST_STATIC_MAX_POINTS)
        return fail(WOST_ERR_INVALID_ARG,
                    "n_points exceeds WOST_STATIC_MAX_POINTS (65536): split the points over several calls");
    if (walks_per_point < 1) return fail(WOST_ERR_INVALID_ARG, "walks_per_point must be >= 1");
    if (!(epsilon > 0) || !std::isfinite(epsilon)) return fail(WOST_ERR_INVALID_ARG, "epsilon must be > 0");
    const float rmin = r_min == 0 ? epsilon : r_min;
    if (!(rmin > 0) || rmin > epsilon) return fail(WOST_ERR_INVALID_ARG, "need 0 < r_min <= epsilon");
    if (max_steps < 1) return fail(WOST_ERR_INVALID_ARG, "max_steps must be >= 1");
    if (scene->host.n_dirichlet == 0)
        return fail(WOST_ERR_INVALID_ARG, "a scene without Dirichlet primitives needs sigma > 0: use wost_solve");
    cudaStream_t stream = (cudaStream_t)stream_arg;
    CK(cudaSetDevice(scene->device), "cudaSetDevice");
    unsigned char *s = nullptr;
    CK(scratch_address(&s), "cudaGetSymbolAddress");
    const size_t n = (size_t)n_points;
    // the array keeps the previous call's contents: clear the counters and
    // the first n entries of each accumulator array
    CK(cudaMemsetAsync(s, 0, kHeader, stream), "cudaMemsetAsync");
    for (int a = 0; a < 4; ++a) CK(cudaMemsetAsync(s + kHeader + a * kArray, 0, 8 * n, stream), "cudaMemsetAsync");
    SolveParams sp{};
    sp.points = points;
    sp.n_points = n_points;
    sp.walks_per_point = walks_per_point;
    sp.first_walk = first_walk;
    sp.epsilon = epsilon;
    sp.r_min = rmin;
    sp.max_steps = max_steps;
    sp.key0 = (uint32_t)seed;
    sp.key1 = (uint32_t)(seed >> 32);
    sp.offset = 1e-6f;
    sp.vis_tmax = 1.f - 1e-4f;
    sp.stack_depth = scene->stack_depth;
    Accumulators acc{};
    acc.sum = (double *)(s + kHeader);
    acc.sumsq = (double *)(s + kHeader + kArray);
    acc.walks = (unsigned long long *)(s + kHeader + 2 * kArray);
    acc.steps = (unsigned long long *)(s + kHeader + 3 * kArray);
    acc.capped = (unsigned long long *)s;
    acc.next_walk = (unsigned long long *)(s + 8);
    acc.guard = (unsigned int *)(s + 16);
    acc.cancel = (int *)(s + 20);
    const int block = scene->tuned_block ? scene->tuned_block : 128;
    int blocks = 0;
    CK(persistent_grid(scene->view.dim, block, sp.stack_depth, &blocks), "occupancy");
    CK(launch_walk_persistent(scene->view, sp, acc, block, blocks, stream), "kernel launch");
    k_static_finish<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(s, n_points, mean_out, stderr_out);
    CK(cudaGetLastError(), "kernel launch");
    return WOST_OK;
}
