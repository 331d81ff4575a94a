// Poisson walk kernels (the SCR = false instantiations of wost_walk.cuh),
// the per-solve summary kernel, the batched query kernels (Q.1-Q.4 over
// arrays of queries, through the same query code as the walks) and their
// launchers (sm_103a).  A solve with sigma > 0 is passed on to the screened
// translation unit, wost_kernels_scr.cu.
#include <cuda_runtime.h>

#include <algorithm>

#include "wost_walk.cuh"

namespace wost {

// Per-solve summary of the FP64 accumulators (serving engine): largest
// per-point sample variance, smallest per-point walk count, and the sums of
// steps and walks.  grid.y = solve, grid.x strides over points.
__global__ void k_request_stats(const StatJob *jobs, int n_jobs, unsigned int *max_var_bits,
                                unsigned long long *min_walks, unsigned long long *steps_sum,
                                unsigned long long *walks_sum) {
    int j = blockIdx.y;
    if (j >= n_jobs) return;
    const StatJob J = jobs[j];
    float mv = 0.f;
    unsigned long long mw = ~0ull, ss = 0, ws = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < J.n; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long w = J.walks[i];
        double c = (double)w;
        float var = 3.0e38f;
        if (w > 1) {
            double m = J.sum[i] / c;
            var = (float)fmax(0.0, (J.sumsq[i] - c * m * m) / (c - 1.0));
        }
        mv = fmaxf(mv, var);
        mw = w < mw ? w : mw;
        ss += J.steps[i];
        ws += w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mv = fmaxf(mv, __shfl_xor_sync(0xffffffffu, mv, o));
        unsigned long long t = __shfl_xor_sync(0xffffffffu, mw, o);
        mw = t < mw ? t : mw;
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        ws += __shfl_xor_sync(0xffffffffu, ws, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(max_var_bits + j, __float_as_uint(mv));  // non-negative floats order like their bits
        atomicMin(min_walks + j, mw);
        atomicAdd(steps_sum + j, ss);
        atomicAdd(walks_sum + j, ws);
    }
}

cudaError_t launch_request_stats(const StatJob *jobs, int n_jobs, int64_t max_points, unsigned int *max_var_bits,
                                 unsigned long long *min_walks, unsigned long long *steps_sum,
                                 unsigned long long *walks_sum, cudaStream_t s) {
    if (n_jobs <= 0) return cudaSuccess;
    const int block = 256;
    int gx = (int)std::min<int64_t>((max_points + block - 1) / block, 128);
    dim3 grid(gx > 0 ? gx : 1, n_jobs);
    k_request_stats<<<grid, block, 0, s>>>(jobs, n_jobs, max_var_bits, min_walks, steps_sum, walks_sum);
    return cudaGetLastError();
}

// ------------------------------- queries ---------------------------------
// one team per query; the team's leader writes the answer
template <int D>
__global__ void k_query_closest(const SceneView sc, int64_t n, const float *pts, float *dist, float *closest,
                                int32_t *prim, int depth, unsigned int *guard) {
    Cnt<false> cnt;
    auto q = make_q<D, false>(depth, guard, cnt);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    P3 x = load_point<D>(pts, i);
    Closest c = q.closest(sc.D, x, INFINITY);
    if (!make_team<1>().leader()) return;
    dist[i] = sqrtf(c.d2);
    closest[D * i] = c.p.x;
    closest[D * i + 1] = c.p.y;
    if (D == 3) closest[D * i + 2] = c.p.z;
    prim[i] = c.rec >= 0 ? __ldg(sc.D.ids + c.rec) : -1;
}

template <int D>
__global__ void k_query_silhouette(const SceneView sc, int64_t n, const float *pts, const float *rmax, float *dist,
                                   int depth, unsigned int *guard) {
    Cnt<false> cnt;
    auto q = make_q<D, false>(depth, guard, cnt);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float d = q.silhouette(sc.S, load_point<D>(pts, i), rmax[i]);
    if (make_team<1>().leader()) dist[i] = d;
}

template <int D>
__global__ void k_query_ray(const SceneView sc, int64_t n, const float *o, const float *v, const float *tmax,
                            const int32_t *skip, const int32_t *rec_of_id, int64_t n_ids, int32_t *hit, float *t,
                            int32_t *prim, int depth, unsigned int *guard) {
    Cnt<false> cnt;
    auto q = make_q<D, false>(depth, guard, cnt);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int sk = -1;
    if (skip && skip[i] >= 0 && skip[i] < n_ids) sk = rec_of_id[skip[i]];
    float tt;
    int r = q.ray(sc.N, load_point<D>(o, i), load_point<D>(v, i), tmax[i], sk, false, tt);
    if (!make_team<1>().leader()) return;
    hit[i] = r >= 0;
    t[i] = r >= 0 ? tt : tmax[i];
    prim[i] = r >= 0 ? __ldg(sc.N.ids + r) : -1;
}

template <int D>
__global__ void k_query_sample(const SceneView sc, int64_t n, const float *pts, const float *r, uint32_t k0,
                               uint32_t k1, uint32_t c1, uint32_t c2, float *z, float *pdf, int32_t *prim) {
    Cnt<false> cnt;
    auto q = make_q<D, false>(0, nullptr, cnt);  // Q.4 keeps no stack
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Stream rng;
    rng.init(k0, k1, (uint32_t)i, c1, c2);
    NSample s = q.sample(sc.N, load_point<D>(pts, i), r[i], rng);
    if (!make_team<1>().leader()) return;
    z[D * i] = s.z.x;
    z[D * i + 1] = s.z.y;
    if (D == 3) z[D * i + 2] = s.z.z;
    pdf[i] = s.rec >= 0 ? s.pdf : 0.f;
    prim[i] = s.rec >= 0 ? __ldg(sc.N.ids + s.rec) : -1;
}

// ------------------------------- launchers --------------------------------
cudaError_t launch_walk_plain(const SceneView &sc, const SolveParams &sp, const Accumulators &acc, int block,
                              cudaStream_t s) {
    if (sp.sigma > 0.f) return launch_walk_plain_scr(sc, sp, acc, block, s);
    return walk_plain_launch<false>(sc, sp, acc, block, s);
}

cudaError_t launch_walk_count(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                              unsigned long long *stats, int block, cudaStream_t s) {
    if (sp.sigma > 0.f) return launch_walk_count_scr(sc, sp, acc, stats, block, s);
    return walk_count_launch<false>(sc, sp, acc, stats, block, s);
}

// The grids of the persistent kernels are sized for the Poisson
// instantiation; the screened one runs under the same register cap and
// shared memory, so the same number of its blocks is resident.
// lanes = 8: the team form over the 8-wide trees (Poisson only; the
// screened solves and the other kernels use one lane per walk)
cudaError_t persistent_grid(int dim, int block, int depth, int *blocks_out, int lanes) {
    if (lanes == WOST_WIDE) return persistent_grid_team(dim, block, depth, blocks_out);
    return resident_grid(dim == 2 ? (const void *)k_walk_persistent<2, false, 1>
                                  : (const void *)k_walk_persistent<3, false, 1>,
                         block, depth, blocks_out);
}

cudaError_t launch_walk_persistent(const SceneView &sc, const SolveParams &sp, const Accumulators &acc, int block,
                                   int blocks, cudaStream_t s, int lanes) {
    if (sp.sigma > 0.f) return launch_walk_persistent_scr(sc, sp, acc, block, blocks, s);
    if (lanes == WOST_WIDE) return launch_walk_persistent_team(sc, sp, acc, block, blocks, s);
    return walk_persistent_launch<false, 1>(sc, sp, acc, block, blocks, s);
}

// the resumable kernels share the persistent ones' occupancy (same body)
cudaError_t resume_grid(int dim, int block, int depth, int *blocks_out, int lanes) {
    if (lanes == WOST_WIDE) return persistent_grid_team(dim, block, depth, blocks_out);
    return resident_grid(dim == 2 ? (const void *)k_walk_resume<2, false, 1> : (const void *)k_walk_resume<3, false, 1>,
                         block, depth, blocks_out);
}

int64_t resume_slots(int block, int blocks, int lanes) { return (int64_t)blocks * (block / lanes); }

cudaError_t launch_walk_resume(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                               const ResumeState &rs, int iters, int block, int blocks, cudaStream_t s, int lanes) {
    if (sp.sigma > 0.f) return launch_walk_resume_scr(sc, sp, acc, rs, iters, block, blocks, s);
    if (lanes == WOST_WIDE) return launch_walk_resume_team(sc, sp, acc, rs, iters, block, blocks, s);
    return walk_resume_launch<false, 1>(sc, sp, acc, rs, iters, block, blocks, s);
}

static cudaError_t query_smem(const void *fn, size_t bytes) {
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

cudaError_t launch_query_closest(const SceneView &sc, int64_t n, const float *pts, float *dist, float *closest,
                                 int32_t *prim, int depth, unsigned int *guard, cudaStream_t s) {
    const int block = 128;
    unsigned grid = (unsigned)((n + block - 1) / block);
    size_t sm = smem_bytes(depth, block);
    if (sc.dim == 2) {
        cudaError_t e = query_smem((const void *)k_query_closest<2>, sm);
        if (e != cudaSuccess) return e;
        k_query_closest<2><<<grid, block, sm, s>>>(sc, n, pts, dist, closest, prim, depth, guard);
    } else {
        cudaError_t e = query_smem((const void *)k_query_closest<3>, sm);
        if (e != cudaSuccess) return e;
        k_query_closest<3><<<grid, block, sm, s>>>(sc, n, pts, dist, closest, prim, depth, guard);
    }
    return cudaGetLastError();
}

cudaError_t launch_query_silhouette(const SceneView &sc, int64_t n, const float *pts, const float *rmax, float *dist,
                                    int depth, unsigned int *guard, cudaStream_t s) {
    const int block = 128;
    unsigned grid = (unsigned)((n + block - 1) / block);
    size_t sm = smem_bytes(depth, block);
    if (sc.dim == 2) {
        cudaError_t e = query_smem((const void *)k_query_silhouette<2>, sm);
        if (e != cudaSuccess) return e;
        k_query_silhouette<2><<<grid, block, sm, s>>>(sc, n, pts, rmax, dist, depth, guard);
    } else {
        cudaError_t e = query_smem((const void *)k_query_silhouette<3>, sm);
        if (e != cudaSuccess) return e;
        k_query_silhouette<3><<<grid, block, sm, s>>>(sc, n, pts, rmax, dist, depth, guard);
    }
    return cudaGetLastError();
}

cudaError_t launch_query_ray(const SceneView &sc, int64_t n, const float *o, const float *v, const float *tmax,
                             const int32_t *skip, const int32_t *rec_of_id, int64_t n_ids, int32_t *hit, float *t,
                             int32_t *prim, int depth, unsigned int *guard, cudaStream_t s) {
    const int block = 128;
    unsigned grid = (unsigned)((n + block - 1) / block);
    size_t sm = smem_bytes(depth, block);
    if (sc.dim == 2) {
        cudaError_t e = query_smem((const void *)k_query_ray<2>, sm);
        if (e != cudaSuccess) return e;
        k_query_ray<2><<<grid, block, sm, s>>>(sc, n, o, v, tmax, skip, rec_of_id, n_ids, hit, t, prim, depth, guard);
    } else {
        cudaError_t e = query_smem((const void *)k_query_ray<3>, sm);
        if (e != cudaSuccess) return e;
        k_query_ray<3><<<grid, block, sm, s>>>(sc, n, o, v, tmax, skip, rec_of_id, n_ids, hit, t, prim, depth, guard);
    }
    return cudaGetLastError();
}

cudaError_t launch_query_sample(const SceneView &sc, int64_t n, const float *pts, const float *r, uint32_t k0,
                                uint32_t k1, uint32_t c1, uint32_t c2, float *z, float *pdf, int32_t *prim,
                                cudaStream_t s) {
    const int block = 128;
    unsigned grid = (unsigned)((n + block - 1) / block);
    if (sc.dim == 2)
        k_query_sample<2><<<grid, block, 0, s>>>(sc, n, pts, r, k0, k1, c1, c2, z, pdf, prim);
    else
        k_query_sample<3><<<grid, block, 0, s>>>(sc, n, pts, r, k0, k1, c1, c2, z, pdf, prim);
    return cudaGetLastError();
}

}  // namespace wost
