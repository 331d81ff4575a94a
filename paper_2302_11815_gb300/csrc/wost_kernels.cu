// Walk kernels and batched query kernels (sm_103a).
//
//   k_walk_plain       one thread per walk, one launch per solve; a warp holds
//                      its lanes until its longest walk ends.
//   k_walk_persistent  one resident grid; each lane runs one walk step per
//                      iteration and, when its walk ends, takes the next walk
//                      from a global counter (warp ballot + one atomicAdd per
//                      warp), so finished lanes are refilled at once.
//   k_query_*          Q.1-Q.4 over arrays of queries (parity checks, reuse).
//
// Traversal stacks live in dynamic shared memory: stack_depth entries of
// (node ref, key) per thread, laid out [entry][thread] so that a warp's
// accesses fall in distinct banks.
#include <cuda_runtime.h>

#include <algorithm>

#include "wost_device.cuh"
#include "wost_kernels.h"

// Minimum resident 256-thread blocks per SM the walk kernels are compiled for
// (bounds their registers: 1 -> no bound, 4 -> 64 registers, 5 -> 51).  A
// build-time occupancy knob, chosen by measurement.
#ifndef WOST_WALK_MIN_BLOCKS
#define WOST_WALK_MIN_BLOCKS 1
#endif

namespace wost {

__device__ __forceinline__ Stack make_stack(int depth, unsigned int *guard) {
    extern __shared__ int2 smem_stack[];
    Stack s;
    s.base = smem_stack + threadIdx.x;
    s.stride = blockDim.x;
    s.cap = depth;
    s.guard = guard;
    return s;
}

__device__ __forceinline__ void accumulate(const Accumulators &acc, const Walk &w) {
    double v = (double)w.acc;
    atomicAdd(acc.sum + w.point, v);
    atomicAdd(acc.sumsq + w.point, v * v);
    atomicAdd(acc.walks + w.point, 1ull);
    atomicAdd(acc.steps + w.point, (unsigned long long)w.steps);
    if (w.capped) atomicAdd(acc.capped, 1ull);
}

template <int D>
__global__ void __launch_bounds__(256, WOST_WALK_MIN_BLOCKS) k_walk_plain(const SceneView sc, const SolveParams sp, const Accumulators acc,
                                                    int warp_uniform_points) {
    Stack st = make_stack(sp.stack_depth, acc.guard);
    const uint64_t total = (uint64_t)sp.n_points * (uint64_t)sp.walks_per_point;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = gid < total && *(volatile int *)acc.cancel == 0;
    Walk w;
    if (active) {
        int64_t pt = (int64_t)(gid / (uint64_t)sp.walks_per_point);
        uint32_t j = (uint32_t)(gid % (uint64_t)sp.walks_per_point) + sp.first_walk;
        walk_init<D>(sp, w, pt, j);
    }
    // the warp reconverges after every step (see k_walk_persistent)
    bool done = !active;
    while (__any_sync(0xffffffffu, !done)) {
        if (!done) {
            Cnt<false> cnt;
            done = walk_step<D>(sc, sp, w, st, cnt);
        }
        __syncwarp();
    }
    if (warp_uniform_points) {
        // every lane of this warp estimates the same point: reduce first
        unsigned mask = __ballot_sync(0xffffffffu, active);
        if (!mask) return;
        double v = active ? (double)w.acc : 0.0, v2 = v * v;
        unsigned long long s = active ? (unsigned long long)w.steps : 0ull, c = (active && w.capped) ? 1ull : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v += __shfl_xor_sync(0xffffffffu, v, o);
            v2 += __shfl_xor_sync(0xffffffffu, v2, o);
            s += __shfl_xor_sync(0xffffffffu, s, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        int lead = __ffs(mask) - 1;
        if ((int)(threadIdx.x & 31) == lead) {
            uint32_t pt = w.point;
            atomicAdd(acc.sum + pt, v);
            atomicAdd(acc.sumsq + pt, v2);
            atomicAdd(acc.walks + pt, (unsigned long long)__popc(mask));
            atomicAdd(acc.steps + pt, s);
            if (c) atomicAdd(acc.capped, c);
        }
    } else if (active) {
        accumulate(acc, w);
    }
}

template <int D>
__global__ void __launch_bounds__(256, WOST_WALK_MIN_BLOCKS) k_walk_persistent(const SceneView sc, const SolveParams sp,
                                                         const Accumulators acc) {
    Stack st = make_stack(sp.stack_depth, acc.guard);
    const uint64_t total = (uint64_t)sp.n_points * (uint64_t)sp.walks_per_point;
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    Walk w;
    bool have = false, drained = false;
    // All 32 lanes stay in this loop until the warp runs out of work and meet
    // at __syncwarp() after every walk step, so the warp starts each step
    // converged (without it, independent thread scheduling lets the lanes
    // drift apart and issue alone).
    for (;;) {
        // regeneration: lanes without a walk take the next ones
        unsigned need = __ballot_sync(FULL, !have && !drained);
        if (need) {
            int lead = __ffs(need) - 1;
            unsigned long long base = 0;
            if (lane == lead) {
                bool stop = *(volatile int *)acc.cancel != 0;
                base = stop ? total : atomicAdd(acc.next_walk, (unsigned long long)__popc(need));
            }
            base = __shfl_sync(FULL, base, lead);
            if (!have && !drained) {
                unsigned long long my = base + __popc(need & ((1u << lane) - 1u));
                if (my < total) {
                    int64_t pt = (int64_t)(my / (uint64_t)sp.walks_per_point);
                    uint32_t j = (uint32_t)(my % (uint64_t)sp.walks_per_point) + sp.first_walk;
                    walk_init<D>(sp, w, pt, j);
                    have = true;
                } else {
                    drained = true;
                }
            }
        }
        if (!__any_sync(FULL, have)) break;
        if (have) {
            Cnt<false> cnt;
            if (walk_step<D>(sc, sp, w, st, cnt)) {
                accumulate(acc, w);
                have = false;
            }
        }
        __syncwarp();
    }
}

// Batched persistent kernel: many solves (scenes, point sets, walk counts,
// parameters) in one launch.  The walk index space is the concatenation of
// the jobs' walks; a lane maps its next index to a job by binary search over
// the jobs' first indices and runs that job's walk on that job's scene.
template <int D>
__global__ void __launch_bounds__(256, WOST_WALK_MIN_BLOCKS) k_walk_batch(const BatchHeader *__restrict__ hdr,
                                                    const BatchJob *__restrict__ jobs, unsigned long long *counter,
                                                    unsigned int *guard, int stack_depth, const int *cancel) {
    const int n_jobs = hdr->n_jobs;
    const unsigned long long total = hdr->total;
    if (n_jobs <= 0) return;
    Stack st = make_stack(stack_depth, guard);
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    Walk w;
    int job = -1;
    bool drained = false;  // the launch's counter has run past `total`
    // as in k_walk_persistent: the whole warp stays in the loop and
    // reconverges after every step
    for (;;) {
        unsigned need = __ballot_sync(FULL, job < 0 && !drained);
        if (need) {
            int lead = __ffs(need) - 1;
            unsigned long long base = 0;
            if (lane == lead) {
                bool stop = cancel && *(volatile const int *)cancel != 0;
                base = stop ? total : atomicAdd(counter, (unsigned long long)__popc(need));
            }
            base = __shfl_sync(FULL, base, lead);
            if (job < 0 && !drained) {
                unsigned long long my = base + __popc(need & ((1u << lane) - 1u));
                if (my >= total) {
                    drained = true;
                } else {
                    int lo = 0, hi = n_jobs - 1;
                    while (lo < hi) {
                        int mid = (lo + hi + 1) >> 1;
                        if (jobs[mid].walk_begin <= my) lo = mid;
                        else hi = mid - 1;
                    }
                    // a cancelled solve's remaining walks are skipped: the
                    // lane takes another index at the next iteration
                    if (*(volatile const int *)jobs[lo].acc.cancel == 0) {
                        job = lo;
                        const SolveParams &sp = jobs[job].sp;
                        unsigned long long local = my - jobs[job].walk_begin;
                        int64_t pt = sp.point_begin + (int64_t)(local / (uint64_t)sp.walks_per_point);
                        uint32_t j = (uint32_t)(local % (uint64_t)sp.walks_per_point) + sp.first_walk;
                        walk_init<D>(sp, w, pt, j);
                    }
                }
            }
        }
        if (!__any_sync(FULL, job >= 0 || !drained)) break;
        if (job >= 0) {
            Cnt<false> cnt;
            if (walk_step<D>(*jobs[job].scene, jobs[job].sp, w, st, cnt)) {
                accumulate(jobs[job].acc, w);
                job = -1;
            }
        }
        __syncwarp();
    }
}

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

// Counting variant of the plain kernel: same walks, plus per-query node
// visits and primitive tests summed into stats[2 * C_NQ] (nodes then prims).
template <int D>
__global__ void __launch_bounds__(256) k_walk_count(const SceneView sc, const SolveParams sp, const Accumulators acc,
                                                    unsigned long long *stats) {
    Stack st = make_stack(sp.stack_depth, acc.guard);
    const uint64_t total = (uint64_t)sp.n_points * (uint64_t)sp.walks_per_point;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    Walk w;
    int64_t pt = (int64_t)(gid / (uint64_t)sp.walks_per_point);
    uint32_t j = (uint32_t)(gid % (uint64_t)sp.walks_per_point) + sp.first_walk;
    walk_init<D>(sp, w, pt, j);
    Cnt<true> cnt;
    while (!walk_step<D, true>(sc, sp, w, st, cnt)) {
    }
    accumulate(acc, w);
    for (int q = 0; q < C_NQ; ++q) {
        atomicAdd(stats + q, (unsigned long long)cnt.nodes[q]);
        atomicAdd(stats + C_NQ + q, (unsigned long long)cnt.prims[q]);
    }
}

// ------------------------------- queries ---------------------------------
template <int D>
__global__ void k_query_closest(const SceneView sc, int64_t n, const float *pts, float *dist, float *closest,
                                int32_t *prim, int depth, unsigned int *guard) {
    Stack st = make_stack(depth, guard);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    P3 x = load_point<D>(pts, i);
    Cnt<false> cnt;
    Closest c = q_closest<D>(sc.D, x, st, cnt);
    dist[i] = sqrtf(c.d2);
    closest[D * i] = c.p.x;
    closest[D * i + 1] = c.p.y;
    if (D == 3) closest[D * i + 2] = c.p.z;
    prim[i] = c.rec >= 0 ? __ldg(sc.D.ids + c.rec) : -1;
}

template <int D>
__global__ void k_query_silhouette(const SceneView sc, int64_t n, const float *pts, const float *rmax, float *dist,
                                   int depth, unsigned int *guard) {
    Stack st = make_stack(depth, guard);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Cnt<false> cnt;
    dist[i] = q_silhouette<D>(sc.S, load_point<D>(pts, i), rmax[i], st, cnt);
}

template <int D>
__global__ void k_query_ray(const SceneView sc, int64_t n, const float *o, const float *v, const float *tmax,
                            const int32_t *skip, const int32_t *rec_of_id, int64_t n_ids, int32_t *hit, float *t,
                            int32_t *prim, int depth, unsigned int *guard) {
    Stack st = make_stack(depth, guard);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int sk = -1;
    if (skip && skip[i] >= 0 && skip[i] < n_ids) sk = rec_of_id[skip[i]];
    float tt;
    Cnt<false> cnt;
    int r = q_ray<D>(sc.N, load_point<D>(o, i), load_point<D>(v, i), tmax[i], sk, false, tt, st, cnt);
    hit[i] = r >= 0;
    t[i] = r >= 0 ? tt : tmax[i];
    prim[i] = r >= 0 ? __ldg(sc.N.ids + r) : -1;
}

template <int D>
__global__ void k_query_sample(const SceneView sc, int64_t n, const float *pts, const float *r, uint32_t k0,
                               uint32_t k1, uint32_t c1, uint32_t c2, float *z, float *pdf, int32_t *prim) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Stream rng;
    rng.init(k0, k1, (uint32_t)i, c1, c2);
    Cnt<false> cnt;
    NSample s = q_sample<D>(sc.N, load_point<D>(pts, i), r[i], rng, cnt);
    z[D * i] = s.z.x;
    z[D * i + 1] = s.z.y;
    if (D == 3) z[D * i + 2] = s.z.z;
    pdf[i] = s.rec >= 0 ? s.pdf : 0.f;
    prim[i] = s.rec >= 0 ? __ldg(sc.N.ids + s.rec) : -1;
}

// ------------------------------- launchers --------------------------------
static size_t smem_bytes(int depth, int block) { return (size_t)depth * block * sizeof(int2); }

template <int D>
static cudaError_t set_smem_attrs(size_t bytes) {
    cudaError_t e = cudaSuccess;
    if (bytes > 48 * 1024) {
        e = cudaFuncSetAttribute(k_walk_plain<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_walk_persistent<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    }
    return e;
}

cudaError_t launch_walk_plain(const SceneView &sc, const SolveParams &sp, const Accumulators &acc, int block,
                              cudaStream_t s) {
    uint64_t total = (uint64_t)sp.n_points * (uint64_t)sp.walks_per_point;
    uint64_t grid = (total + block - 1) / block;
    if (grid > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
    size_t sm = smem_bytes(sp.stack_depth, block);
    int uniform = (sp.walks_per_point % 32 == 0) && (block % 32 == 0);
    cudaError_t e = sc.dim == 2 ? set_smem_attrs<2>(sm) : set_smem_attrs<3>(sm);
    if (e != cudaSuccess) return e;
    if (sc.dim == 2)
        k_walk_plain<2><<<(unsigned)grid, block, sm, s>>>(sc, sp, acc, uniform);
    else
        k_walk_plain<3><<<(unsigned)grid, block, sm, s>>>(sc, sp, acc, uniform);
    return cudaGetLastError();
}

cudaError_t launch_walk_count(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                              unsigned long long *stats, int block, cudaStream_t s) {
    uint64_t total = (uint64_t)sp.n_points * (uint64_t)sp.walks_per_point;
    uint64_t grid = (total + block - 1) / block;
    if (grid > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
    size_t sm = smem_bytes(sp.stack_depth, block);
    if (sm > 48 * 1024) {
        cudaError_t e = sc.dim == 2 ? cudaFuncSetAttribute(k_walk_count<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                                    : cudaFuncSetAttribute(k_walk_count<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    if (sc.dim == 2)
        k_walk_count<2><<<(unsigned)grid, block, sm, s>>>(sc, sp, acc, stats);
    else
        k_walk_count<3><<<(unsigned)grid, block, sm, s>>>(sc, sp, acc, stats);
    return cudaGetLastError();
}

cudaError_t batch_grid(int dim, int block, int depth, int *blocks_out) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t sm = smem_bytes(depth, block);
    if (e == cudaSuccess && sm > 48 * 1024)
        e = dim == 2 ? cudaFuncSetAttribute(k_walk_batch<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                     : cudaFuncSetAttribute(k_walk_batch<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)
        e = dim == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_batch<2>, block, sm)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_batch<3>, block, sm);
    if (e != cudaSuccess) return e;
    *blocks_out = sms * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

cudaError_t launch_walk_batch(int dim, const BatchHeader *hdr, const BatchJob *jobs, unsigned long long *counter,
                              unsigned int *guard, int depth, const int *cancel, int block, int blocks,
                              cudaStream_t s) {
    size_t sm = smem_bytes(depth, block);
    if (dim == 2)
        k_walk_batch<2><<<blocks, block, sm, s>>>(hdr, jobs, counter, guard, depth, cancel);
    else
        k_walk_batch<3><<<blocks, block, sm, s>>>(hdr, jobs, counter, guard, depth, cancel);
    return cudaGetLastError();
}

cudaError_t persistent_grid(int dim, int block, int depth, int *blocks_out) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t sm = smem_bytes(depth, block);
    if (e == cudaSuccess) e = dim == 2 ? set_smem_attrs<2>(sm) : set_smem_attrs<3>(sm);
    if (e == cudaSuccess)
        e = dim == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_persistent<2>, block, sm)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_persistent<3>, block, sm);
    if (e != cudaSuccess) return e;
    *blocks_out = sms * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

cudaError_t launch_walk_persistent(const SceneView &sc, const SolveParams &sp, const Accumulators &acc, int block,
                                   int blocks, cudaStream_t s) {
    size_t sm = smem_bytes(sp.stack_depth, block);
    if (sc.dim == 2)
        k_walk_persistent<2><<<blocks, block, sm, s>>>(sc, sp, acc);
    else
        k_walk_persistent<3><<<blocks, block, sm, s>>>(sc, sp, acc);
    return cudaGetLastError();
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
