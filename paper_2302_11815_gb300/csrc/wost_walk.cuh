// Walk kernels (templates), shared by the Poisson translation unit
// (wost_kernels.cu: the SCR = false instantiations) and the screened one
// (wost_kernels_scr.cu: SCR = true and the batched kernel).  Keeping the
// screened instantiations and the Bessel functions out of the Poisson
// module keeps that module's code as compact as before they existed.
//
// A walk is carried by a team of T lanes (1: a lane per walk over the binary
// trees; 8: a team per walk over the 8-wide trees, see wost_group.cuh).  All
// lanes of a team hold the same walk state.  The persistent and resumable
// kernels come in both forms, chosen at run time (the autotuner picks one per
// scene); the other kernels use one lane per walk.
//
//   k_walk_plain       one team per walk, one launch per solve; a warp holds
//                      its teams until its longest walk ends.
//   k_walk_persistent  one resident grid; each team runs one walk step per
//                      iteration and, when its walk ends, takes the next walk
//                      from a global counter (warp ballot + one atomicAdd per
//                      warp), so finished teams are refilled at once.
//   k_walk_resume      the persistent loop for a bounded number of steps,
//                      unfinished walks saved for the next launch.
//   k_walk_batch       the persistent kernel over many solves (wost_batch.cuh).
//   k_walk_count       the plain kernel with work counters.
//
// Traversal stacks live in dynamic shared memory, stack_depth entries of
// (node ref, key) per team: [entry][thread] for single lanes (a warp's
// accesses fall in distinct banks), [team][entry] for teams of 8 (odd
// stack_depth spreads the teams of a warp over the banks).
#pragma once

#include <cuda_runtime.h>

#include "wost_device.cuh"
#include "wost_group.cuh"
#include "wost_kernels.h"

// Register caps of the walk kernels (2D and 3D instantiations).  They are
// latency-bound (dependent node fetches, divergent traversals): more
// resident warps beat the few spills a lower cap costs.  Measured with the
// warp-synchronous step and the fused Q.3/visibility traversal, 128-thread
// blocks, steady state of the resumable kernel: Koch workload (2D) 48 ->
// 7.8e8 steps/s, 56 -> 8.2e8, 64 -> 8.4e8, 72 -> 8.2e8; cube + torus (3D)
// 64 -> 1.04e8, 72 -> 1.01e8, 80 -> 0.97e8.  Build-time knobs; 255 = no cap.
#ifndef WOST_WALK_REGS_2D
#define WOST_WALK_REGS_2D 64
#endif
#ifndef WOST_WALK_REGS_3D
#define WOST_WALK_REGS_3D 64
#endif
#define WOST_WALK_BOUNDS __maxnreg__(D == 2 ? WOST_WALK_REGS_2D : WOST_WALK_REGS_3D)

namespace wost {

template <int T>
__device__ __forceinline__ Group make_team() {
    static_assert(T == 1 || T == WOST_WIDE, "a team is one lane or one lane per wide child");
    Group g;
    int lane = threadIdx.x & 31;
    g.gl = lane & (T - 1);
    g.base = lane - g.gl;
    g.mask = (T == 32 ? 0xffffffffu : ((1u << T) - 1u)) << g.base;
    return g;
}

template <int D, bool CN, int T>
struct PolicyOf;
template <int D, bool CN>
struct PolicyOf<D, CN, 1> {
    using type = LaneQ<D, CN>;
};
template <int D, bool CN>
struct PolicyOf<D, CN, WOST_WIDE> {
    using type = GroupQ<D, CN>;
};

// the query policy of this thread's team, with its shared-memory stack
template <int D, bool CN, int T = 1>
__device__ __forceinline__ typename PolicyOf<D, CN, T>::type make_q(int depth, unsigned int *guard, Cnt<CN> &cnt,
                                                                    uint32_t visit_limit = 0u) {
    extern __shared__ int2 smem_stack[];
    if constexpr (T == 1) {
        Stack s{smem_stack + threadIdx.x, (int)blockDim.x, depth, guard, visit_limit};
        return LaneQ<D, CN>{s, cnt};
    } else {
        GStack s{smem_stack + (threadIdx.x / T) * depth, depth, guard};
        return GroupQ<D, CN>{make_team<T>(), s, cnt};
    }
}

// host-set flag read once per team (every lane of a team must take the same
// branch), null = not set
__device__ __forceinline__ bool team_flag(const Group &g, const int *flag) {
    int v = (g.leader() && flag) ? *(volatile const int *)flag : 0;
    return __shfl_sync(g.mask, v, g.base) != 0;
}

__device__ __forceinline__ void accumulate(const Accumulators &acc, const Walk &w) {
    double v = (double)w.acc;
    atomicAdd(acc.sum + w.point, v);
    atomicAdd(acc.sumsq + w.point, v * v);
    atomicAdd(acc.walks + w.point, 1ull);
    atomicAdd(acc.steps + w.point, (unsigned long long)w.steps);
    if (w.capped) atomicAdd(acc.capped, 1ull);
}

template <int D, bool SCR>
__global__ void WOST_WALK_BOUNDS k_walk_plain(const SceneView sc, const SolveParams sp, const Accumulators acc,
                                                    int warp_uniform_points) {
    Cnt<false> cnt;
    auto q = make_q<D, false>(sp.stack_depth, acc.guard, cnt, sp.visit_limit);
    const Group g = make_team<1>();
    const uint64_t total = (uint64_t)sp.n_points * (uint64_t)sp.walks_per_point;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = gid < total && !team_flag(g, acc.cancel);
    Walk w{};
    if (active) {
        int64_t pt = (int64_t)(gid / (uint64_t)sp.walks_per_point);
        uint32_t j = (uint32_t)(gid % (uint64_t)sp.walks_per_point) + sp.first_walk;
        walk_init<D>(sp, w, pt, j);
    }
    // the whole warp steps together (walk_step is warp-synchronous)
    bool done = !active;
    while (__any_sync(0xffffffffu, !done)) {
        if (walk_step<D, SCR>(sc, sp, w, q, !done)) done = true;
        __syncwarp();
    }
    const bool own = active && g.leader();  // one lane reports each walk
    if (warp_uniform_points) {
        // every team of this warp estimates the same point: reduce first
        unsigned mask = __ballot_sync(0xffffffffu, own);
        if (!mask) return;
        double v = own ? (double)w.acc : 0.0, v2 = v * v;
        unsigned long long s = own ? (unsigned long long)w.steps : 0ull, c = (own && w.capped) ? 1ull : 0ull;
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
    } else if (own) {
        accumulate(acc, w);
    }
}

template <int D, bool SCR, int T>
__global__ void WOST_WALK_BOUNDS k_walk_persistent(const SceneView sc, const SolveParams sp,
                                                         const Accumulators acc) {
    Cnt<false> cnt;
    auto q = make_q<D, false, T>(sp.stack_depth, acc.guard, cnt, sp.visit_limit);
    const Group g = make_team<T>();
    const uint64_t total = (uint64_t)sp.n_points * (uint64_t)sp.walks_per_point;
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    Walk w{};
    bool have = false, drained = false;  // uniform within a team
    // All 32 lanes stay in this loop until the warp runs out of work, call
    // the warp-synchronous walk_step together (lanes without a walk take part
    // in its meetings only) and meet at __syncwarp() after every walk step,
    // so the warp starts each step and each query converged (without it,
    // independent thread scheduling lets the lanes drift apart and issue
    // alone).
    for (;;) {
        // regeneration: teams without a walk take the next ones (one ballot
        // bit per team, on its leader)
        unsigned need = __ballot_sync(FULL, g.leader() && !have && !drained);
        if (need) {
            int lead = __ffs(need) - 1;
            unsigned long long base = 0;
            if (lane == lead) {
                bool stop = *(volatile int *)acc.cancel != 0;
                base = stop ? total : atomicAdd(acc.next_walk, (unsigned long long)__popc(need));
            }
            base = __shfl_sync(FULL, base, lead);
            if ((need >> g.base) & 1u) {
                unsigned long long my = base + __popc(need & ((1u << g.base) - 1u));
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
        if (walk_step<D, SCR>(sc, sp, w, q, have)) {
            if (g.leader()) accumulate(acc, w);
            have = false;
        }
        __syncwarp();
    }
}

// Resumable persistent kernel: as k_walk_persistent, but each launch runs at
// most `iters` loop iterations (one walk step each) and then saves the walk
// its team holds into the team's slot; the next launch resumes it.  A solve
// is a sequence of such launches over a fixed grid, so no launch waits for
// the longest walks of the solve: their steps spill into later launches
// while the rest of the grid keeps drawing new walks.
template <int D, bool SCR, int T>
__global__ void WOST_WALK_BOUNDS k_walk_resume(const SceneView sc, const SolveParams sp,
                                                     const Accumulators acc, const ResumeState rs, int iters) {
    Cnt<false> cnt;
    auto q = make_q<D, false, T>(sp.stack_depth, acc.guard, cnt, sp.visit_limit);
    const Group g = make_team<T>();
    const uint64_t total = (uint64_t)sp.n_points * (uint64_t)sp.walks_per_point;
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    float4 *slot = rs.slots + 3 * (((size_t)blockIdx.x * blockDim.x + threadIdx.x) / T);
    Walk w{};
    bool have = false, drained = false;  // uniform within a team
    {
        float4 c = slot[2];
        uint32_t flags = __float_as_uint(c.w);
        if (flags & 1u) {
            float4 a = slot[0], b = slot[1];
            w.x = mk(a.x, a.y, a.z);
            w.acc = a.w;
            w.n = mk(b.x, b.y, b.z);
            w.dbound = b.w;
            w.steps = (int)__float_as_uint(c.x);
            w.point = __float_as_uint(c.y);
            w.index = __float_as_uint(c.z);
            w.onN = (flags & 2u) != 0;
            w.capped = (flags & 4u) != 0;
            have = true;
        }
    }
    unsigned long long ran = 0;
    for (int it = 0; it < iters; ++it) {
        unsigned need = __ballot_sync(FULL, g.leader() && !have && !drained);
        if (need) {
            int lead = __ffs(need) - 1;
            unsigned long long base = 0;
            if (lane == lead) {
                bool stop = *(volatile int *)acc.cancel != 0;
                base = stop ? total : atomicAdd(acc.next_walk, (unsigned long long)__popc(need));
            }
            base = __shfl_sync(FULL, base, lead);
            if ((need >> g.base) & 1u) {
                unsigned long long my = base + __popc(need & ((1u << g.base) - 1u));
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
        if (have) ++ran;
        if (walk_step<D, SCR>(sc, sp, w, q, have)) {
            if (g.leader()) accumulate(acc, w);
            have = false;
        }
        __syncwarp();
    }
    if (g.leader()) {
        if (have) {
            uint32_t flags = 1u | (w.onN ? 2u : 0u) | (w.capped ? 4u : 0u);
            slot[0] = make_float4(w.x.x, w.x.y, w.x.z, w.acc);
            slot[1] = make_float4(w.n.x, w.n.y, w.n.z, w.dbound);
            slot[2] = make_float4(__uint_as_float((uint32_t)w.steps), __uint_as_float(w.point),
                                  __uint_as_float(w.index), __uint_as_float(flags));
        } else {
            slot[2] = make_float4(0.f, 0.f, 0.f, 0.f);  // flags 0: empty
        }
    }
    // launch totals: steps run (one count per team) and walks saved
    unsigned long long r = g.leader() ? ran : 0ull;
    unsigned saved = __popc(__ballot_sync(FULL, g.leader() && have));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(FULL, r, o);
    if (lane == 0) {
        if (r) atomicAdd(rs.steps_run, r);
        if (saved) atomicAdd(rs.live, saved);
    }
}

// Counting variant of the plain kernel: same walks, plus per-query node
// visits and primitive tests summed into stats[2 * C_NQ] (nodes then prims).
template <int D, bool SCR>
__global__ void __launch_bounds__(256) k_walk_count(const SceneView sc, const SolveParams sp, const Accumulators acc,
                                                    unsigned long long *stats) {
    Cnt<true> cnt;
    auto q = make_q<D, true>(sp.stack_depth, acc.guard, cnt, sp.visit_limit);
    const Group g = make_team<1>();
    const uint64_t total = (uint64_t)sp.n_points * (uint64_t)sp.walks_per_point;
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = gid < total;
    Walk w{};
    if (active) {
        int64_t pt = (int64_t)(gid / (uint64_t)sp.walks_per_point);
        uint32_t j = (uint32_t)(gid % (uint64_t)sp.walks_per_point) + sp.first_walk;
        walk_init<D>(sp, w, pt, j);
    }
    bool done = !active;
    while (__any_sync(0xffffffffu, !done)) {
        if (walk_step<D, SCR>(sc, sp, w, q, !done)) done = true;
        __syncwarp();
    }
    if (!active || !g.leader()) return;
    accumulate(acc, w);
    for (int c = 0; c < C_NQ; ++c) {
        atomicAdd(stats + c, (unsigned long long)cnt.nodes[c]);
        atomicAdd(stats + C_NQ + c, (unsigned long long)cnt.prims[c]);
    }
}

// ------------------------------- launch helpers ---------------------------
static size_t smem_bytes(int depth, int block, int lanes = 1) { return (size_t)depth * (block / lanes) * sizeof(int2); }

// sets the dynamic shared-memory limit of kernel k when above the default
static cudaError_t smem_limit(const void *k, size_t bytes) {
    return bytes > 48 * 1024 ? cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
                             : cudaSuccess;
}

template <bool SCR>
static cudaError_t walk_plain_launch(const SceneView &sc, const SolveParams &sp, const Accumulators &acc, int block,
                                     cudaStream_t s) {
    uint64_t total = (uint64_t)sp.n_points * (uint64_t)sp.walks_per_point;
    uint64_t grid = (total + block - 1) / block;
    if (grid > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
    size_t sm = smem_bytes(sp.stack_depth, block);
    int uniform = (sp.walks_per_point % 32 == 0) && (block % 32 == 0);
    const void *k = sc.dim == 2 ? (const void *)k_walk_plain<2, SCR> : (const void *)k_walk_plain<3, SCR>;
    cudaError_t e = smem_limit(k, sm);
    if (e != cudaSuccess) return e;
    if (sc.dim == 2)
        k_walk_plain<2, SCR><<<(unsigned)grid, block, sm, s>>>(sc, sp, acc, uniform);
    else
        k_walk_plain<3, SCR><<<(unsigned)grid, block, sm, s>>>(sc, sp, acc, uniform);
    return cudaGetLastError();
}

template <bool SCR>
static cudaError_t walk_count_launch(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                                     unsigned long long *stats, int block, cudaStream_t s) {
    uint64_t total = (uint64_t)sp.n_points * (uint64_t)sp.walks_per_point;
    uint64_t grid = (total + block - 1) / block;
    if (grid > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
    size_t sm = smem_bytes(sp.stack_depth, block);
    const void *k = sc.dim == 2 ? (const void *)k_walk_count<2, SCR> : (const void *)k_walk_count<3, SCR>;
    cudaError_t e = smem_limit(k, sm);
    if (e != cudaSuccess) return e;
    if (sc.dim == 2)
        k_walk_count<2, SCR><<<(unsigned)grid, block, sm, s>>>(sc, sp, acc, stats);
    else
        k_walk_count<3, SCR><<<(unsigned)grid, block, sm, s>>>(sc, sp, acc, stats);
    return cudaGetLastError();
}

// resident blocks of kernel k per SM times the SM count, its shared-memory
// limit set
static cudaError_t resident_grid(const void *k, int block, int depth, int *blocks_out, int lanes = 1) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t sm = smem_bytes(depth, block, lanes);
    if (e == cudaSuccess) e = smem_limit(k, sm);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, sm);
    if (e != cudaSuccess) return e;
    *blocks_out = sms * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

template <bool SCR, int T>
static cudaError_t walk_persistent_launch(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                                          int block, int blocks, cudaStream_t s) {
    size_t sm = smem_bytes(sp.stack_depth, block, T);
    const void *k =
        sc.dim == 2 ? (const void *)k_walk_persistent<2, SCR, T> : (const void *)k_walk_persistent<3, SCR, T>;
    cudaError_t e = smem_limit(k, sm);
    if (e != cudaSuccess) return e;
    if (sc.dim == 2)
        k_walk_persistent<2, SCR, T><<<blocks, block, sm, s>>>(sc, sp, acc);
    else
        k_walk_persistent<3, SCR, T><<<blocks, block, sm, s>>>(sc, sp, acc);
    return cudaGetLastError();
}

template <bool SCR, int T>
static cudaError_t walk_resume_launch(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                                      const ResumeState &rs, int iters, int block, int blocks, cudaStream_t s) {
    size_t sm = smem_bytes(sp.stack_depth, block, T);
    const void *k = sc.dim == 2 ? (const void *)k_walk_resume<2, SCR, T> : (const void *)k_walk_resume<3, SCR, T>;
    cudaError_t e = smem_limit(k, sm);
    if (e != cudaSuccess) return e;
    if (sc.dim == 2)
        k_walk_resume<2, SCR, T><<<blocks, block, sm, s>>>(sc, sp, acc, rs, iters);
    else
        k_walk_resume<3, SCR, T><<<blocks, block, sm, s>>>(sc, sp, acc, rs, iters);
    return cudaGetLastError();
}

// screened instantiations, defined in wost_kernels_scr.cu
cudaError_t launch_walk_plain_scr(const SceneView &sc, const SolveParams &sp, const Accumulators &acc, int block,
                                  cudaStream_t s);
cudaError_t launch_walk_count_scr(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                                  unsigned long long *stats, int block, cudaStream_t s);
cudaError_t launch_walk_persistent_scr(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                                       int block, int blocks, cudaStream_t s);
cudaError_t launch_walk_resume_scr(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                                   const ResumeState &rs, int iters, int block, int blocks, cudaStream_t s);
// 8-lane team instantiations (Poisson), defined in wost_kernels_team.cu
cudaError_t persistent_grid_team(int dim, int block, int depth, int *blocks_out);
cudaError_t launch_walk_persistent_team(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                                        int block, int blocks, cudaStream_t s);
cudaError_t launch_walk_resume_team(const SceneView &sc, const SolveParams &sp, const Accumulators &acc,
                                    const ResumeState &rs, int iters, int block, int blocks, cudaStream_t s);

}  // namespace wost
