// The batched persistent walk kernel (wost_solve_batch and the serving
// engine's rounds), instantiated in wost_kernels_batch.cu in two forms:
// SCR = true when a job of the batch is screened, SCR = false (the smaller
// Poisson-only code) when none is.
#pragma once

#include "wost_walk.cuh"

namespace wost {

// Batched persistent kernel: many solves (scenes, point sets, walk counts,
// parameters) in one launch.  The walk index space is the concatenation of
// the jobs' walks; a team maps its next index to a job by binary search over
// the jobs' first indices and runs that job's walk on that job's scene.
// steps_out (may be null) receives the walk steps of the finished walks.
template <int D, bool SCR>
__global__ void WOST_WALK_BOUNDS k_walk_batch(const BatchHeader *__restrict__ hdr,
                                                    const BatchJob *__restrict__ jobs, unsigned long long *counter,
                                                    unsigned int *guard, int stack_depth, const int *cancel,
                                                    unsigned long long *steps_out) {
    const int n_jobs = hdr->n_jobs;
    const unsigned long long total = hdr->total;
    if (n_jobs <= 0) return;
    Cnt<false> cnt;
    auto q = make_q<D, false>(stack_depth, guard, cnt);
    const Group g = make_team<1>();
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    Walk w{};
    int job = -1;
    unsigned int ran = 0;  // steps of this lane's finished walks
    bool drained = false;  // the launch's counter has run past `total`
    // as in k_walk_persistent: the whole warp stays in the loop and
    // reconverges after every step
    for (;;) {
        unsigned need = __ballot_sync(FULL, g.leader() && job < 0 && !drained);
        if (need) {
            int lead = __ffs(need) - 1;
            unsigned long long base = 0;
            if (lane == lead) {
                bool stop = cancel && *(volatile const int *)cancel != 0;
                base = stop ? total : atomicAdd(counter, (unsigned long long)__popc(need));
            }
            base = __shfl_sync(FULL, base, lead);
            if ((need >> g.base) & 1u) {
                unsigned long long my = base + __popc(need & ((1u << g.base) - 1u));
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
                    // team takes another index at the next iteration
                    if (!team_flag(g, jobs[lo].acc.cancel)) {
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
        // lanes without a job step a dummy reference to job 0 (inactive)
        const BatchJob &J = jobs[job >= 0 ? job : 0];
        if (walk_step<D, SCR>(*J.scene, J.sp, w, q, job >= 0)) {
            if (g.leader()) {
                accumulate(J.acc, w);
                ran += (unsigned int)w.steps;
            }
            job = -1;
        }
        __syncwarp();
    }
    if (steps_out) {
        unsigned long long r = ran;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(FULL, r, o);
        if (lane == 0 && r) atomicAdd(steps_out, r);
    }
}

}  // namespace wost
