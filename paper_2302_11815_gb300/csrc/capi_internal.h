// Internal objects behind the C ABI handles, shared by wost_capi.cpp and
// wost_engine.cpp.
#pragma once

#include <cuda_runtime.h>

#include <chrono>
#include <memory>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/wost.h"
#include "scene_build.h"
#include "wost_kernels.h"

namespace wost {

// records the thread-local error message and returns s
wost_status fail(wost_status s, const std::string &msg);
wost_status cuda_fail(cudaError_t e, const char *what);
#define CK(expr, what)                                     \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return wost::cuda_fail(_e, what); \
    } while (0)

// device allocation owned by a scene or solve
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t n) {
        bytes = n;
        return n ? cudaMalloc(&p, n) : cudaSuccess;
    }
    // stream-ordered allocation / release: neither waits for the device,
    // unlike cudaMalloc / cudaFree, which synchronise with all work in flight
    cudaError_t alloc_async(size_t n, cudaStream_t s, cudaMemPool_t pool = nullptr) {
        bytes = n;
        if (!n) return cudaSuccess;
        return pool ? cudaMallocFromPoolAsync(&p, n, pool, s) : cudaMallocAsync(&p, n, s);
    }
    void release_async(cudaStream_t s) {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
    }
};

template <class T>
cudaError_t upload(DevBuf &b, const std::vector<T> &v) {
    cudaError_t e = b.alloc(v.size() * sizeof(T));
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

// resources shared by the solves of one batched launch
struct BatchShared {
    DevBuf jobs[2], counters;  // counters: next walk (2D), next walk (3D), guard
    unsigned long long total[2] = {0, 0};
    cudaEvent_t ev_start = nullptr, ev_done = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;  // the 3D launch's side stream
    cudaStream_t own_stream = nullptr, side = nullptr;
    ~BatchShared() {
        if (ev_done) cudaEventSynchronize(ev_done);
        if (ev_start) cudaEventDestroy(ev_start);
        if (ev_done) cudaEventDestroy(ev_done);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
        if (own_stream) cudaStreamDestroy(own_stream);
    }
};

}  // namespace wost

struct wost_engine;

struct wost_scene {
    int device = 0;
    wost::HostScene host;
    wost::SceneView view{};
    wost::DevBuf bufs[16];
    wost::DevBuf wbufs[6];  // wide layout: nodes and cones of the three trees
    wost::DevBuf sbufs[4];  // double-sided records (App. B): - side data and flags of D and N
    wost::DevBuf n_rec_of_id;
    unsigned int *guard = nullptr;        // device guard word for query kernels
    wost::SceneView *view_dev = nullptr;  // device copy of `view` (batched launches)
    wost_scene_info info{};
    int stack_depth = 0;                  // traversal stack entries per walk, one lane per walk
    int stack_depth_team = 0;             // ... per 8-lane team over the 8-wide trees
    int tuned_block = 0;                  // set by wost_scene_autotune (0 = not tuned)
    int tuned_lanes = 1;                  // lanes per walk chosen by wost_scene_autotune
    std::mutex mu;
    ~wost_scene() {
        if (guard) cudaFree(guard);
        if (view_dev) cudaFree(view_dev);
    }
};

struct wost_solve_handle {
    wost_scene *scene = nullptr;
    int device = 0;
    int dim = 2;
    int64_t n_points = 0;
    int32_t walks = 0;
    int block = 128;
    int lanes = 1;                        // lanes per walk (persistent / resumable kernels)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t poll_stream = nullptr;
    bool own_poll_stream = true;  // engine requests share the engine's poll streams
    cudaEvent_t ev_start = nullptr, ev_done = nullptr;
    bool own_events = false;
    std::shared_ptr<wost::BatchShared> batch;  // set for solves started by wost_solve_batch
    unsigned int *batch_guard = nullptr;
    wost_engine *engine = nullptr;             // set for solves submitted to an engine
    wost::SolveParams sp{};
    wost::Accumulators acc{};
    wost::DevBuf points, normals, onN;
    wost::DevBuf sum, sumsq, walks_done, steps, globals;  // globals: capped, next_walk, guard
    wost::DevBuf counts;                                   // counting kernel only
    // resumable solves: saved-walk slots of the fixed grid, launch counters
    // (steps_run u64, live u32), launches enqueued so far
    wost::DevBuf slots, rstate;
    int resume_blocks = 0;
    uint64_t launches = 0;
    bool resumable() const { return kernel == WOST_KERNEL_RESUMABLE; }
    int kernel = 0;
    int *cancel_host = nullptr;                            // mapped pinned (engine requests: plain host)
    int *cancel_dev = nullptr;
    // engine requests: device buffers come from the stream-ordered allocator
    // and the cancel flag is plain host memory (the engine reads it on the
    // host), so that destroying a request never waits for the device, whose
    // queue the engine keeps full
    bool engine_buffers = false;
    cudaMemPool_t pool = nullptr;  // the engine's memory pool (engine requests)
    // engine requests: set once a round holding some of the request's walks
    // has completed; until then a poll reports no walks without reading
    // the device (its buffers may still be being set up)
    std::atomic<bool> engine_ready{false};
    std::chrono::steady_clock::time_point t_launch;
    double elapsed_done = -1;
    bool done = false;
    wost_status final_status = WOST_OK;                    // engine requests
    std::mutex mu;
    ~wost_solve_handle() {
        if (ev_done) cudaEventSynchronize(ev_done);
        else if (stream) cudaStreamSynchronize(stream);
        if (own_events && ev_start) cudaEventDestroy(ev_start);
        if (own_events && ev_done) cudaEventDestroy(ev_done);
        if (engine_buffers) {
            for (wost::DevBuf *b : {&points, &normals, &onN, &sum, &sumsq, &walks_done, &steps, &globals})
                b->release_async(poll_stream);
            delete cancel_host;
        } else if (cancel_host) {
            cudaFreeHost(cancel_host);
        }
        if (poll_stream && own_poll_stream) cudaStreamDestroy(poll_stream);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace wost {
// Layout fields of a scene's info for `lanes` lanes per walk.
void set_layout_info(wost_scene *s, int lanes);
// Validates a solve description, allocates and fills the solve's device
// buffers on `stream`, fills h->sp and h->acc.  Does not launch.  With
// fill false the buffers are only allocated: the caller uploads the points,
// normals and flags and clears the accumulators (the serving engine does
// both on streams of its own).
wost_status prepare_solve(wost_scene *scene, const wost_solve_desc *d, cudaStream_t stream, wost_solve_handle *h,
                          bool fill = true);
// Zeroes a solve's accumulators and counters on `stream`.
cudaError_t clear_accumulators(wost_solve_handle *h, cudaStream_t stream);
// Blocks until the work queued so far on `stream` (the input copies) is done.
wost_status wait_for_copies(cudaStream_t stream);
// Engine side of wost_solve_destroy / wost_cancel for engine requests.
void engine_detach(wost_engine *e, wost_solve_handle *h);
}  // namespace wost
