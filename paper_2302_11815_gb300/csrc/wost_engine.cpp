// Serving engine (include/wost.h, wost_engine_*): continuous batching of
// walk-on-stars solves with target standard errors on one device.
//
// One scheduler thread per engine.  Each scheduling round is one batched
// persistent launch (k_walk_batch, one per dimension present) over "pieces"
// -- point ranges x walk ranges -- of every active request, sized so that a
// round takes about round_seconds of GPU time (the walk-step budget adapts to
// the measured round times), but never less than a few walks per resident
// lane (min_round_steps).  Every round slot has streams of its own and up
// to three rounds are in flight: a round lasts until its longest walk ends,
// and the next rounds' blocks take the SMs that its finished blocks free, so
// the tail of one round overlaps the bulk of the next and the host prepares
// rounds while the GPU runs earlier ones.  Requests are admitted FIFO by
// device-memory budget, run in stages of walks per point, and are checked
// after each stage with the per-solve summary kernel (k_request_stats) on a
// high-priority stream (its blocks go first when SMs free up).  A check is
// asynchronous: the scheduler issues it and reads its results once its event
// has completed, so it never waits for the device with the engine's lock
// held (submissions and new rounds go on meanwhile).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <new>
#include <thread>
#include <unordered_map>

#include "capi_internal.h"

using namespace wost;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    wost_solve_handle *h = nullptr;
    wost_scene *scene = nullptr;
    std::vector<float> pts, nrm;  // host copies of the inputs until admission
    std::vector<uint8_t> onN;
    wost_solve_desc desc{};
    double target = 0;
    int cap = 0;
    int64_t bytes = 0;
    Clock::time_point t_submit;
    int stage_begin = 0, stage_end = 0;  // walks per point of the current stage
    int64_t cursor = 0;                  // next point of the stage to issue
    int outstanding = 0;                 // pieces in flight
    double mean_steps = 64.0;            // running estimate of steps per walk (from its scene's at admission)
    bool admitted = false, finished = false, started = false;
};

struct Piece {
    Request *r;
    int64_t p0, np;
    int w0, nw;
};

// One scheduling slot: device job tables (BatchHeader + jobs, per
// dimension), their pinned staging copies, and the CUDA graph of one round:
// reset counters, upload both tables, launch the 2D and the 3D batched
// kernels as parallel branches (a kernel whose table is empty returns at
// once), copy the round's walk-step count to the host.  A round replays the
// graph on the slot's own stream; it is re-captured only when a table
// outgrows its capacity or a deeper scene needs a larger traversal stack.
struct Slot {
    DevBuf jobs[2];
    unsigned char *host[2] = {nullptr, nullptr};
    size_t cap[2] = {0, 0};    // jobs per table
    int depth[2] = {0, 0};     // stack entries the graph was captured with
    bool scr[2] = {true, true};  // the kernels' form: screened, or Poisson only
    DevBuf counters;           // next walk 2D, next walk 3D, guard, walk steps run
    unsigned long long *steps_host = nullptr;  // pinned copy of the walk-step count
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t stream = nullptr, side = nullptr;  // the round; its 3D branch
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool busy = false;
    ~Slot() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (auto *h : host)
            if (h) cudaFreeHost(h);
        if (steps_host) cudaFreeHost(steps_host);
        for (cudaEvent_t ev : {fork, join, ev0, ev1})
            if (ev) cudaEventDestroy(ev);
        for (cudaStream_t st : {stream, side})
            if (st) cudaStreamDestroy(st);
    }
};

constexpr int kSlots = 3;  // rounds in flight at most

size_t table_bytes(size_t jobs) { return sizeof(BatchHeader) + jobs * sizeof(BatchJob); }

struct Round {
    int slot;
    std::vector<Piece> pieces;
};

// One stage check in flight: the summary kernel's inputs and outputs for the
// requests whose stage completed, on the device and in pinned host memory.
// Outputs, cap entries each: max variance (FP32 bits, u32), then min walks,
// steps and walks (u64) at byte offsets 8, 16 and 24 times cap.
struct CheckSet {
    DevBuf jobs, out;
    StatJob *host_jobs = nullptr;
    unsigned char *host_out = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    std::vector<Request *> reqs;
    bool busy = false;
    ~CheckSet() {
        if (host_jobs) cudaFreeHost(host_jobs);
        if (host_out) cudaFreeHost(host_out);
        if (ev) cudaEventDestroy(ev);
    }
};

constexpr int kChecks = 4;  // stage checks in flight at most
constexpr int kStage = 8;                  // pinned staging slots for request inputs
constexpr int kPollStreams = 8;            // poll streams shared by the engine's requests
constexpr size_t kStageBytes = 8u << 20;   // bytes per slot

}  // namespace

struct wost_engine {
    int device = 0;
    cudaStream_t stream = nullptr, check_stream = nullptr;  // admissions; stage checks
    cudaEvent_t ev_ready = nullptr;                   // orders a round after the admissions before it
    cudaStream_t copy_stream = nullptr;               // submissions' copies of device inputs
    // requests poll on these (creating a stream per request waits for the
    // device: measured up to 2 s with rounds resident)
    cudaStream_t poll[kPollStreams] = {};
    int poll_next = 0;
    // request buffers come from the engine's own pool, which keeps what is
    // freed (no trimming, so no remapping on later allocations)
    cudaMemPool_t pool = nullptr;
    // admissions: allocations and input uploads on `stream` (copies only, no
    // kernels, so they complete while rounds fill the SMs), the zeroing of
    // the accumulators on `zero_stream` (high priority); rounds wait for both
    cudaStream_t zero_stream = nullptr;
    cudaEvent_t ev_alloc = nullptr;
    cudaEvent_t ev_detach = nullptr;  // orders a released request's frees after its set-up
    // pinned staging slots the inputs are uploaded from (a copy from
    // pageable memory is synchronous and may wait on the device); a slot is
    // free again once its event has completed, and an admission that finds
    // none free waits for a later pass of the scheduler
    unsigned char *stage = nullptr;
    cudaEvent_t stage_ev[kStage] = {};
    bool stage_busy[kStage] = {};
    int64_t budget = 0, used = 0;
    double round_seconds = 0.02;
    double max_wait = 0;              // seconds a request may wait for its first walks (0: no limit)
    // resident lanes of the batched kernel per traversal stack depth (the
    // shared memory per block sets the grid), for the rounds' walk-step
    // floor (min_round_steps)
    std::unordered_map<int, double> lanes_at_depth[2];
    int min_walks = 16, cap = 65536, block = 128;
    std::mutex mu;
    std::mutex copy_mu;  // the copy stream (submissions from several threads)
    std::condition_variable cv, done_cv;
    std::deque<Request *> pending;
    std::vector<Request *> active;
    std::unordered_map<wost_solve_handle *, Request *> by_handle;
    std::deque<Round> inflight;
    Slot slots[kSlots];
    double round_budget_steps = 4e6;
    wost_engine_stats st{};
    bool stop = false;
    std::thread th;
    CheckSet checks[kChecks];
    std::deque<int> check_order;  // busy check sets, oldest first
    // steps per walk measured on each scene (moving average over stage
    // checks): a new request's cost estimate, so that rounds hold the walk
    // steps their budget pays for from the first stage on
    std::unordered_map<const wost_scene *, double> scene_steps;
};

namespace {

double since(Clock::time_point t) { return std::chrono::duration<double>(Clock::now() - t).count(); }

void finish(wost_engine *e, Request *r, wost_status status) {
    if (r->finished) return;
    r->finished = true;
    {
        std::lock_guard<std::mutex> lk(r->h->mu);
        r->h->done = true;
        r->h->elapsed_done = since(r->t_submit);
        r->h->final_status = status;
    }
    if (status == WOST_OK) e->st.completed++;
    else if (status == WOST_ERR_CANCELLED) e->st.cancelled++;
    e->active.erase(std::remove(e->active.begin(), e->active.end(), r), e->active.end());
    e->done_cv.notify_all();
}

bool cancelled(const Request *r) { return *(volatile int *)r->h->cancel_host != 0; }

// A free staging slot (-1: none now).
int free_stage(wost_engine *e) {
    for (int i = 0; i < kStage; ++i) {
        if (e->stage_busy[i] && cudaEventQuery(e->stage_ev[i]) != cudaErrorNotReady) e->stage_busy[i] = false;
        if (!e->stage_busy[i]) return i;
    }
    return -1;
}

// Allocates a request's buffers, uploads its inputs from a staging slot
// (or, for inputs larger than a slot, straight from its host copy) and
// clears its accumulators.  Polls read the buffers only once a round with
// the request's walks has completed, and rounds run after all of this.
wost_status set_up(wost_engine *e, Request *r, int slot) {
    r->h->poll_stream = e->poll[e->poll_next];
    r->h->own_poll_stream = false;
    e->poll_next = (e->poll_next + 1) % kPollStreams;
    wost_status s = prepare_solve(r->scene, &r->desc, e->stream, r->h, false);
    r->h->stream = nullptr;  // the engine's streams are not the handle's to synchronize
    if (s != WOST_OK) return s;
    wost_solve_handle *h = r->h;
    const size_t n = (size_t)h->n_points, pb = n * h->dim * sizeof(float);
    const bool has_n = !r->nrm.empty();
    cudaError_t er = cudaSuccess;
    auto put = [&](void *dst, const void *src, size_t bytes, size_t &off) {
        if (er != cudaSuccess) return;
        if (slot >= 0) {
            unsigned char *buf = e->stage + (size_t)slot * kStageBytes + off;
            std::memcpy(buf, src, bytes);
            er = cudaMemcpyAsync(dst, buf, bytes, cudaMemcpyHostToDevice, e->stream);
            off += (bytes + 15) & ~(size_t)15;
        } else {
            er = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, e->stream);
        }
    };
    size_t off = 0;
    put(h->points.p, r->pts.data(), pb, off);
    if (has_n) {
        put(h->normals.p, r->nrm.data(), pb, off);
        put(h->onN.p, r->onN.data(), n, off);
    }
    if (er == cudaSuccess && slot >= 0 && (er = cudaEventRecord(e->stage_ev[slot], e->stream)) == cudaSuccess)
        e->stage_busy[slot] = true;
    if (er == cudaSuccess) er = cudaEventRecord(e->ev_alloc, e->stream);
    if (er == cudaSuccess) er = cudaStreamWaitEvent(e->zero_stream, e->ev_alloc, 0);
    if (er == cudaSuccess) er = clear_accumulators(h, e->zero_stream);
    return er == cudaSuccess ? WOST_OK : fail(WOST_ERR_CUDA, "setting up a request");
}

size_t input_bytes(const Request *r) {
    const size_t b = r->pts.size() * sizeof(float) + r->nrm.size() * sizeof(float) + r->onN.size();
    return b + 32;  // alignment of the second and third arrays
}

void admit(wost_engine *e) {
    while (!e->pending.empty()) {
        Request *r = e->pending.front();
        if (cancelled(r)) {
            e->pending.pop_front();
            finish(e, r, WOST_ERR_CANCELLED);
            continue;
        }
        if (e->used + r->bytes > e->budget) break;  // FIFO: later requests wait too
        int slot = -1;
        if (input_bytes(r) <= kStageBytes && (slot = free_stage(e)) < 0) break;  // no slot free yet
        e->pending.pop_front();
        wost_status s;
        {
            std::lock_guard<std::mutex> hl(r->h->mu);  // pollers see either nothing or a complete state
            s = set_up(e, r, slot);
        }
        r->pts.clear();
        r->pts.shrink_to_fit();
        r->nrm.clear();
        r->nrm.shrink_to_fit();
        r->onN.clear();
        r->onN.shrink_to_fit();
        if (s != WOST_OK) {
            finish(e, r, s);
            continue;
        }
        r->h->t_launch = Clock::now();
        auto known = e->scene_steps.find(r->scene);
        if (known != e->scene_steps.end()) r->mean_steps = known->second;
        r->admitted = true;
        e->used += r->bytes;
        e->st.admitted++;
        r->stage_begin = 0;
        r->stage_end = std::min(r->cap, e->min_walks);
        r->cursor = 0;
        e->active.push_back(r);
    }
}

// Stage decisions from a completed check: finish the request (target met,
// walk cap reached, cancelled) or size its next stage from its variance.
void apply_check(wost_engine *e, CheckSet &cs, cudaError_t err) {
    const size_t cap = cs.cap;
    const unsigned int *hv = (const unsigned int *)cs.host_out;
    const unsigned long long *hs = (const unsigned long long *)(cs.host_out + 16 * cap);
    const unsigned long long *hw = (const unsigned long long *)(cs.host_out + 24 * cap);
    for (size_t i = 0; i < cs.reqs.size(); ++i) {
        Request *r = cs.reqs[i];
        r->outstanding--;
        if (err != cudaSuccess) {
            finish(e, r, WOST_ERR_CUDA);
            continue;
        }
        float mv;
        std::memcpy(&mv, &hv[i], 4);
        if (hw[i]) {
            r->mean_steps = std::max(1.0, (double)hs[i] / (double)hw[i]);
            auto ins = e->scene_steps.emplace(r->scene, r->mean_steps);
            if (!ins.second) ins.first->second = 0.75 * ins.first->second + 0.25 * r->mean_steps;
        }
        int W = r->stage_end;
        double t2 = r->target * r->target;
        bool met = r->target > 0 && (double)mv <= t2 * W;
        if (cancelled(r)) {
            finish(e, r, WOST_ERR_CANCELLED);
        } else if (met || W >= r->cap) {
            if (!met && r->target > 0) e->st.capped++;
            finish(e, r, WOST_OK);
        } else {
            double need = (double)mv / t2;
            int next = (int)std::min<double>(r->cap, std::max(W + W / 2.0, std::ceil(1.05 * need / 16.0) * 16.0));
            r->stage_begin = W;
            r->stage_end = std::max(next, W + 1);
            r->cursor = 0;
        }
    }
    cs.reqs.clear();
    cs.busy = false;
}

// Applies the checks whose results have arrived (all of them, waiting for
// the device, if wait is set).
void complete_checks(wost_engine *e, bool wait) {
    while (!e->check_order.empty()) {
        CheckSet &cs = e->checks[e->check_order.front()];
        cudaError_t q = wait ? cudaEventSynchronize(cs.ev) : cudaEventQuery(cs.ev);
        if (q == cudaErrorNotReady) return;
        e->check_order.pop_front();
        apply_check(e, cs, q);
    }
}

// Issues the stage check of the requests whose current stage has fully
// completed; each counts as outstanding until its check is applied.
void issue_check(wost_engine *e, std::vector<Request *> &ready) {
    if (ready.empty()) return;
    int ci = -1;
    for (int i = 0; i < kChecks && ci < 0; ++i)
        if (!e->checks[i].busy) ci = i;
    if (ci < 0) {  // all sets in flight: the oldest is applied first
        int oldest = e->check_order.front();
        CheckSet &o = e->checks[oldest];
        cudaError_t q = cudaEventSynchronize(o.ev);
        e->check_order.pop_front();
        apply_check(e, o, q);
        ci = oldest;
    }
    CheckSet &cs = e->checks[ci];
    const size_t n = ready.size();
    cudaError_t err = cudaSuccess;
    if (n > cs.cap) {
        size_t nc = std::max<size_t>(n, 2 * cs.cap);
        if (cs.host_jobs) cudaFreeHost(cs.host_jobs);
        if (cs.host_out) cudaFreeHost(cs.host_out);
        cs.host_jobs = nullptr;
        cs.host_out = nullptr;
        cs.cap = 0;
        cs.jobs.release_async(e->check_stream);
        cs.out.release_async(e->check_stream);
        if ((err = cudaMallocHost((void **)&cs.host_jobs, nc * sizeof(StatJob))) == cudaSuccess &&
            (err = cudaMallocHost((void **)&cs.host_out, nc * 32)) == cudaSuccess &&
            (err = cs.jobs.alloc_async(nc * sizeof(StatJob), e->check_stream, e->pool)) == cudaSuccess &&
            (err = cs.out.alloc_async(nc * 32, e->check_stream, e->pool)) == cudaSuccess)
            cs.cap = nc;
    }
    if (err == cudaSuccess && !cs.ev) err = cudaEventCreateWithFlags(&cs.ev, cudaEventDisableTiming);
    if (err != cudaSuccess) {
        for (Request *r : ready) finish(e, r, WOST_ERR_CUDA);
        return;
    }
    const size_t cap = cs.cap;
    int64_t maxn = 0;
    for (size_t i = 0; i < n; ++i) {
        const Accumulators &a = ready[i]->h->acc;
        cs.host_jobs[i] = StatJob{a.sum, a.sumsq, a.walks, a.steps, ready[i]->h->n_points};
        maxn = std::max(maxn, ready[i]->h->n_points);
    }
    unsigned char *out = (unsigned char *)cs.out.p;
    unsigned int *mvar = (unsigned int *)out;
    unsigned long long *minw = (unsigned long long *)(out + 8 * cap);
    unsigned long long *ssum = minw + cap, *wsum = ssum + cap;
    cudaStream_t s = e->check_stream;
    cudaMemcpyAsync(cs.jobs.p, cs.host_jobs, n * sizeof(StatJob), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(mvar, 0, n * 4, s);
    cudaMemsetAsync(minw, 0xFF, n * 8, s);
    cudaMemsetAsync(ssum, 0, n * 8, s);
    cudaMemsetAsync(wsum, 0, n * 8, s);
    launch_request_stats((const StatJob *)cs.jobs.p, (int)n, maxn, mvar, minw, ssum, wsum, s);
    cudaMemcpyAsync(cs.host_out, mvar, n * 4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(cs.host_out + 16 * cap, ssum, n * 8, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(cs.host_out + 24 * cap, wsum, n * 8, cudaMemcpyDeviceToHost, s);
    cudaEventRecord(cs.ev, s);
    cs.reqs = ready;
    for (Request *r : ready) r->outstanding++;
    cs.busy = true;
    e->check_order.push_back(ci);
}

void retire(wost_engine *e, size_t i) {
    Round rd = std::move(e->inflight[i]);
    e->inflight.erase(e->inflight.begin() + (std::ptrdiff_t)i);
    Slot &sl = e->slots[rd.slot];
    float ms = 0;
    cudaEventElapsedTime(&ms, sl.ev0, sl.ev1);
    sl.busy = false;
    e->st.rounds++;
    e->st.gpu_seconds += ms * 1e-3;
    e->st.walk_steps += *(volatile unsigned long long *)sl.steps_host;
    if (ms > 0.05f) {
        double f = std::min(2.0, std::max(0.5, e->round_seconds * 1e3 / ms));
        e->round_budget_steps = std::min(2e10, std::max(1e5, e->round_budget_steps * f));
    }
    std::vector<Request *> ready;
    e->done_cv.notify_all();
    for (auto &p : rd.pieces) {
        p.r->h->engine_ready.store(true);
        p.r->outstanding--;
        if (!p.r->finished && p.r->outstanding == 0 && p.r->cursor >= p.r->h->n_points &&
            std::find(ready.begin(), ready.end(), p.r) == ready.end())
            ready.push_back(p.r);
    }
    issue_check(e, ready);
}

void process_cancels(wost_engine *e) {
    std::vector<Request *> done;
    for (Request *r : e->active)
        if (!r->finished && r->outstanding == 0 && (cancelled(r) || e->stop)) done.push_back(r);
    for (Request *r : done) finish(e, r, WOST_ERR_CANCELLED);
}

// (Re)captures the slot's round graph if its tables are too small for this
// round, a scene needs a deeper stack than the graph was captured with, or
// the round needs the other kernel form (a screened job, or none).
cudaError_t ensure_graph(wost_engine *e, Slot &sl, const size_t cnt[2], const int depth[2], const bool scr[2]) {
    bool rebuild = sl.exec == nullptr;
    cudaError_t er;
    for (int di = 0; di < 2; ++di) {
        if (cnt[di] > sl.cap[di] || !sl.host[di]) {
            size_t nc = std::max<size_t>(std::max<size_t>(cnt[di], 2 * sl.cap[di]), 16);
            if (sl.host[di]) cudaFreeHost(sl.host[di]);
            sl.host[di] = nullptr;
            if ((er = cudaMallocHost((void **)&sl.host[di], table_bytes(nc))) != cudaSuccess) return er;
            std::memset(sl.host[di], 0, sizeof(BatchHeader));
            sl.jobs[di].~DevBuf();
            new (&sl.jobs[di]) DevBuf();
            if ((er = sl.jobs[di].alloc(table_bytes(nc))) != cudaSuccess) return er;
            sl.cap[di] = nc;
            rebuild = true;
        }
        int want = std::max(depth[di], 2);
        if (want > sl.depth[di]) {
            sl.depth[di] = want;
            rebuild = true;
        }
        if (cnt[di] && scr[di] != sl.scr[di]) {
            sl.scr[di] = scr[di];
            rebuild = true;
        }
    }
    if (!sl.counters.p) {
        if ((er = sl.counters.alloc(4 * 8)) != cudaSuccess) return er;
        if ((er = cudaMallocHost((void **)&sl.steps_host, 8)) != cudaSuccess) return er;
        *sl.steps_host = 0;
        rebuild = true;
    }
    if (!rebuild) return cudaSuccess;
    if (sl.exec) cudaGraphExecDestroy(sl.exec);
    if (sl.graph) cudaGraphDestroy(sl.graph);
    sl.exec = nullptr;
    sl.graph = nullptr;
    int blocks[2];
    for (int di = 0; di < 2; ++di)
        if ((er = batch_grid(di + 2, e->block, sl.depth[di], &blocks[di])) != cudaSuccess) return er;
    unsigned long long *ctr = (unsigned long long *)sl.counters.p;
    if ((er = cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return er;
    cudaMemsetAsync(sl.counters.p, 0, 4 * 8, sl.stream);
    for (int di = 0; di < 2; ++di)
        cudaMemcpyAsync(sl.jobs[di].p, sl.host[di], table_bytes(sl.cap[di]), cudaMemcpyHostToDevice, sl.stream);
    // the 2D and 3D kernels are parallel branches of the graph (the 3D one
    // on the side stream, forked and joined inside the capture), so each
    // fills the SMs the other's tail leaves idle
    cudaEventRecord(sl.fork, sl.stream);
    cudaStreamWaitEvent(sl.side, sl.fork, 0);
    for (int di = 0; di < 2; ++di) {
        const unsigned char *base = (const unsigned char *)sl.jobs[di].p;
        launch_walk_batch(di + 2, (const BatchHeader *)base, (const BatchJob *)(base + sizeof(BatchHeader)), ctr + di,
                          (unsigned int *)(ctr + 2), sl.depth[di], nullptr, e->block, blocks[di],
                          di == 0 ? sl.stream : sl.side, ctr + 3, sl.scr[di]);
    }
    cudaEventRecord(sl.join, sl.side);
    cudaStreamWaitEvent(sl.stream, sl.join, 0);
    cudaMemcpyAsync(sl.steps_host, ctr + 3, 8, cudaMemcpyDeviceToHost, sl.stream);
    er = cudaStreamEndCapture(sl.stream, &sl.graph);
    if (er != cudaSuccess) return er;
    return cudaGraphInstantiate(&sl.exec, sl.graph, 0);
}

// Overload shedding: requests that waited too long for their first walks,
// admitted or still queued for memory, finish with BUDGET (checked on every
// pass of the scheduler, not only when a round slot is free).
void shed_late(wost_engine *e) {
    if (e->max_wait <= 0) return;
    std::vector<Request *> late;
    for (Request *r : e->active)
        if (!r->finished && !r->started && r->outstanding == 0 && since(r->t_submit) > e->max_wait)
            late.push_back(r);
    std::deque<Request *> keep;
    for (Request *r : e->pending) {
        if (!r->finished && since(r->t_submit) > e->max_wait) late.push_back(r);
        else keep.push_back(r);
    }
    e->pending.swap(keep);
    for (Request *r : late) {
        e->st.rejected++;
        finish(e, r, WOST_ERR_BUDGET);
    }
}

#ifndef WOST_ROUND_WALKS
#define WOST_ROUND_WALKS 4
#endif

// Resident lanes of the batched kernel for a dimension at a stack depth.
double lanes_at(wost_engine *e, int dim, int depth) {
    auto &m = e->lanes_at_depth[dim - 2];
    auto it = m.find(depth);
    if (it != m.end()) return it->second;
    int blocks = 0;
    double lanes = batch_grid(dim, e->block, std::max(depth, 2), &blocks) == cudaSuccess ? (double)blocks * e->block
                                                                                           : 0.0;
    m[depth] = lanes;
    return lanes;
}

// The round's walk-step floor: WOST_ROUND_WALKS walks of 64 steps for every
// resident lane (the deepest stack of each dimension sets that dimension's
// grid; 2D and 3D kernels share the SMs, so the larger grid counts).
double min_round_steps(wost_engine *e, const std::vector<Request *> &iss) {
    int depth[2] = {0, 0};
    for (const Request *r : iss) depth[r->h->dim - 2] = std::max(depth[r->h->dim - 2], r->scene->stack_depth);
    double lanes = 0;
    for (int di = 0; di < 2; ++di)
        if (depth[di]) lanes = std::max(lanes, lanes_at(e, di + 2, depth[di]));
    return (double)WOST_ROUND_WALKS * 64.0 * lanes;
}

bool launch_round(wost_engine *e) {
    int si = -1;
    for (int i = 0; i < kSlots; ++i)
        if (!e->slots[i].busy) {
            si = i;
            break;
        }
    if (si < 0) return false;
    // active requests with work left in their current stage, least
    // remaining stage work first (admission order among equals): under
    // overload the cheapest finish and the rest wait, instead of every
    // request advancing slowly and none finishing
    std::vector<Request *> iss;
    for (Request *r : e->active)
        if (!r->finished && r->cursor < r->h->n_points && !cancelled(r)) iss.push_back(r);
    if (iss.empty()) return false;
    auto left_work = [](const Request *r) {
        return (double)(r->h->n_points - r->cursor) * (double)(r->stage_end - r->stage_begin) * r->mean_steps;
    };
    std::stable_sort(iss.begin(), iss.end(),
                     [&](const Request *a, const Request *b) { return left_work(a) < left_work(b); });
    Round rd;
    rd.slot = si;
    // the round's budget goes down that order: each request takes as many
    // points of its current stage as the remaining budget pays for (at
    // least one point, so every round makes progress)
    double remaining = std::max(e->round_budget_steps, min_round_steps(e, iss));
    for (Request *r : iss) {
        if (remaining <= 0) break;
        int64_t left = r->h->n_points - r->cursor;
        double cost = (double)(r->stage_end - r->stage_begin) * r->mean_steps;
        int64_t np = std::max<int64_t>(1, std::min<int64_t>((int64_t)(remaining / cost), left));
        rd.pieces.push_back(Piece{r, r->cursor, np, r->stage_begin, r->stage_end - r->stage_begin});
        r->cursor += np;
        r->outstanding++;
        r->started = true;
        remaining -= (double)np * cost;
    }
    // job tables per dimension, written into the slot's pinned staging
    Slot &sl = e->slots[si];
    size_t cnt[2] = {0, 0};
    int depth[2] = {0, 0};
    bool scr[2] = {false, false};
    for (auto &p : rd.pieces) {
        int di = p.r->h->dim - 2;
        cnt[di]++;
        depth[di] = std::max(depth[di], p.r->scene->stack_depth);
        scr[di] = scr[di] || p.r->h->sp.sigma > 0.f;
    }
    cudaError_t err = ensure_graph(e, sl, cnt, depth, scr);
    if (err != cudaSuccess) {
        for (auto &p : rd.pieces) finish(e, p.r, WOST_ERR_CUDA);
        return false;
    }
    unsigned long long total[2] = {0, 0};
    size_t fill[2] = {0, 0};
    BatchJob *tab[2] = {(BatchJob *)(sl.host[0] + sizeof(BatchHeader)),
                        (BatchJob *)(sl.host[1] + sizeof(BatchHeader))};
    for (auto &p : rd.pieces) {
        int di = p.r->h->dim - 2;
        BatchJob j;
        j.scene = p.r->scene->view_dev;
        j.sp = p.r->h->sp;
        j.sp.point_begin = p.p0;
        j.sp.n_points = p.np;
        j.sp.walks_per_point = p.nw;
        j.sp.first_walk = p.r->h->sp.first_walk + (uint32_t)p.w0;
        j.sp.stack_depth = sl.depth[di];
        j.acc = p.r->h->acc;
        j.walk_begin = total[di];
        total[di] += (unsigned long long)p.np * (unsigned long long)p.nw;
        tab[di][fill[di]++] = j;
    }
    for (int di = 0; di < 2; ++di) {
        BatchHeader hd{(int)cnt[di], 0, total[di]};
        std::memcpy(sl.host[di], &hd, sizeof hd);
    }
    // the round runs after the admissions (uploads, zeroing) issued before it
    err = cudaEventRecord(e->ev_ready, e->stream);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(sl.stream, e->ev_ready, 0);
    if (err == cudaSuccess) err = cudaEventRecord(e->ev_ready, e->zero_stream);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(sl.stream, e->ev_ready, 0);
    if (err == cudaSuccess) err = cudaEventRecord(sl.ev0, sl.stream);
    if (err == cudaSuccess) err = cudaGraphLaunch(sl.exec, sl.stream);
    if (err == cudaSuccess) err = cudaEventRecord(sl.ev1, sl.stream);
    if (err != cudaSuccess) {
        for (auto &p : rd.pieces) finish(e, p.r, WOST_ERR_CUDA);
        cudaStreamSynchronize(sl.stream);
        return false;
    }
    e->st.graph_launches++;
    sl.busy = true;
    e->inflight.push_back(std::move(rd));
    return true;
}

void engine_loop(wost_engine *e) {
    cudaSetDevice(e->device);
    std::unique_lock<std::mutex> lk(e->mu);
    for (;;) {
        // rounds on different streams may finish in any order
        for (size_t i = 0; i < e->inflight.size();) {
            if (cudaEventQuery(e->slots[e->inflight[i].slot].ev1) != cudaErrorNotReady) retire(e, i);
            else ++i;
        }
        complete_checks(e, false);
        process_cancels(e);
        if (e->stop && e->inflight.empty() && e->check_order.empty()) break;
        if (!e->stop) {
            admit(e);
            shed_late(e);
        }
        if (!e->stop && (int)e->inflight.size() < kSlots && launch_round(e)) continue;
        // nothing to launch: wake on a submission or cancellation, or poll
        // the rounds in flight again after a short sleep
        e->cv.wait_for(lk, std::chrono::milliseconds(e->inflight.empty() ? 2 : 1));
    }
    // stopped: whatever is left is cancelled
    std::vector<Request *> left(e->active.begin(), e->active.end());
    for (Request *r : left) finish(e, r, WOST_ERR_CANCELLED);
    while (!e->pending.empty()) {
        Request *r = e->pending.front();
        e->pending.pop_front();
        finish(e, r, WOST_ERR_CANCELLED);
    }
}

}  // namespace

namespace wost {

void engine_detach(wost_engine *e, wost_solve_handle *h) {
    std::unique_lock<std::mutex> lk(e->mu);
    auto it = e->by_handle.find(h);
    if (it == e->by_handle.end()) return;
    Request *r = it->second;
    if (!r->finished) {
        *(volatile int *)h->cancel_host = 1;
        e->cv.notify_all();
    }
    e->done_cv.wait(lk, [&] { return r->finished && r->outstanding == 0; });
    // a request none of whose rounds ran may still have its set-up queued:
    // its buffers are freed on its poll stream after that work
    if (r->admitted && !h->engine_ready.load()) {
        for (cudaStream_t st : {e->stream, e->zero_stream})
            if (cudaEventRecord(e->ev_detach, st) == cudaSuccess) cudaStreamWaitEvent(h->poll_stream, e->ev_detach, 0);
    }
    if (r->admitted) e->used -= r->bytes;
    e->pending.erase(std::remove(e->pending.begin(), e->pending.end(), r), e->pending.end());
    e->by_handle.erase(it);
    delete r;
    e->cv.notify_all();
}

}  // namespace wost

extern "C" {

wost_status wost_engine_create(const wost_engine_desc *d, wost_engine **out) {
    try {
        if (!d || !out) return fail(WOST_ERR_INVALID_ARG, "null argument");
        *out = nullptr;
        if (d->memory_budget_bytes < 0 || d->round_seconds < 0 || d->min_walks < 0 || d->max_walks_per_point < 0)
            return fail(WOST_ERR_INVALID_ARG, "negative engine parameter");
        int block = d->block_size ? d->block_size : 128;
        if (block < 32 || block > 256 || block % 32) return fail(WOST_ERR_INVALID_ARG, "block_size must be 32..256, multiple of 32");
        int ndev = 0;
        CK(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
        if (d->device < 0 || d->device >= ndev) return fail(WOST_ERR_INVALID_ARG, "device ordinal out of range");
        CK(cudaSetDevice(d->device), "cudaSetDevice");
        std::unique_ptr<wost_engine> e(new wost_engine);
        e->device = d->device;
        e->round_seconds = d->round_seconds > 0 ? d->round_seconds : 0.02;
        if (!(d->max_wait_seconds >= 0)) return fail(WOST_ERR_INVALID_ARG, "max_wait_seconds must be >= 0");
        e->max_wait = d->max_wait_seconds;
        e->min_walks = d->min_walks ? d->min_walks : 16;
        e->cap = d->max_walks_per_point ? d->max_walks_per_point : 65536;
        e->block = block;
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
        e->budget = d->memory_budget_bytes ? d->memory_budget_bytes : (int64_t)(fr / 4);
        int prio_low = 0, prio_high = 0;
        CK(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high), "cudaDeviceGetStreamPriorityRange");
        CK(cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        CK(cudaStreamCreateWithPriority(&e->check_stream, cudaStreamNonBlocking, prio_high), "cudaStreamCreate");
        CK(cudaEventCreateWithFlags(&e->ev_ready, cudaEventDisableTiming), "cudaEventCreate");
        CK(cudaStreamCreateWithFlags(&e->copy_stream, cudaStreamNonBlocking), "cudaStreamCreate");
        for (auto &ps : e->poll) CK(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking), "cudaStreamCreate");
        {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = d->device;
            CK(cudaMemPoolCreate(&e->pool, &props), "cudaMemPoolCreate");
            uint64_t keep_all = ~0ull;
            CK(cudaMemPoolSetAttribute(e->pool, cudaMemPoolAttrReleaseThreshold, &keep_all), "cudaMemPoolSetAttribute");
        }
        CK(cudaMallocHost((void **)&e->stage, kStage * kStageBytes), "cudaMallocHost");
        for (auto &ev : e->stage_ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "cudaEventCreate");
        CK(cudaEventCreateWithFlags(&e->ev_alloc, cudaEventDisableTiming), "cudaEventCreate");
        CK(cudaEventCreateWithFlags(&e->ev_detach, cudaEventDisableTiming), "cudaEventCreate");
        CK(cudaStreamCreateWithPriority(&e->zero_stream, cudaStreamNonBlocking, prio_high), "cudaStreamCreate");
        for (auto &s : e->slots) {
            CK(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking), "cudaStreamCreate");
            CK(cudaStreamCreateWithFlags(&s.side, cudaStreamNonBlocking), "cudaStreamCreate");
            CK(cudaEventCreateWithFlags(&s.fork, cudaEventDisableTiming), "cudaEventCreate");
            CK(cudaEventCreateWithFlags(&s.join, cudaEventDisableTiming), "cudaEventCreate");
            CK(cudaEventCreate(&s.ev0), "cudaEventCreate");
            CK(cudaEventCreate(&s.ev1), "cudaEventCreate");
        }
        e->st.budget_bytes = e->budget;
        wost_engine *raw = e.release();
        raw->th = std::thread(engine_loop, raw);
        *out = raw;
        return WOST_OK;
    } catch (const std::exception &ex) {
        return fail(WOST_ERR_INTERNAL, ex.what());
    }
}

wost_status wost_engine_submit(wost_engine *e, wost_scene *scene, const wost_solve_desc *d, double target_se,
                               wost_solve_handle **out) {
    try {
        if (!e || !scene || !d || !out) return fail(WOST_ERR_INVALID_ARG, "null argument");
        *out = nullptr;
        if (scene->device != e->device) return fail(WOST_ERR_INVALID_ARG, "scene on another device");
        if (!(target_se >= 0) || !std::isfinite(target_se)) return fail(WOST_ERR_INVALID_ARG, "target_se must be >= 0");
        if (d->n_points < 1 || !d->points) return fail(WOST_ERR_INVALID_ARG, "points missing");
        if (d->n_points > 0xFFFFFFFFll) return fail(WOST_ERR_INVALID_ARG, "more than 2^32-1 points");
        if (d->walks_per_point < 0) return fail(WOST_ERR_INVALID_ARG, "walks_per_point must be >= 0");
        if (!(d->epsilon > 0)) return fail(WOST_ERR_INVALID_ARG, "epsilon must be > 0");
        float rmin = d->r_min == 0 ? d->epsilon : d->r_min;
        if (!(rmin > 0) || rmin > d->epsilon) return fail(WOST_ERR_INVALID_ARG, "need 0 < r_min <= epsilon");
        if (d->max_steps < 1) return fail(WOST_ERR_INVALID_ARG, "max_steps must be >= 1");
        if (d->memory != WOST_MEM_HOST && d->memory != WOST_MEM_DEVICE)
            return fail(WOST_ERR_INVALID_ARG, "memory must be HOST or DEVICE");
        const int dim = scene->view.dim;
        const size_t n = (size_t)d->n_points;
        std::unique_ptr<Request> r(new Request);
        r->scene = scene;
        r->target = target_se;
        r->cap = (d->walks_per_point > 0 && d->walks_per_point < e->cap) ? d->walks_per_point : e->cap;
        bool has_n = d->normals && d->on_neumann;
        r->bytes = (int64_t)(n * (dim * 4 + 32 + (has_n ? dim * 4 + 1 : 0)) + 64);
        if (r->bytes > e->budget) {
            std::lock_guard<std::mutex> lk(e->mu);
            e->st.rejected++;
            return fail(WOST_ERR_BUDGET, "request exceeds the engine's memory budget");
        }
        CK(cudaSetDevice(e->device), "cudaSetDevice");
        // the inputs are copied before return: host arrays with memcpy (a
        // CUDA host-to-host copy goes through the legacy stream and may wait
        // on the device), device arrays on the engine's copy stream
        auto copy_in = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
            if (d->memory == WOST_MEM_HOST) {
                std::memcpy(dst, src, bytes);
                return cudaSuccess;
            }
            std::lock_guard<std::mutex> ck(e->copy_mu);
            cudaError_t er = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, e->copy_stream);
            return er == cudaSuccess ? cudaStreamSynchronize(e->copy_stream) : er;
        };
        r->pts.resize(n * dim);
        CK(copy_in(r->pts.data(), d->points, n * dim * 4), "copy points");
        if (has_n) {
            r->nrm.resize(n * dim);
            r->onN.resize(n);
            CK(copy_in(r->nrm.data(), d->normals, n * dim * 4), "copy normals");
            CK(copy_in(r->onN.data(), d->on_neumann, n), "copy on_neumann");
        }
        r->desc = *d;
        r->desc.points = r->pts.data();
        r->desc.normals = has_n ? r->nrm.data() : nullptr;
        r->desc.on_neumann = has_n ? r->onN.data() : nullptr;
        r->desc.memory = WOST_MEM_HOST;
        r->desc.walks_per_point = r->cap;
        r->desc.kernel = WOST_KERNEL_PERSISTENT;
        r->desc.block_size = e->block;
        r->desc.stream = nullptr;
        std::unique_ptr<wost_solve_handle> h(new wost_solve_handle);
        h->engine = e;
        h->scene = scene;
        h->device = e->device;
        h->dim = dim;
        h->n_points = d->n_points;
        h->walks = r->cap;
        // the cancel flag exists before admission so that queued requests can
        // be cancelled; the engine reads it on the host (it stops issuing the
        // request's pieces), so it is plain host memory, and the request's
        // device buffers are stream-ordered (no device-wide wait on destroy)
        h->engine_buffers = true;
        h->pool = e->pool;
        h->cancel_host = new int(0);
        h->cancel_dev = nullptr;
        r->h = h.get();
        r->t_submit = Clock::now();
        {
            std::lock_guard<std::mutex> lk(e->mu);
            if (e->stop) return fail(WOST_ERR_CANCELLED, "engine is shutting down");
            e->pending.push_back(r.get());
            e->by_handle[h.get()] = r.get();
            e->st.submitted++;
        }
        r.release();
        e->cv.notify_all();
        *out = h.release();
        return WOST_OK;
    } catch (const std::bad_alloc &) {
        return fail(WOST_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (const std::exception &ex) {
        return fail(WOST_ERR_INTERNAL, ex.what());
    }
}

wost_status wost_engine_get_stats(wost_engine *e, wost_engine_stats *out) {
    if (!e || !out) return fail(WOST_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(e->mu);
    *out = e->st;
    out->queued = (int32_t)e->pending.size();
    out->active = (int32_t)e->active.size();
    out->budget_bytes = e->budget;
    out->used_bytes = e->used;
    out->round_budget_steps = e->round_budget_steps;
    return WOST_OK;
}

wost_status wost_engine_destroy(wost_engine *e) {
    if (!e) return fail(WOST_ERR_INVALID_ARG, "null engine");
    {
        std::lock_guard<std::mutex> lk(e->mu);
        e->stop = true;
        for (auto &kv : e->by_handle) *(volatile int *)kv.first->cancel_host = 1;
    }
    e->cv.notify_all();
    if (e->th.joinable()) e->th.join();
    cudaSetDevice(e->device);
    cudaStreamSynchronize(e->stream);
    for (auto &s : e->slots)
        if (s.stream) cudaStreamSynchronize(s.stream);
    for (auto &kv : e->by_handle) {
        kv.first->engine = nullptr;  // the handle outlives the engine
        if (!kv.first->own_poll_stream) {  // and needs a poll stream of its own
            std::lock_guard<std::mutex> hl(kv.first->mu);
            if (cudaStreamCreateWithFlags(&kv.first->poll_stream, cudaStreamNonBlocking) != cudaSuccess)
                kv.first->poll_stream = nullptr;
            kv.first->own_poll_stream = true;
        }
        delete kv.second;
    }
    e->by_handle.clear();
    cudaStreamSynchronize(e->check_stream);
    cudaStreamDestroy(e->check_stream);
    cudaEventDestroy(e->ev_ready);
    cudaStreamSynchronize(e->zero_stream);
    for (cudaEvent_t ev : e->stage_ev)
        if (ev) cudaEventDestroy(ev);
    cudaEventDestroy(e->ev_alloc);
    cudaEventDestroy(e->ev_detach);
    if (e->stage) cudaFreeHost(e->stage);
    cudaStreamDestroy(e->zero_stream);
    cudaStreamDestroy(e->copy_stream);
    for (cudaStream_t ps : e->poll) {
        cudaStreamSynchronize(ps);
        cudaStreamDestroy(ps);
    }
    cudaStreamDestroy(e->stream);
    cudaMemPool_t pool = e->pool;
    delete e;  // the slots release their graphs, streams and events
    // a pool with allocations outstanding (handles that outlive the engine)
    // is released once they are freed
    if (pool) cudaMemPoolDestroy(pool);
    return WOST_OK;
}

}  // extern "C"
