// C ABI of libwost (include/wost.h): scenes, solves, queries, errors.
//
// Nothing throws across the ABI: every entry point catches, records a
// thread-local message and returns a status.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "capi_internal.h"

using namespace wost;

namespace wost {

static thread_local std::string g_last_error;

wost_status fail(wost_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}
wost_status cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? WOST_ERR_OUT_OF_MEMORY : WOST_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace wost

extern "C" {

const char *wost_last_error(void) { return g_last_error.c_str(); }
int32_t wost_abi_version(void) { return WOST_ABI_VERSION; }

wost_status wost_scene_create(const wost_scene_desc *desc, wost_scene **out) {
    try {
        if (!desc || !out) return fail(WOST_ERR_INVALID_ARG, "null argument");
        *out = nullptr;
        if (desc->device < 0) return fail(WOST_ERR_INVALID_ARG, "device ordinal out of range");
        std::unique_ptr<wost_scene> s(new wost_scene);
        s->device = desc->device;
        // host-side validation and build first: bad input is rejected without
        // touching the device
        std::string err = build_scene(*desc, s->host);
        if (!err.empty()) return fail(WOST_ERR_INVALID_ARG, err);
        int ndev = 0;
        CK(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
        if (desc->device >= ndev) return fail(WOST_ERR_INVALID_ARG, "device ordinal out of range");
        CK(cudaSetDevice(s->device), "cudaSetDevice");
        HostScene &H = s->host;
        HostTree *trees[3] = {&H.D, &H.N, &H.S};
        TreeView *views[3] = {&s->view.D, &s->view.N, &s->view.S};
        int64_t bytes = 0;
        for (int t = 0; t < 3; ++t) {
            HostTree &T = *trees[t];
            DevBuf *b = &s->bufs[5 * t];
            CK(upload(b[0], T.nodes), "upload nodes");
            CK(upload(b[1], T.cones), "upload cones");
            CK(upload(b[2], T.prims), "upload prims");
            CK(upload(b[3], T.data), "upload data");
            CK(upload(b[4], T.ids), "upload ids");
            for (int k = 0; k < 5; ++k) bytes += (int64_t)b[k].bytes;
            TreeView &V = *views[t];
            V.nodes = (const float4 *)b[0].p;
            V.cones = (const float4 *)b[1].p;
            V.prims = (const float4 *)b[2].p;
            V.data = (const float4 *)b[3].p;
            V.ids = (const int32_t *)b[4].p;
            V.root = T.root;
            for (int a = 0; a < 3; ++a) {
                V.root_lo[a] = T.root_lo[a];
                V.root_hi[a] = T.root_hi[a];
            }
            V.root_cone = T.root_cone;
            V.n_prims = T.n_prims;
            V.n_nodes = T.n_nodes;
            V.depth = T.depth;
            DevBuf *w = &s->wbufs[2 * t];
            CK(upload(w[0], T.wnodes), "upload wide nodes");
            CK(upload(w[1], T.wcones), "upload wide cones");
            bytes += (int64_t)(w[0].bytes + w[1].bytes);
            V.wnodes = (const float4 *)w[0].p;
            V.wcones = (const float4 *)w[1].p;
            V.wroot = T.wroot;
            V.wn_nodes = T.wn_nodes;
            V.wdepth = T.wdepth;
        }
        for (int t = 0; t < 2; ++t) {  // double-sided records of D and N
            HostTree &T = *trees[t];
            CK(upload(s->sbufs[2 * t], T.data_minus), "upload data");
            CK(upload(s->sbufs[2 * t + 1], T.sided), "upload flags");
            bytes += (int64_t)(s->sbufs[2 * t].bytes + s->sbufs[2 * t + 1].bytes);
            views[t]->data_minus = (const float4 *)s->sbufs[2 * t].p;
            views[t]->sided = (const uint8_t *)s->sbufs[2 * t + 1].p;
        }
        CK(upload(s->bufs[15], H.grid), "upload grid");
        bytes += (int64_t)s->bufs[15].bytes;
        std::vector<int32_t> rec_of_id((size_t)desc->n_prims, -1);
        for (size_t k = 0; k < H.N.ids.size(); ++k) rec_of_id[H.N.ids[k]] = (int32_t)k;
        CK(upload(s->n_rec_of_id, rec_of_id), "upload map");
        CK(cudaMalloc(&s->guard, sizeof(unsigned int)), "cudaMalloc guard");
        CK(cudaMemset(s->guard, 0, sizeof(unsigned int)), "cudaMemset guard");
        s->view.dim = H.dim;
        s->view.g = H.g;
        s->view.h = H.h;
        s->view.f = H.f;
        s->view.f.grid = (const float *)s->bufs[15].p;
        {
            float m = 0.f;
            for (int a = 0; a < H.dim; ++a) m = std::max(m, H.hi[a] - H.lo[a]);
            float d2 = 0.f;
            for (int a = 0; a < 3; ++a) {
                s->view.out_lo[a] = H.lo[a] - m;
                s->view.out_hi[a] = H.hi[a] + m;
                if (a < H.dim) d2 += (H.hi[a] - H.lo[a]) * (H.hi[a] - H.lo[a]);
            }
            s->view.rmax = std::sqrt(d2);
        }
        // binary trees: one pending subtree per level
        s->stack_depth = std::max(H.D.depth, std::max(H.N.depth, H.S.depth)) + 2;
        // 8-wide trees: at most 7 pending subtrees per level; odd, so that
        // the teams of a warp start in different shared-memory banks
        s->stack_depth_team = ((WOST_WIDE - 1) * std::max(H.D.wdepth, std::max(H.N.wdepth, H.S.wdepth)) + 1) | 1;
        CK(cudaMalloc(&s->view_dev, sizeof(SceneView)), "cudaMalloc view");
        CK(cudaMemcpy(s->view_dev, &s->view, sizeof(SceneView), cudaMemcpyHostToDevice), "copy view");
        wost_scene_info &I = s->info;
        I.dim = H.dim;
        I.n_dirichlet = H.n_dirichlet;
        I.n_neumann = H.n_neumann;
        I.n_silhouette = H.n_silhouette;
        I.n_dropped = H.n_dropped;
        I.nodes_dirichlet = H.D.n_nodes;
        I.nodes_neumann = H.N.n_nodes;
        I.nodes_silhouette = H.S.n_nodes;
        I.depth_dirichlet = H.D.depth;
        I.depth_neumann = H.N.depth;
        I.depth_silhouette = H.S.depth;
        I.wide_nodes_dirichlet = H.D.wn_nodes;
        I.wide_nodes_neumann = H.N.wn_nodes;
        I.wide_nodes_silhouette = H.S.wn_nodes;
        I.wide_depth_dirichlet = H.D.wdepth;
        I.wide_depth_neumann = H.N.wdepth;
        I.wide_depth_silhouette = H.S.wdepth;
        I.device_bytes = bytes;
        I.build_seconds = H.build_seconds;
        I.device = s->device;
        set_layout_info(s.get(), 1);
        for (int a = 0; a < 3; ++a) {
            I.bbox_lo[a] = H.lo[a];
            I.bbox_hi[a] = H.hi[a];
        }
        *out = s.release();
        return WOST_OK;
    } catch (const std::bad_alloc &) {
        return fail(WOST_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(WOST_ERR_INTERNAL, e.what());
    }
}

wost_status wost_scene_validate(const wost_scene_desc *desc, wost_scene_info *out) {
    try {
        if (!desc || !out) return fail(WOST_ERR_INVALID_ARG, "null argument");
        HostScene H;
        std::string err = build_scene(*desc, H);
        if (!err.empty()) return fail(WOST_ERR_INVALID_ARG, err);
        err = check_scene(H);
        if (!err.empty()) return fail(WOST_ERR_INTERNAL, err);
        wost_scene_info I{};
        I.dim = H.dim;
        I.n_dirichlet = H.n_dirichlet;
        I.n_neumann = H.n_neumann;
        I.n_silhouette = H.n_silhouette;
        I.n_dropped = H.n_dropped;
        I.nodes_dirichlet = H.D.n_nodes;
        I.nodes_neumann = H.N.n_nodes;
        I.nodes_silhouette = H.S.n_nodes;
        I.depth_dirichlet = H.D.depth;
        I.depth_neumann = H.N.depth;
        I.depth_silhouette = H.S.depth;
        I.lanes_per_walk = 1;
        I.wide_nodes_dirichlet = H.D.wn_nodes;
        I.wide_nodes_neumann = H.N.wn_nodes;
        I.wide_nodes_silhouette = H.S.wn_nodes;
        I.wide_depth_dirichlet = H.D.wdepth;
        I.wide_depth_neumann = H.N.wdepth;
        I.wide_depth_silhouette = H.S.wdepth;
        I.build_seconds = H.build_seconds;
        I.device = desc->device;
        I.stack_depth = std::max(H.D.depth, std::max(H.N.depth, H.S.depth)) + 2;
        I.node_bytes = H.dim == 2 ? 48 : 64;
        I.cone_bytes = 32;
        for (int a = 0; a < 3; ++a) {
            I.bbox_lo[a] = H.lo[a];
            I.bbox_hi[a] = H.hi[a];
        }
        *out = I;
        return WOST_OK;
    } catch (const std::bad_alloc &) {
        return fail(WOST_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(WOST_ERR_INTERNAL, e.what());
    }
}

wost_status wost_scene_destroy(wost_scene *scene) {
    if (!scene) return fail(WOST_ERR_INVALID_ARG, "null scene");
    cudaSetDevice(scene->device);
    delete scene;
    return WOST_OK;
}

wost_status wost_scene_get_info(const wost_scene *scene, wost_scene_info *out) {
    if (!scene || !out) return fail(WOST_ERR_INVALID_ARG, "null argument");
    *out = scene->info;
    return WOST_OK;
}

}  // extern "C"

void wost::set_layout_info(wost_scene *s, int lanes) {
    wost_scene_info &I = s->info;
    I.lanes_per_walk = lanes;
    I.node_bytes = lanes == 1 ? (s->host.dim == 2 ? 48 : 64) : 2 * WOST_WIDE * 16;
    I.cone_bytes = lanes == 1 ? 32 : WOST_WIDE * 16;
    I.stack_depth = lanes == 1 ? s->stack_depth : s->stack_depth_team;
}

// Validates a solve description, allocates and fills the solve's device
// buffers on `stream`, and fills h->sp / h->acc.  Does not launch.
cudaError_t wost::clear_accumulators(wost_solve_handle *h, cudaStream_t stream) {
    const size_t n = (size_t)h->n_points;
    cudaError_t e = cudaSuccess;
    for (DevBuf *b : {&h->sum, &h->sumsq, &h->walks_done, &h->steps})
        if (e == cudaSuccess) e = cudaMemsetAsync(b->p, 0, n * 8, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->globals.p, 0, 4 * 8, stream);
    return e;
}

wost_status wost::prepare_solve(wost_scene *scene, const wost_solve_desc *d, cudaStream_t stream,
                                 wost_solve_handle *h, bool fill) {
    if (!scene || !d) return fail(WOST_ERR_INVALID_ARG, "null argument");
    if (d->n_points < 1 || !d->points) return fail(WOST_ERR_INVALID_ARG, "points missing");
    if (d->n_points > 0xFFFFFFFFll) return fail(WOST_ERR_INVALID_ARG, "more than 2^32-1 points");
    if (d->walks_per_point < 1) return fail(WOST_ERR_INVALID_ARG, "walks_per_point must be >= 1");
    if (!(d->epsilon > 0) || !std::isfinite(d->epsilon)) return fail(WOST_ERR_INVALID_ARG, "epsilon must be > 0");
    float rmin = d->r_min == 0 ? d->epsilon : d->r_min;
    if (!(rmin > 0) || rmin > d->epsilon) return fail(WOST_ERR_INVALID_ARG, "need 0 < r_min <= epsilon");
    if (d->max_steps < 1) return fail(WOST_ERR_INVALID_ARG, "max_steps must be >= 1");
    if (!(d->sigma >= 0) || !std::isfinite(d->sigma)) return fail(WOST_ERR_INVALID_ARG, "sigma must be >= 0");
    if (d->screen_after < 0) return fail(WOST_ERR_INVALID_ARG, "screen_after must be >= 0");
    if (d->stack_depth < 0 || d->stack_depth > 4096)
        return fail(WOST_ERR_INVALID_ARG, "stack_depth must be 0 (the scene's) or 1..4096");
    if (d->visit_limit < 0) return fail(WOST_ERR_INVALID_ARG, "visit_limit must be >= 0");
    if (scene->host.n_dirichlet == 0 && !(d->sigma > 0))
        return fail(WOST_ERR_INVALID_ARG, "a scene without Dirichlet primitives needs sigma > 0 (Tikhonov "
                                          "regularisation of the pure Neumann problem)");
    if (d->memory != WOST_MEM_HOST && d->memory != WOST_MEM_DEVICE)
        return fail(WOST_ERR_INVALID_ARG, "memory must be HOST or DEVICE");
    if (d->kernel != WOST_KERNEL_PLAIN && d->kernel != WOST_KERNEL_PERSISTENT && d->kernel != WOST_KERNEL_COUNTING &&
        d->kernel != WOST_KERNEL_RESUMABLE)
        return fail(WOST_ERR_INVALID_ARG, "unknown kernel");
    int block = d->block_size ? d->block_size : (scene->tuned_block ? scene->tuned_block : 128);
    if (block < 32 || block > 256 || block % 32)
        return fail(WOST_ERR_INVALID_ARG, "block_size must be 32..256, multiple of 32");
    if (d->lanes_per_walk != 0 && d->lanes_per_walk != 1 && d->lanes_per_walk != WOST_WIDE)
        return fail(WOST_ERR_INVALID_ARG, "lanes_per_walk must be 0, 1 or 8");
    // 8-lane teams: persistent and resumable Poisson solves only; the tuned
    // choice applies where it can, an explicit request elsewhere is an error
    const bool team_ok = (d->kernel == WOST_KERNEL_PERSISTENT || d->kernel == WOST_KERNEL_RESUMABLE) && !(d->sigma > 0);
    if (d->lanes_per_walk == WOST_WIDE && !team_ok)
        return fail(WOST_ERR_INVALID_ARG, "8 lanes per walk: persistent or resumable Poisson solves only");
    const int lanes = d->lanes_per_walk ? d->lanes_per_walk : (team_ok ? scene->tuned_lanes : 1);
    CK(cudaSetDevice(scene->device), "cudaSetDevice");
    h->scene = scene;
    h->device = scene->device;
    h->dim = scene->view.dim;
    h->n_points = d->n_points;
    h->walks = d->walks_per_point;
    h->kernel = d->kernel;
    h->block = block;
    h->lanes = lanes;
    h->stream = stream;
    const int dim = h->dim;
    if (!h->poll_stream) {  // (the serving engine assigns one of its own)
        CK(cudaStreamCreateWithFlags(&h->poll_stream, cudaStreamNonBlocking), "cudaStreamCreate");
        h->own_poll_stream = true;
    }
    const size_t n = (size_t)d->n_points;
    // engine requests allocate on the engine's stream without waiting for it
    auto alloc = [&](DevBuf &b, size_t bytes) {
        return h->engine_buffers ? b.alloc_async(bytes, stream, h->pool) : b.alloc(bytes);
    };
    CK(alloc(h->points, n * dim * sizeof(float)), "cudaMalloc points");
    cudaMemcpyKind kind = d->memory == WOST_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (fill) CK(cudaMemcpyAsync(h->points.p, d->points, n * dim * sizeof(float), kind, stream), "copy points");
    if (d->normals && d->on_neumann) {
        CK(alloc(h->normals, n * dim * sizeof(float)), "cudaMalloc normals");
        CK(alloc(h->onN, n), "cudaMalloc on_neumann");
        if (fill) {
            CK(cudaMemcpyAsync(h->normals.p, d->normals, n * dim * sizeof(float), kind, stream), "copy normals");
            CK(cudaMemcpyAsync(h->onN.p, d->on_neumann, n, kind, stream), "copy on_neumann");
        }
    }
    CK(alloc(h->sum, n * 8), "cudaMalloc accumulators");
    CK(alloc(h->sumsq, n * 8), "cudaMalloc accumulators");
    CK(alloc(h->walks_done, n * 8), "cudaMalloc accumulators");
    CK(alloc(h->steps, n * 8), "cudaMalloc accumulators");
    CK(alloc(h->globals, 4 * 8), "cudaMalloc accumulators");
    if (fill) CK(clear_accumulators(h, stream), "memset");
    if (!h->cancel_host) {
        CK(cudaHostAlloc((void **)&h->cancel_host, sizeof(int), cudaHostAllocMapped), "cudaHostAlloc");
        *h->cancel_host = 0;
        CK(cudaHostGetDevicePointer((void **)&h->cancel_dev, h->cancel_host, 0), "cudaHostGetDevicePointer");
    }
    SolveParams &sp = h->sp;
    sp = SolveParams{};
    sp.points = (const float *)h->points.p;
    sp.normals = (const float *)h->normals.p;
    sp.on_neumann = (const uint8_t *)h->onN.p;
    sp.n_points = d->n_points;
    sp.walks_per_point = d->walks_per_point;
    sp.first_walk = d->first_walk;
    sp.epsilon = d->epsilon;
    sp.r_min = rmin;
    sp.max_steps = d->max_steps;
    sp.key0 = (uint32_t)d->seed;
    sp.key1 = (uint32_t)(d->seed >> 32);
    sp.offset = 1e-6f;
    sp.vis_tmax = 1.f - 1e-4f;
    sp.stack_depth = d->stack_depth ? d->stack_depth : (lanes == 1 ? scene->stack_depth : scene->stack_depth_team);
    sp.visit_limit = (uint32_t)d->visit_limit;
    sp.sigma = d->sigma;
    sp.sqrt_sigma = std::sqrt(d->sigma);
    sp.screen_after = d->screen_after;
    Accumulators &acc = h->acc;
    acc = Accumulators{};
    acc.sum = (double *)h->sum.p;
    acc.sumsq = (double *)h->sumsq.p;
    acc.walks = (unsigned long long *)h->walks_done.p;
    acc.steps = (unsigned long long *)h->steps.p;
    unsigned long long *g = (unsigned long long *)h->globals.p;
    acc.capped = g;
    acc.next_walk = g + 1;
    acc.guard = (unsigned int *)(g + 2);
    acc.cancel = h->cancel_dev;
    return WOST_OK;
}

// The caller's arrays may be released once a solve call returns.
wost_status wost::wait_for_copies(cudaStream_t stream) {
    cudaEvent_t copied;
    CK(cudaEventCreateWithFlags(&copied, cudaEventDisableTiming), "cudaEventCreate");
    cudaEventRecord(copied, stream);
    cudaError_t ce = cudaEventSynchronize(copied);
    cudaEventDestroy(copied);
    if (ce != cudaSuccess) return cuda_fail(ce, "input copy");
    return WOST_OK;
}

extern "C" {

wost_status wost_solve(wost_scene *scene, const wost_solve_desc *d, wost_solve_handle **out) {
    try {
        if (!scene || !d || !out) return fail(WOST_ERR_INVALID_ARG, "null argument");
        *out = nullptr;
        CK(cudaSetDevice(scene->device), "cudaSetDevice");
        std::unique_ptr<wost_solve_handle> h(new wost_solve_handle);
        cudaStream_t stream = (cudaStream_t)d->stream;
        if (!stream) {
            CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking), "cudaStreamCreate");
            h->own_stream = true;
            h->stream = stream;
        }
        wost_status st = prepare_solve(scene, d, stream, h.get());
        if (st != WOST_OK) return st;
        CK(cudaEventCreate(&h->ev_start), "cudaEventCreate");
        CK(cudaEventCreate(&h->ev_done), "cudaEventCreate");
        h->own_events = true;
        if (d->kernel == WOST_KERNEL_RESUMABLE) {
            // state only; the launches come from wost_solve_advance
            CK(resume_grid(h->dim, h->block, h->sp.stack_depth, &h->resume_blocks, h->lanes), "occupancy");
            CK(h->slots.alloc((size_t)resume_slots(h->block, h->resume_blocks, h->lanes) * 3 * sizeof(float4)),
               "cudaMalloc slots");
            CK(h->rstate.alloc(16), "cudaMalloc counters");
            CK(cudaMemsetAsync(h->slots.p, 0, h->slots.bytes, stream), "memset");
            CK(cudaMemsetAsync(h->rstate.p, 0, 16, stream), "memset");
            if ((st = wait_for_copies(stream)) != WOST_OK) return st;
            *out = h.release();
            return WOST_OK;
        }
        if ((st = wait_for_copies(stream)) != WOST_OK) return st;
        const SolveParams &sp = h->sp;
        const Accumulators &acc = h->acc;
        h->t_launch = std::chrono::steady_clock::now();
        CK(cudaEventRecord(h->ev_start, stream), "cudaEventRecord");
        cudaError_t le;
        if (d->kernel == WOST_KERNEL_PLAIN) {
            le = launch_walk_plain(scene->view, sp, acc, h->block, stream);
        } else if (d->kernel == WOST_KERNEL_COUNTING) {
            le = h->counts.alloc(10 * 8);
            if (le == cudaSuccess) le = cudaMemsetAsync(h->counts.p, 0, 10 * 8, stream);
            if (le == cudaSuccess)
                le = launch_walk_count(scene->view, sp, acc, (unsigned long long *)h->counts.p, h->block, stream);
        } else {
            int blocks = 0;
            le = persistent_grid(h->dim, h->block, sp.stack_depth, &blocks, h->lanes);
            if (le == cudaSuccess) le = launch_walk_persistent(scene->view, sp, acc, h->block, blocks, stream, h->lanes);
        }
        if (le != cudaSuccess) return cuda_fail(le, "kernel launch");
        CK(cudaEventRecord(h->ev_done, stream), "cudaEventRecord");
        h->launches = 1;
        *out = h.release();
        return WOST_OK;
    } catch (const std::bad_alloc &) {
        return fail(WOST_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(WOST_ERR_INTERNAL, e.what());
    }
}

wost_status wost_solve_batch(int32_t n, wost_scene *const *scenes, const wost_solve_desc *descs, void *stream_arg,
                             wost_solve_handle **out) {
    try {
        if (n < 1 || !scenes || !descs || !out) return fail(WOST_ERR_INVALID_ARG, "null argument or n < 1");
        for (int32_t i = 0; i < n; ++i) {
            out[i] = nullptr;
            if (!scenes[i]) return fail(WOST_ERR_INVALID_ARG, "null scene");
            if (scenes[i]->device != scenes[0]->device) return fail(WOST_ERR_INVALID_ARG, "scenes on different devices");
        }
        CK(cudaSetDevice(scenes[0]->device), "cudaSetDevice");
        auto shared = std::make_shared<BatchShared>();
        cudaStream_t stream = (cudaStream_t)stream_arg;
        if (!stream) {
            CK(cudaStreamCreateWithFlags(&shared->own_stream, cudaStreamNonBlocking), "cudaStreamCreate");
            stream = shared->own_stream;
        }
        std::vector<std::unique_ptr<wost_solve_handle>> hs(n);
        int block = descs[0].block_size ? descs[0].block_size
                                        : (scenes[0]->tuned_block ? scenes[0]->tuned_block : 128);
        for (int32_t i = 0; i < n; ++i) {
            hs[i].reset(new wost_solve_handle);
            wost_solve_desc d = descs[i];
            if (d.kernel == WOST_KERNEL_COUNTING) return fail(WOST_ERR_INVALID_ARG, "counting kernel in a batch");
            d.block_size = block;
            wost_status st = prepare_solve(scenes[i], &d, stream, hs[i].get());
            if (st != WOST_OK) return st;
            hs[i]->kernel = WOST_KERNEL_PERSISTENT;
            hs[i]->launches = 1;
        }
        // jobs per dimension, in the caller's order
        std::vector<BatchJob> jobs[2];
        int depth[2] = {0, 0};
        for (int32_t i = 0; i < n; ++i) {
            wost_solve_handle *h = hs[i].get();
            int di = h->dim - 2;
            BatchJob j;
            j.scene = scenes[i]->view_dev;
            j.sp = h->sp;
            j.acc = h->acc;
            j.walk_begin = shared->total[di];
            shared->total[di] += (unsigned long long)h->n_points * (unsigned long long)h->walks;
            depth[di] = std::max(depth[di], scenes[i]->stack_depth);
            jobs[di].push_back(j);
        }
        // device layout per dimension: BatchHeader, then the jobs
        std::vector<unsigned char> staging[2];
        for (int di = 0; di < 2; ++di) {
            for (auto &j : jobs[di]) j.sp.stack_depth = depth[di];
            BatchHeader hd{(int)jobs[di].size(), 0, shared->total[di]};
            staging[di].resize(sizeof(BatchHeader) + jobs[di].size() * sizeof(BatchJob));
            std::memcpy(staging[di].data(), &hd, sizeof hd);
            if (!jobs[di].empty())
                std::memcpy(staging[di].data() + sizeof hd, jobs[di].data(), jobs[di].size() * sizeof(BatchJob));
            CK(shared->jobs[di].alloc(staging[di].size()), "cudaMalloc jobs");
            CK(cudaMemcpyAsync(shared->jobs[di].p, staging[di].data(), staging[di].size(), cudaMemcpyHostToDevice,
                               stream), "copy jobs");
        }
        CK(shared->counters.alloc(4 * 8), "cudaMalloc counters");
        CK(cudaMemsetAsync(shared->counters.p, 0, 4 * 8, stream), "memset");
        CK(cudaEventCreate(&shared->ev_start), "cudaEventCreate");
        CK(cudaEventCreate(&shared->ev_done), "cudaEventCreate");
        wost_status st = wait_for_copies(stream);
        if (st != WOST_OK) return st;
        auto t0 = std::chrono::steady_clock::now();
        CK(cudaEventRecord(shared->ev_start, stream), "cudaEventRecord");
        unsigned long long *ctr = (unsigned long long *)shared->counters.p;
        // 2D and 3D jobs run in two kernels (each dimension its own register
        // budget, no warp mixing both), launched CONCURRENTLY: the 3D one on a
        // side stream forked from and joined back into the caller's, so each
        // fills the SMs the other's tail leaves idle
        const bool both = !jobs[0].empty() && !jobs[1].empty();
        if (both) {
            CK(cudaStreamCreateWithFlags(&shared->side, cudaStreamNonBlocking), "cudaStreamCreate");
            CK(cudaEventCreateWithFlags(&shared->ev_fork, cudaEventDisableTiming), "cudaEventCreate");
            CK(cudaEventCreateWithFlags(&shared->ev_join, cudaEventDisableTiming), "cudaEventCreate");
            CK(cudaEventRecord(shared->ev_fork, stream), "cudaEventRecord");
            CK(cudaStreamWaitEvent(shared->side, shared->ev_fork, 0), "cudaStreamWaitEvent");
        }
        for (int di = 0; di < 2; ++di) {
            if (jobs[di].empty()) continue;
            int blocks = 0;
            CK(batch_grid(di + 2, block, depth[di], &blocks), "occupancy");
            const unsigned char *base = (const unsigned char *)shared->jobs[di].p;
            cudaStream_t ls = (both && di == 1) ? shared->side : stream;
            const bool scr = std::any_of(jobs[di].begin(), jobs[di].end(),
                                         [](const BatchJob &j) { return j.sp.sigma > 0.f; });
            CK(launch_walk_batch(di + 2, (const BatchHeader *)base, (const BatchJob *)(base + sizeof(BatchHeader)),
                                 ctr + di, (unsigned int *)(ctr + 2), depth[di], nullptr, block, blocks, ls, nullptr,
                                 scr),
               "kernel launch");
        }
        if (both) {
            CK(cudaEventRecord(shared->ev_join, shared->side), "cudaEventRecord");
            CK(cudaStreamWaitEvent(stream, shared->ev_join, 0), "cudaStreamWaitEvent");
        }
        CK(cudaEventRecord(shared->ev_done, stream), "cudaEventRecord");
        for (int32_t i = 0; i < n; ++i) {
            hs[i]->batch = shared;
            hs[i]->ev_start = shared->ev_start;
            hs[i]->ev_done = shared->ev_done;
            hs[i]->t_launch = t0;
            hs[i]->batch_guard = (unsigned int *)(ctr + 2);
        }
        for (int32_t i = 0; i < n; ++i) out[i] = hs[i].release();
        return WOST_OK;
    } catch (const std::bad_alloc &) {
        return fail(WOST_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(WOST_ERR_INTERNAL, e.what());
    }
}

// Resumable solve whose latest launch has completed: finished when that
// launch saved no walk and no walk is left to draw (or the solve was
// cancelled, which stops the drawing).
static wost_status resumable_finished(wost_solve_handle *h, bool *finished) {
    unsigned long long g[4] = {0, 0, 0, 0};
    unsigned int st[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(g, h->globals.p, sizeof g, cudaMemcpyDeviceToHost, h->poll_stream), "poll copy");
    CK(cudaMemcpyAsync(st, h->rstate.p, sizeof st, cudaMemcpyDeviceToHost, h->poll_stream), "poll copy");
    CK(cudaStreamSynchronize(h->poll_stream), "poll sync");
    const uint64_t total = (uint64_t)h->n_points * (uint64_t)h->walks;
    *finished = st[2] == 0 && (g[1] >= total || *(volatile int *)h->cancel_host != 0);
    return WOST_OK;
}

static wost_status check_done(wost_solve_handle *h) {
    if (h->done || !h->ev_done) return WOST_OK;  // engine requests are marked done by the engine
    if (h->resumable() && h->launches == 0) return WOST_OK;  // nothing launched yet
    cudaError_t q = cudaEventQuery(h->ev_done);
    if (q == cudaSuccess && h->resumable()) {
        bool fin = false;
        wost_status st = resumable_finished(h, &fin);
        if (st != WOST_OK) return st;
        if (!fin) return WOST_OK;
    }
    if (q == cudaSuccess) {
        h->done = true;
        float ms = 0;
        cudaEventElapsedTime(&ms, h->ev_start, h->ev_done);
        h->elapsed_done = ms * 1e-3;
        return WOST_OK;
    }
    if (q != cudaErrorNotReady) return cuda_fail(q, "solve");
    return WOST_OK;
}

wost_status wost_poll(wost_solve_handle *h, double *mean, double *se, uint64_t *walks_done, wost_progress *pr) {
    try {
        if (!h) return fail(WOST_ERR_INVALID_ARG, "null solve");
        std::lock_guard<std::mutex> lk(h->mu);
        CK(cudaSetDevice(h->device), "cudaSetDevice");
        wost_status st = check_done(h);
        if (st != WOST_OK) return st;
        bool was_done = h->done;
        const size_t n = (size_t)h->n_points;
        // an engine request not admitted yet, or none of whose rounds has
        // completed: nothing accumulated
        if (!h->sum.p || (h->engine_buffers && !h->engine_ready.load())) {
            for (size_t i = 0; i < n; ++i) {
                if (mean) mean[i] = 0;
                if (se) se[i] = 0;
                if (walks_done) walks_done[i] = 0;
            }
            if (pr) {
                std::memset(pr, 0, sizeof *pr);
                pr->done = was_done ? 1 : 0;
                pr->elapsed_seconds = h->elapsed_done > 0 ? h->elapsed_done : 0.0;
            }
            return WOST_OK;
        }
        std::vector<double> s(n), q(n);
        std::vector<unsigned long long> w(n), stp(n), glob(4);
        CK(cudaMemcpyAsync(s.data(), h->sum.p, n * 8, cudaMemcpyDeviceToHost, h->poll_stream), "poll copy");
        CK(cudaMemcpyAsync(q.data(), h->sumsq.p, n * 8, cudaMemcpyDeviceToHost, h->poll_stream), "poll copy");
        CK(cudaMemcpyAsync(w.data(), h->walks_done.p, n * 8, cudaMemcpyDeviceToHost, h->poll_stream), "poll copy");
        if (pr) CK(cudaMemcpyAsync(stp.data(), h->steps.p, n * 8, cudaMemcpyDeviceToHost, h->poll_stream), "poll copy");
        CK(cudaMemcpyAsync(glob.data(), h->globals.p, 4 * 8, cudaMemcpyDeviceToHost, h->poll_stream), "poll copy");
        unsigned int bg = 0;
        if (h->batch_guard)
            CK(cudaMemcpyAsync(&bg, h->batch_guard, sizeof bg, cudaMemcpyDeviceToHost, h->poll_stream), "poll copy");
        unsigned long long rs[2] = {0, 0};
        if (h->resumable())
            CK(cudaMemcpyAsync(rs, h->rstate.p, sizeof rs, cudaMemcpyDeviceToHost, h->poll_stream), "poll copy");
        CK(cudaStreamSynchronize(h->poll_stream), "poll sync");
        uint64_t tw = 0, ts = 0;
        for (size_t i = 0; i < n; ++i) {
            double c = (double)w[i];
            double m = c > 0 ? s[i] / c : 0.0;
            if (mean) mean[i] = m;
            if (se) {
                double var = c > 1 ? std::max(0.0, (q[i] - c * m * m) / (c - 1.0)) : 0.0;
                se[i] = c > 0 ? std::sqrt(var / c) : 0.0;
            }
            if (walks_done) walks_done[i] = w[i];
            tw += w[i];
            if (pr) ts += stp[i];
        }
        if (pr) {
            pr->done = was_done ? 1 : 0;
            pr->walks_done = tw;
            pr->total_steps = ts;
            pr->capped_walks = glob[0];
            pr->guard_flags = (uint32_t)glob[2] | bg;
            pr->elapsed_seconds = was_done ? h->elapsed_done
                                           : std::chrono::duration<double>(std::chrono::steady_clock::now() - h->t_launch).count();
            if (h->resumable() && h->launches == 0) pr->elapsed_seconds = 0;
            pr->steps_run = h->resumable() ? rs[0] : ts;
            pr->launches = h->launches;
        }
        if ((uint32_t)glob[2] | bg) return fail(WOST_ERR_INTERNAL, "device guard fired (traversal stack overflow or visit limit)");
        return WOST_OK;
    } catch (const std::exception &e) {
        return fail(WOST_ERR_INTERNAL, e.what());
    }
}

// One launch of a resumable solve (caller holds h->mu).
static wost_status advance_locked(wost_solve_handle *h, int iters, cudaStream_t s) {
    if (h->launches == 0) {
        h->t_launch = std::chrono::steady_clock::now();
        CK(cudaEventRecord(h->ev_start, s), "cudaEventRecord");
    }
    unsigned int *live = (unsigned int *)((char *)h->rstate.p + 8);
    CK(cudaMemsetAsync(live, 0, sizeof(unsigned int), s), "memset");
    ResumeState rs{(float4 *)h->slots.p, (unsigned long long *)h->rstate.p, live};
    CK(launch_walk_resume(h->scene->view, h->sp, h->acc, rs, iters, h->block, h->resume_blocks, s, h->lanes),
       "kernel launch");
    CK(cudaEventRecord(h->ev_done, s), "cudaEventRecord");
    h->launches++;
    return WOST_OK;
}

wost_status wost_solve_advance(wost_solve_handle *h, int32_t iterations, void *stream) {
    try {
        if (!h) return fail(WOST_ERR_INVALID_ARG, "null solve");
        if (!h->resumable()) return fail(WOST_ERR_INVALID_ARG, "solve was not started with the resumable kernel");
        if (iterations < 1) return fail(WOST_ERR_INVALID_ARG, "iterations must be >= 1");
        std::lock_guard<std::mutex> lk(h->mu);
        CK(cudaSetDevice(h->device), "cudaSetDevice");
        if (h->done) return WOST_OK;
        return advance_locked(h, iterations, stream ? (cudaStream_t)stream : h->stream);
    } catch (const std::exception &e) {
        return fail(WOST_ERR_INTERNAL, e.what());
    }
}

wost_status wost_wait(wost_solve_handle *h, double timeout_s) {
    if (!h) return fail(WOST_ERR_INVALID_ARG, "null solve");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(h->mu);
            wost_status st = check_done(h);
            if (st != WOST_OK) return st;
            if (h->done) break;
            // a resumable solve advances while its caller waits: the next
            // launch as soon as the previous one has completed
            if (h->resumable() && (h->launches == 0 || cudaEventQuery(h->ev_done) == cudaSuccess))
                if ((st = advance_locked(h, 2048, h->stream)) != WOST_OK) return st;
        }
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (timeout_s >= 0 && el >= timeout_s) return fail(WOST_ERR_TIMEOUT, "solve not finished");
        std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 20 : 500));
    }
    if (h->engine || !h->ev_done) {  // engine request: its outcome was recorded by the engine
        if (h->final_status == WOST_ERR_CANCELLED) return fail(WOST_ERR_CANCELLED, "solve was cancelled");
        if (h->final_status != WOST_OK) return fail(h->final_status, "engine request failed");
        return WOST_OK;
    }
    unsigned long long glob[4];
    CK(cudaMemcpy(glob, h->globals.p, sizeof glob, cudaMemcpyDeviceToHost), "copy guard");
    unsigned int bg = 0;
    if (h->batch_guard) CK(cudaMemcpy(&bg, h->batch_guard, sizeof bg, cudaMemcpyDeviceToHost), "copy guard");
    if ((uint32_t)glob[2] | bg) return fail(WOST_ERR_INTERNAL, "device guard fired (traversal stack overflow or visit limit)");
    if (*(volatile int *)h->cancel_host) return fail(WOST_ERR_CANCELLED, "solve was cancelled");
    return WOST_OK;
}

wost_status wost_cancel(wost_solve_handle *h) {
    if (!h) return fail(WOST_ERR_INVALID_ARG, "null solve");
    *(volatile int *)h->cancel_host = 1;
    return WOST_OK;
}

wost_status wost_solve_destroy(wost_solve_handle *h) {
    if (!h) return fail(WOST_ERR_INVALID_ARG, "null solve");
    cudaSetDevice(h->device);
    if (h->engine) engine_detach(h->engine, h);  // waits until no round uses it
    delete h;
    return WOST_OK;
}

wost_status wost_solve_device_accumulators(wost_solve_handle *h, const double **sum, const double **sumsq,
                                           const uint64_t **walks, const uint64_t **steps) {
    if (!h) return fail(WOST_ERR_INVALID_ARG, "null solve");
    if (sum) *sum = (const double *)h->sum.p;
    if (sumsq) *sumsq = (const double *)h->sumsq.p;
    if (walks) *walks = (const uint64_t *)h->walks_done.p;
    if (steps) *steps = (const uint64_t *)h->steps.p;
    return WOST_OK;
}

wost_status wost_solve_work_counts(wost_solve_handle *h, uint64_t counts[10]) {
    if (!h || !counts) return fail(WOST_ERR_INVALID_ARG, "null argument");
    if (h->kernel != WOST_KERNEL_COUNTING) return fail(WOST_ERR_INVALID_ARG, "solve was not started with the counting kernel");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    CK(cudaEventSynchronize(h->ev_done), "solve");
    CK(cudaMemcpy(counts, h->counts.p, 10 * 8, cudaMemcpyDeviceToHost), "copy counts");
    return WOST_OK;
}

extern "C" wost_status wost_screened_kernels(int32_t dim, int64_t n, const float *rho, const float *R, float sigma,
                                             float *G, float *Q, void *stream) {
    if (dim != 2 && dim != 3) return fail(WOST_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (n < 0 || (n > 0 && (!rho || !R))) return fail(WOST_ERR_INVALID_ARG, "null argument or negative count");
    if (!(sigma > 0) || !std::isfinite(sigma)) return fail(WOST_ERR_INVALID_ARG, "sigma must be > 0");
    CK(launch_screened_kernels(dim, n, rho, R, sigma, G, Q, (cudaStream_t)stream), "kernel launch");
    return WOST_OK;
}

// ------------------------------- queries ---------------------------------
static wost_status query_prologue(wost_scene *s, int64_t n) {
    if (!s) return fail(WOST_ERR_INVALID_ARG, "null scene");
    if (n < 0) return fail(WOST_ERR_INVALID_ARG, "negative count");
    CK(cudaSetDevice(s->device), "cudaSetDevice");
    return WOST_OK;
}
static wost_status query_epilogue(wost_scene *s, cudaError_t e, cudaStream_t st) {
    if (e != cudaSuccess) return cuda_fail(e, "query launch");
    unsigned int g = 0;
    CK(cudaMemcpyAsync(&g, s->guard, sizeof g, cudaMemcpyDeviceToHost, st), "copy guard");
    CK(cudaStreamSynchronize(st), "query sync");
    if (g) return fail(WOST_ERR_INTERNAL, "device guard fired (traversal stack overflow or visit limit)");
    return WOST_OK;
}

wost_status wost_query_closest_dirichlet(wost_scene *s, int64_t n, const float *pts, float *dist, float *closest,
                                         int32_t *prim, void *stream) {
    wost_status st = query_prologue(s, n);
    if (st != WOST_OK) return st;
    if (!n) return WOST_OK;
    if (!pts || !dist || !closest || !prim) return fail(WOST_ERR_INVALID_ARG, "null array");
    std::lock_guard<std::mutex> lk(s->mu);
    cudaError_t e = launch_query_closest(s->view, n, pts, dist, closest, prim, s->stack_depth, s->guard,
                                         (cudaStream_t)stream);
    return query_epilogue(s, e, (cudaStream_t)stream);
}

wost_status wost_query_silhouette(wost_scene *s, int64_t n, const float *pts, const float *rmax, float *dist,
                                  void *stream) {
    wost_status st = query_prologue(s, n);
    if (st != WOST_OK) return st;
    if (!n) return WOST_OK;
    if (!pts || !rmax || !dist) return fail(WOST_ERR_INVALID_ARG, "null array");
    std::lock_guard<std::mutex> lk(s->mu);
    cudaError_t e = launch_query_silhouette(s->view, n, pts, rmax, dist, s->stack_depth, s->guard, (cudaStream_t)stream);
    return query_epilogue(s, e, (cudaStream_t)stream);
}

wost_status wost_query_intersect_neumann(wost_scene *s, int64_t n, const float *o, const float *v, const float *tmax,
                                         const int32_t *skip, int32_t *hit, float *t, int32_t *prim, void *stream) {
    wost_status st = query_prologue(s, n);
    if (st != WOST_OK) return st;
    if (!n) return WOST_OK;
    if (!o || !v || !tmax || !hit || !t || !prim) return fail(WOST_ERR_INVALID_ARG, "null array");
    std::lock_guard<std::mutex> lk(s->mu);
    cudaError_t e = launch_query_ray(s->view, n, o, v, tmax, skip, (const int32_t *)s->n_rec_of_id.p,
                                     (int64_t)(s->n_rec_of_id.bytes / sizeof(int32_t)), hit, t, prim, s->stack_depth,
                                     s->guard, (cudaStream_t)stream);
    return query_epilogue(s, e, (cudaStream_t)stream);
}

wost_status wost_query_neumann_sample(wost_scene *s, int64_t n, const float *pts, const float *r, uint64_t seed,
                                      uint32_t ctr1, uint32_t ctr2, float *z, float *pdf, int32_t *prim,
                                      void *stream) {
    wost_status st = query_prologue(s, n);
    if (st != WOST_OK) return st;
    if (!n) return WOST_OK;
    if (!pts || !r || !z || !pdf || !prim) return fail(WOST_ERR_INVALID_ARG, "null array");
    if (n > 0xFFFFFFFFll) return fail(WOST_ERR_INVALID_ARG, "too many queries");
    std::lock_guard<std::mutex> lk(s->mu);
    cudaError_t e = launch_query_sample(s->view, n, pts, r, (uint32_t)seed, (uint32_t)(seed >> 32), ctr1, ctr2, z, pdf,
                                        prim, (cudaStream_t)stream);
    return query_epilogue(s, e, (cudaStream_t)stream);
}

wost_status wost_scene_autotune(wost_scene *scene, const float *points, int64_t n, int32_t walks, float epsilon,
                                float r_min, int32_t max_steps, wost_tune_result *out) {
    try {
        if (!scene || !points || !out || n < 1) return fail(WOST_ERR_INVALID_ARG, "null argument or n < 1");
        std::memset(out, 0, sizeof *out);
        CK(cudaSetDevice(scene->device), "cudaSetDevice");
        // an evenly strided sample of the caller's points (a prefix could
        // hold one region of the domain only)
        const int dim = scene->view.dim;
        const int64_t m = std::min<int64_t>(n, 65536), stride = n / m;
        DevBuf sample;
        CK(sample.alloc((size_t)m * dim * sizeof(float)), "cudaMalloc");
        CK(cudaMemcpy2D(sample.p, dim * sizeof(float), points, (size_t)stride * dim * sizeof(float),
                        dim * sizeof(float), (size_t)m, cudaMemcpyDeviceToDevice),
           "sample copy");
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        CK(cudaEventCreate(&e0), "cudaEventCreate");
        CK(cudaEventCreate(&e1), "cudaEventCreate");
        std::unique_ptr<CUevent_st, cudaError_t (*)(cudaEvent_t)> k0(e0, cudaEventDestroy), k1(e1, cudaEventDestroy);
        const int blocks[4] = {64, 128, 192, 256};
        const int iters = 256;  // walk steps per lane per launch
        double best = -1;
        for (int ci = 0; ci < 8; ++ci) {
            const int bi = ci % 4, lanes = ci < 4 ? 1 : WOST_WIDE;
            wost_solve_desc d{};
            d.lanes_per_walk = lanes;
            d.n_points = m;
            d.points = (const float *)sample.p;
            d.memory = WOST_MEM_DEVICE;
            d.walks_per_point = walks > 0 ? walks : 32;
            d.epsilon = epsilon;
            d.r_min = r_min;
            d.max_steps = max_steps;
            d.seed = 0x5EED0000u;
            d.kernel = WOST_KERNEL_RESUMABLE;
            d.block_size = blocks[bi];
            // steady state of the resumable kernel: one launch fills every
            // lane with a walk, the next two are timed (walk steps executed
            // over their device time); a sample too small to keep the lanes
            // busy is timed as it drains, which is then its real regime
            wost_solve_handle *h = nullptr;
            wost_status st = wost_solve(scene, &d, &h);
            if (st != WOST_OK) return st;
            std::unique_ptr<wost_solve_handle, wost_status (*)(wost_solve_handle *)> hk(h, wost_solve_destroy);
            const cudaStream_t s = h->stream;
            unsigned long long before = 0, after = 0;
            if ((st = wost_solve_advance(h, iters, nullptr)) != WOST_OK) return st;
            CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
            CK(cudaMemcpy(&before, h->rstate.p, sizeof before, cudaMemcpyDeviceToHost), "copy steps");
            CK(cudaEventRecord(e0, s), "cudaEventRecord");
            for (int rep = 0; rep < 2; ++rep)
                if ((st = wost_solve_advance(h, iters, nullptr)) != WOST_OK) return st;
            CK(cudaEventRecord(e1, s), "cudaEventRecord");
            CK(cudaEventSynchronize(e1), "cudaEventSynchronize");
            CK(cudaMemcpy(&after, h->rstate.p, sizeof after, cudaMemcpyDeviceToHost), "copy steps");
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
            const double rate = ms > 0 ? (double)(after - before) / (ms * 1e-3) : 0;
            out->tried_block[out->n_tried] = blocks[bi];
            out->tried_lanes[out->n_tried] = lanes;
            out->tried_steps_per_second[out->n_tried] = rate;
            out->n_tried++;
            if (rate > best) {
                best = rate;
                out->block_size = blocks[bi];
                out->lanes_per_walk = lanes;
                out->steps_per_second = rate;
            }
        }
        scene->tuned_block = out->block_size;
        scene->tuned_lanes = out->lanes_per_walk;
        set_layout_info(scene, scene->tuned_lanes);
        return WOST_OK;
    } catch (const std::exception &e) {
        return fail(WOST_ERR_INTERNAL, e.what());
    }
}

}  // extern "C"
