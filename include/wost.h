/*
 * wost.h -- C ABI of the GB300 walk-on-stars library (libwost.so).
 *
 * Method: Sawhney, Miller, Gkioulekas, Crane, "Walk on Stars: A Grid-Free
 * Monte Carlo Method for PDEs with Neumann Boundary Conditions", ACM TOG
 * 42(4), 2023 (arXiv 2302.11815).
 *
 * Problem solved (Sec. 3.2, Eq. PoissonEquation, with the sign convention of
 * the positive Green's functions of App. A.1):
 *
 *     -Lap u = f   in Omega,
 *          u = g   on the Dirichlet boundary,
 *      du/dn = h   on the Neumann boundary (n = outward unit normal),
 *
 * estimated at caller-chosen points by independent random walks (Alg. 1),
 * each step using a star-shaped region whose radius is the smaller of the
 * distance to the Dirichlet boundary (query Q.1) and the distance to the
 * visibility silhouette of the Neumann boundary (Q.2, Sec. 5.1), a ray cast
 * against the Neumann boundary (Q.3) and a hierarchical Neumann sample (Q.4,
 * Sec. 5.2).  Walks run on the GPU in single precision; per-point sums are
 * accumulated in double precision.
 *
 * Conventions for every call:
 *   - Every call returns a wost_status; nothing throws or aborts across the
 *     ABI.  On failure, wost_last_error() gives a message (thread-local).
 *   - The library copies every input array during the call; the caller keeps
 *     ownership and may free its arrays as soon as the call returns.
 *   - Output arrays are caller-owned and sized as stated.
 *   - Handles are opaque; the caller destroys what it creates.
 *   - Geometry: dim = 2 (line segments, 2 vertex indices each) or 3
 *     (triangles, 3 indices).  A 2D segment a->b has outward normal
 *     (t.y, -t.x), t = (b-a)/|b-a|; a 3D triangle a,b,c has outward normal
 *     (b-a)x(c-a)/|..|.  Degenerate primitives (zero length or area) are
 *     dropped and counted.  The boundary need not be watertight (Sec. 5).
 */
#ifndef WOST_H
#define WOST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WOST_ABI_VERSION 4

typedef enum {
    WOST_OK = 0,
    WOST_ERR_INVALID_ARG = 1, /* bad pointer, size, index, value or mode     */
    WOST_ERR_OUT_OF_MEMORY = 2, /* device or host allocation failed          */
    WOST_ERR_BUDGET = 3,      /* the engine rejected the request (memory
                                 budget, or its wait limit ran out)          */
    WOST_ERR_CUDA = 4,        /* a CUDA runtime call failed                  */
    WOST_ERR_TIMEOUT = 5,     /* wost_wait gave up before completion         */
    WOST_ERR_CANCELLED = 6,   /* the solve was cancelled                     */
    WOST_ERR_INTERNAL = 7     /* a device-side guard fired (see progress)    */
} wost_status;

/* ---------------------------------------------------------------------- */
/* Boundary data and source (Sec. 3.2: g on the Dirichlet part, h on the   */
/* Neumann part, f inside).                                                */
/* ---------------------------------------------------------------------- */
typedef enum {
    WOST_DATA_NONE = 0,       /* absent: zero (f only)                         */
    WOST_DATA_PER_VERTEX = 1, /* values[n_vertices], linear on each primitive */
    WOST_DATA_PER_CORNER = 2, /* values[n_prims*dim], one per primitive corner */
    WOST_DATA_ANALYTIC = 3,   /* built-in exact solution `fn`: g = u,
                                 h = grad u . n, f = -Lap u                    */
    WOST_DATA_GRID = 4        /* f only: node-centred grid, dims[0] fastest,
                                 (bi/tri)linear, clamped at the edges          */
} wost_data_kind;

typedef enum {
    WOST_FN_ZERO = 0,
    WOST_FN_EXP_COS = 1,     /* u = e^x cos y                                  */
    WOST_FN_SIN2X_COS3Y = 2, /* u = sin 2x cos 3y (2D), -Lap u = 13 u          */
    WOST_FN_QUAD3 = 3,       /* u = x^2 - y^2 + z/2                            */
    WOST_FN_BUMP = 4,        /* u = (1 - |x|^2)/(2 dim), -Lap u = 1            */
    WOST_FN_LINEAR = 5,      /* u = p0 + p1 x + p2 y + p3 z                    */
    WOST_FN_LOG_RADIAL = 6,  /* 2D p0 + p1 log|x-c|, 3D p0 + p1/|x-c|,
                                c = (p2, p3, p4)                               */
    WOST_FN_EXP_PLANE = 7    /* u = p0 exp(p1 x + p2 y + p3 z): solves the
                                screened equation for sigma = p1^2+p2^2+p3^2   */
} wost_fn;

typedef struct {
    int32_t kind;          /* wost_data_kind                                 */
    const float *values;   /* host array for PER_VERTEX / PER_CORNER / GRID  */
    int32_t fn;            /* ANALYTIC: wost_fn                              */
    float params[8];       /* ANALYTIC parameters                            */
    float origin[3];       /* GRID: position of node (0,0,0)                 */
    float spacing[3];      /* GRID: node spacing (> 0)                       */
    int32_t dims[3];       /* GRID: nodes per axis (>= 1; dims[2] ignored in 2D) */
} wost_field;

/* ---------------------------------------------------------------------- */
/* Scenes: the boundary, its hierarchies (a BVH over the Dirichlet part, a */
/* BVH and a spatialized normal-cone hierarchy over the Neumann part,      */
/* Sec. 5 and 5.1.1) and boundary data, resident on one device.            */
/* ---------------------------------------------------------------------- */
typedef struct wost_scene wost_scene;

/* Double-sided boundaries (App. B): a primitive flagged 2 or 3 bounds the
 * domain on both of its sides (a crack, a thin sheet, an open surface).  Its
 * canonical normal n+ is the outward normal above; the "+" side is the one
 * n+ points away from (as for a one-sided primitive, whose domain lies
 * behind its outward normal), the "-" side the one it points into.  g and h
 * give the + side's data (h = du/dn+), g_minus and h_minus the - side's
 * (h_minus = du/dn-, n- = -n+).  A walk uses the data of the side it is on:
 * the side of x relative to the closest point (Dirichlet), the side it came
 * from when it hits a Neumann sheet (its next direction stays on that side),
 * and the side of the walk's query point relative to a Neumann sample.
 * g_minus / h_minus may be NONE: then g- = g+ and h- = -h+ (a solution
 * continuous across the sheet), which is also what analytic data give. */
typedef struct {
    int32_t dim;               /* 2 or 3                                       */
    int64_t n_vertices;
    const float *vertices;     /* host [n_vertices * dim]                      */
    int64_t n_prims;
    const int32_t *prims;      /* host [n_prims * dim], indices < n_vertices   */
    const uint8_t *flags;      /* host [n_prims]: 0 Dirichlet, 1 Neumann,
                                  2 double-sided Dirichlet, 3 double-sided
                                  Neumann                                      */
    wost_field g, h, f;
    int32_t device;            /* CUDA device ordinal                          */
    int32_t leaf_size;         /* primitives per leaf, 0 = default (4)         */
    wost_field g_minus, h_minus; /* - side data of double-sided primitives:
                                  NONE, PER_VERTEX or PER_CORNER               */
    int32_t silhouette_split;  /* split cost of the silhouette hierarchy:
                                  0 = surface area x orientation (groups
                                  candidates that face alike, Sec. 5.1.1's
                                  suggested improvement), 1 = surface area
                                  only (the paper's own build)                 */
} wost_scene_desc;

typedef struct {
    int32_t dim;
    int64_t n_dirichlet, n_neumann, n_silhouette, n_dropped;
    int64_t nodes_dirichlet, nodes_neumann, nodes_silhouette;
    int32_t depth_dirichlet, depth_neumann, depth_silhouette;
    int64_t device_bytes;      /* bytes of resident scene data               */
    double build_seconds;
    float bbox_lo[3], bbox_hi[3];
    /* layout the walk kernels traverse by default (the scene's tuned choice,
     * else binary): lanes per walk (1: binary trees, one lane per walk; 8:
     * 8-wide trees, 8 cooperating lanes per walk), bytes read per node visit
     * (node record; the silhouette tree adds its child cones), and the wide
     * trees' node counts and depths */
    int32_t lanes_per_walk;
    int32_t node_bytes, cone_bytes;
    int64_t wide_nodes_dirichlet, wide_nodes_neumann, wide_nodes_silhouette;
    int32_t wide_depth_dirichlet, wide_depth_neumann, wide_depth_silhouette;
    int32_t device;            /* CUDA device ordinal the scene lives on       */
    int32_t stack_depth;       /* traversal stack entries per walk (per team)
                                  of that layout                               */
} wost_scene_info;

/* Builds the hierarchies on the host, uploads them, returns a handle.
 * Errors: INVALID_ARG for dim not 2/3, null arrays, an index out of range, a
 * flag > 1, non-finite coordinates, a field whose values are missing;
 * OUT_OF_MEMORY; CUDA.  A scene without Dirichlet primitives (a pure
 * Neumann problem, Sec. 6.4) is accepted; its solves need sigma > 0. */
wost_status wost_scene_create(const wost_scene_desc *desc, wost_scene **out);

/* Builds the hierarchies of a scene on the host only (no device is used),
 * checks their structure -- every child reference reaches a node once or a
 * leaf, every primitive lies in exactly one leaf, every box contains what
 * lies below it, every normal cone of the silhouette hierarchy contains the
 * normals below it, no leaf is deeper than the traversal stacks are sized
 * for; binary and 8-wide forms -- and fills *info (device_bytes = 0).
 * Errors: INVALID_ARG as wost_scene_create; INTERNAL with the violation. */
wost_status wost_scene_validate(const wost_scene_desc *desc, wost_scene_info *info);
wost_status wost_scene_destroy(wost_scene *scene);
wost_status wost_scene_get_info(const wost_scene *scene, wost_scene_info *out);

/* ---------------------------------------------------------------------- */
/* Solves: n points x walks_per_point walks of Alg. 1.                     */
/* ---------------------------------------------------------------------- */
typedef struct wost_solve_handle wost_solve_handle;

typedef enum {
    WOST_MEM_HOST = 0,   /* points / normals / on_neumann are host pointers   */
    WOST_MEM_DEVICE = 1  /* ... are device pointers on the scene's device      */
} wost_memory;

typedef enum {
    WOST_KERNEL_PLAIN = 0,      /* one thread per walk, one launch             */
    WOST_KERNEL_PERSISTENT = 1, /* persistent lanes that regenerate finished
                                   walks from a work counter                   */
    WOST_KERNEL_COUNTING = 2,   /* the plain kernel plus per-query work
                                   counters (see wost_solve_work_counts)       */
    WOST_KERNEL_RESUMABLE = 3   /* persistent lanes over a fixed grid, run as a
                                   sequence of bounded launches that carry
                                   unfinished walks over (wost_solve_advance) */
} wost_kernel;

typedef struct {
    int64_t n_points;
    const float *points;       /* [n_points * dim]                             */
    const float *normals;      /* optional [n_points * dim]: outward normal of
                                  points on the Neumann boundary (Alg. 1 n_x)  */
    const uint8_t *on_neumann; /* optional [n_points]: 1 if on the Neumann part */
    int32_t memory;            /* wost_memory of the three arrays above        */
    int32_t walks_per_point;   /* >= 1                                         */
    float epsilon;             /* epsilon-shell width (> 0)                    */
    float r_min;               /* minimum star radius, 0 < r_min (0 = epsilon) */
    int32_t max_steps;         /* step cap per walk (>= 1)                     */
    uint64_t seed;             /* Philox key                                   */
    uint32_t first_walk;       /* walk index of the first walk of every point  */
    int32_t kernel;            /* wost_kernel                                  */
    int32_t block_size;        /* threads per block, 0 = tuned default         */
    void *stream;              /* cudaStream_t to run on, NULL = library stream */
    float sigma;               /* screening coefficient >= 0 of the screened
                                  Poisson equation -Lap u + sigma u = f
                                  (Sec. 2, App. A.2); 0 = Poisson            */
    int32_t screen_after;      /* steps k >= screen_after solve the screened
                                  equation, earlier ones the Poisson equation:
                                  the Tikhonov switch of Sec. 4.1 for pure
                                  Neumann problems (0 = every step).  Screened
                                  steps end walks by Russian roulette with
                                  the step weight Q of App. A.2              */
    int32_t stack_depth;       /* traversal stack entries per walk, 0 = the
                                  scene's (wost_scene_info.stack_depth, which
                                  no traversal exceeds).  A smaller value saves
                                  shared memory but a traversal that needs more
                                  drops subtrees and sets guard bit 1, making
                                  wost_wait / wost_poll return INTERNAL       */
    int32_t visit_limit;       /* node visits allowed per traversal, 0 = twice
                                  the tree's nodes plus 8 (more than a correct
                                  traversal makes).  A traversal that reaches
                                  the limit stops and sets guard bit 2        */
    int32_t lanes_per_walk;    /* 1: one lane per walk over the binary trees;
                                  8: a team of 8 lanes per walk over the 8-wide
                                  trees (persistent and resumable Poisson
                                  solves); 0: the scene's choice (set by
                                  wost_scene_autotune, else 1)               */
} wost_solve_desc;

typedef struct {
    int32_t done;              /* 1 once every walk has finished               */
    uint64_t walks_done;       /* walks accumulated so far                     */
    uint64_t total_steps;      /* walk steps (each Q.1 evaluation is a step)   */
    uint64_t capped_walks;     /* walks stopped by max_steps                   */
    uint32_t guard_flags;      /* device guards: 1 = traversal stack overflow,
                                  2 = a traversal exceeded its visit limit     */
    double elapsed_seconds;    /* from launch to completion (or to now)        */
    uint64_t steps_run;        /* resumable solves: walk steps executed by the
                                  completed launches, finished walks or not;
                                  other kernels: total_steps                   */
    uint64_t launches;         /* kernel launches of this solve so far          */
} wost_progress;

/* Starts a solve asynchronously on the stream and returns its handle.
 * The caller's arrays are copied before return.  Errors: INVALID_ARG
 * (n_points < 1, walks < 1, epsilon <= 0, r_min > epsilon, max_steps < 1,
 * a null points array, sigma < 0 or not finite, screen_after < 0, sigma = 0
 * on a scene without Dirichlet primitives, stack_depth or visit_limit < 0),
 * OUT_OF_MEMORY, CUDA. */
wost_status wost_solve(wost_scene *scene, const wost_solve_desc *desc, wost_solve_handle **out);

/* Resumable solves (desc->kernel = WOST_KERNEL_RESUMABLE): wost_solve
 * allocates the solve's state, including one saved-walk slot per lane of a
 * fixed resident grid, and launches nothing.  Each wost_solve_advance
 * enqueues ONE launch on `stream` (NULL = the solve's stream) in which every
 * lane runs at most `iterations` walk steps, drawing new walks as its walks
 * end, and saves its unfinished walk for the next launch; the launches of a
 * solve must run in order (one stream, or ordered by the caller).  No
 * launch waits for the longest walks of the solve, which is what keeps
 * the GPU full on workloads whose walk lengths have a long tail.  wost_wait
 * on a resumable solve issues launches of 2048 iterations itself until
 * every walk has finished.  The walks and estimates are those of the other
 * kernels for the same seed.  Errors: INVALID_ARG (not a resumable solve,
 * iterations < 1), CUDA. */
wost_status wost_solve_advance(wost_solve_handle *solve, int32_t iterations, void *stream);

/* Batching: starts n solves (any scenes of one device, any point counts, walk
 * counts and parameters) in ONE persistent launch per dimension present (2D
 * jobs and 3D jobs run in separate launches, back to back on the stream).
 * Lanes take walks from a shared counter across all jobs, so uneven walk
 * lengths do not idle the GPU.  out[i] (n handles) behaves like a handle from
 * wost_solve; all of them complete together.  descs[i].kernel and block_size
 * are taken from descs[0] (the counting kernel is not allowed here).
 * Errors as for wost_solve; on error no handle is returned. */
wost_status wost_solve_batch(int32_t n, wost_scene *const *scenes, const wost_solve_desc *descs, void *stream,
                             wost_solve_handle **out);

/* Snapshot of the running estimates.  mean and stderr_ (host, n_points each)
 * may be NULL.  stderr_ is sqrt(sample variance / walks); walks_done
 * (host, n_points, may be NULL) is the per-point walk count. */
wost_status wost_poll(wost_solve_handle *solve, double *mean, double *stderr_, uint64_t *walks_done,
                      wost_progress *progress);

/* Blocks until the solve finishes or timeout_s elapses (< 0: no limit).
 * Returns TIMEOUT on expiry, INTERNAL if a device guard fired. */
wost_status wost_wait(wost_solve_handle *solve, double timeout_s);

/* Stops a solve at the next walk boundary (walks already accumulated stay). */
wost_status wost_cancel(wost_solve_handle *solve);
wost_status wost_solve_destroy(wost_solve_handle *solve);

/* Device pointers to the per-point FP64 accumulators of a solve (valid until
 * destroy): sum and sum of squares of the walk estimates, walk and step
 * counts. */
wost_status wost_solve_device_accumulators(wost_solve_handle *solve, const double **sum,
                                           const double **sumsq, const uint64_t **walks,
                                           const uint64_t **steps);

/* Work done by a WOST_KERNEL_COUNTING solve (after wost_wait): counts[0..4]
 * are node visits of Q.1, Q.2, Q.3, Q.4 and of the visibility ray of the
 * Neumann sample; counts[5..9] the primitive tests of the same queries.
 * INVALID_ARG for a solve started with another kernel. */
wost_status wost_solve_work_counts(wost_solve_handle *solve, uint64_t counts[10]);

/* The screened-equation functions the walks evaluate (App. A.2): at each
 * of n pairs, G[i] = G^sigma_B(rho[i]) of the ball of radius R[i] (Eq.
 * GreensFnsScreenedPoissonBall) and Q[i] = Q^sigma_B(rho[i]) (Eq.
 * ScreenedPoissonKernelsSphere), 0 < rho[i] <= R[i].  All arrays are device
 * float arrays of the current device (G or Q may be NULL); single precision,
 * the Bessel functions by the approximations of Abramowitz & Stegun 9.8.
 * Enqueued on `stream`.  Errors: INVALID_ARG (dim, sigma <= 0, null rho or
 * R), CUDA. */
wost_status wost_screened_kernels(int32_t dim, int64_t n, const float *rho, const float *R, float sigma, float *G,
                                  float *Q, void *stream);

/* ---------------------------------------------------------------------- */
/* Solve without allocation.  The paper has no counterpart: this is a      */
/* deployment variant of wost_solve.                                      */
/* ---------------------------------------------------------------------- */
#define WOST_STATIC_MAX_POINTS 65536

/* For callers that cannot allocate device memory while they solve (a loop
 * that must not stall on the device synchronisation of cudaMalloc/cudaFree,
 * a process whose device memory is committed under a fixed budget).
 * Enqueues on `stream` (NULL = the legacy default stream) the n_points x
 * walks_per_point walks that wost_solve runs with WOST_KERNEL_PERSISTENT for
 * the same arguments (walk indices first_walk.., Philox key seed) and
 * writes the per-point mean to mean_out and, when
 * stderr_out is not NULL, its standard error sqrt(sample variance / walks).
 * points (device, n_points * dim floats; interior points: no Neumann
 * normals), mean_out and stderr_out (device, n_points floats) belong to the
 * caller and must stay valid until the stream has passed this call.
 * The call allocates nothing: the FP64 accumulators and counters live in one
 * fixed device array of the library (about 2 MiB, held by every device that
 * loads the library until the process exits), which the call clears on
 * `stream` before use.  Hence:
 *   - n_points > WOST_STATIC_MAX_POINTS is rejected with INVALID_ARG;
 *   - calls whose work overlaps on one device (other streams or threads)
 *     share that array and give wrong results: order them;
 *   - every call looks up the array's device address (a device reset or a
 *     recreated context moves it); the first lookup on a device may load the
 *     module: make the first call before any stream capture.
 * If a device guard fires (traversal stack overflow or visit limit), every
 * output is NaN.  Returns once the work is enqueued.  Errors: INVALID_ARG
 * (null scene, points or mean_out; n_points < 1 or above the maximum;
 * walks_per_point < 1; epsilon <= 0; r_min > epsilon; max_steps < 1), CUDA. */
wost_status wost_solve_static(wost_scene *scene, int64_t n_points, const float *points, int32_t walks_per_point,
                              float epsilon, float r_min, int32_t max_steps, uint64_t seed, uint32_t first_walk,
                              float *mean_out, float *stderr_out, void *stream);

/* ---------------------------------------------------------------------- */
/* Serving engine: continuous batching of solves with target errors.       */
/* ---------------------------------------------------------------------- */
/* A background scheduler owns one device stream.  Submitted requests wait
 * in a FIFO until their state (points and FP64 accumulators) fits the
 * engine's device-memory budget, then join the running mix: every
 * scheduling round is one batched persistent launch over pieces (point
 * ranges x walk ranges) of the active requests, sized to about
 * round_seconds of GPU time but never so small that the resident grid runs
 * short of walks; the round's walk-step budget goes to the active requests
 * with the least work left in their current stage first, so under overload
 * the cheapest complete and the rest wait (or are shed by
 * max_wait_seconds).  Up to three rounds run concurrently (each on streams
 * of its own, so one round's last walks overlap the next rounds), and the
 * GPU never waits for the host.  A request runs in stages of walks per point
 * (min_walks, then growing from its own variance estimate); after each
 * stage it completes if its largest per-point standard error is at most its
 * target, or if it reached its walk cap.  A request's walks use its own
 * seed and walk indices, so its result does not depend on what else runs
 * (progressive estimates via wost_poll at any time).  This is the paper's
 * progressive evaluation (Sec. 1) served to many clients. */
typedef struct wost_engine wost_engine;

typedef struct {
    int32_t device;
    int64_t memory_budget_bytes;  /* device bytes for request state; 0 = 1/4 of free memory */
    double round_seconds;         /* target GPU time per round; 0 = 0.02 s                 */
    int32_t min_walks;            /* walks per point of the first stage; 0 = 16           */
    int32_t max_walks_per_point;  /* default walk cap; 0 = 65536                           */
    int32_t block_size;           /* threads per block; 0 = 128                            */
    double max_wait_seconds;      /* a request whose first walks have not started this long
                                     after submission is finished with BUDGET and counted
                                     as rejected (overload shedding); 0 = wait forever    */
} wost_engine_desc;

typedef struct {
    uint64_t submitted, admitted, completed, cancelled, rejected, capped;
    int32_t queued, active;
    uint64_t rounds;
    uint64_t graph_launches;      /* rounds launched by replaying a CUDA graph   */
    double gpu_seconds;           /* summed duration of finished rounds (rounds
                                     overlap on the device: may exceed wall time) */
    int64_t budget_bytes, used_bytes;
    double round_budget_steps;    /* current walk-step budget of one round       */
    uint64_t walk_steps;          /* walk steps of every walk finished by a
                                     finished round (completed, cancelled and
                                     shed requests alike)                        */
} wost_engine_stats;

wost_status wost_engine_create(const wost_engine_desc *desc, wost_engine **out);

/* Submits a request: desc as for wost_solve (points, seed, epsilon, r_min,
 * max_steps; memory HOST or DEVICE; kernel, block_size and stream ignored);
 * desc->walks_per_point is the request's walk cap (0 or larger than the
 * engine's cap: the engine's cap).  target_se > 0: stop once every point's
 * standard error is <= target_se; target_se == 0: run exactly the cap.
 * Inputs are copied before return.  The handle works with wost_poll
 * (no walks reported until a round holding some of the request's walks has
 * completed), wost_wait (CANCELLED for a cancelled request; BUDGET for one
 * shed by the wait limit), wost_cancel and wost_solve_destroy.  Errors: INVALID_ARG; BUDGET if the request alone
 * exceeds the memory budget (it could never be admitted). */
wost_status wost_engine_submit(wost_engine *engine, wost_scene *scene, const wost_solve_desc *desc,
                               double target_se, wost_solve_handle **out);
wost_status wost_engine_get_stats(wost_engine *engine, wost_engine_stats *out);
/* Cancels what is queued or running, waits for the device, joins the
 * scheduler.  Handles of its requests stay valid until destroyed. */
wost_status wost_engine_destroy(wost_engine *engine);

/* ---------------------------------------------------------------------- */
/* Batched geometric queries (Sec. 5, Q.1-Q.4), for checking and reuse.    */
/* All arrays are DEVICE pointers; points/vectors are [n * dim] floats.    */
/* ---------------------------------------------------------------------- */

/* Q.1: distance to the closest Dirichlet point, that point, and the
 * primitive (input index), or +inf and -1 without Dirichlet primitives. */
wost_status wost_query_closest_dirichlet(wost_scene *scene, int64_t n, const float *points,
                                         float *dist, float *closest, int32_t *prim, void *stream);

/* Q.2 (Algs. 2-4): distance to the closest visibility-silhouette point of
 * the Neumann boundary within rmax[i]; rmax[i] if there is none. */
wost_status wost_query_silhouette(wost_scene *scene, int64_t n, const float *points,
                                  const float *rmax, float *dist, void *stream);

/* Q.3: first hit of origin + t dir, 0 < t <= tmax[i], with the Neumann
 * boundary; skip[i] (input index or -1, may be NULL) is ignored.  hit is 0/1,
 * t the distance along dir (unnormalised dir scales t), prim the input
 * index or -1. */
wost_status wost_query_intersect_neumann(wost_scene *scene, int64_t n, const float *origins,
                                         const float *dirs, const float *tmax, const int32_t *skip,
                                         int32_t *hit, float *t, int32_t *prim, void *stream);

/* Q.4 (Algs. 5-6): for ball i (center points[i], radius r[i]) one Neumann
 * sample z (n * dim), its density pdf (0 if none) and primitive (input index
 * or -1), drawn from the Philox stream key = seed, counter = (i, ctr1,
 * ctr2, 1, 2, ...). */
wost_status wost_query_neumann_sample(wost_scene *scene, int64_t n, const float *points,
                                      const float *r, uint64_t seed, uint32_t ctr1, uint32_t ctr2,
                                      float *z, float *pdf, int32_t *prim, void *stream);

/* ---------------------------------------------------------------------- */
/* Autotuning                                                              */
/* ---------------------------------------------------------------------- */
typedef struct {
    int32_t block_size;         /* fastest threads per block                     */
    double steps_per_second;    /* its walk-step rate on the sample              */
    int32_t n_tried;
    int32_t tried_block[8];
    double tried_steps_per_second[8];
    int32_t lanes_per_walk;     /* fastest layout: 1 (binary) or 8 (8-wide teams) */
    int32_t tried_lanes[8];
} wost_tune_result;

/* Times the walk loop in steady state -- the resumable kernel, one launch
 * of 256 steps per lane to fill the lanes, then two timed launches (walk
 * steps executed over device time) -- on an evenly strided sample of the
 * caller's points (device pointer, n points, at most 65,536 used) at
 * walks_per_point (0: 32), for each layout -- one lane per walk over the
 * binary trees, 8-lane teams over the 8-wide trees -- and block sizes
 * 64..256 (8 combinations), and keeps the fastest block size as the
 * scene's default for persistent, batched and engine launches whose
 * block_size is 0, and the fastest layout as its default for persistent and
 * resumable Poisson solves whose lanes_per_walk is 0 (wost_scene_info then
 * reports that layout).  Same validation as wost_solve. */
wost_status wost_scene_autotune(wost_scene *scene, const float *points, int64_t n, int32_t walks_per_point,
                                float epsilon, float r_min, int32_t max_steps, wost_tune_result *out);

/* ---------------------------------------------------------------------- */
/* Measurement helper (no counterpart in the paper)                        */
/* ---------------------------------------------------------------------- */
/* Enqueues on `stream` one read sweep kernel over the caller's device buffer
 * (bytes, 16-byte aligned, a multiple of 16): `passes` sweeps of 16-byte
 * loads that bypass L1, resident grid.  It measures the read bandwidth of
 * the level the buffer lives in -- L2 for a buffer well below the L2 size,
 * HBM for one well above it -- for the roofline of the walk kernels, whose
 * scene data are L2-resident.  The caller times it (CUDA events on
 * `stream`); sink (device, 1 float) receives a value only in a case that
 * cannot occur with finite data.  Allocates nothing.  Errors: INVALID_ARG,
 * CUDA. */
wost_status wost_read_probe(const void *buf, int64_t bytes, int32_t passes, float *sink, void *stream);

/* Thread-local description of the last failure on this thread. */
const char *wost_last_error(void);
int32_t wost_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* WOST_H */
