// Internal data layout shared by the host scene builder and the CUDA kernels.
//
// Three binary hierarchies per scene, each flattened so that a node holds the
// bounding boxes of BOTH children (one 64-byte fetch tests two boxes):
//   D  BVH over the Dirichlet primitives     -> Q.1 closest point (Sec. 5)
//   N  BVH over the Neumann primitives       -> Q.3 rays, Q.4 sampling (Sec. 5.2)
//   S  normal-cone hierarchy over silhouette candidates of the Neumann part
//      (2D: vertices, 3D: edges), each node also holding both children's
//      normal cones                          -> Q.2 silhouette distance (Sec. 5.1)
//
// Node (64 B, float4 x4):
//   2D: q0 = box0 (lo.x lo.y hi.x hi.y), q1 = box1, q2 = (ref0, ref1, -, -) as int bits
//   3D: q0 = (b0.lo.x b0.lo.y b0.lo.z b0.hi.x), q1 = (b0.hi.y b0.hi.z b1.lo.x b1.lo.y),
//       q2 = (b1.lo.z b1.hi.x b1.hi.y b1.hi.z), q3 = (ref0, ref1, -, -)
// Child reference: bit 31 clear -> internal node index; set -> leaf with
//   first primitive (bits 4..30) and count-1 (bits 0..3).
// Cone record (S only, 32 B per node): float4 per child = (axis.xyz, cos(half angle));
//   cos <= 0 means "may always contain a silhouette" (half angle >= 90 deg).
//
// Primitive records, in leaf order:
//   D/N 2D: float4 (a.x a.y b.x b.y)
//   D/N 3D: float4 x3: (a.xyz, area) (b.xyz, 0) (c.xyz, 0)
//   S   2D: float4 x2: (p.x p.y 0 0) (n0.x n0.y n1.x n1.y)
//   S   3D: float4 x3: (a.xyz n0.x) (b.xyz n0.y) (n0.z n1.xyz)
//   A silhouette candidate with one adjacent Neumann primitive (a boundary
//   vertex/edge, always a silhouette, Sec. 5.1) stores n1 = 0, so the
//   predicate (v.n0)(v.n1) <= 0 holds for it without a flag.
// Boundary data per primitive, in leaf order (corner values of g on D, h on N):
//   2D float2, 3D float4 (xyz used).
#pragma once

#include <stdint.h>

#define WOST_LEAF_BIT 0x80000000u
#define WOST_EMPTY_REF 0xFFFFFFFFu
#define WOST_MAX_LEAF 16
#define WOST_MAX_DEPTH 60
#define WOST_WIDE 8  // children per node of the wide layout (= lanes per walk team)

namespace wost {

enum FieldKind { FIELD_NONE = 0, FIELD_CORNER = 2, FIELD_ANALYTIC = 3, FIELD_GRID = 4 };

inline uint32_t leaf_ref(uint32_t first, uint32_t count) {
    return WOST_LEAF_BIT | (first << 4) | (count - 1u);
}

struct FieldView {
    int32_t kind;       // FieldKind (per-vertex data is converted to corners)
    int32_t fn;         // analytic id
    float params[8];
    const float *grid;  // GRID values
    float origin[3], spacing[3];
    int32_t dims[3];
};

struct TreeView {
    const float4 *nodes;    // 4 float4 per node
    const float4 *cones;    // 2 float4 per node (S only)
    const float4 *prims;    // records, see above
    const float4 *data;     // D/N corner data (2D: reinterpret as float2)
    const float4 *data_minus;  // D/N corner data of the - side of double-sided records (or null)
    const uint8_t *sided;   // per record: 1 = double-sided (App. B); null if none is
    const int32_t *ids;     // input index of each record
    uint32_t root;          // child reference of the root (or WOST_EMPTY_REF)
    float root_lo[3], root_hi[3];
    float4 root_cone;       // S only
    int32_t n_prims, n_nodes, depth;
    // 8-wide layout: 16 float4 per node (child c: (lo.xyz, ref), (hi.xyz, 0));
    // S also has 8 float4 of child cones per node
    const float4 *wnodes;
    const float4 *wcones;
    uint32_t wroot;
    int32_t wn_nodes, wdepth;
};

struct SceneView {
    int32_t dim;
    TreeView D, N, S;
    FieldView g, h, f;
    // the boundary's bounding box grown by its largest side on every side: a
    // walk outside it has left the domain (through a rounding gap)
    float out_lo[3], out_hi[3];
    float rmax;  // diagonal of the boundary's bounding box: bound on the star radius
};

struct SolveParams {
    const float *points;        // device [n_points * dim]
    const float *normals;       // device or null
    const uint8_t *on_neumann;  // device or null
    int64_t point_begin;        // first point of this launch/job (batched rounds)
    int64_t n_points;           // points [point_begin, point_begin + n_points)
    int32_t walks_per_point;
    uint32_t first_walk;
    float epsilon, r_min;
    int32_t max_steps;
    uint32_t key0, key1;
    float offset;               // relative ray-origin offset on the boundary
    float vis_tmax;             // visibility ray end for the Neumann sample
    int32_t stack_depth;        // shared-memory stack entries per walk (thread or team)
    uint32_t visit_limit;       // node visits allowed per traversal (0: 2 n_nodes + 8)
    float sigma;                // screening coefficient (0: Poisson)
    float sqrt_sigma;
    int32_t screen_after;       // steps k >= screen_after are screened (Tikhonov switch)
};

struct Accumulators {
    double *sum, *sumsq;
    unsigned long long *walks, *steps;
    unsigned long long *capped;     // [1]
    unsigned long long *next_walk;  // [1] work counter (persistent kernel)
    unsigned int *guard;            // [1] guard flags
    int *cancel;                    // [1] host-set cancel flag (mapped)
};

// Walks carried across the launches of a resumable solve: one slot per team
// of the (fixed) launch grid, 3 float4: (x, acc), (n, dbound), (steps,
// point, walk index, flags) with flags bit 0 = the slot holds a walk, bit 1
// = on the Neumann boundary, bit 2 = capped.
struct ResumeState {
    float4 *slots;
    unsigned long long *steps_run;  // [1] walk steps executed by all launches
    unsigned int *live;             // [1] walks saved by the latest launch (cleared before it)
};

// Accumulators of one solve, for the per-solve summary kernel.
struct StatJob {
    const double *sum, *sumsq;
    const unsigned long long *walks, *steps;
    int64_t n;
};

// Size of a batched launch, read by the kernel from device memory so that a
// captured graph can be replayed with new job tables.
struct BatchHeader {
    int n_jobs;
    int pad;
    unsigned long long total;  // walks in the launch
};

// One entry of a batched launch: a solve's walks [walk_begin, walk_begin +
// n_points * walks_per_point) in the launch's walk index space.
struct BatchJob {
    const SceneView *scene;         // device copy of the scene's view
    SolveParams sp;
    Accumulators acc;
    unsigned long long walk_begin;
};

}  // namespace wost
