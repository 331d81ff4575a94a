// Device code of the walk-on-stars hot path (single precision, sm_103a).
//
// Paper: Sawhney et al., "Walk on Stars", 2023.  One call of walk_step() is
// one iteration of Alg. 1: Q.1 closest Dirichlet point, epsilon-shell test,
// Q.2 silhouette distance within d_D, star radius, direction (hemisphere on
// the Neumann boundary, Sec. 4.4.2), Q.3 first Neumann hit, Q.4 Neumann
// sample with its visibility test (Sec. 4.5, Algs. 5-6), source sample
// reusing the direction (Sec. 4.6), and the move.  Readings of the paper
// used here (also listed in the design notes):
//   R1 each step adds +N + S (App. A's positive Green's functions, outward h);
//   R2 d_sil is the minimum over silhouette candidates within d_D (Alg. 3's
//      Ensure line);
//   R3 r = min(d_D, max(r_min, d_sil));
//   R4 on the Neumann boundary Q.2/Q.3/visibility start at x - delta n_x,
//      delta = offset (1 + |x|_inf); the visibility ray skips z's primitive
//      and stops at vis_tmax;
//   R5 at the step cap the walk ends with g at the closest Dirichlet point;
//   R6 Q.4 child weight 1/d to the child box centre (the 1/(4 pi) of the
//      free-space Green's function cancels in the child probabilities);
//   R7 2D source radius R sqrt(U1 U2), 3D R (1/2 + sin(asin(2U-1)/3));
//   R12 a Neumann sample at distance 0 from x contributes nothing;
//   R13 a walk outside the grown bounding box ends like a capped walk;
//   R14 the star radius is at most the scene's diameter;
//   R15 screened steps (App. A.2): G^sigma_B for the Neumann term, the
//       unscreened source sample reweighted, Russian roulette with Q.
// Random numbers: Philox4x32-10 (Salmon et al., SC'11); key = seed, counter
// = (walk, point, step, slot); slot 0 drives direction and source, slots
// 1, 2, ... the Neumann sampler.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wost_internal.h"

// Postponed-leaf traversals for Q.1, Q.2 and Q.3 + visibility in 2D (1, the
// default) or the per-lane depth-first loops (0).  Build-time knob.
#ifndef WOST_POSTPONE_LEAVES
#define WOST_POSTPONE_LEAVES 1
#endif

namespace wost {

// ---------------------------------------------------------------------------
// vectors (3 components; z stays 0 in 2D)
// ---------------------------------------------------------------------------
struct P3 {
    float x, y, z;
};
__device__ __forceinline__ P3 mk(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ P3 operator+(P3 a, P3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ P3 operator-(P3 a, P3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ P3 operator*(P3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
template <int D>
__device__ __forceinline__ float dotp(P3 a, P3 b) {
    float r = a.x * b.x + a.y * b.y;
    if constexpr (D == 3) r += a.z * b.z;
    return r;
}
__device__ __forceinline__ P3 crossp(P3 a, P3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// ---------------------------------------------------------------------------
// Philox4x32-10
// ---------------------------------------------------------------------------
// One out-of-line copy: it is called from several places per step, and
// inlining it at each one bloats the kernel past the instruction cache.
static __device__ __noinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}
// One out-of-line copy of each library function the walk step needs.  Inlined
// at every call site, their range reductions and slow paths were a fifth of
// the walk kernels' code, and instruction supply is what stalls those
// kernels most (ncu: no_instruction the leading stall reason).  Results come
// back by value: an out-of-line function writing through pointers would put
// the caller's variables in local memory.
static __device__ __noinline__ float m_exp(float a) { return expf(a); }
static __device__ __noinline__ float m_log(float a) { return logf(a); }
static __device__ __noinline__ float m_asin(float a) { return asinf(a); }
static __device__ __noinline__ float2 m_sincos(float a) {
    float s, c;
    sincosf(a, &s, &c);
    return make_float2(s, c);
}
__device__ __forceinline__ float m_sin(float a) { return m_sincos(a).x; }
__device__ __forceinline__ float m_cos(float a) { return m_sincos(a).y; }

// (0,1): top 23 bits plus one half, times 2^-23 (exact in FP32)
__device__ __forceinline__ float u01(uint32_t w) { return ((float)(w >> 9) + 0.5f) * (1.0f / 8388608.0f); }

struct Stream {  // sequential uniforms from slots 1, 2, ... of one (walk, point, step)
    uint4 ctr;
    uint32_t k0, k1;
    uint4 buf;
    int used;
    __device__ __forceinline__ void init(uint32_t key0, uint32_t key1, uint32_t c0, uint32_t c1, uint32_t c2) {
        ctr = make_uint4(c0, c1, c2, 1u);
        k0 = key0;
        k1 = key1;
        used = 4;
    }
    // inline (the refill calls the one out-of-line Philox): an out-of-line
    // member function would keep the stream's state in local memory
    __device__ __forceinline__ float next() {
        if (used == 4) {
            buf = philox10(ctr, k0, k1);
            ctr.w += 1u;
            used = 0;
        }
        uint32_t w = used == 0 ? buf.x : (used == 1 ? buf.y : (used == 2 ? buf.z : buf.w));
        ++used;
        return u01(w);
    }
};

// ---------------------------------------------------------------------------
// work counters (compiled in only for the counting kernel): per query, node
// visits and primitive tests
// ---------------------------------------------------------------------------
enum { C_Q1 = 0, C_Q2 = 1, C_Q3 = 2, C_Q4 = 3, C_VIS = 4, C_NQ = 5 };
template <bool ON>
struct Cnt {
    __device__ __forceinline__ void node(int) {}
    __device__ __forceinline__ void prim(int) {}
    __device__ __forceinline__ void prim_n(int, unsigned) {}
};
template <>
struct Cnt<true> {
    unsigned nodes[C_NQ], prims[C_NQ];
    __device__ __forceinline__ Cnt() {
        for (int i = 0; i < C_NQ; ++i) nodes[i] = prims[i] = 0u;
    }
    __device__ __forceinline__ void node(int q) { ++nodes[q]; }
    __device__ __forceinline__ void prim(int q) { ++prims[q]; }
    __device__ __forceinline__ void prim_n(int q, unsigned n) { prims[q] += n; }
};

// ---------------------------------------------------------------------------
// traversal stack in shared memory: entry i of this thread at base[i*stride]
// ---------------------------------------------------------------------------
struct Stack {
    int2 *base;
    int stride, cap;
    unsigned int *guard;
    unsigned visit_limit;  // 0: 2 n_nodes + 8
};
__device__ __forceinline__ void spush(const Stack &s, int &sp, uint32_t ref, float key) {
    if (sp < s.cap) {
        s.base[sp * s.stride] = make_int2((int)ref, __float_as_int(key));
        ++sp;
    } else {
        atomicOr(s.guard, 1u);  // overflow: recorded, entry dropped (no fault)
    }
}
__device__ __forceinline__ void spop(const Stack &s, int &sp, uint32_t &ref, float &key) {
    --sp;
    int2 e = s.base[sp * s.stride];
    ref = (uint32_t)e.x;
    key = __int_as_float(e.y);
}

// A traversal visits every node and leaf at most once: more visits than
// that (2 n_nodes + 1) mean a corrupt tree.  The traversal then stops and
// records guard bit 2 (guard may be null: not recorded) instead of running on.
// `limit` (nonzero) sets a lower cap chosen by the caller.
__device__ __forceinline__ bool over_visit_limit(unsigned &visits, int n_nodes, unsigned int *guard,
                                                 unsigned limit = 0u) {
    if (++visits <= (limit ? limit : 2u * (unsigned)n_nodes + 8u)) return false;
    if (guard) atomicOr(guard, 2u);
    return true;
}

// ---------------------------------------------------------------------------
// nodes
// ---------------------------------------------------------------------------
template <int D>
struct Node {
    float lo0[3], hi0[3], lo1[3], hi1[3];
    uint32_t r0, r1;
};
template <int D>
__device__ __forceinline__ Node<D> load_node(const float4 *nodes, uint32_t i) {
    Node<D> n;
    const float4 *q = nodes + 4 * (size_t)i;
    float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
    if constexpr (D == 2) {
        n.lo0[0] = a.x; n.lo0[1] = a.y; n.hi0[0] = a.z; n.hi0[1] = a.w;
        n.lo1[0] = b.x; n.lo1[1] = b.y; n.hi1[0] = b.z; n.hi1[1] = b.w;
        n.lo0[2] = n.hi0[2] = n.lo1[2] = n.hi1[2] = 0.f;
        n.r0 = __float_as_uint(c.x);
        n.r1 = __float_as_uint(c.y);
    } else {
        float4 d = __ldg(q + 3);
        n.lo0[0] = a.x; n.lo0[1] = a.y; n.lo0[2] = a.z; n.hi0[0] = a.w;
        n.hi0[1] = b.x; n.hi0[2] = b.y; n.lo1[0] = b.z; n.lo1[1] = b.w;
        n.lo1[2] = c.x; n.hi1[0] = c.y; n.hi1[1] = c.z; n.hi1[2] = c.w;
        n.r0 = __float_as_uint(d.x);
        n.r1 = __float_as_uint(d.y);
    }
    return n;
}
__device__ __forceinline__ bool is_leaf(uint32_t ref) { return (ref & WOST_LEAF_BIT) != 0u; }
__device__ __forceinline__ uint32_t leaf_first(uint32_t ref) { return (ref & 0x7FFFFFFFu) >> 4; }
__device__ __forceinline__ uint32_t leaf_count(uint32_t ref) { return (ref & 15u) + 1u; }

template <int D>
__device__ __forceinline__ float box_dist2(const float lo[3], const float hi[3], P3 x) {
    float dx = fmaxf(fmaxf(lo[0] - x.x, x.x - hi[0]), 0.f);
    float dy = fmaxf(fmaxf(lo[1] - x.y, x.y - hi[1]), 0.f);
    float r = dx * dx + dy * dy;
    if constexpr (D == 3) {
        float dz = fmaxf(fmaxf(lo[2] - x.z, x.z - hi[2]), 0.f);
        r += dz * dz;
    }
    return r;
}

// slab test: entry distance of the ray into the box, +inf if it misses [0, tmax]
template <int D>
__device__ __forceinline__ float box_ray(const float lo[3], const float hi[3], P3 o, P3 inv, float tmax) {
    float t0x = (lo[0] - o.x) * inv.x, t1x = (hi[0] - o.x) * inv.x;
    float t0y = (lo[1] - o.y) * inv.y, t1y = (hi[1] - o.y) * inv.y;
    float tn = fmaxf(fminf(t0x, t1x), fminf(t0y, t1y));
    float tf = fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y));
    if constexpr (D == 3) {
        float t0z = (lo[2] - o.z) * inv.z, t1z = (hi[2] - o.z) * inv.z;
        tn = fmaxf(tn, fminf(t0z, t1z));
        tf = fminf(tf, fmaxf(t0z, t1z));
    }
    tn = fmaxf(tn, 0.f);
    tf = fminf(tf, tmax);
    return tn <= tf ? tn : INFINITY;
}

// ---------------------------------------------------------------------------
// primitives
// ---------------------------------------------------------------------------
template <int D>
struct Prim {
    P3 a, b, c;
    float area;  // 3D only (stored); 2D computed when needed
};
template <int D>
__device__ __forceinline__ Prim<D> load_prim(const float4 *prims, uint32_t k) {
    Prim<D> p;
    if constexpr (D == 2) {
        float4 q = __ldg(prims + k);
        p.a = mk(q.x, q.y, 0.f);
        p.b = mk(q.z, q.w, 0.f);
        p.c = p.b;
        p.area = 0.f;
    } else {
        float4 q0 = __ldg(prims + 3 * (size_t)k), q1 = __ldg(prims + 3 * (size_t)k + 1),
               q2 = __ldg(prims + 3 * (size_t)k + 2);
        p.a = mk(q0.x, q0.y, q0.z);
        p.b = mk(q1.x, q1.y, q1.z);
        p.c = mk(q2.x, q2.y, q2.z);
        p.area = q0.w;
    }
    return p;
}

// closest point on a segment: parameter t in [0,1]
__device__ __forceinline__ float seg_param(P3 a, P3 b, P3 x, int dimz) {
    P3 e = b - a, ap = x - a;
    float ee = e.x * e.x + e.y * e.y + (dimz ? e.z * e.z : 0.f);
    float t = __fdividef(ap.x * e.x + ap.y * e.y + (dimz ? ap.z * e.z : 0.f), ee);
    return fminf(fmaxf(t, 0.f), 1.f);
}

// closest point on triangle abc to p by Voronoi regions of the vertices,
// edges and face (Ericson, Real-Time Collision Detection, 2005, Sec. 5.1.5);
// returns barycentric weights of b and c in (v, w)
__device__ __forceinline__ P3 tri_closest(P3 a, P3 b, P3 c, P3 p, float &v, float &w) {
    P3 ab = b - a, ac = c - a, ap = p - a;
    float d1 = dotp<3>(ab, ap), d2 = dotp<3>(ac, ap);
    if (d1 <= 0.f && d2 <= 0.f) { v = 0.f; w = 0.f; return a; }
    P3 bp = p - b;
    float d3 = dotp<3>(ab, bp), d4 = dotp<3>(ac, bp);
    if (d3 >= 0.f && d4 <= d3) { v = 1.f; w = 0.f; return b; }
    float vc = d1 * d4 - d3 * d2;
    if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
        float t = __fdividef(d1, d1 - d3);
        v = t; w = 0.f;
        return a + ab * t;
    }
    P3 cp = p - c;
    float d5 = dotp<3>(ab, cp), d6 = dotp<3>(ac, cp);
    if (d6 >= 0.f && d5 <= d6) { v = 0.f; w = 1.f; return c; }
    float vb = d5 * d2 - d1 * d6;
    if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
        float t = __fdividef(d2, d2 - d6);
        v = 0.f; w = t;
        return a + ac * t;
    }
    float va = d3 * d6 - d5 * d4;
    if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {
        float t = __fdividef(d4 - d3, (d4 - d3) + (d5 - d6));
        v = 1.f - t; w = t;
        return b + (c - b) * t;
    }
    float den = __fdividef(1.f, va + vb + vc);
    v = vb * den;
    w = vc * den;
    return a + ab * v + ac * w;
}

// closest point of a primitive: returns the point, squared distance and the
// interpolation weights (2D: t along a->b in s0; 3D: weights of b, c)
template <int D>
__device__ __forceinline__ P3 prim_closest(const Prim<D> &p, P3 x, float &s0, float &s1) {
    if constexpr (D == 2) {
        float t = seg_param(p.a, p.b, x, 0);
        s0 = t;
        s1 = 0.f;
        return p.a + (p.b - p.a) * t;
    } else {
        return tri_closest(p.a, p.b, p.c, x, s0, s1);
    }
}

template <int D>
__device__ __forceinline__ P3 prim_normal(const Prim<D> &p) {
    if constexpr (D == 2) {
        P3 t = p.b - p.a;
        float il = rsqrtf(t.x * t.x + t.y * t.y);
        return mk(t.y * il, -t.x * il, 0.f);
    } else {
        P3 n = crossp(p.b - p.a, p.c - p.a);
        return n * rsqrtf(dotp<3>(n, n));
    }
}
template <int D>
__device__ __forceinline__ float prim_area(const Prim<D> &p) {
    if constexpr (D == 2) {
        P3 t = p.b - p.a;
        return sqrtf(t.x * t.x + t.y * t.y);
    } else {
        return p.area;
    }
}

// ray o + t v against a primitive, 0 < t <= tmax.  The edge tests accept a
// margin `tol` in the segment parameter / barycentric coordinates.  Q.3 uses
// kEdgeTol: with exact arithmetic a ray through a vertex shared by two
// primitives hits both, in single precision it can miss both (rounding
// errors of order 1e-5 in these parameters for the short segments of the
// workloads), and the walk would cross the boundary through that gap.  The
// visibility test uses no margin (a margin there would hide samples next to
// a vertex).
constexpr float kEdgeTol = 1e-4f;
template <int D>
__device__ __forceinline__ bool prim_ray(const Prim<D> &p, P3 o, P3 v, float tmax, float &t, float tol) {
    if constexpr (D == 2) {
        P3 e = p.b - p.a, ao = p.a - o;
        float den = v.x * e.y - v.y * e.x;
        if (den == 0.f) return false;
        float inv = __fdividef(1.f, den);
        float tt = (ao.x * e.y - ao.y * e.x) * inv;
        float u = (ao.x * v.y - ao.y * v.x) * inv;
        if (u < -tol || u > 1.f + tol || !(tt > 0.f) || tt > tmax) return false;
        t = tt;
        return true;
    } else {
        P3 e1 = p.b - p.a, e2 = p.c - p.a;
        P3 pv = crossp(v, e2);
        float det = dotp<3>(e1, pv);
        if (det == 0.f) return false;
        float inv = __fdividef(1.f, det);
        P3 tv = o - p.a;
        float u = dotp<3>(tv, pv) * inv;
        if (u < -tol || u > 1.f + tol) return false;
        P3 qv = crossp(tv, e1);
        float w = dotp<3>(v, qv) * inv;
        if (w < -tol || u + w > 1.f + tol) return false;
        float tt = dotp<3>(e2, qv) * inv;
        if (!(tt > 0.f) || tt > tmax) return false;
        t = tt;
        return true;
    }
}

// ---------------------------------------------------------------------------
// Q.1 closest point on the Dirichlet boundary
// ---------------------------------------------------------------------------
struct Closest {
    float d2;
    int rec;
    float s0, s1;
    P3 p;
};

template <int D, bool CN = false>
__device__ Closest q_closest(const TreeView &T, P3 x, const Stack &st, Cnt<CN> &cnt, float bound2 = INFINITY) {
    // bound2: a known upper bound on the squared distance (nodes farther away
    // are pruned from the start); the caller retries without it if nothing
    // lies within the bound
    Closest best;
    best.d2 = bound2;
    best.rec = -1;
    best.s0 = best.s1 = 0.f;
    best.p = x;
    if (T.root == WOST_EMPTY_REF) return best;
    // nearest-first depth-first search: the nearer child is visited next
    // without a stack round trip, only the farther one is pushed
    int sp = 0;
    uint32_t ref = T.root;
    if (box_dist2<D>(T.root_lo, T.root_hi, x) >= best.d2) return best;
    unsigned visits = 0;
    for (;;) {
        if (over_visit_limit(visits, T.n_nodes, st.guard, st.visit_limit)) break;
        if (is_leaf(ref)) {
            uint32_t f = leaf_first(ref), c = leaf_count(ref);
            for (uint32_t k = f; k < f + c; ++k) {
                cnt.prim(C_Q1);
                Prim<D> p = load_prim<D>(T.prims, k);
                float s0, s1;
                P3 q = prim_closest<D>(p, x, s0, s1);
                P3 dq = q - x;
                float d2 = dotp<D>(dq, dq);
                if (d2 < best.d2) {
                    best.d2 = d2;
                    best.rec = (int)k;
                    best.s0 = s0;
                    best.s1 = s1;
                    best.p = q;
                }
            }
        } else {
            cnt.node(C_Q1);
            Node<D> n = load_node<D>(T.nodes, ref);
            float d0 = box_dist2<D>(n.lo0, n.hi0, x), d1 = box_dist2<D>(n.lo1, n.hi1, x);
            bool h0 = d0 < best.d2, h1 = d1 < best.d2;
            if (h0 && h1) {
                bool first0 = d0 <= d1;
                spush(st, sp, first0 ? n.r1 : n.r0, first0 ? d1 : d0);
                ref = first0 ? n.r0 : n.r1;
                continue;
            }
            if (h0 || h1) {
                ref = h0 ? n.r0 : n.r1;
                continue;
            }
        }
        // next pending subtree that can still hold something closer
        float key = INFINITY;
        while (sp > 0) {
            spop(st, sp, ref, key);
            if (key < best.d2) break;
        }
        if (!(key < best.d2)) break;
    }
    return best;
}

// ---------------------------------------------------------------------------
// Q.2 closest visibility-silhouette point within rmax (Algs. 2-4)
// ---------------------------------------------------------------------------
// Alg. 4 HasSilhouette, conservative, without inverse trigonometry: the view
// cone of the box (axis to its centre, half angle asin(rb/l)) and the normal
// cone (axis a, half angle th) contain orthogonal directions iff the angle phi
// between the axes satisfies |phi - pi/2| <= th + th_v, i.e. (when the sum is
// below pi/2) |cos phi| <= sin(th + th_v).
template <int D>
__device__ __forceinline__ bool has_silhouette(const float lo[3], const float hi[3], float4 cone, P3 x) {
    float ct = cone.w;
    if (ct <= 0.f) return true;  // normal cone half angle >= 90 degrees
    P3 c = mk(0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]), 0.5f * (lo[2] + hi[2]));
    P3 av = c - x;
    float l2 = dotp<D>(av, av);
    P3 ext = mk(hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]);
    float rb2 = 0.25f * dotp<D>(ext, ext);
    if (l2 <= rb2 * 1.0001f) return true;  // bounding sphere contains x
    float il = rsqrtf(l2);
    float sv = sqrtf(rb2) * il, cv = sqrtf(fmaxf(0.f, 1.f - sv * sv));
    float st = sqrtf(fmaxf(0.f, 1.f - ct * ct));
    float cos_sum = ct * cv - st * sv;
    if (cos_sum <= 1e-6f) return true;  // combined half angle >= 90 degrees
    float sin_sum = st * cv + ct * sv;
    float cphi = (cone.x * av.x + cone.y * av.y + (D == 3 ? cone.z * av.z : 0.f)) * il;
    return fabsf(cphi) <= sin_sum + 1e-5f;
}

template <int D>
__device__ __forceinline__ float4 load_cone(const float4 *cones, uint32_t i, int which) {
    return __ldg(cones + 2 * (size_t)i + which);
}

// silhouette candidate k: distance from x if it is a silhouette, else +inf
template <int D>
__device__ __forceinline__ float sil_test(const float4 *prims, uint32_t k, P3 x, float r2) {
    P3 pe, n0, n1;
    if constexpr (D == 2) {
        float4 q0 = __ldg(prims + 2 * (size_t)k), q1 = __ldg(prims + 2 * (size_t)k + 1);
        pe = mk(q0.x, q0.y, 0.f);
        n0 = mk(q1.x, q1.y, 0.f);
        n1 = mk(q1.z, q1.w, 0.f);
    } else {
        float4 q0 = __ldg(prims + 3 * (size_t)k), q1 = __ldg(prims + 3 * (size_t)k + 1),
               q2 = __ldg(prims + 3 * (size_t)k + 2);
        P3 a = mk(q0.x, q0.y, q0.z), b = mk(q1.x, q1.y, q1.z);
        n0 = mk(q0.w, q1.w, q2.x);
        n1 = mk(q2.y, q2.z, q2.w);
        float t = seg_param(a, b, x, 1);
        pe = a + (b - a) * t;
    }
    P3 v = pe - x;
    float d2 = dotp<D>(v, v);
    if (d2 >= r2) return INFINITY;
    // Eq. SilhouetteDefinition; n1 = 0 for boundary vertices/edges
    if (dotp<D>(v, n0) * dotp<D>(v, n1) <= 0.f) return d2;
    return INFINITY;
}

template <int D, bool CN = false>
__device__ float q_silhouette(const TreeView &T, P3 x, float rmax, const Stack &st, Cnt<CN> &cnt) {
    float r2 = rmax * rmax;
    if (T.root == WOST_EMPTY_REF) return rmax;
    int sp = 0;
    float d0 = box_dist2<D>(T.root_lo, T.root_hi, x);
    if (d0 >= r2) return rmax;
    if (d0 > 0.f && !has_silhouette<D>(T.root_lo, T.root_hi, T.root_cone, x)) return rmax;
    bool found = false;
    uint32_t ref = T.root;
    unsigned visits = 0;
    for (;;) {
        if (over_visit_limit(visits, T.n_nodes, st.guard, st.visit_limit)) break;
        if (is_leaf(ref)) {
            uint32_t f = leaf_first(ref), c = leaf_count(ref);
            for (uint32_t k = f; k < f + c; ++k) {
                cnt.prim(C_Q2);
                float d2 = sil_test<D>(T.prims, k, x, r2);
                if (d2 < r2) {
                    r2 = d2;
                    found = true;
                }
            }
        } else {
            cnt.node(C_Q2);
            Node<D> n = load_node<D>(T.nodes, ref);
            float e0 = box_dist2<D>(n.lo0, n.hi0, x), e1 = box_dist2<D>(n.lo1, n.hi1, x);
            bool v0 = e0 < r2, v1 = e1 < r2;
            if (v0 && e0 > 0.f) v0 = has_silhouette<D>(n.lo0, n.hi0, load_cone<D>(T.cones, ref, 0), x);
            if (v1 && e1 > 0.f) v1 = has_silhouette<D>(n.lo1, n.hi1, load_cone<D>(T.cones, ref, 1), x);
            if (v0 && v1) {
                bool first0 = e0 <= e1;
                spush(st, sp, first0 ? n.r1 : n.r0, first0 ? e1 : e0);
                ref = first0 ? n.r0 : n.r1;
                continue;
            }
            if (v0 || v1) {
                ref = v0 ? n.r0 : n.r1;
                continue;
            }
        }
        float key = INFINITY;
        while (sp > 0) {
            spop(st, sp, ref, key);
            if (key < r2) break;
        }
        if (!(key < r2)) break;
    }
    return found ? sqrtf(r2) : rmax;
}

// ---------------------------------------------------------------------------
// Q.3 ray against the Neumann boundary (closest hit / any hit)
// ---------------------------------------------------------------------------
// any = true: stop at the first hit found (visibility test).  One out-of-line
// copy serves both uses (code size, see philox10).
template <int D, bool CN = false>
__device__ __noinline__ int q_ray(const TreeView &T, P3 o, P3 v, float tmax, int skip, bool any, float &t_out,
                                  const Stack &st, Cnt<CN> &cnt) {
    const int cq = any ? C_VIS : C_Q3;
    const bool ANY = any;
    const float tol = any ? 0.f : kEdgeTol;
    int hit = -1;
    if (T.root == WOST_EMPTY_REF) return -1;
    P3 inv = mk(1.f / v.x, 1.f / v.y, D == 3 ? 1.f / v.z : 0.f);
    float tb = tmax;
    int sp = 0;
    float t0 = box_ray<D>(T.root_lo, T.root_hi, o, inv, tb);
    if (t0 == INFINITY) return -1;
    uint32_t ref = T.root;
    unsigned visits = 0;
    for (;;) {
        if (over_visit_limit(visits, T.n_nodes, st.guard, st.visit_limit)) break;
        if (is_leaf(ref)) {
            uint32_t f = leaf_first(ref), c = leaf_count(ref);
            for (uint32_t k = f; k < f + c; ++k) {
                if ((int)k == skip) continue;
                cnt.prim(cq);
                Prim<D> p = load_prim<D>(T.prims, k);
                float t;
                if (prim_ray<D>(p, o, v, tb, t, tol)) {
                    tb = t;
                    hit = (int)k;
                    if (ANY) {
                        t_out = tb;
                        return hit;
                    }
                }
            }
        } else {
            cnt.node(cq);
            Node<D> n = load_node<D>(T.nodes, ref);
            float a0 = box_ray<D>(n.lo0, n.hi0, o, inv, tb), a1 = box_ray<D>(n.lo1, n.hi1, o, inv, tb);
            bool h0 = a0 != INFINITY, h1 = a1 != INFINITY;
            if (h0 && h1) {
                bool first0 = a0 <= a1;
                spush(st, sp, first0 ? n.r1 : n.r0, first0 ? a1 : a0);
                ref = first0 ? n.r0 : n.r1;
                continue;
            }
            if (h0 || h1) {
                ref = h0 ? n.r0 : n.r1;
                continue;
            }
        }
        float key = INFINITY;
        while (sp > 0) {
            spop(st, sp, ref, key);
            if (key <= tb) break;
        }
        if (!(key <= tb)) break;
    }
    t_out = tb;
    return hit;
}

// Q.3 and the visibility test of the Neumann sample in ONE traversal of the
// Neumann tree: ray A (o + t va, 0 < t <= tmaxA, closest hit, edge margin
// kEdgeTol) and, if wantB, ray B (o + t vb, 0 < t <= tmaxB, any hit, no
// margin, skipping primitive skipB).  Both start at the same origin; a node
// is visited if either ray still needs it, and each leaf primitive is loaded
// once and tested against both.  Against two separate traversals this saves
// the second loop, which the warp would otherwise run for the few lanes
// whose Neumann sample is valid.  A stack entry keeps A's entry distance
// (+inf if A misses the node) with the sign bit set when B meets the node.
// Returns A's hit record (or -1, t_out = tmaxA) and sets occB.
__device__ __forceinline__ float key_with_b(float ka, bool b) {
    return __uint_as_float(__float_as_uint(ka) | (b ? 0x80000000u : 0u));
}
template <int D, bool CN = false>
__device__ __noinline__ int q_ray2(const TreeView &T, P3 o, P3 va, float tmaxA, float &t_out, bool wantB, P3 vb,
                                   int skipB, float tmaxB, bool &occB, const Stack &st, Cnt<CN> &cnt) {
    int hit = -1;
    float tb = tmaxA;
    bool actB = wantB;
    occB = false;
    t_out = tmaxA;
    if (T.root == WOST_EMPTY_REF) return -1;
    const P3 ia = mk(1.f / va.x, 1.f / va.y, D == 3 ? 1.f / va.z : 0.f);
    const P3 ib = mk(1.f / vb.x, 1.f / vb.y, D == 3 ? 1.f / vb.z : 0.f);
    {
        float a0 = box_ray<D>(T.root_lo, T.root_hi, o, ia, tb);
        float b0 = actB ? box_ray<D>(T.root_lo, T.root_hi, o, ib, tmaxB) : INFINITY;
        if (a0 == INFINITY && b0 == INFINITY) return -1;
    }
    int sp = 0;
    uint32_t ref = T.root;
    unsigned visits = 0;
    for (;;) {
        if (over_visit_limit(visits, T.n_nodes, st.guard, st.visit_limit)) break;
        if (is_leaf(ref)) {
            uint32_t f = leaf_first(ref), c = leaf_count(ref);
            for (uint32_t k = f; k < f + c; ++k) {
                Prim<D> p = load_prim<D>(T.prims, k);
                float t;
                cnt.prim(C_Q3);
                if (prim_ray<D>(p, o, va, tb, t, kEdgeTol)) {
                    tb = t;
                    hit = (int)k;
                }
                if (actB && (int)k != skipB) {
                    cnt.prim(C_VIS);
                    if (prim_ray<D>(p, o, vb, tmaxB, t, 0.f)) {
                        occB = true;
                        actB = false;
                    }
                }
            }
        } else {
            cnt.node(C_Q3);
            Node<D> n = load_node<D>(T.nodes, ref);
            float a0 = box_ray<D>(n.lo0, n.hi0, o, ia, tb), a1 = box_ray<D>(n.lo1, n.hi1, o, ia, tb);
            bool b0 = actB && box_ray<D>(n.lo0, n.hi0, o, ib, tmaxB) != INFINITY;
            bool b1 = actB && box_ray<D>(n.lo1, n.hi1, o, ib, tmaxB) != INFINITY;
            bool h0 = a0 != INFINITY || b0, h1 = a1 != INFINITY || b1;
            if (h0 && h1) {
                bool first0 = a0 <= a1;
                spush(st, sp, first0 ? n.r1 : n.r0, first0 ? key_with_b(a1, b1) : key_with_b(a0, b0));
                ref = first0 ? n.r0 : n.r1;
                continue;
            }
            if (h0 || h1) {
                ref = h0 ? n.r0 : n.r1;
                continue;
            }
        }
        // next pending subtree that either ray still needs
        bool found = false;
        while (sp > 0) {
            float key;
            spop(st, sp, ref, key);
            if (fabsf(key) <= tb || (actB && signbit(key))) {
                found = true;
                break;
            }
        }
        if (!found) break;
    }
    t_out = tb;
    return hit;
}

// ---------------------------------------------------------------------------
// Warp-wide traversals with postponed leaves (Q.1, Q.2, Q.3 + visibility)
// ---------------------------------------------------------------------------
// All 32 lanes of the warp call these together (act = the lane has a query).
// A lane that reaches a leaf does not test it at once: it keeps the leaf
// aside and goes on descending from its stack; the leaves are tested when
// every lane either holds a leaf it cannot put aside (it already has one) or
// has nothing left.  In the node phase all active lanes run node code and in
// the leaf phase all run primitive code, instead of a warp paying for both
// in almost every iteration (a node and a leaf visit of different lanes
// serialise).  The answers are exact: pruning uses the best bound found so
// far, which is never below the true minimum, so postponing a leaf only
// visits some nodes a tighter bound would have pruned (the postponed
// traversal of Aila & Laine, HPG 2009, for nearest-point and ray queries).
// The visitors' methods are all inlined: a visitor whose method stays out of
// line must live in addressable memory, and as it refers to the kernel's
// scene parameter, the compiler then copies ~800 bytes of kernel parameters
// into every thread's local memory (measured: 2D walk kernels 960 -> 96 bytes
// of stack frame, 4.6% more walk steps/s on the Koch workload).
template <class V>
__device__ __forceinline__ bool spop_keep(const Stack &st, int &sp, uint32_t &ref, const V &vis) {
    while (sp > 0) {
        float key;
        spop(st, sp, ref, key);
        if (vis.keep(key)) return true;
    }
    return false;
}

template <int D, class V>
__device__ __forceinline__ void spec_traverse(const TreeView &T, const Stack &st, V &vis, bool alive) {
    constexpr unsigned FULL = 0xffffffffu;
    uint32_t ref = T.root, pend = 0u;
    bool have = alive, hasp = false;
    int sp = 0;
    unsigned visits = 0;
    while (__any_sync(FULL, have || hasp)) {
        for (;;) {
            const bool step = have && !(hasp && is_leaf(ref));
            if (!__any_sync(FULL, step)) break;
            if (step) {
                if (over_visit_limit(visits, T.n_nodes, st.guard, st.visit_limit)) {
                    have = false;
                    sp = 0;
                } else if (is_leaf(ref)) {
                    pend = ref;
                    hasp = true;
                    have = spop_keep(st, sp, ref, vis);
                } else {
                    vis.count_node();
                    Node<D> n = load_node<D>(T.nodes, ref);
                    bool h0, h1;
                    float k0, k1;
                    vis.children(n, ref, h0, h1, k0, k1);
                    if (h0 && h1) {
                        bool first0 = vis.first0(k0, k1);
                        spush(st, sp, first0 ? n.r1 : n.r0, first0 ? k1 : k0);
                        ref = first0 ? n.r0 : n.r1;
                    } else if (h0 || h1) {
                        ref = h0 ? n.r0 : n.r1;
                    } else {
                        have = spop_keep(st, sp, ref, vis);
                    }
                }
            }
        }
        if (hasp) {
            vis.leaf(leaf_first(pend), leaf_count(pend));
            hasp = false;
        }
    }
}

template <int D, bool CN>
struct ClosestVisitor {  // Q.1
    const TreeView &T;
    P3 x;
    Closest best;
    Cnt<CN> &cnt;
    __device__ __forceinline__ bool keep(float key) const { return key < best.d2; }
    __device__ __forceinline__ bool first0(float k0, float k1) const { return k0 <= k1; }
    __device__ __forceinline__ void count_node() { cnt.node(C_Q1); }
    __device__ __forceinline__ void children(const Node<D> &n, uint32_t, bool &h0, bool &h1, float &k0, float &k1) const {
        k0 = box_dist2<D>(n.lo0, n.hi0, x);
        k1 = box_dist2<D>(n.lo1, n.hi1, x);
        h0 = k0 < best.d2;
        h1 = k1 < best.d2;
    }
    __device__ __forceinline__ void leaf(uint32_t f, uint32_t c) {
        for (uint32_t k = f; k < f + c; ++k) {
            cnt.prim(C_Q1);
            Prim<D> p = load_prim<D>(T.prims, k);
            float s0, s1;
            P3 q = prim_closest<D>(p, x, s0, s1);
            P3 dq = q - x;
            float d2 = dotp<D>(dq, dq);
            if (d2 < best.d2) {
                best.d2 = d2;
                best.rec = (int)k;
                best.s0 = s0;
                best.s1 = s1;
                best.p = q;
            }
        }
    }
};

template <int D, bool CN = false>
__device__ Closest q_closest_w(const TreeView &T, P3 x, const Stack &st, Cnt<CN> &cnt, float bound2, bool act) {
    ClosestVisitor<D, CN> vis{T, x, {}, cnt};
    vis.best.d2 = bound2;
    vis.best.rec = -1;
    vis.best.s0 = vis.best.s1 = 0.f;
    vis.best.p = x;
    const bool alive = act && T.root != WOST_EMPTY_REF && box_dist2<D>(T.root_lo, T.root_hi, x) < bound2;
    spec_traverse<D>(T, st, vis, alive);
    return vis.best;
}

template <int D, bool CN>
struct SilhouetteVisitor {  // Q.2
    const TreeView &T;
    P3 x;
    float r2;
    bool found;
    Cnt<CN> &cnt;
    __device__ __forceinline__ bool keep(float key) const { return key < r2; }
    __device__ __forceinline__ bool first0(float k0, float k1) const { return k0 <= k1; }
    __device__ __forceinline__ void count_node() { cnt.node(C_Q2); }
    __device__ __forceinline__ void children(const Node<D> &n, uint32_t ref, bool &h0, bool &h1, float &k0, float &k1) const {
        k0 = box_dist2<D>(n.lo0, n.hi0, x);
        k1 = box_dist2<D>(n.lo1, n.hi1, x);
        h0 = k0 < r2;
        h1 = k1 < r2;
        if (h0 && k0 > 0.f) h0 = has_silhouette<D>(n.lo0, n.hi0, load_cone<D>(T.cones, ref, 0), x);
        if (h1 && k1 > 0.f) h1 = has_silhouette<D>(n.lo1, n.hi1, load_cone<D>(T.cones, ref, 1), x);
    }
    __device__ __forceinline__ void leaf(uint32_t f, uint32_t c) {
        for (uint32_t k = f; k < f + c; ++k) {
            cnt.prim(C_Q2);
            float d2 = sil_test<D>(T.prims, k, x, r2);
            if (d2 < r2) {
                r2 = d2;
                found = true;
            }
        }
    }
};

template <int D, bool CN = false>
__device__ float q_silhouette_w(const TreeView &T, P3 x, float rmax, const Stack &st, Cnt<CN> &cnt, bool act) {
    SilhouetteVisitor<D, CN> vis{T, x, rmax * rmax, false, cnt};
    bool alive = act && T.root != WOST_EMPTY_REF;
    if (alive) {
        float d0 = box_dist2<D>(T.root_lo, T.root_hi, x);
        alive = d0 < vis.r2 && (d0 == 0.f || has_silhouette<D>(T.root_lo, T.root_hi, T.root_cone, x));
    }
    spec_traverse<D>(T, st, vis, alive);
    return vis.found ? sqrtf(vis.r2) : rmax;
}

template <int D, bool CN>
struct Ray2Visitor {  // Q.3 (ray A) and the visibility of the Neumann sample (ray B)
    const TreeView &T;
    P3 o, va, vb, ia, ib;
    float tb, tmaxB;
    int skipB, hit;
    bool actB, occB;
    Cnt<CN> &cnt;
    __device__ __forceinline__ bool keep(float key) const { return fabsf(key) <= tb || (actB && signbit(key)); }
    __device__ __forceinline__ bool first0(float k0, float k1) const { return fabsf(k0) <= fabsf(k1); }
    __device__ __forceinline__ void count_node() { cnt.node(C_Q3); }
    __device__ __forceinline__ void children(const Node<D> &n, uint32_t, bool &h0, bool &h1, float &k0, float &k1) const {
        float a0 = box_ray<D>(n.lo0, n.hi0, o, ia, tb), a1 = box_ray<D>(n.lo1, n.hi1, o, ia, tb);
        bool b0 = actB && box_ray<D>(n.lo0, n.hi0, o, ib, tmaxB) != INFINITY;
        bool b1 = actB && box_ray<D>(n.lo1, n.hi1, o, ib, tmaxB) != INFINITY;
        h0 = a0 != INFINITY || b0;
        h1 = a1 != INFINITY || b1;
        k0 = key_with_b(a0, b0);
        k1 = key_with_b(a1, b1);
    }
    __device__ __forceinline__ void leaf(uint32_t f, uint32_t c) {
        for (uint32_t k = f; k < f + c; ++k) {
            Prim<D> p = load_prim<D>(T.prims, k);
            float t;
            cnt.prim(C_Q3);
            if (prim_ray<D>(p, o, va, tb, t, kEdgeTol)) {
                tb = t;
                hit = (int)k;
            }
            if (actB && (int)k != skipB) {
                cnt.prim(C_VIS);
                if (prim_ray<D>(p, o, vb, tmaxB, t, 0.f)) {
                    occB = true;
                    actB = false;
                }
            }
        }
    }
};

template <int D, bool CN = false>
__device__ int q_ray2_w(const TreeView &T, P3 o, P3 va, float tmaxA, float &t_out, bool wantB, P3 vb, int skipB,
                        float tmaxB, bool &occB, const Stack &st, Cnt<CN> &cnt, bool act) {
    Ray2Visitor<D, CN> vis{T, o, va, vb, mk(1.f / va.x, 1.f / va.y, D == 3 ? 1.f / va.z : 0.f),
                           mk(1.f / vb.x, 1.f / vb.y, D == 3 ? 1.f / vb.z : 0.f), tmaxA, tmaxB, skipB, -1,
                           act && wantB, false, cnt};
    bool alive = act && T.root != WOST_EMPTY_REF;
    if (alive) {
        float a0 = box_ray<D>(T.root_lo, T.root_hi, o, vis.ia, tmaxA);
        bool b0 = vis.actB && box_ray<D>(T.root_lo, T.root_hi, o, vis.ib, tmaxB) != INFINITY;
        alive = a0 != INFINITY || b0;
    }
    spec_traverse<D>(T, st, vis, alive);
    t_out = vis.tb;
    occB = vis.occB;
    return vis.hit;
}

// ---------------------------------------------------------------------------
// Q.4 hierarchical Neumann sample (Algs. 5-6)
// ---------------------------------------------------------------------------
struct NSample {
    int rec;
    float pdf;
    P3 z;
    float s0, s1;  // interpolation weights of z on the primitive
};

template <int D, bool CN = false>
__device__ NSample q_sample(const TreeView &T, P3 x, float r, Stream &rng, Cnt<CN> &cnt) {
    NSample out;
    out.rec = -1;
    out.pdf = 0.f;
    out.z = x;
    out.s0 = out.s1 = 0.f;
    if (T.root == WOST_EMPTY_REF) return out;
    float r2 = r * r;
    if (box_dist2<D>(T.root_lo, T.root_hi, x) > r2) return out;
    uint32_t ref = T.root;
    float pdf = 1.f;
    // Alg. 6: one random child among those whose box meets the ball, weighted
    // by proximity of the box centre (a descent longer than the tree is deep
    // means a corrupt tree: no sample)
    for (int level = 0; !is_leaf(ref); ++level) {
        if (level > WOST_MAX_DEPTH) return out;
        cnt.node(C_Q4);
        Node<D> n = load_node<D>(T.nodes, ref);
        float w0 = 0.f, w1 = 0.f;
        if (box_dist2<D>(n.lo0, n.hi0, x) <= r2) {
            P3 c = mk(0.5f * (n.lo0[0] + n.hi0[0]), 0.5f * (n.lo0[1] + n.hi0[1]), 0.5f * (n.lo0[2] + n.hi0[2]));
            P3 dc = c - x;
            w0 = rsqrtf(fmaxf(dotp<D>(dc, dc), 1e-24f));
        }
        if (box_dist2<D>(n.lo1, n.hi1, x) <= r2) {
            P3 c = mk(0.5f * (n.lo1[0] + n.hi1[0]), 0.5f * (n.lo1[1] + n.hi1[1]), 0.5f * (n.lo1[2] + n.hi1[2]));
            P3 dc = c - x;
            w1 = rsqrtf(fmaxf(dotp<D>(dc, dc), 1e-24f));
        }
        float tot = w0 + w1;
        if (!(tot > 0.f)) return out;
        float p0 = __fdividef(w0, tot);  // the decision and the pdf use this same p0
        if (rng.next() < p0) {
            pdf *= p0;
            ref = n.r0;
        } else {
            pdf *= 1.f - p0;
            ref = n.r1;
        }
    }
    // Alg. 6 leaf: reservoir choice proportional to area among primitives
    // meeting the ball
    uint32_t f = leaf_first(ref), c = leaf_count(ref);
    float total = 0.f;
    int chosen = -1;
    Prim<D> cp;
    for (uint32_t k = f; k < f + c; ++k) {
        cnt.prim(C_Q4);
        Prim<D> p = load_prim<D>(T.prims, k);
        float s0, s1;
        P3 q = prim_closest<D>(p, x, s0, s1);
        P3 dq = q - x;
        if (dotp<D>(dq, dq) <= r2) {
            float A = prim_area<D>(p);
            total += A;
            if (rng.next() * total < A) {
                chosen = (int)k;
                cp = p;
            }
        }
    }
    if (chosen < 0) return out;
    // Alg. 5: uniform point on the chosen primitive
    if constexpr (D == 2) {
        float u = rng.next();
        out.z = cp.a + (cp.b - cp.a) * u;
        out.s0 = u;
        out.s1 = 0.f;
        out.pdf = pdf / total;
    } else {
        float u1 = rng.next(), u2 = rng.next();
        float su = sqrtf(u1);
        float wb = su * (1.f - u2), wc = su * u2;
        out.z = cp.a * (1.f - su) + cp.b * wb + cp.c * wc;
        out.s0 = wb;
        out.s1 = wc;
        out.pdf = pdf / total;
    }
    out.rec = chosen;
    return out;
}

// ---------------------------------------------------------------------------
// exact solutions used as analytic boundary data (g = u, h = grad u . n,
// f = -Lap u)
// ---------------------------------------------------------------------------
template <int D>
__device__ __noinline__ float fn_u(int fn, const float *p, P3 x) {
    switch (fn) {
    case 1: return m_exp(x.x) * m_cos(x.y);
    case 2: return m_sin(2.f * x.x) * m_cos(3.f * x.y);
    case 3: return x.x * x.x - x.y * x.y + 0.5f * x.z;
    case 4: return (1.f - (x.x * x.x + x.y * x.y + x.z * x.z)) / (2.f * D);
    case 5: return p[0] + p[1] * x.x + p[2] * x.y + p[3] * x.z;
    case 6: {
        P3 d = x - mk(p[2], p[3], D == 3 ? p[4] : 0.f);
        float rho = sqrtf(dotp<D>(d, d));
        return D == 2 ? p[0] + p[1] * m_log(rho) : p[0] + p[1] / rho;
    }
    case 7: return p[0] * m_exp(p[1] * x.x + p[2] * x.y + p[3] * x.z);
    default: return 0.f;
    }
}
template <int D>
__device__ __noinline__ P3 fn_grad(int fn, const float *p, P3 x) {
    switch (fn) {
    case 1: {
        float e = m_exp(x.x);
        float2 sc = m_sincos(x.y);
        return mk(e * sc.y, -e * sc.x, 0.f);
    }
    case 2: {
        float2 a2 = m_sincos(2.f * x.x), a3 = m_sincos(3.f * x.y);
        return mk(2.f * a2.y * a3.y, -3.f * a2.x * a3.x, 0.f);
    }
    case 3: return mk(2.f * x.x, -2.f * x.y, 0.5f);
    case 4: return x * (-1.f / D);
    case 5: return mk(p[1], p[2], p[3]);
    case 6: {
        P3 d = x - mk(p[2], p[3], D == 3 ? p[4] : 0.f);
        float rho2 = dotp<D>(d, d);
        return D == 2 ? d * (p[1] / rho2) : d * (-p[1] / (rho2 * sqrtf(rho2)));
    }
    case 7: {
        float u = p[0] * m_exp(p[1] * x.x + p[2] * x.y + p[3] * x.z);
        return mk(u * p[1], u * p[2], u * p[3]);
    }
    default: return mk(0.f, 0.f, 0.f);
    }
}
template <int D>
__device__ __noinline__ float fn_neglap(int fn, const float *p, P3 x) {
    if (fn == 2) return 13.f * m_sin(2.f * x.x) * m_cos(3.f * x.y);
    if (fn == 4) return 1.f;
    if (fn == 7) return -(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]) * p[0] * m_exp(p[1] * x.x + p[2] * x.y + p[3] * x.z);
    return 0.f;
}

// ---------------------------------------------------------------------------
// screened Poisson equation (App. A.2): the ball's Green's function and the
// step weight Q, defined in wost_screened.cuh (screened translation unit only)
// ---------------------------------------------------------------------------
template <int D>
__device__ __noinline__ float screened_green(float rho, float R, float sqs);
template <int D>
__device__ __noinline__ float screened_q(float rho, float R, float sqs);

template <int D>
__device__ __forceinline__ float corner_interp(const float4 *data, int rec, float s0, float s1) {
    if constexpr (D == 2) {
        float2 v = __ldg(reinterpret_cast<const float2 *>(data) + rec);
        return v.x + (v.y - v.x) * s0;
    } else {
        float4 v = __ldg(data + rec);
        return v.x * (1.f - s0 - s1) + v.y * s0 + v.z * s1;
    }
}

template <int D>
__device__ __noinline__ float grid_eval(const FieldView &f, P3 y) {
    float c[3] = {y.x, y.y, y.z};
    int i0[3] = {0, 0, 0};
    float fr[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        int n = f.dims[a];
        float g = (c[a] - f.origin[a]) / f.spacing[a];
        g = fminf(fmaxf(g, 0.f), (float)(n - 1));
        int i = min((int)floorf(g), max(n - 2, 0));
        i0[a] = i;
        fr[a] = n >= 2 ? g - (float)i : 0.f;
    }
    float acc = 0.f;
#pragma unroll
    for (int m = 0; m < (1 << D); ++m) {
        float w = 1.f;
        int idx[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            int bit = (m >> a) & 1;
            idx[a] = i0[a] + (f.dims[a] >= 2 ? bit : 0);
            w *= bit ? fr[a] : 1.f - fr[a];
        }
        size_t lin = (size_t)idx[0] + (size_t)f.dims[0] * ((size_t)idx[1] + (D == 3 ? (size_t)f.dims[1] * idx[2] : 0));
        acc += w * __ldg(f.grid + lin);
    }
    return acc;
}

// ---------------------------------------------------------------------------
// one walk
// ---------------------------------------------------------------------------
struct Walk {
    P3 x, n;
    float acc;
    float dbound;  // upper bound on d_D at x: previous d_D + length of the move
    int steps;
    bool onN, capped;
    uint32_t point, index;
};

__device__ __forceinline__ float maxabs3(P3 a) { return fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z))); }

// Query policy over the binary trees: each lane answers its own walk's
// queries with its own shared-memory stack.
template <int D, bool CN>
struct LaneQ {
    Stack st;
    Cnt<CN> &cnt;
    __device__ Closest closest(const TreeView &T, P3 x, float bound2) { return q_closest<D, CN>(T, x, st, cnt, bound2); }
    __device__ float silhouette(const TreeView &T, P3 x, float rmax) { return q_silhouette<D, CN>(T, x, rmax, st, cnt); }
    __device__ int ray(const TreeView &T, P3 o, P3 v, float tmax, int skip, bool any, float &t) {
        return q_ray<D, CN>(T, o, v, tmax, skip, any, t, st, cnt);
    }
    __device__ NSample sample(const TreeView &T, P3 x, float r, Stream &rng) { return q_sample<D, CN>(T, x, r, rng, cnt); }
    __device__ int ray2(const TreeView &T, P3 o, P3 va, float tmaxA, float &t, bool wantB, P3 vb, int skipB,
                        float tmaxB, bool &occB) {
        return q_ray2<D, CN>(T, o, va, tmaxA, t, wantB, vb, skipB, tmaxB, occB, st, cnt);
    }
    // warp-wide forms: every lane of the warp calls them (act = has a query).
    // Postponed leaves in 2D only: there they gain ~9% on the Koch workload;
    // in 3D (cube + noisy torus) they halve the rate, the silhouette query
    // visiting far more nodes before its bound tightens.
    static constexpr bool kPostpone = WOST_POSTPONE_LEAVES && D == 2;
    __device__ Closest closest_w(const TreeView &T, P3 x, float bound2, bool act) {
        if constexpr (kPostpone) {
            return q_closest_w<D, CN>(T, x, st, cnt, bound2, act);
        } else {
            Closest c;
            c.d2 = bound2;
            c.rec = -1;
            c.s0 = c.s1 = 0.f;
            c.p = x;
            if (act) c = closest(T, x, bound2);
            return c;
        }
    }
    __device__ float silhouette_w(const TreeView &T, P3 x, float rmax, bool act) {
        if constexpr (kPostpone) {
            return q_silhouette_w<D, CN>(T, x, rmax, st, cnt, act);
        } else {
            return act ? silhouette(T, x, rmax) : rmax;
        }
    }
    __device__ int ray2_w(const TreeView &T, P3 o, P3 va, float tmaxA, float &t, bool wantB, P3 vb, int skipB,
                          float tmaxB, bool &occB, bool act) {
        if constexpr (kPostpone) {
            return q_ray2_w<D, CN>(T, o, va, tmaxA, t, wantB, vb, skipB, tmaxB, occB, st, cnt, act);
        } else {
            t = tmaxA;
            occB = false;
            return act ? ray2(T, o, va, tmaxA, t, wantB, vb, skipB, tmaxB, occB) : -1;
        }
    }
};

// R13: inside the grown bounding box (false for a non-finite position)
template <int D>
__device__ __forceinline__ bool in_bounds(const SceneView &sc, P3 x) {
    bool in = x.x >= sc.out_lo[0] && x.x <= sc.out_hi[0] && x.y >= sc.out_lo[1] && x.y <= sc.out_hi[1];
    if constexpr (D == 3) in = in && x.z >= sc.out_lo[2] && x.z <= sc.out_hi[2];
    return in;
}

// One iteration of Alg. 1 for the walk w of this lane (act = the lane holds
// a walk).  Returns true when an active walk has terminated (its estimate is
// then w.acc).  Q answers the geometric queries (LaneQ: one lane per walk;
// GroupQ: 8 cooperating lanes per walk, every lane of the group running this
// same code on the same walk).
//
// Warp-synchronous: all 32 lanes of the warp call it together, and the warp
// meets at a __syncwarp() after every query.  Without those meeting points
// the lanes that finish a traversal early run ahead into the next query
// while the others are still traversing, and the warp splits into small
// groups that each issue the whole step on their own (measured: 5 of 32
// lanes per query call on the Koch workload, 2 in 3D).  Inactive lanes only
// take part in the meetings; every __syncwarp() here is reached by every
// lane (conditions on it are warp-uniform).
//
// SCR: compiled with the screened-equation terms (R15); the Poisson-only
// instantiation keeps them, and their registers, out of the hot loop.
template <int D, bool SCR, class Q>
__device__ bool walk_step(const SceneView &sc, const SolveParams &sp, Walk &w, Q &q, bool act) {
    constexpr unsigned FULL = 0xffffffffu;
    // R13: a walk outside the grown bounding box of the boundary has left the
    // domain through a rounding gap; it ends like a capped walk (R5)
    const bool lost = act && !in_bounds<D>(sc, w.x);
    // distance to the Dirichlet boundary (Q.1).  The closest point of the
    // previous step is at most dbound away (triangle inequality), which
    // prunes the search; the result is the exact closest point either way,
    // and a walk whose bound excluded everything searches again without it.
    const float b = w.dbound * 1.0001f + 1e-6f;
    Closest cl;
    cl.d2 = INFINITY;
    cl.rec = -1;
    cl.s0 = cl.s1 = 0.f;
    cl.p = w.x;
    bool need = act;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {  // one call site keeps the code small
        if (!__any_sync(FULL, need)) break;
        Closest c = q.closest_w(sc.D, w.x, pass == 0 ? b * b : INFINITY, need);
        if (need) {
            cl = c;
            need = cl.rec < 0;
        }
        __syncwarp();
    }
    bool ended = false;
    const float dD = sqrtf(cl.d2);
    if (act) {
        w.steps += 1;
        if (dD < sp.epsilon || w.steps >= sp.max_steps || lost) {
            // epsilon shell: g at the closest point (R5: also at the step cap)
            w.capped = !(dD < sp.epsilon);
            if (cl.rec >= 0) {
                // App. B: on a double-sided primitive, the - side's data if x
                // lies on the side its normal points into
                const float4 *gd = sc.D.data;
                if (sc.D.sided && sc.D.sided[cl.rec] &&
                    !(dotp<D>(cl.p - w.x, prim_normal<D>(load_prim<D>(sc.D.prims, (uint32_t)cl.rec))) > 0.f))
                    gd = sc.D.data_minus;
                float gv = sc.g.kind == FIELD_ANALYTIC ? fn_u<D>(sc.g.fn, sc.g.params, cl.p)
                                                       : corner_interp<D>(gd, cl.rec, cl.s0, cl.s1);
                w.acc += gv;
            }
            ended = true;
        }
    }
    act = act && !ended;
    // R4: query origin off the Neumann boundary
    const float delta = sp.offset * (1.f + maxabs3(w.x));
    const P3 xq = w.onN ? w.x - w.n * delta : w.x;
    // distance to the visibility silhouette (Q.2) within d_D, star radius (R3)
    float dsil = q.silhouette_w(sc.S, xq, dD, act);
    if (!act) dsil = dD;
    __syncwarp();
    float r = fminf(dD, fmaxf(sp.r_min, dsil));
    // R14: at most the scene's diameter, which matters only without Dirichlet
    // data; such scenes are solved with sigma > 0, i.e. in the screened
    // instantiation (with Dirichlet data, r <= d_D <= the diameter anyway)
    if constexpr (SCR) r = fminf(r, sc.rmax);
    // screening of this step (R15: from step screen_after on)
    float sqs = 0.f;
    if constexpr (SCR) sqs = (sp.sigma > 0.f && w.steps - 1 >= sp.screen_after) ? sp.sqrt_sigma : 0.f;
    // direction: uniform, flipped into the hemisphere about -n_x on the boundary
    const uint32_t k = (uint32_t)(w.steps - 1);
    uint4 rb = make_uint4(0u, 0u, 0u, 0u);
    if (act) rb = philox10(make_uint4(w.index, w.point, k, 0u), sp.key0, sp.key1);
    P3 v;
    if constexpr (D == 2) {
        float s, c;
        sincospif(2.f * u01(rb.x), &s, &c);
        v = mk(c, s, 0.f);
    } else {
        float zc = 1.f - 2.f * u01(rb.x);
        float rr = sqrtf(fmaxf(0.f, 1.f - zc * zc));
        float s, c;
        sincospif(2.f * u01(rb.y), &s, &c);
        v = mk(rr * c, rr * s, zc);
    }
    if (w.onN && dotp<D>(w.n, v) > 0.f) v = v * -1.f;
    // Neumann contribution from a separate sample z (Q.4) if h is present
    const bool hzero = sc.h.kind == FIELD_ANALYTIC && sc.h.fn == 0;
    const bool want4 = act && !hzero && sc.N.root != WOST_EMPTY_REF;
    NSample zs;
    zs.rec = -1;
    zs.pdf = 0.f;
    zs.z = w.x;
    zs.s0 = zs.s1 = 0.f;
    if (__any_sync(FULL, want4)) {
        if (want4) {
            Stream rng;
            rng.init(sp.key0, sp.key1, w.index, w.point, k);
            zs = q.sample(sc.N, w.x, r, rng);
        }
        __syncwarp();
    }
    // R12: a sample at zero distance (x and z rounded onto the same point of
    // one primitive) has G = inf and measure zero: skipped
    const P3 dz = zs.z - w.x;
    const float dzl = sqrtf(dotp<D>(dz, dz));
    const bool wantv = want4 && zs.rec >= 0 && zs.pdf > 0.f && dzl < r && dzl > 0.f;
    // first hit with the Neumann part of the star boundary (Q.3) and the
    // visibility of z (one traversal for both rays)
    float th = r;
    bool occ = false;
    int hrec = q.ray2_w(sc.N, xq, v, r, th, wantv, zs.z - xq, zs.rec, sp.vis_tmax, occ, act);
    if (!act) hrec = -1;
    __syncwarp();
    if (!act) return ended;
    P3 p, np = mk(0.f, 0.f, 0.f);
    if (hrec >= 0) {
        p = xq + v * th;
        np = prim_normal<D>(load_prim<D>(sc.N.prims, (uint32_t)hrec));
        // App. B: a double-sided sheet is hit from the side the walk is on;
        // its outward normal there is the one the walk moves along
        if (sc.N.sided && sc.N.sided[hrec] && dotp<D>(v, np) < 0.f) np = np * -1.f;
    } else {
        p = w.x + v * r;
    }
    float Nterm = 0.f;
    if (wantv && !occ) {
        float hv;
        // App. B: the data of the side of a double-sided sheet that faces the
        // query point (offset onto the walk's side when it lies on a sheet)
        const bool minus = sc.N.sided && sc.N.sided[zs.rec] &&
                           !(dotp<D>(zs.z - xq, prim_normal<D>(load_prim<D>(sc.N.prims, (uint32_t)zs.rec))) > 0.f);
        if (sc.h.kind == FIELD_ANALYTIC) {
            P3 nz = prim_normal<D>(load_prim<D>(sc.N.prims, (uint32_t)zs.rec));
            hv = dotp<D>(fn_grad<D>(sc.h.fn, sc.h.params, zs.z), minus ? nz * -1.f : nz);
        } else {
            hv = corner_interp<D>(minus ? sc.N.data_minus : sc.N.data, zs.rec, zs.s0, zs.s1);
        }
        float G = D == 2 ? m_log(__fdividef(r, dzl)) * (0.5f / 3.14159265358979f)
                         : (1.f / dzl - 1.f / r) * (0.25f / 3.14159265358979f);
        if constexpr (SCR) {
            if (sqs > 0.f) G = screened_green<D>(dzl, r, sqs);
        }
        float alpha = w.onN ? 0.5f : 1.f;
        Nterm = G * hv / (alpha * zs.pdf);
    }
    // source contribution, reusing the direction v (Sec. 4.6)
    float Sterm = 0.f;
    if (sc.f.kind != FIELD_NONE) {
        float ts;
        if constexpr (D == 2) {
            ts = r * sqrtf(u01(rb.y) * u01(rb.z));
        } else {
            ts = r * (0.5f + m_sin(m_asin(2.f * u01(rb.z) - 1.f) * (1.f / 3.f)));
        }
        P3 pd = p - w.x;
        if (ts * ts < dotp<D>(pd, pd)) {
            P3 y = w.x + v * ts;
            float fv = sc.f.kind == FIELD_ANALYTIC ? fn_neglap<D>(sc.f.fn, sc.f.params, y) : grid_eval<D>(sc.f, y);
            float wS = (D == 2 ? 0.25f : (1.f / 6.f)) * r * r;
            if constexpr (SCR) {
                if (sqs > 0.f) {  // R15: the unscreened sample reweighted by G^sigma_B / G_B
                    float G0 = D == 2 ? m_log(__fdividef(r, ts)) * (0.5f / 3.14159265358979f)
                                      : (1.f / ts - 1.f / r) * (0.25f / 3.14159265358979f);
                    wS *= screened_green<D>(ts, r, sqs) / G0;
                }
            }
            Sterm = wS * fv;
        }
    }
    // R1: the step adds the Neumann and source terms
    w.acc += Nterm + Sterm;
    P3 mv = p - w.x;
    float moved = sqrtf(dotp<D>(mv, mv));
    // R15: a screened walk goes on to p with probability Q^sigma_B(x, p)
    // (Russian roulette on the fourth uniform of slot 0), else it ends here
    if constexpr (SCR) {
        if (sqs > 0.f && u01(rb.w) >= screened_q<D>(moved, r, sqs)) return true;
    }
    w.dbound = dD + moved;
    w.x = p;
    w.n = np;
    w.onN = hrec >= 0;
    return false;
}

template <int D>
__device__ __forceinline__ P3 load_point(const float *pts, int64_t i) {
    if constexpr (D == 2) {
        return mk(pts[2 * i], pts[2 * i + 1], 0.f);
    } else {
        return mk(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
    }
}

template <int D>
__device__ __forceinline__ void walk_init(const SolveParams &sp, Walk &w, int64_t point, uint32_t index) {
    w.x = load_point<D>(sp.points, point);
    w.onN = sp.on_neumann ? sp.on_neumann[point] != 0 : false;
    w.n = (w.onN && sp.normals) ? load_point<D>(sp.normals, point) : mk(0.f, 0.f, 0.f);
    w.acc = 0.f;
    w.dbound = INFINITY;
    w.steps = 0;
    w.capped = false;
    w.point = (uint32_t)point;
    w.index = index;
}

}  // namespace wost
