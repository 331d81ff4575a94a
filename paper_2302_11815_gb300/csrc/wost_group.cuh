// Group-cooperative queries on the 8-wide trees (Sec. 5 queries Q.1-Q.4).
//
// A walk is owned by a team of 8 consecutive lanes of a warp.  All 8 lanes
// run the same walk code on the same walk state; inside a query, lane j tests
// child j of the current node (or primitives j and j + 8 of the current
// leaf), and the team combines the answers with shuffles inside its 8-lane
// mask.  Every branch that steers the traversal is therefore uniform within
// the team, and divergence is left only between the 4 teams of a warp.  Each
// team has one traversal stack in shared memory; the subtrees other than the
// one visited next are pushed farthest first, so that the nearest is popped
// first.
#pragma once

#include "wost_device.cuh"

namespace wost {

__device__ __forceinline__ bool ref_empty(uint32_t r) { return r == WOST_EMPTY_REF; }

// one team's traversal stack: entry i at base[i]
struct GStack {
    int2 *base;
    int cap;
    unsigned int *guard;
};

struct Group {
    unsigned mask;  // the team's lanes
    int base;       // first lane of the team in the warp
    int gl;         // this lane's index in the team
    __device__ __forceinline__ bool leader() const { return gl == 0; }
};

template <class T>
__device__ __forceinline__ T gshfl(const Group &g, T v, int src) {
    return __shfl_sync(g.mask, v, g.base + src);
}
__device__ __forceinline__ unsigned gballot(const Group &g, bool p) { return __ballot_sync(g.mask, p) >> g.base; }

// index (0..7) of the smallest value over the team; ties: lowest index
__device__ __forceinline__ int gargmin(const Group &g, float v) {
    int who = g.gl;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        float ov = __shfl_xor_sync(g.mask, v, o);
        int ow = __shfl_xor_sync(g.mask, who, o);
        if (ov < v || (ov == v && ow < who)) {
            v = ov;
            who = ow;
        }
    }
    return who;
}

// inclusive prefix sum over the team
__device__ __forceinline__ float gscan(const Group &g, float v) {
#pragma unroll
    for (int o = 1; o < WOST_WIDE; o <<= 1) {
        float t = __shfl_up_sync(g.mask, v, o);
        if (g.gl >= o) v += t;
    }
    return v;
}

// one child slot of a wide node: box and reference
struct WChild {
    float lo[3], hi[3];
    uint32_t ref;
};
__device__ __forceinline__ WChild load_wchild(const float4 *wnodes, uint32_t node, int c) {
    const float4 *q = wnodes + (size_t)node * (2 * WOST_WIDE) + 2 * c;
    float4 a = __ldg(q), b = __ldg(q + 1);
    WChild w;
    w.lo[0] = a.x; w.lo[1] = a.y; w.lo[2] = a.z;
    w.hi[0] = b.x; w.hi[1] = b.y; w.hi[2] = b.z;
    w.ref = __float_as_uint(a.w);
    return w;
}

// Team step at an inner node: among the children with `hit`, goes to the one
// with the smallest key and pushes the others, largest key deepest.  Returns
// false if no child was hit.
__device__ __forceinline__ bool gdescend(const Group &g, const GStack &gs, int &sp, uint32_t &ref, bool hit,
                                         uint32_t cref, float key) {
    unsigned hits = gballot(g, hit);
    if (!hits) return false;
    int next = gargmin(g, hit ? key : INFINITY);
    ref = gshfl(g, cref, next);
    unsigned others = hits & ~(1u << next);
    if (others) {
        // rank among the pushed children by (key, index), descending
        bool mine = (others >> g.gl) & 1u;
        float k = mine ? key : -INFINITY;
        int rank = 0;
#pragma unroll
        for (int o = 1; o < WOST_WIDE; ++o) {
            int j = (g.gl + o) & (WOST_WIDE - 1);
            float kj = __shfl_sync(g.mask, k, g.base + j);
            rank += (kj > k || (kj == k && j > g.gl)) ? 1 : 0;
        }
        int n = __popc(others);
        if (mine) {
            int pos = sp + rank;
            if (pos < gs.cap) gs.base[pos] = make_int2((int)cref, __float_as_int(key));
        }
        if (sp + n > gs.cap) {
            if (g.leader()) atomicOr(gs.guard, 1u);  // overflow: recorded, entries dropped (no fault)
            n = gs.cap - sp;
        }
        sp += n;
        __syncwarp(g.mask);
    }
    return true;
}

// Pops entries until one has key < bound (INCL: key <= bound).  Returns
// false when the stack is exhausted.
template <bool INCL>
__device__ __forceinline__ bool gpop(const GStack &gs, int &sp, uint32_t &ref, float bound) {
    while (sp > 0) {
        --sp;
        int2 e = gs.base[sp];
        float key = __int_as_float(e.y);
        if (INCL ? key <= bound : key < bound) {
            ref = (uint32_t)e.x;
            return true;
        }
    }
    return false;
}

template <int D, bool CN>
struct GroupQ {
    Group g;
    GStack gs;
    Cnt<CN> &cnt;

    // Q.1 closest point on the Dirichlet boundary (bound2: as in q_closest)
    __device__ Closest closest(const TreeView &T, P3 x, float bound2) {
        Closest best;
        best.d2 = bound2;
        best.rec = -1;
        best.s0 = best.s1 = 0.f;
        best.p = x;
        if (ref_empty(T.wroot) || box_dist2<D>(T.root_lo, T.root_hi, x) >= best.d2) return best;
        uint32_t ref = T.wroot;
        int sp = 0;
        unsigned visits = 0;
        for (;;) {
            if (over_visit_limit(visits, T.wn_nodes, g.leader() ? gs.guard : nullptr)) break;
            if (is_leaf(ref)) {
                uint32_t f = leaf_first(ref), c = leaf_count(ref);
                if (g.leader()) cnt.prim_n(C_Q1, c);
                float d2 = INFINITY, s0 = 0.f, s1 = 0.f;
                P3 q = x;
                int rec = -1;
                for (uint32_t j = g.gl; j < c; j += WOST_WIDE) {
                    Prim<D> p = load_prim<D>(T.prims, f + j);
                    float t0, t1;
                    P3 qq = prim_closest<D>(p, x, t0, t1);
                    P3 dq = qq - x;
                    float dd = dotp<D>(dq, dq);
                    if (dd < d2) {
                        d2 = dd;
                        s0 = t0;
                        s1 = t1;
                        q = qq;
                        rec = (int)(f + j);
                    }
                }
                int who = gargmin(g, d2);
                float m = gshfl(g, d2, who);
                if (m < best.d2) {
                    best.d2 = m;
                    best.rec = gshfl(g, rec, who);
                    best.s0 = gshfl(g, s0, who);
                    best.s1 = gshfl(g, s1, who);
                    best.p = mk(gshfl(g, q.x, who), gshfl(g, q.y, who), gshfl(g, q.z, who));
                }
            } else {
                if (g.leader()) cnt.node(C_Q1);
                WChild ch = load_wchild(T.wnodes, ref, g.gl);
                float d = ref_empty(ch.ref) ? INFINITY : box_dist2<D>(ch.lo, ch.hi, x);
                if (gdescend(g, gs, sp, ref, d < best.d2, ch.ref, d)) continue;
            }
            if (!gpop<false>(gs, sp, ref, best.d2)) break;
        }
        return best;
    }

    // Q.2 closest visibility-silhouette point within rmax (Algs. 2-4)
    __device__ float silhouette(const TreeView &T, P3 x, float rmax) {
        float r2 = rmax * rmax;
        if (ref_empty(T.wroot)) return rmax;
        float d0 = box_dist2<D>(T.root_lo, T.root_hi, x);
        if (d0 >= r2) return rmax;
        if (d0 > 0.f && !has_silhouette<D>(T.root_lo, T.root_hi, T.root_cone, x)) return rmax;
        bool found = false;
        uint32_t ref = T.wroot;
        int sp = 0;
        unsigned visits = 0;
        for (;;) {
            if (over_visit_limit(visits, T.wn_nodes, g.leader() ? gs.guard : nullptr)) break;
            if (is_leaf(ref)) {
                uint32_t f = leaf_first(ref), c = leaf_count(ref);
                if (g.leader()) cnt.prim_n(C_Q2, c);
                float d2 = INFINITY;
                for (uint32_t j = g.gl; j < c; j += WOST_WIDE) d2 = fminf(d2, sil_test<D>(T.prims, f + j, x, r2));
                int who = gargmin(g, d2);
                float m = gshfl(g, d2, who);
                if (m < r2) {
                    r2 = m;
                    found = true;
                }
            } else {
                if (g.leader()) cnt.node(C_Q2);
                WChild ch = load_wchild(T.wnodes, ref, g.gl);
                float e = ref_empty(ch.ref) ? INFINITY : box_dist2<D>(ch.lo, ch.hi, x);
                bool hit = e < r2;
                if (hit && e > 0.f)
                    hit = has_silhouette<D>(ch.lo, ch.hi, __ldg(T.wcones + (size_t)ref * WOST_WIDE + g.gl), x);
                if (gdescend(g, gs, sp, ref, hit, ch.ref, e)) continue;
            }
            if (!gpop<false>(gs, sp, ref, r2)) break;
        }
        return found ? sqrtf(r2) : rmax;
    }

    // Q.3 first hit of o + t v, 0 < t <= tmax, with the Neumann boundary
    // (any = true: any hit, for the visibility test of the Neumann sample)
    __device__ int ray(const TreeView &T, P3 o, P3 v, float tmax, int skip, bool any, float &t_out) {
        const int cq = any ? C_VIS : C_Q3;
        const float tol = any ? 0.f : kEdgeTol;
        int hit_rec = -1;
        t_out = tmax;
        if (ref_empty(T.wroot)) return -1;
        P3 inv = mk(1.f / v.x, 1.f / v.y, D == 3 ? 1.f / v.z : 0.f);
        float tb = tmax;
        if (box_ray<D>(T.root_lo, T.root_hi, o, inv, tb) == INFINITY) return -1;
        uint32_t ref = T.wroot;
        int sp = 0;
        unsigned visits = 0;
        for (;;) {
            if (over_visit_limit(visits, T.wn_nodes, g.leader() ? gs.guard : nullptr)) break;
            if (is_leaf(ref)) {
                uint32_t f = leaf_first(ref), c = leaf_count(ref);
                if (g.leader()) cnt.prim_n(cq, c);
                float t = INFINITY;
                int rec = -1;
                for (uint32_t j = g.gl; j < c; j += WOST_WIDE) {
                    int k = (int)(f + j);
                    if (k == skip) continue;
                    Prim<D> p = load_prim<D>(T.prims, (uint32_t)k);
                    float tt;
                    if (prim_ray<D>(p, o, v, fminf(tb, t), tt, tol)) {
                        t = tt;
                        rec = k;
                    }
                }
                int who = gargmin(g, t);
                float m = gshfl(g, t, who);
                if (m < tb) {
                    tb = m;
                    hit_rec = gshfl(g, rec, who);
                    if (any) break;
                }
            } else {
                if (g.leader()) cnt.node(cq);
                WChild ch = load_wchild(T.wnodes, ref, g.gl);
                float a = ref_empty(ch.ref) ? INFINITY : box_ray<D>(ch.lo, ch.hi, o, inv, tb);
                if (gdescend(g, gs, sp, ref, a != INFINITY, ch.ref, a)) continue;
            }
            if (!gpop<true>(gs, sp, ref, tb)) break;
        }
        t_out = tb;
        return hit_rec;
    }

    // Q.4 hierarchical Neumann sample (Algs. 5-6): one child per level,
    // chosen among those whose box meets the ball with probability
    // proportional to 1/(distance to the box centre); in the leaf, one
    // primitive meeting the ball proportionally to its area; then a uniform
    // point on it.  All lanes of the team draw the same uniforms.
    __device__ NSample sample(const TreeView &T, P3 x, float r, Stream &rng) {
        NSample out;
        out.rec = -1;
        out.pdf = 0.f;
        out.z = x;
        out.s0 = out.s1 = 0.f;
        float r2 = r * r;
        if (ref_empty(T.wroot) || box_dist2<D>(T.root_lo, T.root_hi, x) > r2) return out;
        uint32_t ref = T.wroot;
        float pdf = 1.f;
        for (int level = 0; !is_leaf(ref); ++level) {
            if (level > WOST_MAX_DEPTH) return out;
            if (g.leader()) cnt.node(C_Q4);
            WChild ch = load_wchild(T.wnodes, ref, g.gl);
            float w = 0.f;
            if (!ref_empty(ch.ref) && box_dist2<D>(ch.lo, ch.hi, x) <= r2) {
                P3 c = mk(0.5f * (ch.lo[0] + ch.hi[0]), 0.5f * (ch.lo[1] + ch.hi[1]), 0.5f * (ch.lo[2] + ch.hi[2]));
                P3 dc = c - x;
                w = rsqrtf(fmaxf(dotp<D>(dc, dc), 1e-24f));
            }
            float s = gscan(g, w);
            float tot = gshfl(g, s, WOST_WIDE - 1);
            if (!(tot > 0.f)) return out;
            float target = rng.next() * tot;
            unsigned valid = gballot(g, w > 0.f);
            unsigned pick = gballot(g, w > 0.f && s > target);
            // rounding can leave target >= the last partial sum: take the last valid child
            int k = pick ? __ffs(pick) - 1 : 31 - __clz(valid);
            float wk = gshfl(g, w, k);
            ref = gshfl(g, ch.ref, k);
            pdf *= wk / tot;
        }
        uint32_t f = leaf_first(ref), c = leaf_count(ref);
        if (g.leader()) cnt.prim_n(C_Q4, c);
        // areas of primitives gl and gl + 8 (0 unless present and meeting the ball)
        float A[2] = {0.f, 0.f};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t j = g.gl + h * WOST_WIDE;
            if (j < c) {
                Prim<D> p = load_prim<D>(T.prims, f + j);
                float s0, s1;
                P3 q = prim_closest<D>(p, x, s0, s1);
                P3 dq = q - x;
                if (dotp<D>(dq, dq) <= r2) A[h] = prim_area<D>(p);
            }
        }
        float s0 = gscan(g, A[0]);
        float tot0 = gshfl(g, s0, WOST_WIDE - 1);
        float s1 = gscan(g, A[1]) + tot0;
        float total = gshfl(g, s1, WOST_WIDE - 1);
        if (!(total > 0.f)) return out;
        float target = rng.next() * total;
        unsigned pick = gballot(g, A[0] > 0.f && s0 > target) | (gballot(g, A[1] > 0.f && s1 > target) << WOST_WIDE);
        unsigned valid = gballot(g, A[0] > 0.f) | (gballot(g, A[1] > 0.f) << WOST_WIDE);
        int k = pick ? __ffs(pick) - 1 : 31 - __clz(valid);
        Prim<D> cp = load_prim<D>(T.prims, f + (uint32_t)k);
        // Alg. 5: uniform point on primitive k
        if constexpr (D == 2) {
            float u = rng.next();
            out.z = cp.a + (cp.b - cp.a) * u;
            out.s0 = u;
        } else {
            float u1 = rng.next(), u2 = rng.next();
            float su = sqrtf(u1);
            float wb = su * (1.f - u2), wc = su * u2;
            out.z = cp.a * (1.f - su) + cp.b * wb + cp.c * wc;
            out.s0 = wb;
            out.s1 = wc;
        }
        out.pdf = pdf / total;
        out.rec = (int)(f + (uint32_t)k);
        return out;
    }

    // warp-wide forms (every lane of the warp calls them; act is uniform
    // within a team)
    __device__ Closest closest_w(const TreeView &T, P3 x, float bound2, bool act) {
        Closest c;
        c.d2 = bound2;
        c.rec = -1;
        c.s0 = c.s1 = 0.f;
        c.p = x;
        if (act) c = closest(T, x, bound2);
        return c;
    }
    __device__ float silhouette_w(const TreeView &T, P3 x, float rmax, bool act) {
        return act ? silhouette(T, x, rmax) : rmax;
    }
    __device__ int ray2_w(const TreeView &T, P3 o, P3 va, float tmaxA, float &t, bool wantB, P3 vb, int skipB,
                          float tmaxB, bool &occB, bool act) {
        t = tmaxA;
        occB = false;
        return act ? ray2(T, o, va, tmaxA, t, wantB, vb, skipB, tmaxB, occB) : -1;
    }

    // Q.3 and the visibility test: two traversals of the wide tree
    __device__ int ray2(const TreeView &T, P3 o, P3 va, float tmaxA, float &t, bool wantB, P3 vb, int skipB,
                        float tmaxB, bool &occB) {
        int h = ray(T, o, va, tmaxA, -1, false, t);
        occB = false;
        if (wantB) {
            float tv;
            occB = ray(T, o, vb, tmaxB, skipB, true, tv) >= 0;
        }
        return h;
    }
};

}  // namespace wost
