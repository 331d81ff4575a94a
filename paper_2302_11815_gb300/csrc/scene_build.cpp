// Host-side scene construction: validation, silhouette candidates, binned-SAH
// bounding volume hierarchies and normal cones, flattened for the device.
//
// Sec. 5 of the paper: a BVH over the Dirichlet boundary for closest-point
// queries and a spatialized normal cone hierarchy (SNCH, Sec. 5.1.1, after
// Johnson & Cohen) for the Neumann boundary, built with the surface area
// heuristic.  Here the Neumann side is split in two trees with one primitive
// type each: a BVH over Neumann primitives (rays, Q.3; sampling, Q.4) and a
// cone hierarchy over the silhouette candidates (Q.2): vertices in 2D and
// edges in 3D, each carrying the normals of its adjacent Neumann primitives
// (Eq. SilhouetteDefinition).  A node's cone bounds those normals: axis =
// normalised mean normal, half angle = largest deviation from it (Sec. 5.1.1),
// padded for single-precision tests.
#include "scene_build.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>

namespace wost {

namespace {

struct V3 {
    double x, y, z;
};
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator*(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }

struct Item {           // one primitive as seen by the builder
    float lo[3], hi[3]; // bounds
    float c[3];         // centroid
    int rec;            // index into the caller's record list
};

struct BNode {
    float lo[3], hi[3];
    int child[2];       // build-node indices, -1 for a leaf
    int first, count;   // leaf range in the item order
    int depth;
};

inline float area_measure(const float lo[3], const float hi[3], int dim) {
    float ex = std::max(0.f, hi[0] - lo[0]), ey = std::max(0.f, hi[1] - lo[1]);
    if (dim == 2) return ex + ey;
    float ez = std::max(0.f, hi[2] - lo[2]);
    return ex * ey + ey * ez + ez * ex;
}

inline void grow(float lo[3], float hi[3], const float plo[3], const float phi[3]) {
    for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], plo[a]);
        hi[a] = std::max(hi[a], phi[a]);
    }
}
inline void empty_box(float lo[3], float hi[3]) {
    for (int a = 0; a < 3; ++a) {
        lo[a] = INFINITY;
        hi[a] = -INFINITY;
    }
}

// Normal cone of a set of silhouette candidates for the orientation-aware
// split cost: unit axis and half angle theta in [0, pi] (pi: may face any
// way, e.g. a boundary edge, which is always a silhouette).
struct OCone {
    float ax, ay, az, theta;
};

// The smallest cone holding two cones (the union used by the orientation
// heuristic of light hierarchies, Estevez & Kulla 2018, Sec. 4.4).
inline OCone cone_union(const OCone &a, const OCone &b) {
    if (a.theta < 0) return b;  // empty
    if (b.theta < 0) return a;
    const float kPi = 3.14159265f;
    if (a.theta >= kPi || b.theta >= kPi) return {0, 0, 1, kPi};
    float c = std::max(-1.f, std::min(1.f, a.ax * b.ax + a.ay * b.ay + a.az * b.az));
    float d = std::acos(c);
    if (std::min(d + b.theta, kPi) <= a.theta) return a;
    if (std::min(d + a.theta, kPi) <= b.theta) return b;
    float th = 0.5f * (a.theta + d + b.theta);
    if (th >= kPi) return {0, 0, 1, kPi};
    // rotate a's axis toward b's by th - a.theta along their great circle
    float r = th - a.theta, s = std::sin(d);
    if (s < 1e-6f) return {a.ax, a.ay, a.az, th};
    float wa = std::sin(d - r) / s, wb = std::sin(r) / s;
    float x = wa * a.ax + wb * b.ax, y = wa * a.ay + wb * b.ay, z = wa * a.az + wb * b.az;
    float l = std::sqrt(x * x + y * y + z * z);
    return {x / l, y / l, z / l, th};
}

// Fraction of view directions from which a node with normal cone half angle
// theta can hold a silhouette: those within theta of being orthogonal to the
// cone's axis -- a band of the sphere of measure sin(theta) in 3D, 2 theta /
// pi of the circle in 2D -- widened a little for the view cone of a node of
// finite size.
inline float orientation_measure(float theta, int dim) {
    const float kHalfPi = 1.57079633f;
    float t = std::min(theta + 0.05f, kHalfPi);
    return dim == 3 ? std::sin(t) : t / kHalfPi;
}

// Binned SAH over items[first, first+count); reorders items in place.  With
// per-item normal cones (the silhouette candidates) the split cost is the
// surface-area-orientation heuristic: each side's area times its count times
// the orientation measure of its normal cone, so that candidates facing the
// same way are grouped and the traversal's cone test can cull them together
// (Sec. 5.1.1 names this heuristic as the way to improve the hierarchy).
class Builder {
  public:
    Builder(std::vector<Item> &items, int dim, int leaf_size, const std::vector<OCone> *cones = nullptr)
        : it_(items), dim_(dim), leaf_(leaf_size), cones_(cones) {}

    int build() {
        nodes_.reserve(2 * it_.size() + 1);
        return make(0, (int)it_.size(), 0);
    }
    std::vector<BNode> nodes_;
    int max_depth_ = 0;

  private:
    static constexpr int kBins = 32;
    std::vector<Item> &it_;
    int dim_, leaf_;
    const std::vector<OCone> *cones_;
    float measure(const OCone &c) const { return cones_ ? orientation_measure(c.theta, dim_) : 1.f; }

    int make(int first, int count, int depth) {
        int id = (int)nodes_.size();
        nodes_.push_back(BNode{});
        BNode nd;
        empty_box(nd.lo, nd.hi);
        float clo[3], chi[3];
        empty_box(clo, chi);
        for (int i = first; i < first + count; ++i) {
            grow(nd.lo, nd.hi, it_[i].lo, it_[i].hi);
            grow(clo, chi, it_[i].c, it_[i].c);
        }
        nd.child[0] = nd.child[1] = -1;
        nd.first = first;
        nd.count = count;
        nd.depth = depth;
        max_depth_ = std::max(max_depth_, depth);
        nodes_[id] = nd;
        if (count <= 1) return id;

        // best binned SAH split over all axes
        float best_cost = INFINITY;
        int best_axis = -1, best_bin = -1;
        for (int a = 0; a < dim_; ++a) {
            float ext = chi[a] - clo[a];
            if (!(ext > 0)) continue;
            float blo[kBins][3], bhi[kBins][3];
            int bcnt[kBins] = {0};
            OCone bcone[kBins];
            for (int b = 0; b < kBins; ++b) {
                empty_box(blo[b], bhi[b]);
                bcone[b] = {0, 0, 1, -1};
            }
            float scale = kBins / ext;
            for (int i = first; i < first + count; ++i) {
                int b = std::min(kBins - 1, (int)((it_[i].c[a] - clo[a]) * scale));
                bcnt[b]++;
                grow(blo[b], bhi[b], it_[i].lo, it_[i].hi);
                if (cones_) bcone[b] = cone_union(bcone[b], (*cones_)[it_[i].rec]);
            }
            float rlo[3], rhi[3];
            empty_box(rlo, rhi);
            float rarea[kBins];
            int rcnt[kBins];
            int acc = 0;
            OCone rc{0, 0, 1, -1};
            for (int b = kBins - 1; b > 0; --b) {
                grow(rlo, rhi, blo[b], bhi[b]);
                acc += bcnt[b];
                rcnt[b] = acc;
                if (cones_) rc = cone_union(rc, bcone[b]);
                rarea[b] = area_measure(rlo, rhi, dim_) * measure(rc);
            }
            float llo[3], lhi[3];
            empty_box(llo, lhi);
            int lc = 0;
            OCone lcn{0, 0, 1, -1};
            for (int b = 0; b < kBins - 1; ++b) {
                grow(llo, lhi, blo[b], bhi[b]);
                lc += bcnt[b];
                if (cones_) lcn = cone_union(lcn, bcone[b]);
                if (lc == 0 || rcnt[b + 1] == 0) continue;
                float cost = area_measure(llo, lhi, dim_) * measure(lcn) * lc + rarea[b + 1] * rcnt[b + 1];
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = a;
                    best_bin = b;
                }
            }
        }
        float parea = area_measure(nd.lo, nd.hi, dim_);
        if (cones_) {
            OCone pc{0, 0, 1, -1};
            for (int i = first; i < first + count; ++i) pc = cone_union(pc, (*cones_)[it_[i].rec]);
            parea *= measure(pc);
        }
        // leaf if small and splitting does not pay (traversal cost 1, test cost 1)
        if (count <= leaf_ && (best_axis < 0 || 1.0f + best_cost / std::max(parea, 1e-30f) >= (float)count))
            return id;
        int mid;
        if (best_axis < 0 || depth >= WOST_MAX_DEPTH - 8) {
            // degenerate centroids or a deep chain: split by index order halves
            mid = first + count / 2;
            if (best_axis >= 0) {
                int a = best_axis;
                std::nth_element(it_.begin() + first, it_.begin() + mid, it_.begin() + first + count,
                                 [a](const Item &p, const Item &q) { return p.c[a] < q.c[a]; });
            }
        } else {
            int a = best_axis;
            float ext = chi[a] - clo[a];
            float scale = kBins / ext;
            auto pivot = std::partition(it_.begin() + first, it_.begin() + first + count, [&](const Item &p) {
                int b = std::min(kBins - 1, (int)((p.c[a] - clo[a]) * scale));
                return b <= best_bin;
            });
            mid = (int)(pivot - it_.begin());
            if (mid == first || mid == first + count) mid = first + count / 2;
        }
        int l = make(first, mid - first, depth + 1);
        int r = make(mid, first + count - mid, depth + 1);
        nodes_[id].child[0] = l;
        nodes_[id].child[1] = r;
        return id;
    }
};

struct Cone {
    V3 axis;
    double cos_half;  // <= 0: always visit
};

Cone cone_of(const std::vector<V3> &normals, bool always) {
    if (always || normals.empty()) return {{0, 0, 1}, -1.0};
    V3 s{0, 0, 0};
    for (auto &n : normals) s = s + n;
    double l = norm(s);
    if (l < 1e-9) return {{0, 0, 1}, -1.0};
    V3 ax = s * (1.0 / l);
    double mn = 1.0;
    for (auto &n : normals) mn = std::min(mn, dot(ax, n));
    double th = std::acos(std::max(-1.0, std::min(1.0, mn))) + 2e-4;  // padding for FP32 tests
    if (th >= M_PI / 2) return {ax, -1.0};
    return {ax, std::cos(th)};
}

float4 f4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
float ibits(uint32_t v) {
    float f;
    std::memcpy(&f, &v, 4);
    return f;
}

// Flattens a built tree: writes 4 float4 per internal node with both child
// boxes, and returns the child reference of a build node.
struct Flattener {
    const std::vector<BNode> &bn;
    int dim;
    std::vector<float4> &out;
    std::vector<int> flat_of;  // build node -> flat index (internal only)

    uint32_t ref_of(int b) {
        const BNode &n = bn[b];
        if (n.child[0] < 0) return leaf_ref((uint32_t)n.first, (uint32_t)n.count);
        return (uint32_t)flat_of[b];
    }
    void run(int root) {
        flat_of.assign(bn.size(), -1);
        // breadth-first numbering keeps the top levels together in memory
        std::vector<int> order{root};
        for (size_t i = 0; i < order.size(); ++i) {
            const BNode &n = bn[order[i]];
            if (n.child[0] < 0) continue;
            flat_of[order[i]] = 0;
            order.push_back(n.child[0]);
            order.push_back(n.child[1]);
        }
        int k = 0;
        for (int b : order)
            if (bn[b].child[0] >= 0) flat_of[b] = k++;
        out.assign((size_t)k * 4, f4(0, 0, 0, 0));
        for (int b : order) {
            const BNode &n = bn[b];
            if (n.child[0] < 0) continue;
            const BNode &c0 = bn[n.child[0]], &c1 = bn[n.child[1]];
            float4 *q = &out[(size_t)flat_of[b] * 4];
            uint32_t r0 = ref_of(n.child[0]), r1 = ref_of(n.child[1]);
            if (dim == 2) {
                q[0] = f4(c0.lo[0], c0.lo[1], c0.hi[0], c0.hi[1]);
                q[1] = f4(c1.lo[0], c1.lo[1], c1.hi[0], c1.hi[1]);
                q[2] = f4(ibits(r0), ibits(r1), 0, 0);
                q[3] = f4(0, 0, 0, 0);
            } else {
                q[0] = f4(c0.lo[0], c0.lo[1], c0.lo[2], c0.hi[0]);
                q[1] = f4(c0.hi[1], c0.hi[2], c1.lo[0], c1.lo[1]);
                q[2] = f4(c1.lo[2], c1.hi[0], c1.hi[1], c1.hi[2]);
                q[3] = f4(ibits(r0), ibits(r1), 0, 0);
            }
        }
    }
};

// Collapses a binary tree into 8-wide nodes for group-cooperative traversal
// (8 lanes test the 8 children of a node, or the up to 8 primitives of a
// leaf, at once).  A binary subtree holding at most 8 primitives becomes one
// wide leaf (its records are contiguous); otherwise the node's slots are
// filled by repeatedly opening the internal child with the largest surface
// measure.  Node layout (16 float4): per child c, q[2c] = (lo.xyz, ref bits),
// q[2c+1] = (hi.xyz, 0); unused slots hold the empty reference.
struct WideFlattener {
    const std::vector<BNode> &bn;
    int dim;
    std::vector<float4> &out;
    std::vector<std::vector<int>> slots;  // per wide node: binary node ids of its children
    std::vector<int> wide_of;             // binary node -> wide node index (internal)
    int depth = 0;

    bool is_wide_leaf(int b) const { return bn[b].child[0] < 0 || bn[b].count <= WOST_WIDE; }
    uint32_t ref_of(int b) const {
        if (is_wide_leaf(b)) return leaf_ref((uint32_t)bn[b].first, (uint32_t)bn[b].count);
        return (uint32_t)wide_of[b];
    }
    std::vector<int> open(int b) const {
        std::vector<int> ch{bn[b].child[0], bn[b].child[1]};
        while (ch.size() < (size_t)WOST_WIDE) {
            int best = -1;
            float area = -1;
            for (size_t i = 0; i < ch.size(); ++i) {
                if (is_wide_leaf(ch[i])) continue;
                float a = area_measure(bn[ch[i]].lo, bn[ch[i]].hi, dim);
                if (a > area) {
                    area = a;
                    best = (int)i;
                }
            }
            if (best < 0) break;
            int c = ch[best];
            ch[best] = bn[c].child[0];
            ch.insert(ch.begin() + best + 1, bn[c].child[1]);
        }
        return ch;
    }
    // returns the root reference
    uint32_t run(int root) {
        wide_of.assign(bn.size(), -1);
        if (is_wide_leaf(root)) return ref_of(root);
        // breadth-first numbering
        std::vector<std::pair<int, int>> queue{{root, 1}};
        wide_of[root] = 0;
        int k = 1;
        for (size_t i = 0; i < queue.size(); ++i) {
            auto [b, lvl] = queue[i];
            depth = std::max(depth, lvl);
            std::vector<int> ch = open(b);
            slots.push_back(ch);
            for (int c : ch)
                if (!is_wide_leaf(c)) {
                    wide_of[c] = k++;
                    queue.push_back({c, lvl + 1});
                }
        }
        out.assign((size_t)k * 2 * WOST_WIDE, f4(INFINITY, INFINITY, INFINITY, ibits(WOST_EMPTY_REF)));
        for (size_t i = 0; i < queue.size(); ++i) {
            float4 *q = &out[(size_t)wide_of[queue[i].first] * 2 * WOST_WIDE];
            const std::vector<int> &ch = slots[i];
            for (int c = 0; c < WOST_WIDE; ++c) {
                if (c >= (int)ch.size()) {
                    q[2 * c] = f4(INFINITY, INFINITY, INFINITY, ibits(WOST_EMPTY_REF));
                    q[2 * c + 1] = f4(-INFINITY, -INFINITY, -INFINITY, 0);
                    continue;
                }
                const BNode &n = bn[ch[c]];
                q[2 * c] = f4(n.lo[0], n.lo[1], n.lo[2], ibits(ref_of(ch[c])));
                q[2 * c + 1] = f4(n.hi[0], n.hi[1], n.hi[2], 0);
            }
        }
        return 0;
    }
};

// Builds one tree over `items` (records 0..n-1) and returns the leaf order of
// the records (perm[k] = record stored at position k).
std::vector<int> build_tree(std::vector<Item> &items, int dim, int leaf, HostTree &t,
                            std::vector<BNode> *keep_nodes, int *root_out, const std::vector<OCone> *cones = nullptr) {
    t.n_prims = (int)items.size();
    std::vector<int> perm(items.size());
    if (items.empty()) {
        t.root = WOST_EMPTY_REF;
        t.n_nodes = 0;
        t.depth = 0;
        for (int a = 0; a < 3; ++a) t.root_lo[a] = t.root_hi[a] = 0;
        return perm;
    }
    Builder b(items, dim, leaf, cones);
    int root = b.build();
    for (size_t k = 0; k < items.size(); ++k) perm[k] = items[k].rec;
    Flattener fl{b.nodes_, dim, t.nodes, {}};
    fl.run(root);
    t.root = fl.ref_of(root);
    t.n_nodes = (int)(t.nodes.size() / 4);
    t.depth = b.max_depth_ + 1;
    WideFlattener wf{b.nodes_, dim, t.wnodes, {}, {}};
    t.wroot = wf.run(root);
    t.wn_nodes = (int)(t.wnodes.size() / (2 * WOST_WIDE));
    t.wdepth = wf.depth + 1;
    t.wslots = wf.slots;
    t.wide_of = wf.wide_of;
    for (int a = 0; a < 3; ++a) {
        t.root_lo[a] = b.nodes_[root].lo[a];
        t.root_hi[a] = b.nodes_[root].hi[a];
    }
    if (keep_nodes) *keep_nodes = b.nodes_;
    if (root_out) *root_out = root;
    return perm;
}

}  // namespace

std::string build_scene(const wost_scene_desc &d, HostScene &S) {
    auto t0 = std::chrono::steady_clock::now();
    if (d.dim != 2 && d.dim != 3) return "dim must be 2 or 3";
    const int dim = d.dim;
    if (d.n_vertices < 1 || !d.vertices) return "vertices missing";
    if (d.n_prims < 1 || !d.prims || !d.flags) return "primitives or flags missing";
    if (d.n_prims >= (int64_t)1 << 27) return "too many primitives (limit 2^27)";
    if (d.leaf_size < 0 || d.leaf_size > WOST_MAX_LEAF) return "leaf_size must be in [0, 16]";
    if (d.silhouette_split != 0 && d.silhouette_split != 1) return "silhouette_split must be 0 or 1";
    const int leaf = d.leaf_size ? d.leaf_size : 4;
    for (int64_t i = 0; i < d.n_vertices * dim; ++i)
        if (!std::isfinite(d.vertices[i])) return "non-finite vertex coordinate";
    for (int64_t i = 0; i < d.n_prims * dim; ++i)
        if (d.prims[i] < 0 || d.prims[i] >= d.n_vertices) return "primitive index out of range";
    for (int64_t i = 0; i < d.n_prims; ++i)
        if (d.flags[i] > 3)
            return "flag must be 0 (Dirichlet), 1 (Neumann), 2 or 3 (double-sided Dirichlet or Neumann)";
    auto check_field = [&](const wost_field &f, bool is_source) -> std::string {
        switch (f.kind) {
        case WOST_DATA_NONE: return "";
        case WOST_DATA_PER_VERTEX:
        case WOST_DATA_PER_CORNER: {
            if (is_source) return "f must be NONE, ANALYTIC or GRID";
            if (!f.values) return "field values missing";
            int64_t n = f.kind == WOST_DATA_PER_VERTEX ? d.n_vertices : d.n_prims * dim;
            for (int64_t i = 0; i < n; ++i)
                if (!std::isfinite(f.values[i])) return "non-finite field value";
            return "";
        }
        case WOST_DATA_ANALYTIC:
            if (f.fn < WOST_FN_ZERO || f.fn > WOST_FN_EXP_PLANE) return "unknown analytic function id";
            return "";
        case WOST_DATA_GRID: {
            if (!is_source) return "GRID is only valid for f";
            if (!f.values) return "grid values missing";
            int64_t n = 1;
            for (int a = 0; a < dim; ++a) {
                if (f.dims[a] < 1 || !(f.spacing[a] > 0)) return "grid dims and spacing must be positive";
                n *= f.dims[a];
            }
            for (int64_t i = 0; i < n; ++i)
                if (!std::isfinite(f.values[i])) return "non-finite grid value";
            return "";
        }
        default: return "unknown field kind";
        }
    };
    std::string e;
    if (!(e = check_field(d.g, false)).empty()) return "g: " + e;
    if (!(e = check_field(d.h, false)).empty()) return "h: " + e;
    if (!(e = check_field(d.f, true)).empty()) return "f: " + e;
    for (const wost_field *m : {&d.g_minus, &d.h_minus}) {
        if (m->kind != WOST_DATA_NONE && m->kind != WOST_DATA_PER_VERTEX && m->kind != WOST_DATA_PER_CORNER)
            return "g_minus / h_minus must be NONE, PER_VERTEX or PER_CORNER";
        if (!(e = check_field(*m, false)).empty()) return (m == &d.g_minus ? "g_minus: " : "h_minus: ") + e;
    }

    S.dim = dim;
    auto V = [&](int64_t v) -> V3 {
        return {d.vertices[v * dim], d.vertices[v * dim + 1], dim == 3 ? (double)d.vertices[v * dim + 2] : 0.0};
    };
    auto corner = [&](int64_t p, int k) { return V(d.prims[p * dim + k]); };

    // live primitives, normals, areas
    const int64_t np = d.n_prims;
    std::vector<V3> nrm(np);
    std::vector<double> area(np);
    std::vector<int64_t> Dl, Nl;
    for (int64_t p = 0; p < np; ++p) {
        V3 a = corner(p, 0), b = corner(p, 1);
        if (dim == 2) {
            V3 t = b - a;
            double l = norm(t);
            area[p] = l;
            nrm[p] = l > 0 ? V3{t.y / l, -t.x / l, 0} : V3{0, 0, 0};
        } else {
            V3 c = cross(b - a, corner(p, 2) - a);
            double l = norm(c);
            area[p] = 0.5 * l;
            nrm[p] = l > 0 ? c * (1.0 / l) : V3{0, 0, 0};
        }
        if (!(area[p] > 0)) {
            S.n_dropped++;
            continue;
        }
        (d.flags[p] & 1 ? Nl : Dl).push_back(p);
    }

    // scene bounds
    for (int a = 0; a < 3; ++a) {
        S.lo[a] = INFINITY;
        S.hi[a] = -INFINITY;
    }
    for (int64_t v = 0; v < d.n_vertices; ++v) {
        V3 q = V(v);
        double c[3] = {q.x, q.y, q.z};
        for (int a = 0; a < 3; ++a) {
            S.lo[a] = std::min(S.lo[a], (float)c[a]);
            S.hi[a] = std::max(S.hi[a], (float)c[a]);
        }
    }

    auto prim_item = [&](int64_t p, int rec) {
        Item it;
        empty_box(it.lo, it.hi);
        for (int k = 0; k < dim; ++k) {
            V3 q = corner(p, k);
            float c[3] = {(float)q.x, (float)q.y, (float)q.z};
            grow(it.lo, it.hi, c, c);
        }
        for (int a = 0; a < 3; ++a) it.c[a] = 0.5f * (it.lo[a] + it.hi[a]);
        it.rec = rec;
        return it;
    };

    // corner values of a boundary field on primitive p
    auto corner_vals = [&](const wost_field &f, int64_t p, float out[3]) {
        for (int k = 0; k < 3; ++k) out[k] = 0;
        if (f.kind == WOST_DATA_PER_VERTEX)
            for (int k = 0; k < dim; ++k) out[k] = f.values[d.prims[p * dim + k]];
        else if (f.kind == WOST_DATA_PER_CORNER)
            for (int k = 0; k < dim; ++k) out[k] = f.values[p * dim + k];
    };

    // primitive records of a D or N tree in leaf order; double-sided records
    // (flags 2, 3) also get their - side corner data (NONE: the + side's data
    // for g, negated for h, i.e. a solution continuous across the sheet)
    auto fill_prims = [&](const std::vector<int64_t> &list, const std::vector<int> &perm, const wost_field &fld,
                          const wost_field &minus, bool negate_plus, HostTree &t) {
        size_t n = list.size();
        t.prims.assign(n * (dim == 2 ? 1 : 3), f4(0, 0, 0, 0));
        t.data.assign(dim == 2 ? (n + 1) / 2 : n, f4(0, 0, 0, 0));
        t.ids.resize(n);
        bool any_sided = false;
        for (int64_t p : list) any_sided = any_sided || d.flags[p] >= 2;
        if (any_sided) {
            t.sided.assign(n, 0);
            t.data_minus.assign(t.data.size(), f4(0, 0, 0, 0));
        }
        float *dat = reinterpret_cast<float *>(t.data.data());
        float *datm = any_sided ? reinterpret_cast<float *>(t.data_minus.data()) : nullptr;
        for (size_t k = 0; k < n; ++k) {
            int64_t p = list[perm[k]];
            t.ids[k] = (int32_t)p;
            V3 a = corner(p, 0), b = corner(p, 1);
            if (dim == 2) {
                t.prims[k] = f4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
            } else {
                V3 c = corner(p, 2);
                t.prims[3 * k] = f4((float)a.x, (float)a.y, (float)a.z, (float)area[p]);
                t.prims[3 * k + 1] = f4((float)b.x, (float)b.y, (float)b.z, 0);
                t.prims[3 * k + 2] = f4((float)c.x, (float)c.y, (float)c.z, 0);
            }
            float cv[3];
            corner_vals(fld, p, cv);
            const int stride = dim == 2 ? 2 : 4;
            for (int c = 0; c < dim; ++c) dat[stride * k + c] = cv[c];
            if (any_sided && d.flags[p] >= 2) {
                t.sided[k] = 1;
                float mv[3];
                if (minus.kind == WOST_DATA_NONE) {
                    for (int c = 0; c < 3; ++c) mv[c] = negate_plus ? -cv[c] : cv[c];
                } else {
                    corner_vals(minus, p, mv);
                }
                for (int c = 0; c < dim; ++c) datm[stride * k + c] = mv[c];
            }
        }
    };

    // --- Dirichlet BVH ---
    {
        std::vector<Item> items(Dl.size());
        for (size_t i = 0; i < Dl.size(); ++i) items[i] = prim_item(Dl[i], (int)i);
        auto perm = build_tree(items, dim, leaf, S.D, nullptr, nullptr);
        fill_prims(Dl, perm, d.g, d.g_minus, false, S.D);
    }
    // --- Neumann BVH ---
    {
        std::vector<Item> items(Nl.size());
        for (size_t i = 0; i < Nl.size(); ++i) items[i] = prim_item(Nl[i], (int)i);
        auto perm = build_tree(items, dim, leaf, S.N, nullptr, nullptr);
        fill_prims(Nl, perm, d.h, d.h_minus, true, S.N);
    }
    // --- silhouette candidates and their cone hierarchy ---
    struct Sil {
        int64_t a, b;     // vertex ids (b = -1 in 2D)
        int64_t f0, f1;   // adjacent Neumann primitives (f1 = -1 if one; -2 if > 2)
    };
    std::vector<Sil> sil;
    if (dim == 2) {
        std::vector<int64_t> f0(d.n_vertices, -1), f1(d.n_vertices, -1);
        std::vector<int> cnt(d.n_vertices, 0);
        for (int64_t p : Nl)
            for (int k = 0; k < 2; ++k) {
                int64_t v = d.prims[p * 2 + k];
                if (cnt[v] == 0) f0[v] = p;
                else if (cnt[v] == 1) f1[v] = p;
                cnt[v]++;
            }
        for (int64_t v = 0; v < d.n_vertices; ++v)
            if (cnt[v]) sil.push_back({v, -1, f0[v], cnt[v] == 2 ? f1[v] : (cnt[v] > 2 ? -2 : -1)});
    } else {
        struct E {
            int64_t a, b, t;
        };
        std::vector<E> es;
        es.reserve(Nl.size() * 3);
        for (int64_t p : Nl)
            for (int k = 0; k < 3; ++k) {
                int64_t a = d.prims[p * 3 + k], b = d.prims[p * 3 + (k + 1) % 3];
                es.push_back({std::min(a, b), std::max(a, b), p});
            }
        std::sort(es.begin(), es.end(), [](const E &x, const E &y) {
            return x.a != y.a ? x.a < y.a : (x.b != y.b ? x.b < y.b : x.t < y.t);
        });
        for (size_t i = 0; i < es.size();) {
            size_t j = i;
            while (j < es.size() && es[j].a == es[i].a && es[j].b == es[i].b) ++j;
            size_t c = j - i;
            sil.push_back({es[i].a, es[i].b, es[i].t, c == 2 ? es[i + 1].t : (c > 2 ? -2 : -1)});
            i = j;
        }
    }
    {
        std::vector<Item> items(sil.size());
        for (size_t i = 0; i < sil.size(); ++i) {
            Item it;
            empty_box(it.lo, it.hi);
            V3 pa = V(sil[i].a);
            float ca[3] = {(float)pa.x, (float)pa.y, (float)pa.z};
            grow(it.lo, it.hi, ca, ca);
            if (sil[i].b >= 0) {
                V3 pb = V(sil[i].b);
                float cb[3] = {(float)pb.x, (float)pb.y, (float)pb.z};
                grow(it.lo, it.hi, cb, cb);
            }
            for (int a = 0; a < 3; ++a) it.c[a] = 0.5f * (it.lo[a] + it.hi[a]);
            it.rec = (int)i;
            items[i] = it;
        }
        // per-candidate normal cones for the orientation-aware split cost
        std::vector<OCone> icones(sil.size());
        for (size_t i = 0; i < sil.size(); ++i) {
            V3 n0 = nrm[sil[i].f0];
            if (sil[i].f1 < 0) {
                icones[i] = {(float)n0.x, (float)n0.y, (float)n0.z, 3.14159265f};  // always a silhouette
                continue;
            }
            V3 n1 = nrm[sil[i].f1];
            V3 s = n0 + n1;
            double l = norm(s);
            double half = 0.5 * std::acos(std::max(-1.0, std::min(1.0, dot(n0, n1))));
            if (l < 1e-9) icones[i] = {(float)n0.x, (float)n0.y, (float)n0.z, 3.14159265f};
            else icones[i] = {(float)(s.x / l), (float)(s.y / l), (float)(s.z / l), (float)half};
        }
        std::vector<BNode> bn;
        int root = -1;
        auto perm = build_tree(items, dim, leaf, S.S, &bn, &root, d.silhouette_split == 1 ? nullptr : &icones);
        size_t n = sil.size();
        S.S.prims.assign(n * (dim == 2 ? 2 : 3), f4(0, 0, 0, 0));
        S.S.ids.resize(n);
        for (size_t k = 0; k < n; ++k) {
            const Sil &s = sil[perm[k]];
            S.S.ids[k] = (int32_t)s.a;
            V3 n0 = nrm[s.f0];
            V3 n1 = s.f1 >= 0 ? nrm[s.f1] : V3{0, 0, 0};
            V3 pa = V(s.a);
            if (dim == 2) {
                S.S.prims[2 * k] = f4((float)pa.x, (float)pa.y, 0, 0);
                S.S.prims[2 * k + 1] = f4((float)n0.x, (float)n0.y, (float)n1.x, (float)n1.y);
            } else {
                V3 pb = V(s.b);
                S.S.prims[3 * k] = f4((float)pa.x, (float)pa.y, (float)pa.z, (float)n0.x);
                S.S.prims[3 * k + 1] = f4((float)pb.x, (float)pb.y, (float)pb.z, (float)n0.y);
                S.S.prims[3 * k + 2] = f4((float)n0.z, (float)n1.x, (float)n1.y, (float)n1.z);
            }
        }
        // cones: per build node, over the normals of its candidates
        if (!bn.empty()) {
            std::vector<Cone> cones(bn.size());
            std::vector<V3> ns;
            for (size_t b = 0; b < bn.size(); ++b) {
                ns.clear();
                bool always = false;
                for (int k = bn[b].first; k < bn[b].first + bn[b].count; ++k) {
                    const Sil &s = sil[perm[k]];
                    ns.push_back(nrm[s.f0]);
                    if (s.f1 >= 0) ns.push_back(nrm[s.f1]);
                    else always = true;
                }
                cones[b] = cone_of(ns, always);
            }
            auto cf = [](const Cone &c) {
                return f4((float)c.axis.x, (float)c.axis.y, (float)c.axis.z, (float)c.cos_half);
            };
            Flattener fl{bn, dim, S.S.nodes, {}};
            fl.run(root);  // same numbering as build_tree's flattening
            S.S.cones.assign((size_t)S.S.n_nodes * 2, f4(0, 0, 0, -1));
            for (size_t b = 0; b < bn.size(); ++b) {
                if (bn[b].child[0] < 0) continue;
                int fi = fl.flat_of[b];
                S.S.cones[2 * fi] = cf(cones[bn[b].child[0]]);
                S.S.cones[2 * fi + 1] = cf(cones[bn[b].child[1]]);
            }
            S.S.root_cone = cf(cones[root]);
            // wide layout: the cone of every child slot
            S.S.wcones.assign((size_t)S.S.wn_nodes * WOST_WIDE, f4(0, 0, 1, -1));
            for (size_t i = 0; i < S.S.wslots.size(); ++i) {  // wide node i = i-th in breadth-first order
                const std::vector<int> &ch = S.S.wslots[i];
                for (size_t c = 0; c < ch.size(); ++c) S.S.wcones[i * WOST_WIDE + c] = cf(cones[ch[c]]);
            }
        } else {
            S.S.root_cone = f4(0, 0, 1, -1);
        }
    }

    // fields
    auto view = [&](const wost_field &f, FieldView &v, std::vector<float> &store, bool boundary) {
        std::memset(&v, 0, sizeof v);
        if (f.kind == WOST_DATA_ANALYTIC) {
            v.kind = FIELD_ANALYTIC;
            v.fn = f.fn;
            std::memcpy(v.params, f.params, sizeof v.params);
        } else if (f.kind == WOST_DATA_GRID) {
            v.kind = FIELD_GRID;
            int64_t n = 1;
            for (int a = 0; a < dim; ++a) n *= f.dims[a];
            store.assign(f.values, f.values + n);
            for (int a = 0; a < 3; ++a) {
                v.origin[a] = f.origin[a];
                v.spacing[a] = a < dim ? f.spacing[a] : 1.f;
                v.dims[a] = a < dim ? f.dims[a] : 1;
            }
        } else if (f.kind == WOST_DATA_PER_VERTEX || f.kind == WOST_DATA_PER_CORNER) {
            v.kind = FIELD_CORNER;
        } else {
            v.kind = boundary ? FIELD_CORNER : FIELD_NONE;  // absent boundary data: zero corners
        }
    };
    view(d.g, S.g, S.grid_unused, true);
    view(d.h, S.h, S.grid_unused, true);
    view(d.f, S.f, S.grid, false);
    S.n_dirichlet = (int64_t)Dl.size();
    S.n_neumann = (int64_t)Nl.size();
    S.n_silhouette = (int64_t)sil.size();
    S.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return "";
}

}  // namespace wost
