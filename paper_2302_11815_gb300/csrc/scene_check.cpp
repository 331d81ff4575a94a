// Structural checks of the hierarchies built on the host (binary and 8-wide
// forms of the D, N and S trees), run by wost_scene_validate without a GPU:
//   - every child reference is a leaf or an internal node visited once (no
//     cycles, no shared subtrees), and every primitive record lies in
//     exactly one leaf;
//   - every box contains the boxes below it and the primitives of its leaves;
//   - every normal cone of the silhouette tree contains the normals of all
//     candidates below it (a cone with cos <= 0 contains every direction);
//   - no leaf is deeper than the depth the traversal stacks are sized for.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "scene_build.h"

namespace wost {
namespace {

struct Box {
    float lo[3], hi[3];
};

bool contains(const Box &outer, const Box &inner, int dim, float tol) {
    for (int a = 0; a < dim; ++a)
        if (inner.lo[a] < outer.lo[a] - tol || inner.hi[a] > outer.hi[a] + tol) return false;
    return true;
}

// bounding box of record k and its (up to two) normals
struct Rec {
    Box box;
    float n[2][3];
    int n_normals;
};

Rec record(const HostTree &T, int dim, bool sil, int k) {
    Rec r{};
    auto set_pts = [&](const float *pts, int m) {
        for (int a = 0; a < 3; ++a) {
            r.box.lo[a] = INFINITY;
            r.box.hi[a] = -INFINITY;
        }
        for (int i = 0; i < m; ++i)
            for (int a = 0; a < dim; ++a) {
                r.box.lo[a] = std::fmin(r.box.lo[a], pts[3 * i + a]);
                r.box.hi[a] = std::fmax(r.box.hi[a], pts[3 * i + a]);
            }
    };
    if (!sil) {
        if (dim == 2) {
            float4 q = T.prims[k];
            float p[6] = {q.x, q.y, 0, q.z, q.w, 0};
            set_pts(p, 2);
        } else {
            float4 a = T.prims[3 * k], b = T.prims[3 * k + 1], c = T.prims[3 * k + 2];
            float p[9] = {a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z};
            set_pts(p, 3);
        }
        return r;
    }
    if (dim == 2) {
        float4 q0 = T.prims[2 * k], q1 = T.prims[2 * k + 1];
        float p[3] = {q0.x, q0.y, 0};
        set_pts(p, 1);
        float n[2][3] = {{q1.x, q1.y, 0}, {q1.z, q1.w, 0}};
        for (int i = 0; i < 2; ++i)
            for (int a = 0; a < 3; ++a) r.n[i][a] = n[i][a];
    } else {
        float4 q0 = T.prims[3 * k], q1 = T.prims[3 * k + 1], q2 = T.prims[3 * k + 2];
        float p[6] = {q0.x, q0.y, q0.z, q1.x, q1.y, q1.z};
        set_pts(p, 2);
        float n[2][3] = {{q0.w, q1.w, q2.x}, {q2.y, q2.z, q2.w}};
        for (int i = 0; i < 2; ++i)
            for (int a = 0; a < 3; ++a) r.n[i][a] = n[i][a];
    }
    r.n_normals = 0;
    for (int i = 0; i < 2; ++i) {
        float l = r.n[i][0] * r.n[i][0] + r.n[i][1] * r.n[i][1] + r.n[i][2] * r.n[i][2];
        if (l > 0) {
            if (i != r.n_normals)
                for (int a = 0; a < 3; ++a) r.n[r.n_normals][a] = r.n[i][a];
            r.n_normals++;
        }
    }
    return r;
}

bool cone_holds(const float4 &cone, const Rec &r) {
    if (cone.w <= 0.f) return true;
    for (int i = 0; i < r.n_normals; ++i) {
        float d = cone.x * r.n[i][0] + cone.y * r.n[i][1] + cone.z * r.n[i][2];
        if (d < cone.w - 1e-5f) return false;
    }
    return true;
}

struct Item {
    uint32_t ref;
    Box box;
    int depth;
    int cone;  // innermost cone on the path to this subtree (index into the cone list), -1 = none
};

// the cones on a path, innermost first: a list of (cone, enclosing entry)
struct ConeLink {
    float4 cone;
    int up;
};

// children of binary node i: boxes and references (layout in wost_internal.h)
void binary_children(const HostTree &T, int dim, uint32_t i, Box b[2], uint32_t r[2]) {
    const float4 *q = &T.nodes[4 * (size_t)i];
    auto bits = [](float f) {
        uint32_t u;
        std::memcpy(&u, &f, 4);
        return u;
    };
    for (int c = 0; c < 2; ++c)
        for (int a = 0; a < 3; ++a) b[c].lo[a] = b[c].hi[a] = 0.f;
    if (dim == 2) {
        b[0] = Box{{q[0].x, q[0].y, 0}, {q[0].z, q[0].w, 0}};
        b[1] = Box{{q[1].x, q[1].y, 0}, {q[1].z, q[1].w, 0}};
        r[0] = bits(q[2].x);
        r[1] = bits(q[2].y);
    } else {
        b[0] = Box{{q[0].x, q[0].y, q[0].z}, {q[0].w, q[1].x, q[1].y}};
        b[1] = Box{{q[1].z, q[1].w, q[2].x}, {q[2].y, q[2].z, q[2].w}};
        r[0] = bits(q[3].x);
        r[1] = bits(q[3].y);
    }
}

// Walks one form of a tree.  wide = false: binary nodes and T.cones; wide =
// true: 8-wide nodes and T.wcones.
std::string check_form(const HostTree &T, int dim, bool sil, bool wide, float tol) {
    const char *name = wide ? "wide tree" : "binary tree";
    const int n = T.n_prims;
    const uint32_t root = wide ? T.wroot : T.root;
    if (n == 0) return root == WOST_EMPTY_REF ? "" : std::string(name) + ": root of an empty tree";
    if (root == WOST_EMPTY_REF) return std::string(name) + ": empty root";
    const int n_nodes = wide ? T.wn_nodes : T.n_nodes;
    const int max_depth = wide ? T.wdepth : T.depth;
    std::vector<int> covered((size_t)n, 0);
    std::vector<char> visited((size_t)std::max(n_nodes, 1), 0);
    std::vector<ConeLink> cones;
    std::vector<Item> stack;
    Box root_box{{T.root_lo[0], T.root_lo[1], T.root_lo[2]}, {T.root_hi[0], T.root_hi[1], T.root_hi[2]}};
    int root_cone = -1;
    if (sil) {
        cones.push_back({T.root_cone, -1});
        root_cone = 0;
    }
    stack.push_back({root, root_box, 1, root_cone});
    auto bits = [](float f) {
        uint32_t u;
        std::memcpy(&u, &f, 4);
        return u;
    };
    while (!stack.empty()) {
        Item it = stack.back();
        stack.pop_back();
        if (it.depth > max_depth + 1) return std::string(name) + ": deeper than its recorded depth";
        if (it.ref & WOST_LEAF_BIT) {
            uint32_t first = (it.ref & 0x7FFFFFFFu) >> 4, count = (it.ref & 15u) + 1u;
            if ((int64_t)first + count > n) return std::string(name) + ": leaf beyond the records";
            for (uint32_t k = first; k < first + count; ++k) {
                covered[k]++;
                Rec r = record(T, dim, sil, (int)k);
                if (!contains(it.box, r.box, dim, tol)) return std::string(name) + ": a record outside its leaf box";
                for (int c = it.cone; c >= 0; c = cones[(size_t)c].up)
                    if (!cone_holds(cones[(size_t)c].cone, r))
                        return std::string(name) + ": a normal outside an ancestor's cone";
            }
            continue;
        }
        if ((int)it.ref >= n_nodes) return std::string(name) + ": node index out of range";
        if (visited[it.ref]) return std::string(name) + ": a node reached twice";
        visited[it.ref] = 1;
        const int fan = wide ? WOST_WIDE : 2;
        Box bb[2];
        uint32_t rr[2];
        if (!wide) binary_children(T, dim, it.ref, bb, rr);
        for (int c = 0; c < fan; ++c) {
            Box b;
            uint32_t r;
            if (wide) {
                const float4 *q = &T.wnodes[(size_t)it.ref * 2 * WOST_WIDE + 2 * c];
                r = bits(q[0].w);
                if (r == WOST_EMPTY_REF) continue;
                b = Box{{q[0].x, q[0].y, q[0].z}, {q[1].x, q[1].y, q[1].z}};
            } else {
                b = bb[c];
                r = rr[c];
            }
            if (!contains(it.box, b, dim, tol)) return std::string(name) + ": a child box outside its parent's";
            int link = it.cone;
            if (sil) {
                float4 cone = wide ? T.wcones[(size_t)it.ref * WOST_WIDE + c] : T.cones[2 * (size_t)it.ref + c];
                cones.push_back({cone, it.cone});
                link = (int)cones.size() - 1;
            }
            stack.push_back({r, b, it.depth + 1, link});
        }
    }
    for (int k = 0; k < n; ++k)
        if (covered[k] != 1) return std::string(name) + ": a record in " + std::to_string(covered[k]) + " leaves";
    return "";
}

}  // namespace

std::string check_scene(const HostScene &S) {
    float ext = 0.f;
    for (int a = 0; a < S.dim; ++a) ext = std::fmax(ext, S.hi[a] - S.lo[a]);
    const float tol = 1e-5f * (ext > 0 ? ext : 1.f);
    const HostTree *trees[3] = {&S.D, &S.N, &S.S};
    const char *names[3] = {"Dirichlet ", "Neumann ", "silhouette "};
    for (int t = 0; t < 3; ++t)
        for (int wide = 0; wide < 2; ++wide) {
            std::string e = check_form(*trees[t], S.dim, t == 2, wide != 0, tol);
            if (!e.empty()) return names[t] + e;
        }
    return "";
}

}  // namespace wost
