// Host BVH build for the stackless GPU traversal: binned SAH (16 bins per
// axis over centroid bounds), leaves of at most 4 triangles (up to 15 when
// the depth limit forces a leaf), depth <= 60 so a 64-bit trail holds a path.
//
// Node layout (64 bytes = 4 x float4, child boxes stored in the parent so one
// fetch tests both children):
//   n0 = (left.lo.xyz,  left child)    n1 = (left.hi.xyz,  right child)
//   n2 = (right.lo.xyz, 0)             n3 = (right.hi.xyz, 0)
// child >= 0 is an internal node index; child < 0 is a leaf with
// v = -child - 1, first = v >> 4 (index into the leaf-ordered triangle
// arrays), count = v & 15. parent[] and sibling[] drive the backtracking.
#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <cstring>
#include <vector>

#include "pb_bvh.h"

namespace {

struct Box {
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX};
    float hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    void grow(const float *p) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], p[a]);
            hi[a] = std::max(hi[a], p[a]);
        }
    }
    void grow(const Box &b) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], b.lo[a]);
            hi[a] = std::max(hi[a], b.hi[a]);
        }
    }
    double area() const {
        if (lo[0] > hi[0]) return 0.0;
        double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

struct Build {
    const float *V;
    const int32_t *T;
    std::vector<Box> tbox;
    std::vector<float> cen;   // 3 per tri
    std::vector<int32_t> idx;
    std::vector<float> nodes;  // 16 floats per node
    std::vector<int32_t> parent, sibling;
};

int32_t leaf_code(int first, int count) { return -(first * 16 + count) - 1; }

void set_child(Build &b, int node, int side, const Box &bx, int32_t code) {
    float *n = &b.nodes[(size_t)node * 16];
    float *lo = side == 0 ? n + 0 : n + 8;
    float *hi = side == 0 ? n + 4 : n + 12;
    for (int a = 0; a < 3; ++a) {
        lo[a] = bx.lo[a];
        hi[a] = bx.hi[a];
    }
    int32_t *w = reinterpret_cast<int32_t *>(side == 0 ? n + 3 : n + 7);
    *w = code;
}

struct Task { int node, side, first, count, depth; };

Box range_box(const Build &b, int first, int count) {
    Box bx;
    for (int i = first; i < first + count; ++i) bx.grow(b.tbox[b.idx[i]]);
    return bx;
}

// choose a split of idx[first, first+count); returns split position or -1 for a leaf
int split(Build &b, int first, int count, int depth) {
    const int maxleaf = 4;
    if (count <= maxleaf) return -1;
    Box cb;
    for (int i = first; i < first + count; ++i) cb.grow(&b.cen[3 * (size_t)b.idx[i]]);
    const int NB = 16;
    double best = DBL_MAX;
    int best_axis = -1, best_bin = -1;
    for (int a = 0; a < 3; ++a) {
        float ext = cb.hi[a] - cb.lo[a];
        if (!(ext > 0.0f)) continue;
        Box bins[NB];
        int cnt[NB] = {0};
        for (int i = first; i < first + count; ++i) {
            int t = b.idx[i];
            int k = (int)((b.cen[3 * (size_t)t + a] - cb.lo[a]) / ext * NB);
            k = std::min(std::max(k, 0), NB - 1);
            cnt[k]++;
            bins[k].grow(b.tbox[t]);
        }
        double la[NB], ra[NB];
        int lc[NB], rc[NB];
        Box acc;
        int c = 0;
        for (int k = 0; k < NB; ++k) {
            acc.grow(bins[k]);
            c += cnt[k];
            la[k] = acc.area();
            lc[k] = c;
        }
        acc = Box();
        c = 0;
        for (int k = NB - 1; k >= 0; --k) {
            acc.grow(bins[k]);
            c += cnt[k];
            ra[k] = acc.area();
            rc[k] = c;
        }
        for (int k = 0; k < NB - 1; ++k) {
            if (lc[k] == 0 || rc[k + 1] == 0) continue;
            double cost = la[k] * lc[k] + ra[k + 1] * rc[k + 1];
            if (cost < best) {
                best = cost;
                best_axis = a;
                best_bin = k;
            }
        }
    }
    Box pb = range_box(b, first, count);
    double leaf_cost = pb.area() * count;
    bool force = depth >= 58 || best_axis < 0;
    if (!force && count <= 15 && leaf_cost <= best + pb.area() * 1.0) return -1;
    int mid;
    if (best_axis >= 0 && !(depth >= 58)) {
        float ext = cb.hi[best_axis] - cb.lo[best_axis];
        auto it = std::stable_partition(b.idx.begin() + first, b.idx.begin() + first + count, [&](int t) {
            int k = (int)((b.cen[3 * (size_t)t + best_axis] - cb.lo[best_axis]) / ext * NB);
            k = std::min(std::max(k, 0), NB - 1);
            return k <= best_bin;
        });
        mid = (int)(it - b.idx.begin());
    } else {
        // degenerate centroids or depth limit: median split by index
        if (count <= 15) return -1;
        mid = first + count / 2;
    }
    if (mid <= first || mid >= first + count) mid = first + count / 2;
    return mid;
}

}  // namespace

int pb_bvh_build(const float *verts, int nv, const int32_t *tris, int nt, PbBvh *out) {
    (void)nv;
    Build b;
    b.V = verts;
    b.T = tris;
    b.tbox.resize(nt);
    b.cen.resize(3 * (size_t)nt);
    b.idx.resize(nt);
    for (int t = 0; t < nt; ++t) {
        Box bx;
        for (int k = 0; k < 3; ++k) bx.grow(&verts[3 * (size_t)tris[3 * (size_t)t + k]]);
        b.tbox[t] = bx;
        for (int a = 0; a < 3; ++a) b.cen[3 * (size_t)t + a] = 0.5f * (bx.lo[a] + bx.hi[a]);
        b.idx[t] = t;
    }
    b.nodes.reserve(16 * (size_t)std::max(1, nt));
    b.nodes.assign(16, 0.0f);
    b.parent.push_back(-1);
    b.sibling.push_back(-1);
    // root is always an internal node; its children come from splitting all triangles
    std::vector<Task> stack;
    int mid = split(b, 0, nt, 0);
    if (mid < 0) {
        set_child(b, 0, 0, range_box(b, 0, nt), leaf_code(0, nt));
        set_child(b, 0, 1, Box(), leaf_code(0, 0));
    } else {
        stack.push_back({0, 1, mid, nt - mid, 1});
        stack.push_back({0, 0, 0, mid, 1});
    }
    std::vector<int> child_of[2];
    while (!stack.empty()) {
        Task tk = stack.back();
        stack.pop_back();
        Box bx = range_box(b, tk.first, tk.count);
        int m = split(b, tk.first, tk.count, tk.depth);
        if (m < 0) {
            set_child(b, tk.node, tk.side, bx, leaf_code(tk.first, tk.count));
            continue;
        }
        int id = (int)(b.nodes.size() / 16);
        b.nodes.resize(b.nodes.size() + 16, 0.0f);
        b.parent.push_back(tk.node);
        b.sibling.push_back(-1);
        set_child(b, tk.node, tk.side, bx, id);
        stack.push_back({id, 1, m, tk.first + tk.count - m, tk.depth + 1});
        stack.push_back({id, 0, tk.first, m - tk.first, tk.depth + 1});
    }
    int nn = (int)(b.nodes.size() / 16);
    // sibling of each internal child
    for (int n = 0; n < nn; ++n) {
        const int32_t *w = reinterpret_cast<const int32_t *>(&b.nodes[(size_t)n * 16]);
        int32_t l = w[3], r = w[7];
        if (l >= 0 && r >= 0) {
            b.sibling[l] = r;
            b.sibling[r] = l;
        } else if (l >= 0) {
            b.sibling[l] = -1;
        } else if (r >= 0) {
            b.sibling[r] = -1;
        }
    }
    out->nodes = std::move(b.nodes);
    out->parent = std::move(b.parent);
    out->sibling = std::move(b.sibling);
    out->order = std::move(b.idx);
    return nn;
}
