// Host BVH build for the stackless GPU traversal: binned SAH (16 bins per
// axis over centroid bounds), leaves of at most 4 triangles (up to 15 when
// the depth limit forces a leaf), depth <= 60 so a 64-bit trail holds a path.
//
// The build runs on the host's cores: the two subtrees of a node are built on
// separate threads near the root, and a range of at least 2^16 triangles
// computes its bounds, bins and stable partition in parallel parts (min/max
// and counts reduce exactly). The split of a range depends only on the range,
// so the tree is the same for any thread count, and internal nodes are
// numbered in pre-order (a node, then its left subtree, then its right).
//
// Node layout (64 bytes = 4 x float4, child boxes stored in the parent so one
// fetch tests both children):
//   n0 = (left.lo.xyz,  left child)    n1 = (left.hi.xyz,  right child)
//   n2 = (right.lo.xyz, 0)             n3 = (right.hi.xyz, 0)
// child >= 0 is an internal node index; child < 0 is a leaf with
// v = -child - 1, first = v >> 4 (index into the leaf-ordered triangle
// arrays), count = v & 15. parent[] and sibling[] drive the backtracking.
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cstdint>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <system_error>
#include <thread>
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

constexpr int PAR_MIN = 1 << 16;     // ranges at least this long split their passes over threads
constexpr int SPAWN_MIN = 1 << 13;   // subtrees at least this large may start a thread
constexpr int NB = 16;                // SAH bins per axis

struct Build {
    const float *V;
    const int32_t *T;
    std::vector<Box> tbox;
    std::vector<float> cen;   // 3 per tri
    std::vector<int32_t> idx, tmp;
    int nth;                  // threads the build may use
    std::atomic<int> running{1};   // threads working now (one waiting on a join does not count)
};

int32_t leaf_code(int first, int count) { return -(first * 16 + count) - 1; }

// f(part, lo, hi) over [0, n) in `parts` contiguous parts, parts > 1 on threads
template <class F>
void par_parts(int parts, int n, F f) {
    if (parts <= 1) {
        f(0, 0, n);
        return;
    }
    std::vector<std::thread> th;
    int q = 1;
    try {
        for (; q < parts; ++q)
            th.emplace_back(f, q, (int)((int64_t)n * q / parts), (int)((int64_t)n * (q + 1) / parts));
    } catch (const std::system_error &) {   // no thread to be had: the remaining parts run here
    }
    for (int r = q; r < parts; ++r) f(r, (int)((int64_t)n * r / parts), (int)((int64_t)n * (r + 1) / parts));
    f(0, 0, (int)((int64_t)n / parts));
    for (auto &t : th) t.join();
}

int parts_for(int count, int nt) { return count >= PAR_MIN ? std::max(1, std::min(nt, count / (PAR_MIN / 4))) : 1; }
// threads for one range's passes: the idle ones plus the caller
int range_threads(Build &b) { return std::max(1, b.nth - b.running.load() + 1); }

Box range_box(const Build &b, int first, int count, int nt) {
    const int parts = parts_for(count, nt);
    std::vector<Box> part(parts);
    par_parts(parts, count, [&](int q, int lo, int hi) {
        for (int i = first + lo; i < first + hi; ++i) part[q].grow(b.tbox[b.idx[i]]);
    });
    Box bx;
    for (const Box &x : part) bx.grow(x);
    return bx;
}

inline int bin_of(float c, float lo, float ext) {
    int k = (int)((c - lo) / ext * NB);
    return std::min(std::max(k, 0), NB - 1);
}

struct Bins {
    Box box[3][NB];
    int cnt[3][NB];
};

void bin_range(const Build &b, int lo, int hi, const Box &cb, const float *ext, Bins &B) {
    std::memset(B.cnt, 0, sizeof(B.cnt));
    for (int i = lo; i < hi; ++i) {
        const int t = b.idx[i];
        const Box &tb = b.tbox[t];
        for (int a = 0; a < 3; ++a) {
            if (!(ext[a] > 0.0f)) continue;
            const int k = bin_of(b.cen[3 * (size_t)t + a], cb.lo[a], ext[a]);
            B.cnt[a][k]++;
            B.box[a][k].grow(tb);
        }
    }
}

// choose a split of idx[first, first+count), whose triangles' bounds are pb;
// returns the split position or -1 for a leaf
int split(Build &b, int first, int count, int depth, int nt, const Box &pb) {
    const int maxleaf = 4;
    if (count <= maxleaf) return -1;
    const int parts = parts_for(count, nt);
    // centroid bounds
    Box cb;
    if (parts == 1) {
        for (int i = first; i < first + count; ++i) cb.grow(&b.cen[3 * (size_t)b.idx[i]]);
    } else {
        std::vector<Box> pcb(parts);
        par_parts(parts, count, [&](int q, int lo, int hi) {
            for (int i = first + lo; i < first + hi; ++i) pcb[q].grow(&b.cen[3 * (size_t)b.idx[i]]);
        });
        for (const Box &x : pcb) cb.grow(x);
    }
    // bins of all three axes (per part, then reduced)
    float ext[3];
    for (int a = 0; a < 3; ++a) ext[a] = cb.hi[a] - cb.lo[a];
    Bins one;
    std::vector<Bins> pb_(parts > 1 ? parts : 0);
    if (parts == 1) bin_range(b, first, first + count, cb, ext, one);
    else par_parts(parts, count, [&](int q, int lo, int hi) { bin_range(b, first + lo, first + hi, cb, ext, pb_[q]); });
    const Bins *bins_of = parts == 1 ? &one : pb_.data();
    double best = DBL_MAX;
    int best_axis = -1, best_bin = -1;
    for (int a = 0; a < 3; ++a) {
        if (!(ext[a] > 0.0f)) continue;
        Box bins[NB];
        int cnt[NB] = {0};
        for (int q = 0; q < parts; ++q)
            for (int k = 0; k < NB; ++k) {
                bins[k].grow(bins_of[q].box[a][k]);
                cnt[k] += bins_of[q].cnt[a][k];
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
    double leaf_cost = pb.area() * count;
    bool force = depth >= 58 || best_axis < 0;
    if (!force && count <= 15 && leaf_cost <= best + pb.area() * 1.0) return -1;
    int mid;
    if (best_axis >= 0 && !(depth >= 58)) {
        const int a = best_axis;
        auto left = [&](int t) { return bin_of(b.cen[3 * (size_t)t + a], cb.lo[a], ext[a]) <= best_bin; };
        if (parts == 1) {
            auto it = std::stable_partition(b.idx.begin() + first, b.idx.begin() + first + count, left);
            mid = (int)(it - b.idx.begin());
        } else {
            // stable partition in parts: count, place by prefix sums, copy back
            std::vector<int> nl(parts, 0);
            par_parts(parts, count, [&](int q, int lo, int hi) {
                int c = 0;
                for (int i = first + lo; i < first + hi; ++i) c += left(b.idx[i]) ? 1 : 0;
                nl[q] = c;
            });
            int tot = 0;
            std::vector<int> lb(parts), rb(parts);
            for (int q = 0; q < parts; ++q) {
                lb[q] = tot;
                tot += nl[q];
            }
            for (int q = 0, r = 0; q < parts; ++q) {
                rb[q] = tot + r;
                r += (int)((int64_t)count * (q + 1) / parts - (int64_t)count * q / parts) - nl[q];
            }
            par_parts(parts, count, [&](int q, int lo, int hi) {
                int l = first + lb[q], r = first + rb[q];
                for (int i = first + lo; i < first + hi; ++i) {
                    int t = b.idx[i];
                    if (left(t)) b.tmp[l++] = t;
                    else b.tmp[r++] = t;
                }
            });
            par_parts(parts, count, [&](int, int lo, int hi) {
                std::memcpy(&b.idx[first + lo], &b.tmp[first + lo], sizeof(int32_t) * (size_t)(hi - lo));
            });
            mid = first + tot;
        }
    } else {
        // degenerate centroids or depth limit: median split by index
        if (count <= 15) return -1;
        mid = first + count / 2;
    }
    if (mid <= first || mid >= first + count) mid = first + count / 2;
    return mid;
}

// The tree before numbering: a child is a leaf code or an internal node held
// in the arena of the thread that built it.
struct TNode;
struct Arena {
    std::vector<TNode> v;
};
struct Ref {
    Box box;
    int32_t code;   // leaf code when ar == nullptr
    Arena *ar;
    int ix;
};
struct TNode {
    Ref ch[2];
    int size;   // internal nodes of the subtree, this one included
};
inline int subtree_size(const Ref &c) { return c.ar ? c.ar->v[c.ix].size : 0; }

struct Arenas {
    std::mutex mu;
    std::deque<std::unique_ptr<Arena>> all;
    Arena *make() {
        std::lock_guard<std::mutex> g(mu);
        all.push_back(std::make_unique<Arena>());
        return all.back().get();
    }
};

// the subtree over idx[first, first+count) at `depth`; the left subtree of a
// large range goes to a new thread while fewer than nth threads are running
Ref build(Build &b, Arenas &as, Arena *ar, int first, int count, int depth) {
    Ref r;
    const int nt = count >= PAR_MIN ? range_threads(b) : 1;
    r.box = range_box(b, first, count, nt);
    r.ar = nullptr;
    r.ix = -1;
    int m = split(b, first, count, depth, nt, r.box);
    if (m < 0) {
        r.code = leaf_code(first, count);
        return r;
    }
    TNode nd;
    bool spawn = false;
    if (std::min(m - first, first + count - m) >= SPAWN_MIN) {
        int cur = b.running.load();
        while (cur < b.nth && !b.running.compare_exchange_weak(cur, cur + 1)) {
        }
        spawn = cur < b.nth;
    }
    std::thread t;
    if (spawn) {
        Arena *la = as.make();
        try {
            t = std::thread([&nd, &b, &as, la, first, m, depth]() {
                nd.ch[0] = build(b, as, la, first, m - first, depth + 1);
                b.running.fetch_sub(1);
            });
        } catch (const std::system_error &) {   // no thread to be had: build both sides here
            b.running.fetch_sub(1);
            spawn = false;
        }
    }
    if (spawn) {
        nd.ch[1] = build(b, as, ar, m, first + count - m, depth + 1);
        b.running.fetch_sub(1);   // idle while it waits
        t.join();
        b.running.fetch_add(1);
    } else {
        nd.ch[0] = build(b, as, ar, first, m - first, depth + 1);
        nd.ch[1] = build(b, as, ar, m, first + count - m, depth + 1);
    }
    nd.size = 1 + subtree_size(nd.ch[0]) + subtree_size(nd.ch[1]);
    ar->v.push_back(nd);
    r.code = 0;
    r.ar = ar;
    r.ix = (int)ar->v.size() - 1;
    return r;
}

struct Emit {
    std::vector<float> nodes;  // 16 floats per node
    std::vector<int32_t> parent, sibling;
};

void set_child(Emit &e, int node, int side, const Box &bx, int32_t code) {
    float *n = &e.nodes[(size_t)node * 16];
    float *lo = side == 0 ? n + 0 : n + 8;
    float *hi = side == 0 ? n + 4 : n + 12;
    for (int a = 0; a < 3; ++a) {
        lo[a] = bx.lo[a];
        hi[a] = bx.hi[a];
    }
    int32_t *w = reinterpret_cast<int32_t *>(side == 0 ? n + 3 : n + 7);
    *w = code;
}

// Writes the 64-byte layout of the subtree whose root gets index id, in
// pre-order: the left child (if internal) is id + 1, the right one follows
// the left subtree. Subtrees of large nodes near the root are written on
// their own threads; the indices do not depend on the order of writing.
constexpr int EMIT_PAR = 1 << 14;
void emit(Emit &e, const TNode &nd, int id, int parent, int depth) {
    e.parent[id] = parent;
    const int ids[2] = {id + 1, id + 1 + subtree_size(nd.ch[0])};
    for (int s = 0; s < 2; ++s) set_child(e, id, s, nd.ch[s].box, nd.ch[s].ar ? ids[s] : nd.ch[s].code);
    const Ref &l = nd.ch[0], &r = nd.ch[1];
    if (l.ar && r.ar && depth < 5 && nd.size >= EMIT_PAR) {
        std::thread t;
        try {
            t = std::thread([&e, &l, &ids, id, depth]() { emit(e, l.ar->v[l.ix], ids[0], id, depth + 1); });
        } catch (const std::system_error &) {   // no thread to be had: write both sides here
        }
        if (t.joinable()) {
            emit(e, r.ar->v[r.ix], ids[1], id, depth + 1);
            t.join();
            return;
        }
    }
    if (l.ar) emit(e, l.ar->v[l.ix], ids[0], id, depth + 1);
    if (r.ar) emit(e, r.ar->v[r.ix], ids[1], id, depth + 1);
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
    b.tmp.resize(nt);
    const int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    b.nth = nth;
    par_parts(parts_for(nt, nth), nt, [&](int, int lo, int hi) {
        for (int t = lo; t < hi; ++t) {
            Box bx;
            for (int k = 0; k < 3; ++k) bx.grow(&verts[3 * (size_t)tris[3 * (size_t)t + k]]);
            b.tbox[t] = bx;
            for (int a = 0; a < 3; ++a) b.cen[3 * (size_t)t + a] = 0.5f * (bx.lo[a] + bx.hi[a]);
            b.idx[t] = t;
        }
    });
    Emit e;
    // the root is always an internal node; its children come from splitting all triangles
    Arenas as;
    Arena *root_ar = as.make();
    Ref root = build(b, as, root_ar, 0, nt, 0);
    if (!root.ar) {
        e.nodes.assign(16, 0.0f);
        e.parent.push_back(-1);
        e.sibling.push_back(-1);
        set_child(e, 0, 0, root.box, leaf_code(0, nt));
        set_child(e, 0, 1, Box(), leaf_code(0, 0));
    } else {
        const TNode &rn = root.ar->v[root.ix];
        e.nodes.assign(16 * (size_t)rn.size, 0.0f);
        e.parent.assign((size_t)rn.size, -1);
        e.sibling.assign((size_t)rn.size, -1);
        emit(e, rn, 0, -1, 0);
    }
    int nn = (int)(e.nodes.size() / 16);
    // sibling of each internal child
    for (int n = 0; n < nn; ++n) {
        const int32_t *w = reinterpret_cast<const int32_t *>(&e.nodes[(size_t)n * 16]);
        int32_t l = w[3], r = w[7];
        if (l >= 0 && r >= 0) {
            e.sibling[l] = r;
            e.sibling[r] = l;
        } else if (l >= 0) {
            e.sibling[l] = -1;
        } else if (r >= 0) {
            e.sibling[r] = -1;
        }
    }
    out->nodes = std::move(e.nodes);
    out->parent = std::move(e.parent);
    out->sibling = std::move(e.sibling);
    out->order = std::move(b.idx);
    return nn;
}
