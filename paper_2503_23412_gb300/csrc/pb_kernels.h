// Shared declarations of the renderer's kernels and their device buffers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pb_device.cuh"

// Accumulators of the table-learning eye passes (null when rendering).
struct LearnAcc {
    float *conn;        // KT*KS: unweighted connection contribution luminance per (T, S)
    float *proxy;       // KT*KSp: unweighted proxy contribution luminance per (T, S')
    float *tile_all;    // per tile: weighted contribution luminance
    float *tile_proxy;  // per tile: weighted proxy contribution luminance
};

// Render parameters as the kernels see them.
// Learned light-subspace proposal. The feature pass traces the camera
// sub-paths once, stores every eye vertex's hit (replayed by the eye pass
// instead of tracing again) and appends one network input row per vertex
// that makes a subspace connection. Dense index of a connecting vertex:
// ((slot * A) + a - 1) * npix + pix for a = 1..A; of a hit:
// ((slot * max_depth) + a - 1) * npix + pix for a = 1..max_depth.
struct MlpRows {
    uint16_t *rows;         // compact: bf16[16] network input per row
    int32_t *rowT;          // compact: eye subspace T of the row
    int32_t *rowPos;        // compact: dense index of the row's vertex
    unsigned int *count;    // rows appended
    int cap;                // rows the compact arrays hold
    int4 *hits;             // dense: the eye vertex's hit (tri, t, b1, b2), tri = -1: the path left the scene
    const int32_t *sel;     // dense: selected light subspace (-1: none)
    const float *selq;      // dense: its proposal probability Q(S | x)
    const uint16_t *emb;    // bf16[KT][4] embedding of T
    int A;                  // eye vertices with a row per pixel (max_depth - 2)
};

// Training samples of the proposal: one per connection with a non-zero
// contribution (raw features, T, S, unweighted contribution luminance).
struct SampleSink {
    float *raw;             // [cap][10]
    int32_t *T, *S;
    float *w;
    unsigned int *count;
    int cap;
};

// Buffers of the wavefront estimator (pb_light.cu): per chain (one per
// (entry, repeat) of the wave) its window of nodes this round, per node its
// chain, pre-order index, answered queries, pending query and result.
// a query of the replay tracer (pb_estimator.cuh): kind 0 closest hit, 1
// closest hit that only counts on an emitter, 2 occlusion of the segment o -> d
struct WfQuery {
    float3 o, d;
    int skip, skip2, kind;
};
// its answer: closest hit (tri, barycentrics; tri -1 for none) or, for an
// occlusion query, tri = 1 occluded / 0 visible
struct WfResult {
    int tri;
    float b1, b2;
};
constexpr int WF_MAXQ = 5;   // at most u = 4 closest hits and one occlusion per node
constexpr int WF_ROUNDS = 40;   // wavefront rounds launched per wave (idle rounds exit at once)

struct WfBufs {
    int32_t *ch_w, *ch_off, *ch_win;   // per chain: nodes this round, first node, window size
    uint8_t *ch_done;
    int32_t *node_chain, *node_v, *node_nq;
    struct WfResult *node_res;         // WF_MAXQ per node
    struct WfQuery *node_q;
    float *node_g;                     // g and children under the estimate's own bound
    int32_t *node_n;
    float *node_x, *node_u;            // f/q and the RRS uniform (the walk under a raised bound)
    int32_t *list[2];                  // nodes that need a step (ping-pong)
    int32_t *ctl;                      // counters (WF_CTL_* in pb_light.cu)
    int node_cap;
    // pilot of the per-entry bound, run as the same stages: per entry
    int32_t *pil_next;                 // draws evaluated so far
    float *pil_best, *pil_sum;         // largest f/q and sum of f/q over the counted draws
    int32_t *pil_draws;                // draws counted (whole blocks of 32 before the stop)
};

// Occlusion queries of the eye pass (the camera-side wavefront): one pass
// replays the camera sub-paths and appends every NEE, connection and
// proxy-entry visibility query (warp-aggregated), a traversal-only kernel
// answers them, and the shading pass reads the answers. Dense vertex index:
// ((slot * max_depth) + a - 1) * npix + pix; kinds 0 NEE, 1 connection,
// 2 the proxy's first segment z -> y_{s-1}.
struct EyeQueries {
    float4 *qa, *qb;        // segment a -> b: a.xyz and a's skip triangle, b.xyz and b's (int bits in .w)
    int32_t *dst;           // per query: dense vertex index * 4 + kind
    unsigned int *count;    // queries appended this wave
    int cap;                // queries the arrays hold (every vertex's at most: no overflow)
    uint8_t *vis;           // [kind][dense]: 1 the segment is unoccluded
    size_t plane;           // bytes per kind: slots * max_depth * npix
};
constexpr int EYE_INLINE = 0, EYE_EMIT = 1, EYE_READ = 2;

struct KParams {
    uint32_t seed;
    int max_depth, M, M_p, repeats, proxy, conn, trial_cap;
    int L;          // light-path vertex slots = max_depth - 1
    int npix;
    int count;      // 1: count traversal work (node fetches, triangle tests, rays)
    int handoff;    // estimator nodes walked by a warp before a block continues the chain
    int pilot_min, pilot_max;   // per-entry B pilot draws (multiples of 32; pilot_max 0 = off)
    float side_in;              // cosine draws at a dielectric y_{s-1} on the side of y_{s-2}
    int estimator;              // 0: wavefront; 1: warp and block phases
    float booth;                // > 0: Booth's roulette of this scale (wavefront only); 0: the paper's RRS
    int trace;                  // wavefront trace stages: 0 a query per thread; 1 persistent warps, lane refill
    int film;                   // strategies reaching the film: 0 all, 1 the proxy strategy only, 2 all but it
    uint32_t split;             // first pre-order estimator node without splitting (split limit)
    int fixed_bound;            // 1: one B per estimate; 0: the raise rule (est_child_invB)
    LearnAcc acc;
    MlpRows mlp;            // rows != nullptr: write rows (feature pass); sel != nullptr: select with them
    MlpRows mlpp;           // the proxy strategy's network: rows at the proxy's vertex, its S' selections
    SampleSink smp;         // raw != nullptr: record proposal training samples
    SampleSink smpp;        // raw != nullptr: record the proxy network's training samples
    int proposal;           // 0 table rows; 1 learned connection; 2 learned connection and proxy
    EyeQueries q;           // the eye pass's occlusion queries and answers (vis == nullptr: traced inline)
    const uint32_t *iter_dev;   // non-null (graph replay): iteration numbers are *iter_dev + the launch's base
};

// rounds of the wavefront pilot: windows pilot_min, then doubling, until pilot_max
__host__ __device__ inline int wf_pilot_rounds(const KParams &P) {
    if (P.pilot_max <= 0) return 0;
    int nr = 1;
    for (int tot = P.pilot_min, w = P.pilot_min; tot < P.pilot_max; w *= 2) {
        tot += w;
        ++nr;
    }
    return nr;
}

// g = 1 - (f/q) / B of an estimator node, given 1/B, with one rounding (a fused
// multiply-add written out): every kernel that evaluates a node gets the same
// bits, whatever the compiler would contract at each site
__device__ __forceinline__ float est_g(float x, float invB) { return __fmaf_rn(-x, invB, 1.0f); }

// Children of an estimator node (Alg. I~ with the split limit): the paper's
// r = |g|, i.e. floor(|g|) + Bernoulli(frac) children entering with weight
// sign(g); from pre-order node `split` on, a node with |g| > 1 has one child
// entering with weight g. The estimator is unbiased for any such rule (each
// child's estimate has the same expectation); trees that would split without
// end (a bound far below some f/q) become chains.
__device__ __forceinline__ int est_children(float g, float u, uint32_t v, uint32_t split) {
    const float r = fabsf(g);
    if (r > 1.0f && v >= split) return 1;
    int n = (int)floorf(r);
    if (u < r - (float)n) n += 1;
    return n;
}
__device__ __forceinline__ float est_child_weight(float g, uint32_t v, uint32_t split) {
    return (fabsf(g) > 1.0f && v >= split) ? g : (g > 0.0f ? 1.0f : -1.0f);
}

// The bound a node hands its children. The paper keeps one B for a whole
// estimate; here a node that splits (|g| > 1, i.e. f/q > 2B) gives its
// children the bound B' = its own f/q. The estimate of 1/beta stays
// unbiased under any bound fixed before a node's draw (1/beta = 1/B +
// (1 - beta/B) / beta holds for every B, node by node), and the node's term
// becomes g / B', the expected own term of its children, each of which
// enters with 1 / B'. Chains whose draws stay below 2B never raise the
// bound, so they are the paper's walk exactly; a tree that would split
// without end under a low B grows only as far as its own ratios allow.
__device__ __forceinline__ float est_child_invB(float g, float x, float invB, int fixed) {
    return (!fixed && fabsf(g) > 1.0f) ? 1.0f / x : invB;
}

// One node of the exact walk on the stack form: frames of pending children
// that share a weight and a bound; children whose weight and bound match the
// frame on top join it. g0, n0 are the node's g and children under the
// estimate's own bound invB0 (x = f/q, u = the node's RRS uniform), reused
// while the current bound is that one.
struct EstStep {
    float g, cw, cib;   // g under the current bound; the children's weight and inverse bound
    int n;
    bool push;          // the children need a frame of their own
};
template <class St>
__device__ __forceinline__ EstStep est_step(const St &st, float x, float u, float g0, int n0, float invB0, uint32_t v,
                                            const KParams &P) {
    EstStep e;
    if (st.cur_ib == invB0) {
        e.g = g0;
        e.n = n0;
    } else {
        e.g = est_g(x, st.cur_ib);
        e.n = est_children(e.g, u, v, P.split);
    }
    e.cib = est_child_invB(e.g, x, st.cur_ib, P.fixed_bound);
    e.cw = st.cur_sign * est_child_weight(e.g, v, P.split);
    e.push = e.n >= 1 && !(st.sp > 0 && st.fr_sign[st.sp - 1] == e.cw && st.fr_ib[st.sp - 1] == e.cib);
    return e;
}
// Takes the node: adds its term and its children, then moves to the next
// pending node. Returns 0 to go on, 1 when the chain has ended, 2 when the
// children needed a frame beyond CAP or their weight left the float range
// (a truncated estimate).
template <int CAP, class St>
__device__ __forceinline__ int est_take(St &st, const EstStep &e, double &sum_t) {
    sum_t += (double)(st.cur_sign * e.g * e.cib);
    if (e.n >= 1) {
        if (!e.push) {
            st.fr_rem[st.sp - 1] += e.n;
        } else {
            if (st.sp >= CAP || !isfinite(e.cw)) return 2;
            st.fr_sign[st.sp] = e.cw;
            st.fr_ib[st.sp] = e.cib;
            st.fr_rem[st.sp] = e.n;
            st.sp++;
        }
    }
    if (st.sp == 0) return 1;
    st.cur_sign = st.fr_sign[st.sp - 1];
    st.cur_ib = st.fr_ib[st.sp - 1];
    if (--st.fr_rem[st.sp - 1] == 0) st.sp--;
    return 0;
}
// Whether the walk state is on the count form: every pending node has
// weight +1 under the estimate's own bound. pend = pending nodes, the
// current one included.
template <class St>
__device__ __forceinline__ bool est_count_form(const St &st, float invB0, int &pend) {
    bool pos = st.cur_sign == 1.0f && st.cur_ib == invB0;
    pend = 1;
    for (int f = 0; f < st.sp; ++f) {
        pos = pos && st.fr_sign[f] == 1.0f && st.fr_ib[f] == invB0;
        pend += st.fr_rem[f];
    }
    return pos;
}
// Whether the walk state is on the uniform count form: every pending node
// (the current one and all frames) has one weight w and one inverse bound ib.
// A run of nodes with g >= 0 under ib then keeps that form (their children
// enter with weight w and bound ib), so the walk reduces to pending counts
// and terms w g ib. pend = pending nodes, the current one included.
template <class St>
__device__ __forceinline__ bool est_uniform_form(const St &st, float &w, float &ib, int &pend) {
    w = st.cur_sign;
    ib = st.cur_ib;
    pend = 1;
    bool ok = true;
    for (int f = 0; f < st.sp; ++f) {
        ok = ok && st.fr_sign[f] == w && st.fr_ib[f] == ib;
        pend += st.fr_rem[f];
    }
    return ok;
}
// the uniform form with `pend` pending nodes as a stack of at most one frame
template <class St>
__device__ __forceinline__ void est_from_uniform(St &st, int pend, float w, float ib) {
    st.cur_sign = w;
    st.cur_ib = ib;
    st.sp = 0;
    if (pend - 1 > 0) {
        st.fr_sign[0] = w;
        st.fr_ib[0] = ib;
        st.fr_rem[0] = pend - 1;
        st.sp = 1;
    }
}
// The top region of the walk state: the current node and the frames on top
// that share its weight w and inverse bound ib. Until those pending nodes and
// their descendants are walked, the frames below are not touched, so a run of
// nodes with g >= 0 under ib is a pending-count walk of the region alone.
// est_take_top removes the region from the stack and returns its pending
// count; est_put_top pushes it back (one frame, which differs from the frame
// below it); est_pop_below moves to the first pending node under an exhausted
// region (false: none is left, the chain has ended).
template <class St>
__device__ __forceinline__ int est_take_top(St &st, float &w, float &ib) {
    w = st.cur_sign;
    ib = st.cur_ib;
    int pend = 1;
    while (st.sp > 0 && st.fr_sign[st.sp - 1] == w && st.fr_ib[st.sp - 1] == ib) {
        pend += st.fr_rem[st.sp - 1];
        st.sp--;
    }
    return pend;
}
// (false: the region needs a frame beyond CAP, a truncated estimate)
template <int CAP, class St>
__device__ __forceinline__ bool est_put_top(St &st, int pend, float w, float ib) {
    st.cur_sign = w;
    st.cur_ib = ib;
    if (pend - 1 > 0) {
        if (st.sp >= CAP) return false;
        st.fr_sign[st.sp] = w;
        st.fr_ib[st.sp] = ib;
        st.fr_rem[st.sp] = pend - 1;
        st.sp++;
    }
    return true;
}
template <class St>
__device__ __forceinline__ bool est_pop_below(St &st) {
    if (st.sp == 0) return false;
    st.cur_sign = st.fr_sign[st.sp - 1];
    st.cur_ib = st.fr_ib[st.sp - 1];
    if (--st.fr_rem[st.sp - 1] == 0) st.sp--;
    return true;
}
// g and children of a node under the inverse bound ib, as est_step computes
// them (the values drawn under the estimate's own bound invB0 are reused)
__device__ __forceinline__ void est_gn(float x, float u, float g0, int n0, float invB0, float ib, uint32_t v,
                                       uint32_t split, float &g, int &n) {
    if (ib == invB0) {
        g = g0;
        n = n0;
    } else {
        g = est_g(x, ib);
        n = est_children(g, u, v, split);
    }
}
// the count form with `pend` pending nodes as a stack of at most one frame
template <class St>
__device__ __forceinline__ void est_from_count(St &st, int pend, float invB0) {
    st.cur_sign = 1.0f;
    st.cur_ib = invB0;
    st.sp = 0;
    if (pend - 1 > 0) {
        st.fr_sign[0] = 1.0f;
        st.fr_ib[0] = invB0;
        st.fr_rem[0] = pend - 1;
        st.sp = 1;
    }
}

__device__ __forceinline__ uint32_t eff_iter(const KParams &P, uint32_t iter_base) {
    return P.iter_dev ? iter_base + *P.iter_dev : iter_base;
}

// Walk state of a reciprocal estimate handed from a warp to a block: the next
// pre-order node index, the running sums, the sign of the next node and the
// stack of pending sibling groups (sign, remaining count).
#define PB_MAXF 48
struct ChainState {
    int slot, k, rep, next;
    double sum_t;
    float cur_sign, cur_ib;   // the current node's weight and inverse bound
    int sp;
    float fr_sign[PB_MAXF];   // frames of pending children: weight, inverse bound, count
    float fr_ib[PB_MAXF];
    int fr_rem[PB_MAXF];
    double prod, surv;   // Booth's roulette: product of g so far, product of the continuation probabilities
};

// Device buffers of the iterations in flight ("slots"). Per-light-vertex
// arrays are indexed [slot][l * L + e].
struct Pool {
    int slots, ML;  // ML = M * L
    int32_t *gtri;  // geometry
    float2 *gbary;
    float4 *vpos;    // p.xyz, material (int bits)
    float4 *vnrm;    // n.xyz, triangle (int bits)
    float4 *vwl;     // w_light.xyz (toward y_{e-1}), fwd_e
    float4 *valpha;  // alpha rgb (f_y/p_y up to y_e), Lpart = Lsum_{e-2}
    float4 *vmis;    // fwd_{e-1}, cos_{e-1}, d2(y_{e-1}, y_e), availability bits
    int32_t *vlabel; // light subspace S of a connectable vertex, else -1
    int32_t *elabel; // specular subspace S' of an incomplete sub-path end, else -1
    int32_t *einfo;  // u | type << 3 | C << 4
    int32_t *pool_idx, *bstart, *bitems, *npool;   // connection pool, (l,e) order and by S
    int32_t *ent_idx, *estart, *eitems, *nent;     // incomplete sub-paths, (l,e) order and by S'
    float *cdfC, *ZC, *cdfP, *ZP;                  // selection CDF rows per eye subspace
    float *rep, *repn;                             // per (entry, repeat): estimate, nodes
    int32_t *reptr;
    float *rhat;                                   // per entry: averaged reciprocal estimate
    float *eB;                                     // per entry: bound B of its estimates
    float *eMu;                                    // per entry: expected nodes per estimate, B / mean(f/q) (0: unknown)
    uint32_t *esig;
    int32_t *work;                                 // work counters, per-slot work offsets
    struct ChainState *chains;                     // estimates continued by whole blocks
    int chain_cap;
    int32_t *scratch;                              // 2 * slots * ML ints for the bucket sort
    unsigned long long *counters;                  // stats
};

enum {
    CNT_ENTRIES = 0, CNT_TRUNC, CNT_NODES, CNT_CONN, CNT_PROXY, CNT_PROXY_OK, CNT_NFETCH, CNT_TTEST,
    CNT_EYE_NODES, CNT_EYE_TRIS, CNT_EYE_RAYS, CNT_REC_NODES, CNT_REC_TRIS, CNT_REC_RAYS,
    CNT_CAM_NODES, CNT_CAM_TRIS, CNT_CAM_RAYS, CNT_SHD_NODES, CNT_SHD_TRIS, CNT_SHD_RAYS, CNT_N
};

void launch_light_pass(const DScene &S, const KParams &P, const Pool &B, int slots, uint32_t iter_base,
                       cudaStream_t st);
void launch_pool_build(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots,
                       cudaStream_t st);
void launch_recip(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots,
                  uint32_t iter_base, int num_sms, cudaStream_t st, const WfBufs *wf = nullptr);
// the estimator's per-entry bound B (the pilot, or the table values when the
// pilot is off) and its warp/block schedule (estimator = 1)
void launch_recip_bounds(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots,
                         uint32_t iter_base, int num_sms, cudaStream_t st, bool count);
void launch_recip_phases(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots,
                         uint32_t iter_base, int num_sms, cudaStream_t st);
// phase 2 of that schedule, without and with traversal counting
void launch_recip_long_plain(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots,
                             uint32_t iter_base, int num_sms, cudaStream_t st);
void launch_recip_long_counting(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots,
                                uint32_t iter_base, int num_sms, cudaStream_t st);
// the wavefront schedule of the estimator (pilot rounds when P.pilot_max > 0,
// node rounds, finisher); launch_recip brackets it with the offsets, the
// table-bound kernel when there is no pilot, and the repeat averages
void launch_recip_wavefront(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots,
                            uint32_t iter_base, int num_sms, cudaStream_t st, const WfBufs &W);
// the eye pass: mode EYE_INLINE traces its occlusion queries itself;
// EYE_EMIT appends them to P.q and writes nothing else; EYE_READ reads
// their answers from P.q.vis
void launch_eye(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots, uint32_t iter_base,
                float4 *Lbuf, uint32_t *sigbuf, cudaStream_t st, int mode = EYE_INLINE);
// traversal-only answers of the queries the EYE_EMIT pass appended
// fetch: a device counter for the persistent variant (KParams.trace = 1; nullptr: one query per thread)
void launch_eye_occ(const DScene &S, const KParams &P, const Pool &B, int num_sms, cudaStream_t st,
                    unsigned int *fetch = nullptr);
void launch_eye_feat(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots, uint32_t iter_base,
                     cudaStream_t st);
void launch_film_add(const KParams &P, int slots, const float4 *Lbuf, float *film, cudaStream_t st);
void launch_trace(const DScene &S, const float *rays, int n, float *hits, int count, unsigned long long *counters,
                  cudaStream_t st);
void launch_occluded(const DScene &S, const float *seg, int n, int32_t *out, cudaStream_t st);
