// The reciprocal estimator's wavefront schedule (Sec. 4.2, App. Alg. I~, and
// App. "Optimal value for B" for the per-entry pilot):
//   k_wfp_*          the pilot of B as wavefront rounds
//   k_wf_init/plan   windows of pre-order nodes per chain and round
//   k_wf_nodes       the (chain, node) list of a round
//   k_wf_step        replay of each node's draw up to its next ray query
//   k_wf_trace       traversal-only answers to the recorded queries
//   k_wf_trace_pt    the same with persistent warps that refill idle lanes
//   k_wf_walk        the paper's RRS walk per chain (warp scans)
//   k_wf_walk_booth  Booth's roulette per chain (the RR ablation's baseline)
//   k_wf_finish_rest chains still open after the last round
#include <cstdio>

#include <cooperative_groups.h>

#include "pb_entry.cuh"

namespace cg = cooperative_groups;

namespace {

// ---------------------------------------------------------------------------
// Wavefront estimator. Every (entry, repeat) of the wave is a chain. Each
// round gives every unfinished chain a window of consecutive pre-order nodes
// (sized from the entry's expected chain length, doubling while the chain
// lasts), then evaluates all nodes of all windows in stages: a step kernel
// replays a node's draw (entry_ratio with the replay tracer) up to its next
// ray query, a traversal-only kernel answers the queries, and so on until
// every node has its f/q. A walk per chain then consumes its window in
// pre-order exactly as the sequential definition does. Node values depend
// only on (entry, repeat, node), so the estimates are those of the warp and
// block phases.
enum { WF_CTL_ITEMS = 0, WF_CTL_NODES, WF_CTL_ACTIVE, WF_CTL_ERR, WF_CTL_CNT0 };   // CNT0 .. CNT0 + WF_MAXQ + 1
constexpr int WF_WIN_MAX = 1 << 18;   // a window doubles per round up to this many nodes

__global__ void k_wf_init(KParams P, Pool B, WfBufs W, int slots) {
    const int32_t *offs = B.work + 1;
    int total = offs[slots];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        W.ctl[WF_CTL_ITEMS] = min(total, B.chain_cap);
        W.ctl[WF_CTL_ACTIVE] = min(total, B.chain_cap);
        W.ctl[WF_CTL_ERR] = total > B.chain_cap ? 1 : 0;
    }
    int items = min(total, B.chain_cap);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < items; c += gridDim.x * blockDim.x) {
        int slot = 0;
        while (c >= offs[slot + 1]) ++slot;
        int local = c - offs[slot];
        ChainState st;
        st.slot = slot;
        st.k = local / P.repeats;
        st.rep = local % P.repeats;
        st.next = 0;
        st.sum_t = 0.0;
        st.cur_sign = 1.0f;
        st.cur_ib = 1.0f / B.eB[(size_t)slot * B.ML + st.k];
        st.sp = 0;
        st.prod = 1.0;
        st.surv = 1.0;
        B.chains[c] = st;
        W.ch_done[c] = 0;
        // first window: about half the expected chain length, 64 .. 2048 nodes
        float mu = B.eMu[(size_t)slot * B.ML + st.k];
        int win = 256;
        if (mu > 0.0f) {
            win = 64;
            while (win < 2048 && (float)win < 0.5f * mu) win <<= 1;
        }
        W.ch_win[c] = win;
    }
}

// one block: windows of this round and their node offsets (exclusive scan)
__global__ void __launch_bounds__(1024) k_wf_plan(KParams P, Pool B, WfBufs W) {
    // 64-bit sums: windows of up to WF_WIN_MAX nodes over all chains exceed int
    __shared__ long long part[1024];
    const int items = W.ctl[WF_CTL_ITEMS];
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid <= WF_MAXQ + 1) W.ctl[WF_CTL_CNT0 + tid] = 0;
    if (W.ctl[WF_CTL_ACTIVE] == 0) {
        if (tid == 0) W.ctl[WF_CTL_NODES] = 0;
        return;
    }
    const int per = (items + nt - 1) / nt;
    const int c0 = tid * per, c1 = min(items, c0 + per);
    long long acc = 0;
    for (int c = c0; c < c1; ++c) {
        int w = 0;
        if (!W.ch_done[c]) w = max(0, min(W.ch_win[c], P.trial_cap - B.chains[c].next));
        W.ch_w[c] = w;
        acc += w;
    }
    part[tid] = acc;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        long long x = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += x;
        __syncthreads();
    }
    long long run = part[tid] - acc;
    for (int c = c0; c < c1; ++c) {
        int w = W.ch_w[c];
        if (run + w > (long long)W.node_cap) w = 0;   // no room this round: the chain waits
        W.ch_w[c] = w;
        W.ch_off[c] = (int)min(run, (long long)W.node_cap);
        run += w;
    }
    __syncthreads();
    if (tid == nt - 1) W.ctl[WF_CTL_NODES] = (int)min(part[nt - 1], (long long)W.node_cap);
}

template <bool PILOT>
__global__ void k_wf_nodes(Pool B, WfBufs W) {
    const int items = W.ctl[WF_CTL_ITEMS], nodes = W.ctl[WF_CTL_NODES];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nodes; i += gridDim.x * blockDim.x) {
        // the last chain whose window starts at or before i (chains with an
        // empty window share the offset of the next one and come before it)
        int lo = 0, hi = items - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (W.ch_off[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        W.node_chain[i] = lo;
        W.node_v[i] = (PILOT ? W.pil_next[lo] : B.chains[lo].next) + (i - W.ch_off[lo]);
        W.node_nq[i] = 0;
        W.list[0][i] = i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) W.ctl[WF_CTL_CNT0] = nodes;
}

// the (slot, entry) of the e-th entry of the wave
__device__ __forceinline__ void wave_entry(const Pool &B, const KParams &P, int slots, int e, int &slot, int &k) {
    const int32_t *offs = B.work + 1;   // per slot: first (entry, repeat) item
    slot = 0;
    while (e * P.repeats >= offs[slot + 1] && slot < slots - 1) ++slot;
    k = e - offs[slot] / P.repeats;
}

// stage s: replay each listed node up to its next query (or to its f/q).
// PILOT: the node is draw v of the pilot of entry node_chain (stream PILOT),
// and its result is f/q itself.
template <bool PILOT>
__global__ void __launch_bounds__(128) k_wf_step(DScene S, KParams P, Pool B, WfBufs W, int s, uint32_t iter_base,
                                                 int slots) {
    iter_base = eff_iter(P, iter_base);
    const int n = W.ctl[WF_CTL_CNT0 + s];
    const int32_t *in = W.list[s & 1];
    int32_t *out = W.list[(s + 1) & 1];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int i = in[idx];
        int slot, k, rep = 0;
        if (PILOT) {
            wave_entry(B, P, slots, W.node_chain[i], slot, k);
        } else {
            const ChainState &st = B.chains[W.node_chain[i]];
            slot = st.slot;
            k = st.k;
            rep = st.rep;
        }
        int Sp, C;
        Entry E = load_entry(S, P, B, slot, k, Sp, C);
        const float invB = PILOT ? 0.0f : 1.0f / B.eB[(size_t)slot * B.ML + k];
        const int v = W.node_v[i];
        Rng R;
        if (PILOT) R.init(P.seed, K_PILOT, iter_base + slot, (uint32_t)k, (uint32_t)v);
        else R.init(P.seed, K_RECIP, iter_base + slot, (uint32_t)(k * 8 + rep), (uint32_t)v);
        ReplayTracer T;
        T.res = W.node_res + (size_t)WF_MAXQ * i;
        T.nres = W.node_nq[i];
        T.next = 0;
        T.susp = false;
        float ratio = entry_ratio_t<false>(S, E, R, T);
        if (T.susp && s == WF_MAXQ) {   // cannot happen (u <= 4): keep the walk defined and report
            atomicExch(&W.ctl[WF_CTL_ERR], 2);
            W.node_g[i] = 1.0f;
            W.node_n[i] = 0;
            W.node_x[i] = 0.0f;
            W.node_u[i] = 1.0f;
        } else if (T.susp) {
            W.node_q[i] = T.q;
            cg::coalesced_group g = cg::coalesced_threads();
            int base = 0;
            if (g.thread_rank() == 0) base = atomicAdd(&W.ctl[WF_CTL_CNT0 + s + 1], (int)g.size());
            out[g.shfl(base, 0) + g.thread_rank()] = i;
        } else if (PILOT) {
            W.node_g[i] = ratio;
        } else {
            const float gv = est_g(ratio, invB), u18 = R.u(18);
            W.node_g[i] = gv;
            W.node_n[i] = est_children(gv, u18, (uint32_t)W.node_v[i], P.split);
            W.node_x[i] = ratio;
            W.node_u[i] = u18;
        }
    }
}

// pilot: entries of the wave, first window pilot_min draws
__global__ void k_wfp_init(KParams P, Pool B, WfBufs W, int slots) {
    const int32_t *offs = B.work + 1;
    const int ents = min(offs[slots] / P.repeats, B.chain_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        W.ctl[WF_CTL_ITEMS] = ents;
        W.ctl[WF_CTL_ACTIVE] = ents;
    }
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ents; e += gridDim.x * blockDim.x) {
        W.pil_next[e] = 0;
        W.pil_best[e] = 0.0f;
        W.pil_sum[e] = 0.0f;
        W.pil_draws[e] = 0;
        W.ch_done[e] = 0;
        W.ch_win[e] = P.pilot_min;
    }
}

// one block: pilot windows of this round and their node offsets
__global__ void __launch_bounds__(1024) k_wfp_plan(KParams P, WfBufs W) {
    __shared__ int part[1024];
    const int items = W.ctl[WF_CTL_ITEMS];
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid <= WF_MAXQ + 1) W.ctl[WF_CTL_CNT0 + tid] = 0;
    const int per = (items + nt - 1) / nt;
    const int c0 = tid * per, c1 = min(items, c0 + per);
    int acc = 0;
    for (int c = c0; c < c1; ++c) {
        int w = W.ch_done[c] ? 0 : max(0, min(W.ch_win[c], P.pilot_max - W.pil_next[c]));
        W.ch_w[c] = w;
        acc += w;
    }
    part[tid] = acc;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        int x = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += x;
        __syncthreads();
    }
    int run = part[tid] - acc;
    for (int c = c0; c < c1; ++c) {
        int w = W.ch_w[c];
        if (run + w > W.node_cap) w = 0;   // no room this round
        W.ch_w[c] = w;
        W.ch_off[c] = run;
        run += w;
    }
    __syncthreads();
    if (tid == nt - 1) W.ctl[WF_CTL_NODES] = min(part[nt - 1], W.node_cap);
}

// one warp per entry: the pilot's stopping rule over this round's draws, in
// blocks of 32 (stop at the first block boundary >= pilot_min once some
// draw had f > 0; draws evaluated past the stop are not counted)
__global__ void __launch_bounds__(128) k_wfp_reduce(DScene S, KParams P, Pool B, DTables T, WfBufs W, int slots,
                                                    int last_round) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int items = W.ctl[WF_CTL_ITEMS];
    for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < items; e += warps) {
        if (W.ch_done[e]) continue;
        const int w = W.ch_w[e], off = W.ch_off[e];
        int next = W.pil_next[e];
        float best = W.pil_best[e], sum = W.pil_sum[e];
        int draws = W.pil_draws[e];
        bool stop = false;
        for (int b = 0; b < w; b += 32) {
            if (next + b >= P.pilot_min && best > 0.0f) {
                stop = true;
                break;
            }
            float x = W.node_g[off + b + lane];
            float m = x, t = x;
            for (int o = 16; o > 0; o >>= 1) {
                m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                t += __shfl_xor_sync(0xffffffffu, t, o);
            }
            best = fmaxf(best, m);
            sum += t;
            draws += 32;
        }
        next += w;
        if (!stop && next >= P.pilot_min && best > 0.0f) stop = true;
        if (!stop && (next >= P.pilot_max || last_round)) stop = true;
        if (lane == 0) {
            W.pil_next[e] = next;
            W.pil_best[e] = best;
            W.pil_sum[e] = sum;
            W.pil_draws[e] = draws;
            if (stop) {
                int slot, k;
                wave_entry(B, P, slots, e, slot, k);
                int Sp, C;
                Entry E = load_entry(S, P, B, slot, k, Sp, C);
                float Bv = best > 0.0f ? best : T.Bt[((E.u - 1) * T.KSp + Sp) * (T.KC + 1) + C];
                B.eB[(size_t)slot * B.ML + k] = Bv;
                B.eMu[(size_t)slot * B.ML + k] = sum > 0.0f ? Bv * (float)draws / sum : 0.0f;
                W.ch_done[e] = 1;
            } else {
                W.ch_win[e] = 2 * W.ch_win[e];
            }
        }
    }
}

// stage s: answer the queries the step kernel recorded
template <bool COUNT>
__global__ void __launch_bounds__(128) k_wf_trace(DScene S, KParams P, Pool B, WfBufs W, int s) {
    TravCount tc{0, 0, 0};
    const int n = W.ctl[WF_CTL_CNT0 + s + 1];
    const int32_t *lst = W.list[(s + 1) & 1];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int i = lst[idx];
        const WfQuery q = W.node_q[i];
        WfResult res;
        if (q.kind == 2) {
            res.tri = occluded<COUNT>(S, q.o, q.d, q.skip, q.skip2, &tc) ? 1 : 0;
            res.b1 = res.b2 = 0.0f;
        } else {
            Hit h = (q.kind == 1 && S.ne <= PB_EMITTER_LIST_MAX) ? closest_emitter_hit<COUNT>(S, q.o, q.d, q.skip, &tc)
                                                                  : closest_hit<COUNT>(S, q.o, q.d, q.skip, &tc);
            res.tri = h.tri;
            res.b1 = h.b1;
            res.b2 = h.b2;
        }
        int nq = W.node_nq[i];
        if (nq < WF_MAXQ) {
            W.node_res[(size_t)WF_MAXQ * i + nq] = res;
            W.node_nq[i] = nq + 1;
        }
    }
    if (COUNT) {
        atomicAdd(&B.counters[CNT_REC_NODES], (unsigned long long)tc.nodes);
        atomicAdd(&B.counters[CNT_REC_TRIS], (unsigned long long)tc.tris);
        atomicAdd(&B.counters[CNT_REC_RAYS], (unsigned long long)tc.rays);
    }
}

// Persistent variant of k_wf_trace (KParams.trace = 1). A warp keeps its 32
// lanes busy: whenever a lane's traversal ends, the lane takes the next query
// of the stage from a counter (ray replacement), and each trip advances every
// busy lane by up to PT_STEPS node visits. Each query runs the same
// traversal as in k_wf_trace, node for node, so the answers are identical;
// only the assignment of queries to lanes changes. The loop ends: every trip
// advances a traversal (each is capped at 2^22 node visits, as in
// trav_closest / trav_occluded) or takes or refuses a query (at most n plus
// 32 per warp).
constexpr int WF_CTL_FETCH0 = WF_CTL_CNT0 + WF_MAXQ + 2;   // per trace stage: queries taken
static_assert(WF_CTL_FETCH0 + WF_MAXQ <= 16, "ctl holds 16 counters");

// starts query q; true if it is answered without a traversal
template <bool COUNT>
__device__ __forceinline__ bool pt_start(const DScene &S, const WfQuery &q, PtRay &r, TravCount *tc) {
    r.o = q.o;
    r.s1 = q.skip;
    r.s2 = q.skip2;
    r.node = 0;
    r.trail = 0ull;
    r.steps = 0;
    r.h.tri = -1;
    r.h.t = INFINITY;
    r.h.b1 = r.h.b2 = 0.0f;
    if (q.kind == 2) {
        r.kind = 2;
        r.d = q.d - q.o;
    } else {
        r.d = q.d;
        r.kind = 0;
        if (q.kind == 1 && S.ne <= PB_EMITTER_LIST_MAX) {
            r.kind = 3;
            r.h = emitter_candidate(S, q.o, q.d, q.skip);
            if (r.h.tri < 0) return true;
        }
    }
    r.inv = safe_inv(r.d);
    if (COUNT) tc->rays++;
    return false;
}

// the answer of node i's pending query, stored as k_wf_trace stores it
__device__ __forceinline__ void pt_finish(const DScene &S, const WfBufs &W, int i, const PtRay &r) {
    WfResult res;
    if (r.kind == 2) {
        res.tri = r.h.tri >= 0 ? 1 : 0;
        res.b1 = res.b2 = 0.0f;
    } else {
        res.tri = r.h.tri;
        res.b1 = r.h.b1;
        res.b2 = r.h.b2;
        if (r.kind == 3 && r.h.tri >= 0 && __float_as_int(S.stri[4 * (size_t)r.h.tri + 3].w) < 0) res.tri = -1;
    }
    int nq = W.node_nq[i];
    if (nq < WF_MAXQ) {
        W.node_res[(size_t)WF_MAXQ * i + nq] = res;
        W.node_nq[i] = nq + 1;
    }
}

template <bool COUNT>
__global__ void __launch_bounds__(128) k_wf_trace_pt(DScene S, KParams P, Pool B, WfBufs W, int s) {
    const unsigned FULL = 0xffffffffu;
    TravCount tc{0, 0, 0};
    const TravView V = trav_view(S);
    const int n = W.ctl[WF_CTL_CNT0 + s + 1];
    const int32_t *lst = W.list[(s + 1) & 1];
    int32_t *fetch = W.ctl + WF_CTL_FETCH0 + s;
    const int lane = threadIdx.x & 31;
    int i = -1;
    bool drained = false;
    PtRay r;
    for (;;) {
        const bool need = i < 0 && !drained;
        const unsigned m = __ballot_sync(FULL, need);
        if (m) {
            const int leader = __ffs(m) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(fetch, __popc(m));
            base = __shfl_sync(FULL, base, leader);
            if (need) {
                const int k = base + __popc(m & ((1u << lane) - 1u));
                if (k < n) {
                    i = lst[k];
                    if (pt_start<COUNT>(S, W.node_q[i], r, &tc)) {
                        pt_finish(S, W, i, r);
                        i = -1;
                    }
                } else {
                    drained = true;
                }
            }
        }
        if (!__any_sync(FULL, i >= 0)) {
            if (__all_sync(FULL, drained)) break;
            continue;
        }
        if (i >= 0) {
            for (int st = 0; st < PT_STEPS; ++st) {
                if (pt_step<COUNT>(V, r, &tc)) {
                    pt_finish(S, W, i, r);
                    i = -1;
                    break;
                }
            }
        }
    }
    if (COUNT) {
        atomicAdd(&B.counters[CNT_REC_NODES], (unsigned long long)tc.nodes);
        atomicAdd(&B.counters[CNT_REC_TRIS], (unsigned long long)tc.tris);
        atomicAdd(&B.counters[CNT_REC_RAYS], (unsigned long long)tc.rays);
    }
}

// the exact sequential walk over cnt consecutive nodes (g, children, f/q and
// RRS uniform of each), on the stack form (one thread)
__device__ __forceinline__ void walk_seq_arr(const KParams &P, ChainState &st, const float *g, const int32_t *n,
                                             const float *x, const float *u, int cnt, float invB, int &next,
                                             double &sum_t, int &done, int &trunc) {
    for (int q = 0; q < cnt; ++q) {
        const EstStep e = est_step(st, x[q], u[q], g[q], n[q], invB, (uint32_t)next, P);
        next += 1;
        const int r = est_take<PB_MAXF>(st, e, sum_t);
        if (r) {
            done = 1;
            trunc = r == 2;
            return;
        }
    }
}
// the same over nodes [o, o + cnt) of a window, read from the node arrays
__device__ __forceinline__ void walk_seq(const KParams &P, const WfBufs &W, ChainState &gst, int o, int cnt, float invB,
                                         int &next, double &sum_t, int &done, int &trunc) {
    walk_seq_arr(P, gst, W.node_g + o, W.node_n + o, W.node_x + o, W.node_u + o, cnt, invB, next, sum_t, done, trunc);
}

// windows at least this long are walked by a whole block (k_wf_walk_long)
constexpr int WF_WALK_LONG = 8192;

// one warp per chain: the walk over this round's window (below WF_WALK_LONG
// nodes) in chunks of 32. While every pending node shares one weight and one
// bound (est_uniform_form) and the chunk has no negative g under that bound,
// the walk reduces to counts (pending_v = pending - 1 + n_v; the chain ends
// at the first node where pending reaches 0), a warp scan; otherwise lane 0
// replays the exact sequential walk over the chunk.
__global__ void __launch_bounds__(128) k_wf_walk(KParams P, Pool B, WfBufs W) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int items = W.ctl[WF_CTL_ITEMS];
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < items; c += warps) {
        const int w = W.ch_w[c];
        if (W.ch_done[c] || w == 0 || w >= WF_WALK_LONG) continue;
        ChainState &gst = B.chains[c];
        const int slot = gst.slot, k = gst.k, rep = gst.rep;
        const float invB = 1.0f / B.eB[(size_t)slot * B.ML + k];
        const int off = W.ch_off[c];
        int next = gst.next;
        double sum_t = gst.sum_t;
        // pending-count form of the walk state while every pending node has one
        // weight uw and one inverse bound uib
        int pend;
        float uw, uib;
        bool stack_form = !est_uniform_form(gst, uw, uib, pend);   // gst holds the authoritative stack
        int done = 0, trunc = 0;
        // four chunks are loaded ahead of their walk (128 nodes per trip)
        float gq[4];
        int nq4[4];
        for (int j0 = 0; j0 < w && !done; j0 += 32) {
            const int qi = (j0 >> 5) & 3;
            if (qi == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int jj = j0 + 32 * q + lane;
                    gq[q] = jj < w ? W.node_g[off + jj] : 1.0f;
                    nq4[q] = jj < w ? W.node_n[off + jj] : 1;
                }
            }
            const int j = j0 + lane;
            const bool in = j < w;
            float g = gq[0];
            int n = nq4[0];
#pragma unroll
            for (int q = 1; q < 4; ++q)
                if (qi == q) {
                    g = gq[q];
                    n = nq4[q];
                }
            if (!stack_form && uib != invB && in)   // under a raised bound: g and children from f/q
                est_gn(W.node_x[off + j], W.node_u[off + j], g, n, invB, uib, (uint32_t)(next + lane), P.split, g, n);
            const bool anyneg = __any_sync(0xffffffffu, in && g < 0.0f);
            if (!stack_form && !anyneg) {
                // inclusive scan of (n - 1) over the chunk
                int x = in ? n - 1 : 0;
                for (int o = 1; o < 32; o <<= 1) {
                    int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                const unsigned endm = __ballot_sync(0xffffffffu, in && pend + x <= 0);
                const int cnt = min(32, w - j0);
                const int last = endm ? __ffs(endm) - 1 : cnt - 1;   // last node processed
                double t = (in && lane <= last) ? (double)(uw * g * uib) : 0.0;
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                sum_t += t;
                next += last + 1;
                pend += __shfl_sync(0xffffffffu, x, last);
                if (endm) done = 1;
                continue;
            }
            // exact sequential walk of this chunk by lane 0, on the stack form
            if (!stack_form) {
                if (lane == 0) est_from_uniform(gst, pend, uw, uib);
                stack_form = true;
            }
            if (lane == 0) walk_seq(P, W, gst, off + j0, min(32, w - j0), invB, next, sum_t, done, trunc);
            done = __shfl_sync(0xffffffffu, done, 0);
            trunc = __shfl_sync(0xffffffffu, trunc, 0);
            next = __shfl_sync(0xffffffffu, next, 0);
            sum_t = __shfl_sync(0xffffffffu, sum_t, 0);
            __syncwarp();
            // back to the count form when the stack turned uniform again
            int pe;
            float w2, ib2;
            if (est_uniform_form(gst, w2, ib2, pe)) {
                stack_form = false;
                pend = pe;
                uw = w2;
                uib = ib2;
            }
            __syncwarp();
        }
        if (!done && next >= P.trial_cap) {
            done = 1;
            trunc = 1;
        }
        if (lane == 0) {
            if (!stack_form) est_from_uniform(gst, pend, uw, uib);   // store the count form as a one-frame stack
            gst.next = next;
            gst.sum_t = sum_t;
            if (done) {
                size_t o = ((size_t)slot * B.ML + k) * P.repeats + rep;
                B.rep[o] = (float)((double)invB + sum_t);
                B.repn[o] = (float)next;
                B.reptr[o] = trunc;
                W.ch_done[c] = 1;
                atomicSub(&W.ctl[WF_CTL_ACTIVE], 1);
            } else {
                W.ch_win[c] = min(2 * W.ch_win[c], WF_WIN_MAX);
            }
        }
        __syncwarp();
    }
}

// one block per chain whose window holds at least WF_WALK_LONG nodes, in
// tiles of 1024 nodes staged in shared memory together with the chain's walk
// state. The block works on the top region of the state (est_take_top): the
// run of tile nodes up to the first node with a negative g under the region's
// bound is walked in parallel, a block scan of (children - 1) giving each
// node's pending count within the region; where that count reaches 0 the
// region is exhausted, and the walk moves to the pending node below it (or the
// chain ends). The terms w g / B of the run are summed by a block reduction.
// A node with a negative g, and runs of fewer than 64 nodes before one, are
// walked by thread 0 on the full stack.
constexpr int WF_LONG_THREADS = 256;
constexpr int WF_LONG_TILE = 4 * WF_LONG_THREADS;
__global__ void __launch_bounds__(WF_LONG_THREADS) k_wf_walk_long(KParams P, Pool B, WfBufs W) {
    __shared__ ChainState sst;   // the frames below the top region
    __shared__ float t_g[WF_LONG_TILE], t_x[WF_LONG_TILE], t_u[WF_LONG_TILE];
    __shared__ int32_t t_n[WF_LONG_TILE];
    __shared__ int s_wsum[WF_LONG_THREADS / 32];
    __shared__ double s_wpart[WF_LONG_THREADS / 32];
    __shared__ int s_end, s_brk, s_done, s_trunc, s_next, s_pend, s_pos;
    __shared__ float s_w, s_ib;   // the top region: pending count, weight, inverse bound
    __shared__ double s_sum;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int items = W.ctl[WF_CTL_ITEMS];
    for (int c = blockIdx.x; c < items; c += gridDim.x) {
        const int w = W.ch_w[c];
        if (W.ch_done[c] || w < WF_WALK_LONG) continue;   // uniform over the block
        ChainState &gst = B.chains[c];
        const int off = W.ch_off[c];
        if (tid == 0) sst = gst;
        __syncthreads();
        const int slot = sst.slot, k = sst.k, rep = sst.rep;
        const float invB = 1.0f / B.eB[(size_t)slot * B.ML + k];
        if (tid == 0) {
            float w0, ib0;
            s_pend = est_take_top(sst, w0, ib0);
            s_w = w0;
            s_ib = ib0;
            s_next = sst.next;
            s_sum = sst.sum_t;
            s_done = 0;
            s_trunc = 0;
        }
        __syncthreads();
        for (int j0 = 0; j0 < w; j0 += WF_LONG_TILE) {
            if (s_done) break;
            const int cnt = min(WF_LONG_TILE, w - j0);
            // stage the tile: g and children under the estimate's own bound, f/q, uniform
            for (int jj = tid; jj < cnt; jj += WF_LONG_THREADS) {
                t_g[jj] = W.node_g[off + j0 + jj];
                t_n[jj] = W.node_n[off + j0 + jj];
                t_x[jj] = W.node_x[off + j0 + jj];
                t_u[jj] = W.node_u[off + j0 + jj];
            }
            if (tid == 0) s_pos = 0;
            __syncthreads();
            for (;;) {
                const int pos = s_pos;
                if (pos >= cnt || s_done) break;
                const int pend0 = s_pend;
                const float uw = s_w, uib = s_ib;
                const int base_v = s_next - pos;   // pre-order index of tile node 0
                float g[4];
                int n[4];
                int brk = cnt;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int jj = 4 * tid + i;
                    g[i] = 1.0f;
                    n[i] = 1;
                    if (jj >= pos && jj < cnt) {
                        est_gn(t_x[jj], t_u[jj], t_g[jj], t_n[jj], invB, uib, (uint32_t)(base_v + jj), P.split, g[i],
                               n[i]);
                        if (g[i] < 0.0f && jj < brk) brk = jj;
                    }
                }
                if (tid == 0) {
                    s_brk = cnt;
                    s_end = cnt;
                }
                __syncthreads();
                if (brk < cnt) atomicMin(&s_brk, brk);
                __syncthreads();
                const int b = s_brk;   // the run is [pos, b)
                if (b < cnt && b - pos < 64) {
                    // a short run: thread 0 walks it and its breaking node on the full stack
                    if (tid == 0) {
                        int next = s_next, done = 0, trunc = 0;
                        double sum_t = s_sum;
                        if (est_put_top<PB_MAXF>(sst, pend0, uw, uib))
                            walk_seq_arr(P, sst, t_g + pos, t_n + pos, t_x + pos, t_u + pos, b - pos + 1, invB, next,
                                         sum_t, done, trunc);
                        else
                            done = trunc = 1;
                        s_next = next;
                        s_sum = sum_t;
                        s_done = done;
                        s_trunc = trunc;
                        if (!done) {
                            float w2, ib2;
                            s_pend = est_take_top(sst, w2, ib2);
                            s_w = w2;
                            s_ib = ib2;
                        }
                        s_pos = b + 1;
                    }
                    __syncthreads();
                    continue;
                }
                int loc[4], acc = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int jj = 4 * tid + i;
                    if (jj >= pos && jj < b) acc += n[i] - 1;
                    loc[i] = acc;
                }
                int x = acc;
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                if (lane == 31) s_wsum[wid] = x;
                __syncthreads();
                int wbase = 0;
                for (int q = 0; q < wid; ++q) wbase += s_wsum[q];
                const int excl = pend0 + wbase + x - acc;   // the region's pending count before this thread's first node
                int first = cnt;
#pragma unroll
                for (int i = 3; i >= 0; --i) {
                    const int jj = 4 * tid + i;
                    if (jj >= pos && jj < b && excl + loc[i] <= 0) first = jj;
                }
                if (first < cnt) atomicMin(&s_end, first);
                __syncthreads();
                const int end = s_end;   // the node that exhausts the region, or cnt
                const int stop = min(b, end + 1);   // nodes [pos, stop) are taken
                double part = 0.0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int jj = 4 * tid + i;
                    if (jj >= pos && jj < stop) part += (double)(uw * g[i] * uib);
                }
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                if (lane == 0) s_wpart[wid] = part;
                __syncthreads();
                if (tid == 0) {
                    double t = 0.0;
                    int tot = 0;
                    for (int q = 0; q < WF_LONG_THREADS / 32; ++q) {
                        t += s_wpart[q];
                        tot += s_wsum[q];
                    }
                    s_sum += t;
                    s_next += stop - pos;
                    if (end < b) {
                        // the region is exhausted: the next node is the first pending one below it
                        if (!est_pop_below(sst)) {
                            s_done = 1;
                        } else {
                            float w2, ib2;
                            s_pend = est_take_top(sst, w2, ib2);
                            s_w = w2;
                            s_ib = ib2;
                        }
                        s_pos = end + 1;
                    } else {
                        s_pend = pend0 + tot;
                        if (b < cnt) {
                            // the breaking node, on the full stack
                            int next = s_next, done = 0, trunc = 0;
                            double sum_t = s_sum;
                            if (est_put_top<PB_MAXF>(sst, s_pend, uw, uib))
                                walk_seq_arr(P, sst, t_g + b, t_n + b, t_x + b, t_u + b, 1, invB, next, sum_t, done,
                                             trunc);
                            else
                                done = trunc = 1;
                            s_next = next;
                            s_sum = sum_t;
                            s_done = done;
                            s_trunc = trunc;
                            if (!done) {
                                float w2, ib2;
                                s_pend = est_take_top(sst, w2, ib2);
                                s_w = w2;
                                s_ib = ib2;
                            }
                        }
                        s_pos = b < cnt ? b + 1 : cnt;
                    }
                }
                __syncthreads();
            }
        }
        if (tid == 0) {
            int done = s_done, trunc = s_trunc;
            const int next = s_next;
            if (!done && next >= P.trial_cap) {
                done = 1;
                trunc = 1;
            }
            if (!s_done && !est_put_top<PB_MAXF>(sst, s_pend, s_w, s_ib)) {   // the full stack again
                done = 1;
                trunc = 1;
            }
            sst.next = next;
            sst.sum_t = s_sum;
            gst = sst;
            if (done) {
                size_t o = ((size_t)slot * B.ML + k) * P.repeats + rep;
                B.rep[o] = (float)((double)invB + s_sum);
                B.repn[o] = (float)next;
                B.reptr[o] = trunc;
                W.ch_done[c] = 1;
                atomicSub(&W.ctl[WF_CTL_ACTIVE], 1);
            } else {
                W.ch_win[c] = min(2 * W.ch_win[c], WF_WIN_MAX);
            }
        }
        __syncthreads();
    }
}

// Booth's roulette (one chain, no splitting; Sec. 4.2's RR ablation): node j
// of a chain adds prod_{i<=j} g_i over the product of the continuation
// probabilities taken before it, and the chain continues past j with
// probability rho_j = min(1, c |prod_{i<=j} g_i|), drawn with the node's RRS
// uniform. A warp takes 32 consecutive nodes at a time: product scans give
// each lane its prefix product and survival, and a ballot finds the first
// node whose roulette ends the chain.
__global__ void __launch_bounds__(128) k_wf_walk_booth(KParams P, Pool B, WfBufs W, uint32_t iter_base) {
    iter_base = eff_iter(P, iter_base);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int items = W.ctl[WF_CTL_ITEMS];
    const double cb = (double)P.booth;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < items; c += warps) {
        const int w = W.ch_w[c];
        if (W.ch_done[c] || w == 0) continue;
        ChainState &gst = B.chains[c];
        const int slot = gst.slot, k = gst.k, rep = gst.rep;
        const float invB = 1.0f / B.eB[(size_t)slot * B.ML + k];
        const int off = W.ch_off[c];
        int next = gst.next;
        double sum_t = gst.sum_t, prod = gst.prod, surv = gst.surv;
        int done = 0, trunc = 0;
        for (int j0 = 0; j0 < w && !done; j0 += 32) {
            const bool in = j0 + lane < w;
            double pg = in ? (double)W.node_g[off + j0 + lane] : 1.0;
            for (int o = 1; o < 32; o <<= 1) {
                const double y = __shfl_up_sync(FULL, pg, o);
                if (lane >= o) pg *= y;
            }
            const double pr = prod * pg;   // product of g through this node
            const double rho = fmin(1.0, cb * fabs(pr));
            bool stop = false;
            if (in) {
                Rng R;
                R.init(P.seed, K_RECIP, iter_base + slot, (uint32_t)(k * 8 + rep), (uint32_t)(next + lane));
                stop = !((double)R.u(18) < rho);
            }
            double rs = in ? rho : 1.0;    // survival through this node
            for (int o = 1; o < 32; o <<= 1) {
                const double y = __shfl_up_sync(FULL, rs, o);
                if (lane >= o) rs *= y;
            }
            double before = __shfl_up_sync(FULL, rs, 1);
            if (lane == 0) before = 1.0;
            const unsigned stopm = __ballot_sync(FULL, stop);
            const int cnt = min(32, w - j0);
            const int last = stopm ? __ffs(stopm) - 1 : cnt - 1;
            double t = (in && lane <= last) ? pr / (surv * before) * (double)invB : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
            if (!isfinite(t)) {   // the weight left the double range: report the chain as truncated
                done = 1;
                trunc = 1;
                break;
            }
            sum_t += t;
            next += last + 1;
            prod = __shfl_sync(FULL, pr, last);
            surv *= __shfl_sync(FULL, rs, last);
            if (stopm) done = 1;
        }
        if (!done && next >= P.trial_cap) {
            done = 1;
            trunc = 1;
        }
        if (lane == 0) {
            gst.next = next;
            gst.sum_t = sum_t;
            gst.prod = prod;
            gst.surv = surv;
            if (done) {
                size_t o = ((size_t)slot * B.ML + k) * P.repeats + rep;
                B.rep[o] = (float)((double)invB + sum_t);
                B.repn[o] = (float)next;
                B.reptr[o] = trunc;
                W.ch_done[c] = 1;
                atomicSub(&W.ctl[WF_CTL_ACTIVE], 1);
            } else {
                W.ch_win[c] = min(2 * W.ch_win[c], WF_WIN_MAX);
            }
        }
        __syncwarp();
    }
}

// chains the rounds left unfinished (deferred by the node capacity): one
// thread each, inline draws, the same walk; counted in WF_CTL_ERR's high bits
__global__ void k_wf_finish_rest(DScene S, KParams P, Pool B, WfBufs W, uint32_t iter_base) {
    iter_base = eff_iter(P, iter_base);
    const int items = W.ctl[WF_CTL_ITEMS];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < items; c += gridDim.x * blockDim.x) {
        if (W.ch_done[c]) continue;
        atomicAdd(&W.ctl[WF_CTL_ERR], 1 << 8);
        ChainState st = B.chains[c];
        int Sp, C;
        Entry E = load_entry(S, P, B, st.slot, st.k, Sp, C);
        const float invB = 1.0f / B.eB[(size_t)st.slot * B.ML + st.k];
        int done = 0, trunc = 0;
        while (!done && P.booth > 0.0f) {   // Booth's roulette, as k_wf_walk_booth
            if (st.next >= P.trial_cap) {
                done = trunc = 1;
                break;
            }
            Rng R;
            R.init(P.seed, K_RECIP, iter_base + st.slot, (uint32_t)(st.k * 8 + st.rep), (uint32_t)st.next);
            float ratio = entry_ratio<false>(S, E, R, nullptr);
            float gj = est_g(ratio, invB);
            st.prod *= (double)gj;
            const double tb = st.prod / st.surv * (double)invB;
            if (!isfinite(tb)) {   // the weight left the double range: report the chain as truncated
                done = trunc = 1;
                break;
            }
            st.sum_t += tb;
            st.next += 1;
            const double rho = fmin(1.0, (double)P.booth * fabs(st.prod));
            if (!((double)R.u(18) < rho)) done = 1;
            else st.surv *= rho;
        }
        while (!done) {
            if (st.next >= P.trial_cap) {
                done = trunc = 1;
                break;
            }
            Rng R;
            R.init(P.seed, K_RECIP, iter_base + st.slot, (uint32_t)(st.k * 8 + st.rep), (uint32_t)st.next);
            const float ratio = entry_ratio<false>(S, E, R, nullptr), u18 = R.u(18);
            const float gj = est_g(ratio, invB);
            const uint32_t v = (uint32_t)st.next;
            const EstStep e = est_step(st, ratio, u18, gj, est_children(gj, u18, v, P.split), invB, v, P);
            st.next += 1;
            const int r = est_take<PB_MAXF>(st, e, st.sum_t);
            if (r) {
                done = 1;
                trunc = r == 2;
                break;
            }
        }
        size_t o = ((size_t)st.slot * B.ML + st.k) * P.repeats + st.rep;
        B.rep[o] = (float)((double)invB + st.sum_t);
        B.repn[o] = (float)st.next;
        B.reptr[o] = trunc;
        W.ch_done[c] = 1;
        B.chains[c] = st;
    }
}

// one trace stage: a query per thread, or persistent warps that refill lanes
void launch_trace(const DScene &S, const KParams &P, const Pool &B, const WfBufs &W, int s, int num_sms,
                  cudaStream_t st) {
    if (P.trace) {
        cudaMemsetAsync(W.ctl + WF_CTL_FETCH0 + s, 0, sizeof(int32_t), st);
        if (P.count) k_wf_trace_pt<true><<<num_sms * 8, 128, 0, st>>>(S, P, B, W, s);
        else k_wf_trace_pt<false><<<num_sms * 8, 128, 0, st>>>(S, P, B, W, s);
    } else if (P.count) {
        k_wf_trace<true><<<num_sms * 8, 128, 0, st>>>(S, P, B, W, s);
    } else {
        k_wf_trace<false><<<num_sms * 8, 128, 0, st>>>(S, P, B, W, s);
    }
}

}  // namespace

void launch_recip_wavefront(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots,
                            uint32_t iter_base, int num_sms, cudaStream_t st, const WfBufs &W) {
    if (P.pilot_max > 0) {
        // the pilot as wavefront rounds: windows pilot_min, then doubling up to pilot_max
        k_wfp_init<<<num_sms * 2, 256, 0, st>>>(P, B, W, slots);
        const int nr = wf_pilot_rounds(P);
        for (int round = 0; round < nr; ++round) {
            k_wfp_plan<<<1, 1024, 0, st>>>(P, W);
            k_wf_nodes<true><<<num_sms * 8, 256, 0, st>>>(B, W);
            for (int s = 0; s <= WF_MAXQ; ++s) {
                k_wf_step<true><<<num_sms * 8, 128, 0, st>>>(S, P, B, W, s, iter_base, slots);
                if (s == WF_MAXQ) break;
                launch_trace(S, P, B, W, s, num_sms, st);
            }
            k_wfp_reduce<<<num_sms * 16, 128, 0, st>>>(S, P, B, T, W, slots, round == nr - 1 ? 1 : 0);
        }
    }
    k_wf_init<<<num_sms * 2, 256, 0, st>>>(P, B, W, slots);
    for (int round = 0; round < WF_ROUNDS; ++round) {
        k_wf_plan<<<1, 1024, 0, st>>>(P, B, W);
        k_wf_nodes<false><<<num_sms * 8, 256, 0, st>>>(B, W);
        for (int s = 0; s <= WF_MAXQ; ++s) {
            k_wf_step<false><<<num_sms * 8, 128, 0, st>>>(S, P, B, W, s, iter_base, slots);
            if (s == WF_MAXQ) break;
            launch_trace(S, P, B, W, s, num_sms, st);
        }
        if (P.booth > 0.0f) k_wf_walk_booth<<<num_sms * 16, 128, 0, st>>>(P, B, W, iter_base);
        else {
            k_wf_walk<<<num_sms * 16, 128, 0, st>>>(P, B, W);
            k_wf_walk_long<<<num_sms * 2, WF_LONG_THREADS, 0, st>>>(P, B, W);
        }
    }
    k_wf_finish_rest<<<num_sms * 2, 128, 0, st>>>(S, P, B, W, iter_base);
}
