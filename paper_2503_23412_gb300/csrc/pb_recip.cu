// The reciprocal estimator's per-entry bound and its warp/block schedule
// (Sec. 4.2, App. Alg. I~, App. "Optimal value for B"):
//   k_recip_pilot    per-entry B from a pilot (or the learned table value)
//   k_recip          one warp per (entry, repeat): lanes evaluate 32
//                    consecutive pre-order nodes at once, then the warp walks
//   k_recip_long     a block per chain still running, in sorted batches
//                    (pb_recip_long.cuh; one translation unit per variant)
#include <cstdio>

#include "pb_entry.cuh"

namespace {

// Per-entry bound B (App. "Optimal value for B": B = max f/q of the
// integrand being estimated). One warp per entry draws from the entry's
// supporting distribution on stream (kind PILOT, a = iteration, b = entry,
// c = draw), 32 draws per round: at least pilot_min, then rounds until one
// has f > 0, at most pilot_max. B is the largest f/q seen, or the learned
// cell value if every draw had f = 0 or the pilot is off. B depends on none
// of the estimate's own draws, so the estimate stays unbiased.
template <bool COUNT>
__global__ void __launch_bounds__(128) k_recip_pilot(DScene S, DTables T, KParams P, Pool B, int slots,
                                                     uint32_t iter_base) {
    iter_base = eff_iter(P, iter_base);
    int lane = threadIdx.x & 31;
    TravCount tc{0, 0, 0};
    const int32_t *offs = B.work + 1;   // per slot: first (entry, repeat) item
    int32_t *counter = B.work + 4 + slots;
    int total = offs[slots] / P.repeats;
    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        int slot = 0;
        while (item * P.repeats >= offs[slot + 1]) ++slot;
        int k = item - offs[slot] / P.repeats;
        int Sp, C;
        Entry E = load_entry(S, P, B, slot, k, Sp, C);
        float best = 0.0f, sum = 0.0f;
        int draws = 0;
        for (int base = 0; base < P.pilot_max; base += 32) {
            if (base >= P.pilot_min && best > 0.0f) break;   // best is warp-uniform
            Rng R;
            R.init(P.seed, K_PILOT, iter_base + slot, (uint32_t)k, (uint32_t)(base + lane));
            float x = entry_ratio<COUNT>(S, E, R, &tc);
            float m = x, t = x;
            for (int o = 16; o > 0; o >>= 1) {
                m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                t += __shfl_xor_sync(0xffffffffu, t, o);
            }
            best = fmaxf(best, m);
            sum += t;
            draws += 32;
        }
        if (lane == 0) {
            float Bv = best > 0.0f ? best : T.Bt[((E.u - 1) * T.KSp + Sp) * (T.KC + 1) + C];
            B.eB[(size_t)slot * B.ML + k] = Bv;
            // a scheduling hint only: the expected chain length B / mean(f/q) when g stays in [0, 1]
            B.eMu[(size_t)slot * B.ML + k] = sum > 0.0f ? Bv * (float)draws / sum : 0.0f;
        }
    }
    if (COUNT) {
        atomicAdd(&B.counters[CNT_REC_NODES], (unsigned long long)tc.nodes);
        atomicAdd(&B.counters[CNT_REC_TRIS], (unsigned long long)tc.tris);
        atomicAdd(&B.counters[CNT_REC_RAYS], (unsigned long long)tc.rays);
    }
}

#define MAXF PB_MAXF
#define MAXF1 8          // walk frames a warp keeps; deeper walks continue in a block

// the walk state a warp keeps (every lane holds the same copy)
struct WarpStack {
    float cur_sign, cur_ib;
    int sp;
    float fr_sign[MAXF1], fr_ib[MAXF1];
    int fr_rem[MAXF1];
};

// Phase 1: one warp per (entry, repeat). The tree's nodes are numbered in
// pre-order, so node v's sample depends only on v: the 32 lanes draw nodes
// base..base+31 together, then every lane replays the same sequential walk
// (children counts and signs, DFS frames in local memory). Speculative nodes
// past the end are discarded. Chains still running are
// queued for phase 2 with their walk state (after P.handoff nodes).
template <bool COUNT>
__global__ void __launch_bounds__(128) k_recip(DScene S, DTables T, KParams P, Pool B, int slots, uint32_t iter_base) {
    iter_base = eff_iter(P, iter_base);
    int lane = threadIdx.x & 31;
    TravCount tc{0, 0, 0};
    int32_t *counter = B.work;
    int32_t *chain_count = B.work + 2 + slots;
    const int32_t *offs = B.work + 1;   // per slot: first work item, slots+1 entries
    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= offs[slots]) break;
        int slot = 0;
        while (item >= offs[slot + 1]) ++slot;
        int local = item - offs[slot];
        int k = local / P.repeats, rep = local % P.repeats;
        int Sp, C;
        Entry E = load_entry(S, P, B, slot, k, Sp, C);
        float invB = 1.0f / B.eB[(size_t)slot * B.ML + k];
        // chains expected to run far past the hand-off start in the block phase
        const bool long_chain = B.eMu[(size_t)slot * B.ML + k] > 8.0f * (float)P.handoff;
        double sum_t = 0.0;   // long chains add thousands of terms
        int nodes = 0;
        bool done = false, trunc = false, handed = false;
        WarpStack ws;
        ws.cur_sign = 1.0f;
        ws.cur_ib = invB;
        ws.sp = 0;
        bool deep = false;   // the walk needs more frames than a warp keeps
        for (int base = 0; !done; base += 32) {
            if (base >= P.handoff || deep || long_chain) {
                int slot_q = 0;
                if (lane == 0) slot_q = atomicAdd(chain_count, 1);
                slot_q = __shfl_sync(0xffffffffu, slot_q, 0);
                if (slot_q < B.chain_cap) {
                    if (lane == 0) {
                        ChainState &cs = B.chains[slot_q];
                        cs.slot = slot; cs.k = k; cs.rep = rep; cs.next = base;
                        cs.sum_t = sum_t; cs.cur_sign = ws.cur_sign; cs.cur_ib = ws.cur_ib; cs.sp = ws.sp;
                        for (int i = 0; i < ws.sp; ++i) {
                            cs.fr_sign[i] = ws.fr_sign[i];
                            cs.fr_ib[i] = ws.fr_ib[i];
                            cs.fr_rem[i] = ws.fr_rem[i];
                        }
                    }
                    handed = true;
                    break;
                }
                if (deep) {   // no room to hand over a deep walk: stop and report truncation
                    done = true;
                    trunc = true;
                    break;
                }
            }
            int v = base + lane;
            float g = 1.0f, x = 0.0f, u = 1.0f;
            int nch = 0;
            if (v < P.trial_cap) {
                Rng R;
                R.init(P.seed, K_RECIP, iter_base + slot, (uint32_t)(k * 8 + rep), (uint32_t)v);
                x = entry_ratio<COUNT>(S, E, R, &tc);
                u = R.u(18);
                g = est_g(x, invB);
                nch = est_children(g, u, (uint32_t)v, P.split);
            }
            // the walk stops before a node that would need a frame beyond MAXF1;
            // the block phase resumes from that node with the full stack
            int stop = 32;
            for (int j = 0; j < 32; ++j) {
                const float gj = __shfl_sync(0xffffffffu, g, j), xj = __shfl_sync(0xffffffffu, x, j);
                const float uj = __shfl_sync(0xffffffffu, u, j);
                const int nj = __shfl_sync(0xffffffffu, nch, j);
                if (done || j >= stop) continue;
                if (base + j >= P.trial_cap) {
                    done = true;
                    trunc = true;
                    continue;
                }
                const EstStep e = est_step(ws, xj, uj, gj, nj, invB, (uint32_t)(base + j), P);
                if (e.push && ws.sp >= MAXF1) {
                    stop = j;
                    deep = true;
                    continue;
                }
                nodes++;
                const int r = est_take<MAXF1>(ws, e, sum_t);
                if (r) {   // 2: the children's weight left the float range
                    done = true;
                    trunc = r == 2;
                }
            }
            if (deep) base = base + stop - 32;   // resume at node base + stop
        }
        if (lane == 0 && !handed) {
            size_t o = ((size_t)slot * B.ML + k) * P.repeats + rep;
            B.rep[o] = (float)((double)invB + sum_t);
            B.repn[o] = (float)nodes;
            B.reptr[o] = trunc ? 1 : 0;
        }
    }
    if (COUNT) {
        atomicAdd(&B.counters[CNT_REC_NODES], (unsigned long long)tc.nodes);
        atomicAdd(&B.counters[CNT_REC_TRIS], (unsigned long long)tc.tris);
        atomicAdd(&B.counters[CNT_REC_RAYS], (unsigned long long)tc.rays);
    }
}

}  // namespace

void launch_recip_bounds(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots,
                         uint32_t iter_base, int num_sms, cudaStream_t st, bool count) {
    if (count) k_recip_pilot<true><<<num_sms * 4, 128, 0, st>>>(S, T, P, B, slots, iter_base);
    else k_recip_pilot<false><<<num_sms * 4, 128, 0, st>>>(S, T, P, B, slots, iter_base);
}

void launch_recip_phases(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots,
                         uint32_t iter_base, int num_sms, cudaStream_t st) {
    if (P.count) {
        k_recip<true><<<num_sms * 8, 128, 0, st>>>(S, T, P, B, slots, iter_base);
        launch_recip_long_counting(S, T, P, B, slots, iter_base, num_sms, st);
    } else {
        k_recip<false><<<num_sms * 8, 128, 0, st>>>(S, T, P, B, slots, iter_base);
        launch_recip_long_plain(S, T, P, B, slots, iter_base, num_sms, st);
    }
}
