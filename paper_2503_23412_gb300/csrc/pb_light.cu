// Light side of an iteration (Sec. 3.2, 5.1-5.3 of arXiv 2503.23412):
//   k_light_pass     M light sub-paths per iteration, geometry only
//   k_pool_build     per light vertex: throughput f_y/p_y, MIS partial sums,
//                    light-subspace label; incomplete sub-path detection
//                    (L S^u / L D S^u, 1 <= u <= 4) with S' and C labels
//   k_bucket         stable compaction in (path, vertex) order and stable
//                    counting sort by subspace (deterministic pool order)
//   k_cdf            per eye subspace, the selection CDF over non-empty
//                    subspaces (SPCBPT two-stage selection, Sec. 5.5)
//   k_recip          reciprocal estimates (Sec. 4.2, App. Alg. I~): one warp
//                    per (entry, repeat); lanes evaluate 32 consecutive
//                    pre-order nodes at once, then the warp scans the tree
//   k_recip_finish   average of the repeats per entry
#include <cstdio>

#include <cooperative_groups.h>

#include "pb_kernels.h"
#include "pb_estimator.cuh"

namespace cg = cooperative_groups;

namespace {

// ---------------------------------------------------------------------------
__global__ void k_light_pass(DScene S, KParams P, Pool B, uint32_t iter_base) {
    iter_base = eff_iter(P, iter_base);
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    int slot = blockIdx.y;
    if (l >= P.M) return;
    size_t base = (size_t)slot * B.ML + (size_t)l * P.L;
    int32_t *tr = B.gtri + base;
    float2 *ba = B.gbary + base;
    for (int e = 0; e < P.L; ++e) {
        tr[e] = -1;
        ba[e] = make_float2(0.f, 0.f);
    }
    if (P.L < 1) return;
    Rng r;
    r.init(P.seed, K_LIGHT, iter_base + slot, (uint32_t)l, 0);
    int t0;
    float b1, b2;
    if (!sample_light(S, r.u(0), r.u(1), r.u(2), t0, b1, b2)) return;
    tr[0] = t0;
    ba[0] = make_float2(b1, b2);
    Vtx cur = vertex_at(S, t0, b1, b2);
    float3 w = cosine_dir(cur.n, r.u(3), r.u(4));
    for (int e = 1; e < P.L; ++e) {
        Hit h = closest_hit<false>(S, cur.p, w, cur.tri);
        if (h.tri < 0) break;
        Vtx nx = vertex_at(S, h.tri, h.b1, h.b2);
        float3 wl = -w;
        if (absorbing(S, nx, wl)) break;
        tr[e] = h.tri;
        ba[e] = make_float2(h.b1, h.b2);
        if (e + 1 >= P.L) break;
        Rng q;
        q.init(P.seed, K_LIGHT, iter_base + slot, (uint32_t)l, (uint32_t)e);
        float3 ws;
        if (!bsdf_sample(S.mats[nx.mat], nx.n, wl, q.u(0), q.u(1), q.u(2), ws)) break;
        cur = nx;
        w = ws;
    }
}

// Per light path: vertex records for connections, MIS partial sums and
// incomplete sub-paths.
//   fwd_j  light-tracer density of y_j; rev_j eye-tracer density of y_j
//   Lsum_j = (rev_j / fwd_j) (avail_j + Lsum_{j-1}), Lsum_{-1} = 0
// stored per vertex e: Lpart = Lsum_{e-2}; the connection finishes the last
// two terms, whose rev depends on the eye vertex.
__global__ void k_pool_build(DScene S, DTables T, KParams P, Pool B) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    int slot = blockIdx.y;
    if (l >= P.M) return;
    size_t base = (size_t)slot * B.ML + (size_t)l * P.L;
    const int32_t *tr = B.gtri + base;
    const float2 *ba = B.gbary + base;
    Vtx y[16];
    int n = 0;
    for (int e = 0; e < P.L && e < 16; ++e) {
        if (tr[e] < 0) break;
        y[e] = vertex_at(S, tr[e], ba[e].x, ba[e].y);
        n = e + 1;
    }
    for (int e = 0; e < P.L; ++e) {
        B.vlabel[base + e] = -1;
        B.elabel[base + e] = -1;
    }
    if (n == 0) return;
    float fwd_prev = light_pdf(S, y[0].tri);   // fwd_0
    float3 alpha = emitted(S, y[0], n > 1 ? dirto(y[0].p, y[1].p) : y[0].n) * (1.0f / fwd_prev);
    float Lsum_m2 = 0.0f;    // Lsum_{e-2}
    float Lsum_m3 = 0.0f;    // Lsum_{e-3}
    float fwd_m2 = 0.0f;     // fwd_{e-2}
    for (int e = 1; e < n; ++e) {
        float d2;
        float3 w;
        fwd_cos_over_d2(y[e - 1].p, y[e].p, y[e].n, w, d2);
        float fwd_e = fwd_density(S, y, e);
        // throughput to y_e
        if (e == 1) {
            alpha = alpha * PB_PI;
        } else {
            const DMat &m = S.mats[y[e - 1].mat];
            float3 wl = dirto(y[e - 1].p, y[e - 2].p), we = w;
            float pw = bsdf_pdf(m, y[e - 1].n, wl, we);
            float3 rho = bsdf_eval(m, y[e - 1].n, wl, we);
            alpha = pw > 0.0f ? mul(alpha, rho) * (fabsf(dot(y[e - 1].n, we)) / pw) : f3(0, 0, 0);
        }
        // Lsum_{e-2} from Lsum_{e-3}: needs rev_{e-2} (pdf at y_{e-1} given y_e)
        if (e >= 2) {
            int j = e - 2;
            const DMat &m = S.mats[y[j + 1].mat];
            float3 dd = y[j].p - y[j + 1].p;
            float dj2 = len2(dd);
            float3 wj = dd * (1.0f / sqrtf(dj2));
            float rev_j = bsdf_pdf(m, y[j + 1].n, dirto(y[j + 1].p, y[j + 2].p), wj) * fabsf(dot(y[j].n, wj)) / dj2;
            float fwd_j = (j == 0) ? light_pdf(S, y[0].tri) : fwd_m2;
            int avail_j = (j == 0) ? 1 : ((!spec_v(S, y[j - 1]) || j - 1 == 0) && !spec_v(S, y[j]) && (j == 1 || P.conn));
            Lsum_m2 = fwd_j > 0.0f ? (rev_j / fwd_j) * ((float)avail_j + Lsum_m3) : 0.0f;
        }
        float cos_prev = fabsf(dot(y[e - 1].n, w));
        int avail_em1 = (e - 1 == 0) ? 1 : ((e - 2 == 0 || !spec_v(S, y[e - 2])) && !spec_v(S, y[e - 1]) && (e - 1 == 1 || P.conn));
        int avail_e = (e - 1 == 0 || !spec_v(S, y[e - 1])) && !spec_v(S, y[e]) && (e == 1 || P.conn);
        size_t k = base + e;
        B.vpos[k] = make_float4(y[e].p.x, y[e].p.y, y[e].p.z, __int_as_float(y[e].mat));
        B.vnrm[k] = make_float4(y[e].n.x, y[e].n.y, y[e].n.z, __int_as_float(y[e].tri));
        float3 wle = -w;
        B.vwl[k] = make_float4(wle.x, wle.y, wle.z, fwd_e);
        B.valpha[k] = make_float4(alpha.x, alpha.y, alpha.z, (e >= 2) ? Lsum_m2 : 0.0f);
        float fwd_em1 = (e == 1) ? light_pdf(S, y[0].tri) : fwd_prev;
        B.vmis[k] = make_float4(fwd_em1, cos_prev, d2, __int_as_float(avail_em1 | (avail_e << 1)));
        if (!spec_v(S, y[e])) B.vlabel[k] = label_dir(S, y[e], wle, T.KS, T.cS);
        // incomplete light sub-path ending at a specular y_e (first M_p paths)
        if (l < P.M_p && spec_v(S, y[e])) {
            int u = 0, j = e;
            while (j >= 1 && spec_v(S, y[j])) { ++u; --j; }
            if (u >= 1 && u <= 4 && j <= 1) {
                int type = (j == 1);
                int C = type ? label_ctrl(S, T, y[0]) : T.KC;
                B.elabel[k] = label_spec(S, T, y[e]);
                B.einfo[k] = u | (type << 3) | (C << 4);
            }
        }
        // shift
        Lsum_m3 = Lsum_m2;
        fwd_m2 = fwd_prev;
        fwd_prev = fwd_e;
    }
}

// One block per slot, two warps: warp 0 builds the connection pool, warp 1
// the incomplete sub-path list. Stable compaction in (path, vertex) order,
// then a stable counting sort by label.
__device__ void warp_bucket(const int32_t *label, int n, int K, int32_t *idx_out, int32_t *clabel,
                            int32_t *count_out, int32_t *start, int32_t *items, int32_t *run) {
    int lane = threadIdx.x & 31;
    unsigned lt = (1u << lane) - 1u;
    for (int k = lane; k <= K; k += 32) run[k] = 0;
    __syncwarp();
    int cnt = 0;
    for (int b = 0; b < n; b += 32) {
        int i = b + lane;
        int lab = i < n ? label[i] : -1;
        unsigned m = __ballot_sync(0xffffffffu, lab >= 0);
        if (lab >= 0) {
            int pos = cnt + __popc(m & lt);
            idx_out[pos] = i;
            clabel[pos] = lab;
            atomicAdd(&run[lab], 1);
        }
        cnt += __popc(m);
    }
    __syncwarp();
    // exclusive scan of the histogram into start[0..K]
    int carry = 0;
    for (int b = 0; b <= K; b += 32) {
        int k = b + lane;
        int v = k < K ? run[k] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (k <= K) start[k] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    __syncwarp();
    for (int k = lane; k < K; k += 32) run[k] = start[k];
    __syncwarp();
    for (int b = 0; b < cnt; b += 32) {
        int i = b + lane;
        int lab = i < cnt ? clabel[i] : -1 - lane;   // unique dummies never match
        unsigned peers = __match_any_sync(0xffffffffu, lab);
        int rank = __popc(peers & lt);
        int pos = (lab >= 0) ? run[lab] + rank : 0;
        __syncwarp();
        if (lab >= 0) {
            items[pos] = i;
            if (rank == 0) run[lab] += __popc(peers);
        }
        __syncwarp();
    }
    if (lane == 0) *count_out = cnt;
}

__global__ void k_bucket(DTables T, Pool B, int32_t *scratch) {
    extern __shared__ int32_t sh[];
    int slot = blockIdx.x;
    int warp = threadIdx.x >> 5;
    size_t o = (size_t)slot * B.ML;
    if (warp == 0) {
        warp_bucket(B.vlabel + o, B.ML, T.KS, B.pool_idx + o, scratch + o, B.npool + slot,
                    B.bstart + (size_t)slot * (T.KS + 1), B.bitems + o, sh);
    } else {
        warp_bucket(B.elabel + o, B.ML, T.KSp, B.ent_idx + o, scratch + (size_t)B.slots * B.ML + o,
                    B.nent + slot, B.estart + (size_t)slot * (T.KSp + 1), B.eitems + o, sh + T.KS + 1);
    }
}

// selection CDF of row T over the non-empty subspaces of one slot
__global__ void k_cdf(DTables T, Pool B) {
    int row = blockIdx.x, slot = blockIdx.y, which = blockIdx.z;
    int K = which == 0 ? T.KS : T.KSp;
    const float *g = (which == 0 ? T.gC : T.gP) + (size_t)row * K;
    const int32_t *start = which == 0 ? B.bstart + (size_t)slot * (T.KS + 1) : B.estart + (size_t)slot * (T.KSp + 1);
    float *cdf = (which == 0 ? B.cdfC + (size_t)slot * T.KT * T.KS : B.cdfP + (size_t)slot * T.KT * T.KSp) +
                 (size_t)row * K;
    float *Z = (which == 0 ? B.ZC : B.ZP) + (size_t)slot * T.KT + row;
    __shared__ float part[32];
    __shared__ int lastne;
    if (threadIdx.x == 0) lastne = -1;
    __syncthreads();
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float carry = 0.0f;
    for (int b = 0; b < K; b += blockDim.x) {
        int k = b + threadIdx.x;
        float v = 0.0f;
        if (k < K && start[k + 1] > start[k]) {
            v = g[k];
            atomicMax(&lastne, k);
        }
        float x = v;
        for (int s = 1; s < 32; s <<= 1) {
            float y = __shfl_up_sync(0xffffffffu, x, s);
            if (lane >= s) x += y;
        }
        if (lane == 31) part[warp] = x;
        __syncthreads();
        if (warp == 0) {
            float p = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0f;
            for (int s = 1; s < 32; s <<= 1) {
                float y = __shfl_up_sync(0xffffffffu, p, s);
                if (lane >= s) p += y;
            }
            part[lane] = p;
        }
        __syncthreads();
        float incl = x + (warp > 0 ? part[warp - 1] : 0.0f) + carry;
        if (k < K) cdf[k] = incl;
        carry += part[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    float Zv = carry;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float c = Zv > 0.0f ? cdf[k] / Zv : 0.0f;
        if (k >= lastne && lastne >= 0) c = 1.0f;
        cdf[k] = c;
    }
    if (threadIdx.x == 0) *Z = Zv;
}

__device__ __forceinline__ Entry load_entry(const DScene &S, const KParams &P, const Pool &B, int slot, int k,
                                            int &Sp, int &C) {
    size_t o = (size_t)slot * B.ML;
    int fixed = B.ent_idx[o + k];
    int l = fixed / P.L, e = fixed % P.L;
    size_t gb = o + (size_t)l * P.L;
    Entry E;
    E.Y = vertex_at(S, B.gtri[gb + e], B.gbary[gb + e].x, B.gbary[gb + e].y);
    E.H = vertex_at(S, B.gtri[gb], B.gbary[gb].x, B.gbary[gb].y);
    Vtx Yp = vertex_at(S, B.gtri[gb + e - 1], B.gbary[gb + e - 1].x, B.gbary[gb + e - 1].y);
    E.back = dot(E.Y.n, Yp.p - E.Y.p) < 0.0f ? 1 : 0;
    E.pin = P.side_in;
    int info = B.einfo[o + fixed];
    E.u = info & 7;
    E.type = (info >> 3) & 1;
    C = info >> 4;
    Sp = B.elabel[o + fixed];
    return E;
}

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
        float fr_sign[MAXF1];
        int fr_rem[MAXF1];
        int sp = 0;
        float cur_sign = 1.0f;
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
                        cs.sum_t = sum_t; cs.cur_sign = cur_sign; cs.sp = sp;
                        for (int i = 0; i < sp; ++i) { cs.fr_sign[i] = fr_sign[i]; cs.fr_rem[i] = fr_rem[i]; }
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
            float g = 1.0f;
            int nch = 0;
            if (v < P.trial_cap) {
                Rng R;
                R.init(P.seed, K_RECIP, iter_base + slot, (uint32_t)(k * 8 + rep), (uint32_t)v);
                float ratio = entry_ratio<COUNT>(S, E, R, &tc);
                g = 1.0f - ratio * invB;
                float r = fabsf(g);
                nch = (int)floorf(r);
                if (R.u(18) < r - (float)nch) nch += 1;
            }
            // the walk stops before a node that would need a frame beyond MAXF1;
            // the block phase resumes from that node with the full stack
            int stop = 32;
            for (int j = 0; j < 32; ++j) {
                float gj = __shfl_sync(0xffffffffu, g, j);
                int nj = __shfl_sync(0xffffffffu, nch, j);
                if (done || j >= stop) continue;
                if (base + j >= P.trial_cap) {
                    done = true;
                    trunc = true;
                    continue;
                }
                if (nj >= 1 && sp >= MAXF1) {
                    stop = j;
                    deep = true;
                    continue;
                }
                sum_t += (double)(cur_sign * gj * invB);
                nodes++;
                if (nj >= 1) {
                    fr_sign[sp] = cur_sign * (gj > 0.0f ? 1.0f : -1.0f);
                    fr_rem[sp] = nj;
                    ++sp;
                }
                if (sp == 0) {
                    done = true;
                    continue;
                }
                cur_sign = fr_sign[sp - 1];
                if (--fr_rem[sp - 1] == 0) --sp;
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

#define PH2_THREADS 256
#define PH2_NPT 8
#define PH2_BATCH (PH2_THREADS * PH2_NPT)

// Phase 2: a block per long chain. Each batch draws nb = 256 * npt
// consecutive nodes in parallel, npt in {1, 2, 4, 8} sized from the entry's
// expected chain length so that little is drawn past the chain's end. The
// nodes are evaluated grouped by the branch their first uniforms select
// (mixture component, side of the lens), so that whole warps trace alike;
// the walk still consumes them in pre-order. While every pending node has
// sign +1 and the batch has no negative g, the walk reduces to counts:
// pending_v = pending - 1 + n_v per node, the chain ends at the first node
// where pending reaches 0, and the estimate adds g_v / B for the nodes up to
// there -- a block prefix sum. Otherwise one thread replays the exact
// sequential walk over the batch.

// the branch of entry_ratio a node takes before its first ray: 0 / 1 trace
// from y_{s-1} toward the side of y_{s-2} / the other side, 2 the first
// component when u = 1
__device__ __forceinline__ int node_branch(const DScene &S, const Entry &E, Rng &R) {
    if (E.u == 1 && R.u(0) < 0.5f) return 2;
    return (S.mats[E.Y.mat].kind == MK_DIELECTRIC && !(R.u(19) < E.pin)) ? 1 : 0;
}

template <bool COUNT>
__global__ void __launch_bounds__(PH2_THREADS) k_recip_long(DScene S, DTables T, KParams P, Pool B, int slots,
                                                            uint32_t iter_base) {
    iter_base = eff_iter(P, iter_base);
    __shared__ float sg[PH2_BATCH];
    __shared__ int sn[PH2_BATCH];
    __shared__ uint8_t skey[PH2_BATCH];
    __shared__ int16_t sperm[PH2_BATCH];
    __shared__ int s_cnt[4];
    __shared__ int s_item, s_done, s_end, s_neg;
    __shared__ double s_sum;
    __shared__ int s_pending[PH2_THREADS];
    __shared__ double s_part[PH2_THREADS];
    __shared__ ChainState st;
    TravCount tc{0, 0, 0};
    int tid = threadIdx.x;
    int32_t *next_item = B.work + 2 + slots + 1;
    int nitems = min(B.work[2 + slots], B.chain_cap);
    while (true) {
        if (tid == 0) s_item = atomicAdd(next_item, 1);
        __syncthreads();
        int item = s_item;
        if (item >= nitems) break;
        if (tid == 0) st = B.chains[item];
        __syncthreads();
        int slot = st.slot, k = st.k, rep = st.rep;
        int Sp, C;
        Entry E = load_entry(S, P, B, slot, k, Sp, C);
        float invB = 1.0f / B.eB[(size_t)slot * B.ML + k];
        // nodes per thread: about half the expected chain length per batch
        const float mu = B.eMu[(size_t)slot * B.ML + k];
        int npt = PH2_NPT;
        if (mu > 0.0f) {
            npt = 1;
            while (npt < PH2_NPT && (float)(PH2_THREADS * npt) < 0.5f * mu) npt <<= 1;
        }
        const int nb = PH2_THREADS * npt;
        bool trunc = false;
        int done = 0;
        while (!done) {
            int base = st.next;
            // group the batch by branch: counting sort of node indices
            if (tid < 4) s_cnt[tid] = 0;
            __syncthreads();
            for (int j = 0; j < npt; ++j) {
                int idx = tid * npt + j;
                Rng R;
                R.init(P.seed, K_RECIP, iter_base + slot, (uint32_t)(k * 8 + rep), (uint32_t)(base + idx));
                int key = node_branch(S, E, R);
                skey[idx] = (uint8_t)key;
                atomicAdd(&s_cnt[key], 1);
            }
            __syncthreads();
            if (tid == 0) {
                int acc = 0;
                for (int q = 0; q < 4; ++q) {
                    int c = s_cnt[q];
                    s_cnt[q] = acc;
                    acc += c;
                }
            }
            __syncthreads();
            for (int j = 0; j < npt; ++j) {
                int idx = tid * npt + j;
                sperm[atomicAdd(&s_cnt[skey[idx]], 1)] = (int16_t)idx;
            }
            __syncthreads();
            // draw the batch: at step j the block evaluates sorted positions j*256 .. j*256+255
            for (int j = 0; j < npt; ++j) {
                int idx = sperm[j * PH2_THREADS + tid];
                int v = base + idx;
                float g = 1.0f;
                int nch = 0;
                if (v < P.trial_cap) {
                    Rng R;
                    R.init(P.seed, K_RECIP, iter_base + slot, (uint32_t)(k * 8 + rep), (uint32_t)v);
                    float ratio = entry_ratio<COUNT>(S, E, R, &tc);
                    g = 1.0f - ratio * invB;
                    float r = fabsf(g);
                    nch = (int)floorf(r);
                    if (R.u(18) < r - (float)nch) nch += 1;
                }
                sg[idx] = g;
                sn[idx] = nch;
            }
            if (tid == 0) {
                bool pos = st.cur_sign > 0.0f;
                for (int i = 0; i < st.sp; ++i) pos = pos && st.fr_sign[i] > 0.0f;
                s_neg = pos ? 0 : 1;
            }
            __syncthreads();
            // any negative g in the batch?
            int anyneg = 0;
            for (int j = 0; j < npt; ++j) anyneg |= (sg[tid * npt + j] < 0.0f);
            anyneg = __syncthreads_or(anyneg | s_neg);
            if (!anyneg && base + nb <= P.trial_cap) {
                // parallel walk: pending counts by a block prefix sum
                int pend0 = 1;
                for (int i = 0; i < st.sp; ++i) pend0 += st.fr_rem[i];
                int loc[PH2_NPT];
                int acc = 0;
#pragma unroll
                for (int j = 0; j < PH2_NPT; ++j) {
                    if (j < npt) acc += sn[tid * npt + j] - 1;
                    loc[j] = acc;
                }
                s_pending[tid] = acc;
                __syncthreads();
                for (int off = 1; off < PH2_THREADS; off <<= 1) {
                    int x = tid >= off ? s_pending[tid - off] : 0;
                    __syncthreads();
                    s_pending[tid] += x;
                    __syncthreads();
                }
                int excl = pend0 + s_pending[tid] - acc;
                int first = nb;
#pragma unroll
                for (int j = PH2_NPT - 1; j >= 0; --j)
                    if (j < npt && excl + loc[j] <= 0) first = tid * npt + j;
                if (tid == 0) s_end = nb;
                __syncthreads();
                if (first < nb) atomicMin(&s_end, first);
                __syncthreads();
                int end = s_end;   // last node processed (inclusive), or nb if none
                double part = 0.0;
                for (int j = 0; j < npt; ++j) {
                    int idx = tid * npt + j;
                    if (idx <= end && idx < nb) part += (double)(sg[idx] * invB);
                }
                s_part[tid] = part;
                __syncthreads();
                for (int off = PH2_THREADS / 2; off > 0; off >>= 1) {
                    if (tid < off) s_part[tid] += s_part[tid + off];
                    __syncthreads();
                }
                if (tid == 0) {
                    st.sum_t += s_part[0];
                    if (end < nb) {
                        st.next = base + end + 1;
                        s_done = 1;
                    } else {
                        int pend = pend0 + s_pending[PH2_THREADS - 1];
                        st.next = base + nb;
                        st.cur_sign = 1.0f;
                        st.sp = 0;
                        if (pend - 1 > 0) {
                            st.fr_sign[0] = 1.0f;
                            st.fr_rem[0] = pend - 1;
                            st.sp = 1;
                        }
                        s_done = 0;
                    }
                }
            } else if (tid == 0) {
                // exact sequential walk over the batch
                s_done = 0;
                for (int j = 0; j < nb; ++j) {
                    int v = base + j;
                    if (v >= P.trial_cap) {
                        s_done = 1;
                        trunc = true;
                        st.next = v;
                        break;
                    }
                    float gj = sg[j];
                    int nj = sn[j];
                    st.sum_t += (double)(st.cur_sign * gj * invB);
                    if (nj >= 1) {
                        if (st.sp >= MAXF) {
                            s_done = 1;
                            trunc = true;
                            st.next = v + 1;
                            break;
                        }
                        st.fr_sign[st.sp] = st.cur_sign * (gj > 0.0f ? 1.0f : -1.0f);
                        st.fr_rem[st.sp] = nj;
                        st.sp++;
                    }
                    if (st.sp == 0) {
                        s_done = 1;
                        st.next = v + 1;
                        break;
                    }
                    st.cur_sign = st.fr_sign[st.sp - 1];
                    if (--st.fr_rem[st.sp - 1] == 0) st.sp--;
                    st.next = v + 1;
                }
            }
            __syncthreads();
            done = s_done;
            __syncthreads();
        }
        if (tid == 0) {
            size_t o = ((size_t)slot * B.ML + k) * P.repeats + rep;
            B.rep[o] = (float)((double)invB + st.sum_t);
            B.repn[o] = (float)st.next;
            B.reptr[o] = trunc ? 1 : 0;
        }
        __syncthreads();
    }
    if (COUNT) {
        atomicAdd(&B.counters[CNT_REC_NODES], (unsigned long long)tc.nodes);
        atomicAdd(&B.counters[CNT_REC_TRIS], (unsigned long long)tc.tris);
        atomicAdd(&B.counters[CNT_REC_RAYS], (unsigned long long)tc.rays);
    }
}

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
constexpr int WF_WIN_MAX = 16384;

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
    __shared__ int part[1024];
    const int items = W.ctl[WF_CTL_ITEMS];
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid <= WF_MAXQ + 1) W.ctl[WF_CTL_CNT0 + tid] = 0;
    if (W.ctl[WF_CTL_ACTIVE] == 0) {
        if (tid == 0) W.ctl[WF_CTL_NODES] = 0;
        return;
    }
    const int per = (items + nt - 1) / nt;
    const int c0 = tid * per, c1 = min(items, c0 + per);
    int acc = 0;
    for (int c = c0; c < c1; ++c) {
        int w = 0;
        if (!W.ch_done[c]) w = max(0, min(W.ch_win[c], P.trial_cap - B.chains[c].next));
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
        if (run + w > W.node_cap) w = 0;   // no room this round: the chain waits
        W.ch_w[c] = w;
        W.ch_off[c] = run;
        run += w;
    }
    __syncthreads();
    if (tid == nt - 1) W.ctl[WF_CTL_NODES] = min(part[nt - 1], W.node_cap);
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
        } else if (T.susp) {
            W.node_q[i] = T.q;
            cg::coalesced_group g = cg::coalesced_threads();
            int base = 0;
            if (g.thread_rank() == 0) base = atomicAdd(&W.ctl[WF_CTL_CNT0 + s + 1], (int)g.size());
            out[g.shfl(base, 0) + g.thread_rank()] = i;
        } else if (PILOT) {
            W.node_g[i] = ratio;
        } else {
            float gv = 1.0f - ratio * invB;
            float r = fabsf(gv);
            int nch = (int)floorf(r);
            if (R.u(18) < r - (float)nch) nch += 1;
            W.node_g[i] = gv;
            W.node_n[i] = nch;
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

// one warp per chain: the walk over this round's window in chunks of 32
// nodes. While every pending node has sign +1 and the chunk has no negative
// g, the walk reduces to counts (pending_v = pending - 1 + n_v; the chain
// ends at the first node where pending reaches 0), a warp scan; otherwise
// lane 0 replays the exact sequential walk over the chunk.
__global__ void __launch_bounds__(128) k_wf_walk(KParams P, Pool B, WfBufs W) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int items = W.ctl[WF_CTL_ITEMS];
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < items; c += warps) {
        const int w = W.ch_w[c];
        if (W.ch_done[c] || w == 0) continue;
        ChainState &gst = B.chains[c];
        const int slot = gst.slot, k = gst.k, rep = gst.rep;
        const float invB = 1.0f / B.eB[(size_t)slot * B.ML + k];
        const int off = W.ch_off[c];
        int next = gst.next;
        double sum_t = gst.sum_t;
        // pending-count form of the walk state while all signs are +1
        bool pos = gst.cur_sign > 0.0f;
        int pend = 1;
        for (int f = 0; f < gst.sp; ++f) {
            pos = pos && gst.fr_sign[f] > 0.0f;
            pend += gst.fr_rem[f];
        }
        bool stack_form = !pos;   // gst holds the authoritative stack
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
                double t = (in && lane <= last) ? (double)(g * invB) : 0.0;
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                sum_t += t;
                next += last + 1;
                pend += __shfl_sync(0xffffffffu, x, last);
                if (endm) done = 1;
                continue;
            }
            // exact sequential walk of this chunk by lane 0, on the stack form
            if (!stack_form) {
                if (lane == 0) {
                    gst.cur_sign = 1.0f;
                    gst.sp = 0;
                    if (pend - 1 > 0) {
                        gst.fr_sign[0] = 1.0f;
                        gst.fr_rem[0] = pend - 1;
                        gst.sp = 1;
                    }
                }
                stack_form = true;
            }
            if (lane == 0) {
                const int cnt = min(32, w - j0);
                for (int q = 0; q < cnt; ++q) {
                    const float gj = W.node_g[off + j0 + q];
                    const int nj = W.node_n[off + j0 + q];
                    sum_t += (double)(gst.cur_sign * gj * invB);
                    next += 1;
                    if (nj >= 1) {
                        if (gst.sp >= MAXF) {
                            done = 1;
                            trunc = 1;
                            break;
                        }
                        gst.fr_sign[gst.sp] = gst.cur_sign * (gj > 0.0f ? 1.0f : -1.0f);
                        gst.fr_rem[gst.sp] = nj;
                        gst.sp++;
                    }
                    if (gst.sp == 0) {
                        done = 1;
                        break;
                    }
                    gst.cur_sign = gst.fr_sign[gst.sp - 1];
                    if (--gst.fr_rem[gst.sp - 1] == 0) gst.sp--;
                }
            }
            done = __shfl_sync(0xffffffffu, done, 0);
            trunc = __shfl_sync(0xffffffffu, trunc, 0);
            next = __shfl_sync(0xffffffffu, next, 0);
            sum_t = __shfl_sync(0xffffffffu, sum_t, 0);
            __syncwarp();
            // back to the count form when the stack turned all-positive again
            bool p2 = gst.cur_sign > 0.0f;
            int pe = 1;
            for (int f = 0; f < gst.sp; ++f) {
                p2 = p2 && gst.fr_sign[f] > 0.0f;
                pe += gst.fr_rem[f];
            }
            if (p2) {
                stack_form = false;
                pend = pe;
            }
            __syncwarp();
        }
        if (!done && next >= P.trial_cap) {
            done = 1;
            trunc = 1;
        }
        if (lane == 0) {
            if (!stack_form) {   // store the count form as a one-frame stack
                gst.cur_sign = 1.0f;
                gst.sp = 0;
                if (pend - 1 > 0) {
                    gst.fr_sign[0] = 1.0f;
                    gst.fr_rem[0] = pend - 1;
                    gst.sp = 1;
                }
            }
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
            float gj = 1.0f - ratio * invB;
            st.prod *= (double)gj;
            st.sum_t += st.prod / st.surv * (double)invB;
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
            float ratio = entry_ratio<false>(S, E, R, nullptr);
            float gj = 1.0f - ratio * invB;
            float r = fabsf(gj);
            int nj = (int)floorf(r);
            if (R.u(18) < r - (float)nj) nj += 1;
            st.sum_t += (double)(st.cur_sign * gj * invB);
            st.next += 1;
            if (nj >= 1) {
                if (st.sp >= MAXF) {
                    done = trunc = 1;
                    break;
                }
                st.fr_sign[st.sp] = st.cur_sign * (gj > 0.0f ? 1.0f : -1.0f);
                st.fr_rem[st.sp] = nj;
                st.sp++;
            }
            if (st.sp == 0) {
                done = 1;
                break;
            }
            st.cur_sign = st.fr_sign[st.sp - 1];
            if (--st.fr_rem[st.sp - 1] == 0) st.sp--;
        }
        size_t o = ((size_t)st.slot * B.ML + st.k) * P.repeats + st.rep;
        B.rep[o] = (float)((double)invB + st.sum_t);
        B.repn[o] = (float)st.next;
        B.reptr[o] = trunc;
        W.ch_done[c] = 1;
        B.chains[c] = st;
    }
}

__global__ void k_recip_offsets(KParams P, Pool B, int slots) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        B.work[0] = 0;
        B.work[2 + slots] = 0;       // chains handed to phase 2
        B.work[3 + slots] = 0;       // phase-2 work counter
        B.work[4 + slots] = 0;       // pilot work counter
        int acc = 0;
        for (int s = 0; s < slots; ++s) {
            B.work[1 + s] = acc;
            acc += B.nent[s] * P.repeats;
        }
        B.work[1 + slots] = acc;
    }
}

__global__ void k_recip_finish(KParams P, Pool B) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int slot = blockIdx.y;
    if (k >= B.nent[slot]) return;
    size_t o = ((size_t)slot * B.ML + k) * P.repeats;
    double acc = 0.0;
    float nn = 0.0f;
    int tr = 0;
    uint32_t h = 2166136261u;
    for (int r = 0; r < P.repeats; ++r) {
        acc += (double)B.rep[o + r];
        nn += B.repn[o + r];
        tr |= B.reptr[o + r];
        h = (h ^ (uint32_t)B.repn[o + r]) * 16777619u;
    }
    B.rhat[(size_t)slot * B.ML + k] = (float)(acc / (double)P.repeats);
    B.esig[(size_t)slot * B.ML + k] = h;
    atomicAdd(&B.counters[CNT_ENTRIES], 1ull);
    atomicAdd(&B.counters[CNT_TRUNC], (unsigned long long)tr);
    atomicAdd(&B.counters[CNT_NODES], (unsigned long long)nn);
}

}  // namespace

void launch_light_pass(const DScene &S, const KParams &P, const Pool &B, int slots, uint32_t iter_base,
                       cudaStream_t st) {
    dim3 grid((P.M + 127) / 128, slots);
    k_light_pass<<<grid, 128, 0, st>>>(S, P, B, iter_base);
}

void launch_pool_build(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots,
                       cudaStream_t st) {
    dim3 grid((P.M + 127) / 128, slots);
    k_pool_build<<<grid, 128, 0, st>>>(S, T, P, B);
    size_t shb = sizeof(int32_t) * (size_t)(T.KS + 1 + T.KSp + 1);
    k_bucket<<<slots, 64, shb, st>>>(T, B, B.scratch);
    k_cdf<<<dim3(T.KT, slots, 2), 256, 0, st>>>(T, B);
}

void launch_recip(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots, uint32_t iter_base,
                  int num_sms, cudaStream_t st, const WfBufs *wf) {
    k_recip_offsets<<<1, 32, 0, st>>>(P, B, slots);
    if (P.estimator == 0 && wf && wf->node_cap > 0) {
        const WfBufs W = *wf;
        if (P.pilot_max <= 0) {
            // no pilot: the kernel writes the table bounds without drawing
            k_recip_pilot<false><<<num_sms * 4, 128, 0, st>>>(S, T, P, B, slots, iter_base);
        } else {
            // the pilot as wavefront rounds: windows pilot_min, then doubling up to pilot_max
            k_wfp_init<<<num_sms * 2, 256, 0, st>>>(P, B, W, slots);
            const int nr = wf_pilot_rounds(P);
            for (int round = 0; round < nr; ++round) {
                k_wfp_plan<<<1, 1024, 0, st>>>(P, W);
                k_wf_nodes<true><<<num_sms * 8, 256, 0, st>>>(B, W);
                for (int s = 0; s <= WF_MAXQ; ++s) {
                    k_wf_step<true><<<num_sms * 8, 128, 0, st>>>(S, P, B, W, s, iter_base, slots);
                    if (s == WF_MAXQ) break;
                    if (P.count) k_wf_trace<true><<<num_sms * 8, 128, 0, st>>>(S, P, B, W, s);
                    else k_wf_trace<false><<<num_sms * 8, 128, 0, st>>>(S, P, B, W, s);
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
                if (P.count) k_wf_trace<true><<<num_sms * 8, 128, 0, st>>>(S, P, B, W, s);
                else k_wf_trace<false><<<num_sms * 8, 128, 0, st>>>(S, P, B, W, s);
            }
            if (P.booth > 0.0f) k_wf_walk_booth<<<num_sms * 16, 128, 0, st>>>(P, B, W, iter_base);
            else k_wf_walk<<<num_sms * 16, 128, 0, st>>>(P, B, W);
        }
        k_wf_finish_rest<<<num_sms * 2, 128, 0, st>>>(S, P, B, W, iter_base);
        dim3 g2((B.ML + 127) / 128, slots);
        k_recip_finish<<<g2, 128, 0, st>>>(P, B);
        return;
    }
    if (P.count) {
        k_recip_pilot<true><<<num_sms * 4, 128, 0, st>>>(S, T, P, B, slots, iter_base);
        k_recip<true><<<num_sms * 8, 128, 0, st>>>(S, T, P, B, slots, iter_base);
        k_recip_long<true><<<num_sms * 4, PH2_THREADS, 0, st>>>(S, T, P, B, slots, iter_base);
    } else {
        k_recip_pilot<false><<<num_sms * 4, 128, 0, st>>>(S, T, P, B, slots, iter_base);
        k_recip<false><<<num_sms * 8, 128, 0, st>>>(S, T, P, B, slots, iter_base);
        k_recip_long<false><<<num_sms * 4, PH2_THREADS, 0, st>>>(S, T, P, B, slots, iter_base);
    }
    dim3 g2((B.ML + 127) / 128, slots);
    k_recip_finish<<<g2, 128, 0, st>>>(P, B);
}
