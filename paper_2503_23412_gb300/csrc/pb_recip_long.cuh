// Phase 2 of the reciprocal estimator's warp/block schedule (Sec. 4.2, App.
// Alg. I~). Each variant (traversal counting on or off) is compiled in its
// own translation unit, which keeps the build parallel.
#pragma once

#include "pb_entry.cuh"

namespace {

#define PH2_THREADS 256
#define PH2_NPT 8
#define PH2_BATCH (PH2_THREADS * PH2_NPT)

// Phase 2: a block per long chain. Each batch draws nb = 256 * npt
// consecutive nodes in parallel, npt in {1, 2, 4, 8} sized from the entry's
// expected chain length so that little is drawn past the chain's end. The
// nodes are evaluated grouped by the branch their first uniforms select
// (mixture component, side of the lens), so that whole warps trace alike;
// the walk still consumes them in pre-order. While every pending node has
// weight +1 under the estimate's own bound and the batch has no negative g,
// the walk reduces to counts:
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
    __shared__ float sx[PH2_BATCH], su[PH2_BATCH];   // f/q and RRS uniform (the walk under a raised bound)
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
                sg[idx] = g;
                sn[idx] = nch;
                sx[idx] = x;
                su[idx] = u;
            }
            if (tid == 0) {
                int pend;
                s_neg = est_count_form(st, invB, pend) ? 0 : 1;
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
                        est_from_count(st, pend, invB);
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
                    const EstStep e = est_step(st, sx[j], su[j], sg[j], sn[j], invB, (uint32_t)v, P);
                    const int r = est_take<PB_MAXF>(st, e, st.sum_t);
                    st.next = v + 1;
                    if (r) {
                        s_done = 1;
                        trunc = r == 2;
                        break;
                    }
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

}  // namespace
