// Light side of an iteration (Sec. 3.2, 5.1-5.3 of arXiv 2503.23412):
//   k_light_pass     M light sub-paths per iteration, geometry only
//   k_pool_build     per light vertex: throughput f_y/p_y, MIS partial sums,
//                    light-subspace label; incomplete sub-path detection
//                    (L S^u / L D S^u, 1 <= u <= 4) with S' and C labels
//   k_bucket         stable compaction in (path, vertex) order and stable
//                    counting sort by subspace (deterministic pool order)
//   k_cdf            per eye subspace, the selection CDF over non-empty
//                    subspaces (SPCBPT two-stage selection, Sec. 5.5)
//   launch_recip     the reciprocal estimator (Sec. 4.2, App. Alg. I~): the
//                    bound kernels and the warp/block schedule live in
//                    pb_recip.cu, the wavefront schedule in pb_wavefront.cu
//   k_recip_finish   average of the repeats per entry
#include <cstdio>

#include "pb_entry.cuh"

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
                int Sp = label_spec(S, T, y[e]);
                // a cell with MIS scale 0 is left to the other strategies
                if (T.mis[((u - 1) * T.KSp + Sp) * (T.KC + 1) + C] > 0.0f) {
                    B.elabel[k] = Sp;
                    B.einfo[k] = u | (type << 3) | (C << 4);
                }
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
        // no pilot: the bound kernel writes the table bounds without drawing
        if (P.pilot_max <= 0) launch_recip_bounds(S, T, P, B, slots, iter_base, num_sms, st, false);
        launch_recip_wavefront(S, T, P, B, slots, iter_base, num_sms, st, *wf);
    } else {
        launch_recip_bounds(S, T, P, B, slots, iter_base, num_sms, st, P.count != 0);
        launch_recip_phases(S, T, P, B, slots, iter_base, num_sms, st);
    }
    dim3 g2((B.ML + 127) / 128, slots);
    k_recip_finish<<<g2, 128, 0, st>>>(P, B);
}
