// Learning of the frozen subspace tables on the device (Sec. 5.4-5.5 of
// arXiv 2503.23412: subspace statistics feed B and the MIS weight; the
// selection matrix is proportional to expected contribution, learned in the
// first iterations and then frozen). The learning iterations use their own
// iteration indices and are never added to the film.
//
//   centroids  Lloyd k-means (initialised with evenly spaced samples of the
//              valid points in slot order) over: eye vertices of a pretrace
//              (T, 9-d), connectable light vertices (S, 9-d), ends y_{s-1} of
//              incomplete sub-paths (S', 6-d) and their control vertices (C, 3-d)
//   B          b_safety (default 1) x the largest f/q drawn from the supporting
//              distribution per (u, S', C) cell (App. "Optimal value for B")
//   mis        mean(R) / mean(R^2) per cell = 1 / (E[R^2] Pbar), Pbar = 1/E[R]
//   Gamma      0.9 x normalised unweighted contribution per (T, S) + 0.1 uniform
//   pi         1.0 where the proxy share of a 10x10 tile is >= 5 %, else 0.2
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pb_ctx.h"
#include "pb_estimator.cuh"

namespace {

constexpr float B_SAFETY_DEFAULT = 1.0f;
enum : uint32_t { K_PRETRACE = 5 };

__device__ __forceinline__ void put9(float *o, const DScene &S, float3 p, float3 n, float3 w) {
    float3 nn = dot(n, w) >= 0.0f ? n : -n;
    o[0] = (p.x - S.lo.x) / S.ext.x;
    o[1] = (p.y - S.lo.y) / S.ext.y;
    o[2] = (p.z - S.lo.z) / S.ext.z;
    o[3] = nn.x; o[4] = nn.y; o[5] = nn.z;
    o[6] = w.x; o[7] = w.y; o[8] = w.z;
}

// features of the light side of one wave: connectable vertices, incomplete
// sub-path ends and their control vertices; slot-major, fixed positions
__global__ void k_feat_light(DScene S, KParams P, Pool B, int slots, size_t out_off, float *fS, uint8_t *vS,
                             float *fY, uint8_t *vY, float *fC, uint8_t *vC) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)slots * B.ML;
    if (i >= n) return;
    size_t o = out_off + i;
    vS[o] = vY[o] = vC[o] = 0;
    if (B.vlabel[i] >= 0) {
        float4 vp = B.vpos[i], vn = B.vnrm[i], vw = B.vwl[i];
        put9(fS + 9 * o, S, xyz(vp), xyz(vn), xyz(vw));
        vS[o] = 1;
    }
    if (B.elabel[i] >= 0) {
        float4 vp = B.vpos[i], vn = B.vnrm[i];
        float *y = fY + 6 * o;
        y[0] = (vp.x - S.lo.x) / S.ext.x;
        y[1] = (vp.y - S.lo.y) / S.ext.y;
        y[2] = (vp.z - S.lo.z) / S.ext.z;
        y[3] = vn.x; y[4] = vn.y; y[5] = vn.z;
        vY[o] = 1;
        int info = B.einfo[i];
        if ((info >> 3) & 1) {
            size_t slot = i / B.ML, fixed = i % B.ML;
            size_t g0 = slot * B.ML + (fixed / P.L) * P.L;
            Vtx H = vertex_at(S, B.gtri[g0], B.gbary[g0].x, B.gbary[g0].y);
            float *c = fC + 3 * o;
            c[0] = (H.p.x - S.lo.x) / S.ext.x;
            c[1] = (H.p.y - S.lo.y) / S.ext.y;
            c[2] = (H.p.z - S.lo.z) / S.ext.z;
            vC[o] = 1;
        }
    }
}

// eye-vertex pretrace: BSDF-sampled camera paths, features of every
// non-specular vertex (position, normal toward the eye side, eye direction)
__global__ void k_pretrace_eye(DScene S, KParams P, uint32_t iter_base, int slots, size_t out_off, float *fT,
                               uint8_t *vT) {
    int pix = blockIdx.x * blockDim.x + threadIdx.x;
    int slot = blockIdx.y;
    if (pix >= P.npix || slot >= slots) return;
    size_t base = out_off + ((size_t)slot * P.npix + pix) * P.max_depth;
    for (int a = 0; a < P.max_depth; ++a) vT[base + a] = 0;
    uint32_t it = iter_base + slot;
    Rng r;
    r.init(P.seed, K_PRETRACE, it, (uint32_t)pix, 0);
    int px = pix % S.W, py = pix / S.W;
    float sx = 2.0f * ((float)px + r.u(0)) / (float)S.W - 1.0f, sy = 1.0f - 2.0f * ((float)py + r.u(1)) / (float)S.H;
    float3 d = normalize(S.cfwd + (S.cright * (sx * S.tanh_ * S.aspect) + S.cup * (sy * S.tanh_)));
    float3 o = S.cpos;
    int skip = -1;
    for (int a = 0; a < P.max_depth; ++a) {
        Hit h = closest_hit<false>(S, o, d, skip);
        if (h.tri < 0) break;
        Vtx z = vertex_at(S, h.tri, h.b1, h.b2);
        float3 we = -d;
        const DMat &m = S.mats[z.mat];
        if (!m.specular) {
            put9(fT + 9 * (base + a), S, z.p, z.n, we);
            vT[base + a] = 1;
        }
        if (absorbing(S, z, we)) break;
        Rng q;
        q.init(P.seed, K_PRETRACE, it, (uint32_t)pix, (uint32_t)(a + 1));
        float3 wl;
        if (!bsdf_sample(m, z.n, we, q.u(0), q.u(1), q.u(2), wl)) break;
        o = z.p;
        d = wl;
        skip = z.tri;
    }
}

// deterministic compaction of valid point indices (one warp, ballot order)
__global__ void k_compact(const uint8_t *valid, size_t n, int32_t *idx, int32_t *count) {
    int lane = threadIdx.x & 31;
    unsigned lt = (1u << lane) - 1u;
    int cnt = 0;
    for (size_t b = 0; b < n; b += 32) {
        size_t i = b + lane;
        bool v = i < n && valid[i];
        unsigned m = __ballot_sync(0xffffffffu, v);
        if (v) idx[cnt + __popc(m & lt)] = (int32_t)i;
        cnt += __popc(m);
    }
    if (lane == 0) *count = cnt;
}

__global__ void k_km_init(const float *pts, int D, const int32_t *idx, const int32_t *count, int K, float *cent) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    int n = *count;
    for (int d = 0; d < D; ++d) cent[k * D + d] = 0.0f;
    if (n == 0) return;
    int j = n >= K ? (int)(((long long)k * n) / K) : (k % n);
    const float *p = pts + (size_t)D * idx[j];
    for (int d = 0; d < D; ++d) cent[k * D + d] = p[d];
}

__global__ void k_km_assign(const float *pts, int D, const int32_t *idx, const int32_t *count, int K,
                            const float *cent, float *sum, int32_t *cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *count) return;
    const float *p = pts + (size_t)D * idx[i];
    float f[9];
    for (int d = 0; d < D; ++d) f[d] = p[d];
    int best = nearest(f, D, K, cent);
    for (int d = 0; d < D; ++d) atomicAdd(&sum[best * D + d], f[d]);
    atomicAdd(&cnt[best], 1);
}

__global__ void k_km_update(int D, int K, float *cent, const float *sum, const int32_t *cnt) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K || cnt[k] == 0) return;
    for (int d = 0; d < D; ++d) cent[k * D + d] = sum[k * D + d] / (float)cnt[k];
}

// B: largest f/q per cell over n draws per entry (stream kind TRAIN,
// a = iteration, b = entry, c = draw); positive floats compare as ints

__global__ void k_bsample(DScene S, DTables T, KParams P, Pool B, int slots, uint32_t iter_base, int nsamp,
                          unsigned *cell_max) {
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    int slot = blockIdx.y;
    int ne = B.nent[slot];
    if (t >= (size_t)ne * nsamp) return;
    int k = (int)(t / nsamp), smp = (int)(t % nsamp);
    size_t o = (size_t)slot * B.ML;
    int fixed = B.ent_idx[o + k];
    int l = fixed / P.L, e = fixed % P.L;
    size_t gb = o + (size_t)l * P.L;
    Vtx Y = vertex_at(S, B.gtri[gb + e], B.gbary[gb + e].x, B.gbary[gb + e].y);
    Vtx H = vertex_at(S, B.gtri[gb], B.gbary[gb].x, B.gbary[gb].y);
    int info = B.einfo[o + fixed];
    int u = info & 7, type = (info >> 3) & 1, C = info >> 4;
    int Sp = B.elabel[o + fixed];
    Rng R;
    R.init(P.seed, K_TRAIN, iter_base + slot, (uint32_t)k, (uint32_t)smp);
    Entry E;
    E.Y = Y;
    E.H = H;
    E.u = u;
    E.type = type;
    Vtx Yp = vertex_at(S, B.gtri[gb + e - 1], B.gbary[gb + e - 1].x, B.gbary[gb + e - 1].y);
    E.back = dot(Y.n, Yp.p - Y.p) < 0.0f ? 1 : 0;
    E.pin = P.side_in;
    float r = entry_ratio(S, E, R);
    if (r > 0.0f) {
        atomicMax(&cell_max[((u - 1) * T.KSp + Sp) * (T.KC + 1) + C], __float_as_uint(r));
        atomicMax(&cell_max[4 * T.KSp * (T.KC + 1)], __float_as_uint(r));
    }
}

__global__ void k_recip_stats(DTables T, KParams P, Pool B, double *s1, double *s2, double *s3, int32_t *cn) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int slot = blockIdx.y;
    if (k >= B.nent[slot]) return;
    size_t o = (size_t)slot * B.ML;
    int fixed = B.ent_idx[o + k];
    int info = B.einfo[o + fixed];
    int u = info & 7, C = info >> 4;
    int Sp = B.elabel[o + fixed];
    int cell = ((u - 1) * T.KSp + Sp) * (T.KC + 1) + C;
    double R = (double)B.rhat[o + k];
    // estimator nodes of the entry over its repeats; reaching trial_cap in
    // total counts as over any bound
    double nodes = 0.0;
    for (int r = 0; r < P.repeats; ++r) nodes += (double)B.repn[(o + k) * P.repeats + r];
    atomicAdd(&s1[cell], R);
    atomicAdd(&s2[cell], R * R);
    atomicAdd(&s3[cell], nodes >= (double)P.trial_cap ? 1e30 : nodes);
    atomicAdd(&cn[cell], 1);
}

}  // namespace

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return pb_fail(ctx, e_ == cudaErrorMemoryAllocation ? PB_ERR_OOM : PB_ERR_CUDA, \
                           std::string(#call) + ": " + cudaGetErrorString(e_));           \
    } while (0)

namespace {

struct DevBuf {
    std::vector<void *> mem;
    ~DevBuf() {
        for (void *p : mem) cudaFree(p);
    }
    template <class T>
    cudaError_t get(T **p, size_t n) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) {
            mem.push_back(q);
            *p = (T *)q;
        }
        return e;
    }
};

pb_status kmeans(pb_ctx *ctx, DevBuf &tmp, const float *pts, const uint8_t *valid, size_t n, int D, int K, int iters,
                 float *cent_out) {
    int32_t *idx, *count, *cnt;
    float *sum;
    CK(tmp.get(&idx, n));
    CK(tmp.get(&count, 1));
    CK(tmp.get(&cnt, (size_t)K));
    CK(tmp.get(&sum, (size_t)K * D));
    k_compact<<<1, 32, 0, ctx->stream>>>(valid, n, idx, count);
    k_km_init<<<(K + 127) / 128, 128, 0, ctx->stream>>>(pts, D, idx, count, K, cent_out);
    int grid = (int)std::min<size_t>((n + 255) / 256, 1 << 20);
    for (int i = 0; i < iters; ++i) {
        CK(cudaMemsetAsync(sum, 0, sizeof(float) * K * D, ctx->stream));
        CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * K, ctx->stream));
        k_km_assign<<<grid, 256, 0, ctx->stream>>>(pts, D, idx, count, K, cent_out, sum, cnt);
        k_km_update<<<(K + 127) / 128, 128, 0, ctx->stream>>>(D, K, cent_out, sum, cnt);
    }
    CK(cudaGetLastError());
    return PB_OK;
}

}  // namespace

extern "C" pb_status pb_prepare(pb_ctx *ctx, const pb_config *cfg, const pb_learn_desc *ld, pb_stats *stats) {
    if (!ctx) return PB_ERR_ARG;
    if (!ctx->has_scene) return pb_fail(ctx, PB_ERR_STATE, "no scene uploaded");
    if (!cfg || !ld || ld->n_iter < 1 || ld->n_bsamples < 1 || ld->lloyd_iters < 0)
        return pb_fail(ctx, PB_ERR_ARG, "prepare: bad learning description");
    if (ld->keep_centroids && !ctx->has_tables) return pb_fail(ctx, PB_ERR_STATE, "keep_centroids needs uploaded tables");
    CK(cudaSetDevice(ctx->device));
    int W = ctx->S.W, H = ctx->S.H;
    const float b_safety = ld->b_safety > 0.0f ? ld->b_safety : B_SAFETY_DEFAULT;
    // ---- the tables being learned: sizes, bbox, initial contents
    int KT, KS, KSp, KC, tile;
    std::vector<float> cT, cS, cSp, cC, lo(3), hi(3);
    if (ld->keep_centroids) {
        KT = ctx->T.KT; KS = ctx->T.KS; KSp = ctx->T.KSp; KC = ctx->T.KC; tile = ctx->T.tile;
        cT.resize((size_t)KT * 9); cS.resize((size_t)KS * 9); cSp.resize((size_t)KSp * 6); cC.resize((size_t)KC * 3);
        CK(cudaMemcpy(cT.data(), ctx->T.cT, 4 * cT.size(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(cS.data(), ctx->T.cS, 4 * cS.size(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(cSp.data(), ctx->T.cSp, 4 * cSp.size(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(cC.data(), ctx->T.cC, 4 * cC.size(), cudaMemcpyDeviceToHost));
        lo = {ctx->S.lo.x, ctx->S.lo.y, ctx->S.lo.z};
        hi = {ctx->S.lo.x + ctx->S.ext.x, ctx->S.lo.y + ctx->S.ext.y, ctx->S.lo.z + ctx->S.ext.z};
    } else {
        KT = ld->KT; KS = ld->KS; KSp = ld->KSp; KC = ld->KC; tile = ld->tile;
        if (KT <= 0 || KS <= 0 || KSp <= 0 || KC <= 0 || tile <= 0)
            return pb_fail(ctx, PB_ERR_ARG, "prepare: table sizes must be positive");
        cT.assign((size_t)KT * 9, 0.f); cS.assign((size_t)KS * 9, 0.f);
        cSp.assign((size_t)KSp * 6, 0.f); cC.assign((size_t)KC * 3, 0.f);
        lo = {ctx->scene_lo.x, ctx->scene_lo.y, ctx->scene_lo.z};
        hi = {ctx->scene_hi.x, ctx->scene_hi.y, ctx->scene_hi.z};
    }
    int gw = (W + tile - 1) / tile, gh = (H + tile - 1) / tile;
    int ncell = 4 * KSp * (KC + 1);
    std::vector<float> gC((size_t)KT * KS, 1.0f / KS), gP((size_t)KT * KSp, 1.0f / KSp);
    // MIS scale 1 everywhere while learning: every entry stays in the pool
    std::vector<float> Bt(ncell, 1.0f), mis(ncell, 1.0f), pi((size_t)gw * gh, 1.0f);
    auto upload_tables = [&]() -> pb_status {
        pb_tables_desc d{KT, KS, KSp, KC, lo.data(), hi.data(), cT.data(), cS.data(), cSp.data(), cC.data(),
                         gC.data(), gP.data(), Bt.data(), mis.data(), tile, gw, gh, pi.data()};
        return pb_tables_upload(ctx, &d);
    };
    pb_status s = upload_tables();
    if (s != PB_OK) return s;
    KParams P = pb_kparams(ctx, cfg);
    P.booth = 0.0f;   // statistics are learned with the paper's RRS function
    int slots = std::max(1, std::min(ld->n_iter, std::max(1, (1 << 23) / std::max(1, P.npix))));
    s = pb_ensure_pool(ctx, slots, P.M * P.L, P.repeats);
    if (s != PB_OK) return s;
    DevBuf tmp;
    const uint32_t it0 = ld->iter0;
    size_t ML = (size_t)P.M * P.L;
    CK(cudaMemsetAsync(ctx->B.counters, 0, sizeof(unsigned long long) * CNT_N, ctx->stream));
    // ---- 1. centroids
    if (!ld->keep_centroids) {
        size_t nl = (size_t)ld->n_iter * ML, ne = (size_t)ld->n_iter * P.npix * P.max_depth;
        float *fS, *fY, *fC, *fT;
        uint8_t *vS, *vY, *vC, *vT;
        CK(tmp.get(&fS, nl * 9)); CK(tmp.get(&vS, nl));
        CK(tmp.get(&fY, nl * 6)); CK(tmp.get(&vY, nl));
        CK(tmp.get(&fC, nl * 3)); CK(tmp.get(&vC, nl));
        CK(tmp.get(&fT, ne * 9)); CK(tmp.get(&vT, ne));
        for (int done = 0; done < ld->n_iter;) {
            int ns = std::min(slots, ld->n_iter - done);
            launch_light_pass(ctx->S, P, ctx->B, ns, it0 + done, ctx->stream);
            launch_pool_build(ctx->S, ctx->T, P, ctx->B, ns, ctx->stream);
            size_t n = (size_t)ns * ML;
            k_feat_light<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(ctx->S, P, ctx->B, ns, (size_t)done * ML,
                                                                              fS, vS, fY, vY, fC, vC);
            k_pretrace_eye<<<dim3((P.npix + 127) / 128, ns), 128, 0, ctx->stream>>>(
                ctx->S, P, it0 + done, ns, (size_t)done * P.npix * P.max_depth, fT, vT);
            CK(cudaGetLastError());
            done += ns;
        }
        float *dc;
        CK(tmp.get(&dc, (size_t)std::max(std::max(KT, KS) * 9, std::max(KSp * 6, KC * 3))));
        struct Set { const float *f; const uint8_t *v; size_t n; int D, K; std::vector<float> *out; };
        Set sets[4] = {{fT, vT, ne, 9, KT, &cT}, {fS, vS, nl, 9, KS, &cS}, {fY, vY, nl, 6, KSp, &cSp}, {fC, vC, nl, 3, KC, &cC}};
        for (auto &st : sets) {
            s = kmeans(ctx, tmp, st.f, st.v, st.n, st.D, st.K, ld->lloyd_iters, dc);
            if (s != PB_OK) return s;
            CK(cudaMemcpyAsync(st.out->data(), dc, 4 * st.out->size(), cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
        }
        s = upload_tables();
        if (s != PB_OK) return s;
        s = pb_ensure_pool(ctx, slots, P.M * P.L, P.repeats);
        if (s != PB_OK) return s;
    }
    // ---- 2. B from f/q draws
    unsigned *cmax;
    CK(tmp.get(&cmax, (size_t)ncell + 1));
    CK(cudaMemsetAsync(cmax, 0, 4 * ((size_t)ncell + 1), ctx->stream));
    for (int done = 0; done < ld->n_iter;) {
        int ns = std::min(slots, ld->n_iter - done);
        launch_light_pass(ctx->S, P, ctx->B, ns, it0 + done, ctx->stream);
        launch_pool_build(ctx->S, ctx->T, P, ctx->B, ns, ctx->stream);
        size_t n = ML * (size_t)ld->n_bsamples;
        k_bsample<<<dim3((unsigned)((n + 127) / 128), ns), 128, 0, ctx->stream>>>(ctx->S, ctx->T, P, ctx->B, ns,
                                                                                   it0 + done, ld->n_bsamples, cmax);
        CK(cudaGetLastError());
        done += ns;
    }
    std::vector<unsigned> cm(ncell + 1);
    CK(cudaMemcpyAsync(cm.data(), cmax, 4 * cm.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    float gmax;
    memcpy(&gmax, &cm[ncell], 4);
    if (!(gmax > 0.0f)) gmax = 1.0f;
    for (int c = 0; c < ncell; ++c) {
        float v;
        memcpy(&v, &cm[c], 4);
        Bt[c] = b_safety * (v > 0.0f ? v : gmax);
    }
    s = upload_tables();
    if (s != PB_OK) return s;
    s = pb_ensure_pool(ctx, slots, P.M * P.L, P.repeats);
    if (s != PB_OK) return s;
    CK(cudaMemsetAsync(ctx->B.counters, 0, sizeof(unsigned long long) * CNT_N, ctx->stream));
    // ---- 3. MIS scale from reciprocal estimates
    double *s1, *s2, *s3;
    int32_t *cn;
    CK(tmp.get(&s1, (size_t)ncell));
    CK(tmp.get(&s2, (size_t)ncell));
    CK(tmp.get(&s3, (size_t)ncell));
    CK(tmp.get(&cn, (size_t)ncell));
    CK(cudaMemsetAsync(s1, 0, 8 * (size_t)ncell, ctx->stream));
    CK(cudaMemsetAsync(s2, 0, 8 * (size_t)ncell, ctx->stream));
    CK(cudaMemsetAsync(s3, 0, 8 * (size_t)ncell, ctx->stream));
    CK(cudaMemsetAsync(cn, 0, 4 * (size_t)ncell, ctx->stream));
    for (int done = 0; done < ld->n_iter;) {
        int ns = std::min(slots, ld->n_iter - done);
        launch_light_pass(ctx->S, P, ctx->B, ns, it0 + done, ctx->stream);
        launch_pool_build(ctx->S, ctx->T, P, ctx->B, ns, ctx->stream);
        launch_recip(ctx->S, ctx->T, P, ctx->B, ns, it0 + done, ctx->num_sms, ctx->stream);
        k_recip_stats<<<dim3((unsigned)((ML + 127) / 128), ns), 128, 0, ctx->stream>>>(ctx->T, P, ctx->B, s1, s2, s3, cn);
        CK(cudaGetLastError());
        done += ns;
    }
    pb_stats st{};
    {
        unsigned long long c[CNT_N];
        CK(cudaStreamSynchronize(ctx->stream));   // counters are written on the context's stream
        CK(cudaMemcpy(c, ctx->B.counters, sizeof(c), cudaMemcpyDeviceToHost));
        st.n_entries = (int64_t)c[CNT_ENTRIES];   // incomplete sub-paths of the n_iter learning iterations
        st.n_truncated = (int64_t)c[CNT_TRUNC];
        st.n_nodes = (int64_t)c[CNT_NODES];
    }
    std::vector<double> h1(ncell), h2(ncell), h3(ncell);
    std::vector<int32_t> hn(ncell);
    CK(cudaMemcpyAsync(h1.data(), s1, 8 * (size_t)ncell, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(h2.data(), s2, 8 * (size_t)ncell, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(h3.data(), s3, 8 * (size_t)ncell, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hn.data(), cn, 4 * (size_t)ncell, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double t1 = 0, t2 = 0;
    for (int c = 0; c < ncell; ++c) { t1 += h1[c]; t2 += h2[c]; }
    double pooled = (t1 > 0 && t2 > 0) ? t1 / t2 : 1.0;
    const double max_chain = ld->max_chain == 0.0f ? 4096.0 : (double)ld->max_chain;
    for (int c = 0; c < ncell; ++c) {
        mis[c] = (float)((hn[c] > 0 && h1[c] > 0 && h2[c] > 0) ? h1[c] / h2[c] : pooled);
        // learned cost bound: cells whose estimates run too long leave the proxy pool
        if (max_chain > 0.0 && hn[c] > 0 && h3[c] > max_chain * (double)hn[c] * (double)P.repeats) mis[c] = 0.0f;
    }
    s = upload_tables();
    if (s != PB_OK) return s;
    s = pb_ensure_pool(ctx, slots, P.M * P.L, P.repeats);
    if (s != PB_OK) return s;
    // ---- 4. Gamma rows and the tile grid from eye passes with uniform rows
    float *aC, *aP, *tA, *tP;
    CK(tmp.get(&aC, (size_t)KT * KS));
    CK(tmp.get(&aP, (size_t)KT * KSp));
    CK(tmp.get(&tA, (size_t)gw * gh));
    CK(tmp.get(&tP, (size_t)gw * gh));
    CK(cudaMemsetAsync(aC, 0, 4 * (size_t)KT * KS, ctx->stream));
    CK(cudaMemsetAsync(aP, 0, 4 * (size_t)KT * KSp, ctx->stream));
    CK(cudaMemsetAsync(tA, 0, 4 * (size_t)gw * gh, ctx->stream));
    CK(cudaMemsetAsync(tP, 0, 4 * (size_t)gw * gh, ctx->stream));
    KParams PL = P;
    PL.acc = LearnAcc{aC, aP, tA, tP};
    for (int done = 0; done < ld->n_iter;) {
        int ns = std::min(slots, ld->n_iter - done);
        s = pb_run_wave(ctx, PL, ns, it0 + done, true, true, nullptr);
        if (s != PB_OK) return s;
        done += ns;
    }
    std::vector<float> hC((size_t)KT * KS), hP((size_t)KT * KSp), hA((size_t)gw * gh), hT((size_t)gw * gh);
    CK(cudaMemcpyAsync(hC.data(), aC, 4 * hC.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hP.data(), aP, 4 * hP.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hA.data(), tA, 4 * hA.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hT.data(), tP, 4 * hT.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < KT; ++r) {
        double sc = 0, sp = 0;
        for (int c = 0; c < KS; ++c) sc += hC[(size_t)r * KS + c];
        for (int c = 0; c < KSp; ++c) sp += hP[(size_t)r * KSp + c];
        for (int c = 0; c < KS; ++c)
            gC[(size_t)r * KS + c] = (float)(sc > 0 ? 0.9 * hC[(size_t)r * KS + c] / sc + 0.1 / KS : 1.0 / KS);
        for (int c = 0; c < KSp; ++c)
            gP[(size_t)r * KSp + c] = (float)(sp > 0 ? 0.9 * hP[(size_t)r * KSp + c] / sp + 0.1 / KSp : 1.0 / KSp);
    }
    for (size_t i = 0; i < pi.size(); ++i) pi[i] = (hA[i] > 0 && hT[i] / hA[i] >= 0.05f) ? 1.0f : 0.2f;
    s = upload_tables();
    if (s != PB_OK) return s;
    if (stats) *stats = st;
    return PB_OK;
}

extern "C" pb_status pb_tables_readback(pb_ctx *ctx, pb_tables_host *t) {
    if (!ctx || !t) return PB_ERR_ARG;
    if (!ctx->has_tables) return pb_fail(ctx, PB_ERR_STATE, "no tables");
    const DTables &T = ctx->T;
    t->KT = T.KT; t->KS = T.KS; t->KSp = T.KSp; t->KC = T.KC;
    t->tile = T.tile; t->grid_w = T.gw; t->grid_h = T.gh;
    if (!t->cent_T || !t->cent_S || !t->cent_Sp || !t->cent_C || !t->gamma_conn || !t->gamma_proxy || !t->B_tab ||
        !t->mis_tab || !t->pi_grid || !t->bbox_lo || !t->bbox_hi)
        return PB_OK;   // sizes only
    int ncell = 4 * T.KSp * (T.KC + 1);
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(t->cent_T, T.cT, 4 * (size_t)T.KT * 9, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(t->cent_S, T.cS, 4 * (size_t)T.KS * 9, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(t->cent_Sp, T.cSp, 4 * (size_t)T.KSp * 6, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(t->cent_C, T.cC, 4 * (size_t)T.KC * 3, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(t->gamma_conn, T.gC, 4 * (size_t)T.KT * T.KS, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(t->gamma_proxy, T.gP, 4 * (size_t)T.KT * T.KSp, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(t->B_tab, T.Bt, 4 * (size_t)ncell, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(t->mis_tab, T.mis, 4 * (size_t)ncell, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(t->pi_grid, T.pi, 4 * (size_t)T.gw * T.gh, cudaMemcpyDeviceToHost));
    t->bbox_lo[0] = ctx->S.lo.x; t->bbox_lo[1] = ctx->S.lo.y; t->bbox_lo[2] = ctx->S.lo.z;
    t->bbox_hi[0] = ctx->S.lo.x + ctx->S.ext.x;
    t->bbox_hi[1] = ctx->S.lo.y + ctx->S.ext.y;
    t->bbox_hi[2] = ctx->S.lo.z + ctx->S.ext.z;
    return PB_OK;
}
