// C ABI of the renderer (declared in include/proxybdpt.h): context, scene and
// table upload, the render loop over iteration waves, film readback, and the
// single-stage entry points the parity tests drive.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/proxybdpt.h"
#include "pb_bvh.h"
#include "pb_kernels.h"

#include "pb_ctx.h"

namespace {

pb_status fail(pb_ctx *c, pb_status s, const std::string &m) {
    if (c) c->err = m;
    return s;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? PB_ERR_OOM : PB_ERR_CUDA,  \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

template <class T>
cudaError_t dalloc(std::vector<void *> &owner, T **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    owner.push_back(q);
    *p = (T *)q;
    return cudaSuccess;
}

void free_all(std::vector<void *> &v) {
    for (void *p : v) cudaFree(p);
    v.clear();
}

template <class T>
cudaError_t upload(pb_ctx *c, std::vector<void *> &owner, T **dst, const T *src, size_t n) {
    cudaError_t e = dalloc(owner, dst, n);
    if (e != cudaSuccess) return e;
    if (n) e = cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, c->stream);
    return e;
}

pb_status ensure_pool(pb_ctx *ctx, int slots, int ML, int repeats, int npix) {
    const DTables &T = ctx->T;
    if (slots <= ctx->cap_slots && ML <= ctx->cap_ML && repeats <= ctx->cap_rep && T.KT <= ctx->cap_KT &&
        T.KS <= ctx->cap_KS && T.KSp <= ctx->cap_KSp && ctx->Lbuf && slots <= ctx->cap_Lslots &&
        ctx->B.ML == ML) {
        // Lbuf also depends on npix; it is sized at scene upload time
        (void)npix;
        return PB_OK;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    free_graphs(ctx);   // captured renders point into the old buffers
    free_all(ctx->pool_mem);
    // until every buffer below exists, the next call must allocate again
    ctx->cap_slots = ctx->cap_ML = ctx->cap_rep = ctx->cap_Lslots = 0;
    ctx->Lbuf = nullptr;
    ctx->sigbuf = nullptr;
    Pool &B = ctx->B;
    B = Pool{};
    B.slots = slots;
    B.ML = ML;
    size_t n = (size_t)slots * ML;
    auto &o = ctx->pool_mem;
    CK(dalloc(o, &B.gtri, n));
    CK(dalloc(o, &B.gbary, n));
    CK(dalloc(o, &B.vpos, n));
    CK(dalloc(o, &B.vnrm, n));
    CK(dalloc(o, &B.vwl, n));
    CK(dalloc(o, &B.valpha, n));
    CK(dalloc(o, &B.vmis, n));
    CK(dalloc(o, &B.vlabel, n));
    CK(dalloc(o, &B.elabel, n));
    CK(dalloc(o, &B.einfo, n));
    CK(dalloc(o, &B.pool_idx, n));
    CK(dalloc(o, &B.bitems, n));
    CK(dalloc(o, &B.ent_idx, n));
    CK(dalloc(o, &B.eitems, n));
    CK(dalloc(o, &B.bstart, (size_t)slots * (T.KS + 1)));
    CK(dalloc(o, &B.estart, (size_t)slots * (T.KSp + 1)));
    CK(dalloc(o, &B.npool, (size_t)slots));
    CK(dalloc(o, &B.nent, (size_t)slots));
    CK(dalloc(o, &B.cdfC, (size_t)slots * T.KT * T.KS));
    CK(dalloc(o, &B.ZC, (size_t)slots * T.KT));
    CK(dalloc(o, &B.cdfP, (size_t)slots * T.KT * T.KSp));
    CK(dalloc(o, &B.ZP, (size_t)slots * T.KT));
    CK(dalloc(o, &B.rep, n * repeats));
    CK(dalloc(o, &B.repn, n * repeats));
    CK(dalloc(o, &B.reptr, n * repeats));
    CK(dalloc(o, &B.rhat, n));
    CK(dalloc(o, &B.eB, n));
    CK(dalloc(o, &B.eMu, n));
    CK(dalloc(o, &B.esig, n));
    CK(dalloc(o, &B.work, (size_t)slots + 5));
    B.chain_cap = (int)std::min<size_t>(n * repeats, (size_t)1 << 18);
    CK(dalloc(o, &B.chains, (size_t)B.chain_cap));
    CK(dalloc(o, &B.scratch, 2 * n));
    CK(dalloc(o, &B.counters, (size_t)CNT_N));
    CK(dalloc(o, &ctx->Lbuf, (size_t)slots * ctx->S.W * ctx->S.H));
    CK(dalloc(o, &ctx->sigbuf, (size_t)slots * ctx->S.W * ctx->S.H));
    ctx->cap_slots = slots;
    ctx->cap_ML = ML;
    ctx->cap_rep = repeats;
    ctx->cap_KT = T.KT;
    ctx->cap_KS = T.KS;
    ctx->cap_KSp = T.KSp;
    ctx->cap_Lslots = slots;
    return PB_OK;
}

pb_status check_cfg(pb_ctx *ctx, const pb_config *c) {
    if (!ctx->has_scene) return fail(ctx, PB_ERR_STATE, "no scene uploaded");
    if (!ctx->has_tables) return fail(ctx, PB_ERR_STATE, "no tables uploaded");
    if (!c) return fail(ctx, PB_ERR_ARG, "null config");
    if (c->max_depth < 2 || c->max_depth > 16) return fail(ctx, PB_ERR_ARG, "max_depth must be in [2, 16]");
    if (c->M < 1 || c->M > (1 << 22)) return fail(ctx, PB_ERR_ARG, "M out of range");
    if (c->repeats < 1 || c->repeats > 8) return fail(ctx, PB_ERR_ARG, "repeats must be in [1, 8]");
    if (c->trial_cap < 1) return fail(ctx, PB_ERR_ARG, "trial_cap must be positive");
    if (c->spp < 0) return fail(ctx, PB_ERR_ARG, "spp must be >= 0");
    if (c->proposal < 0 || c->proposal > 2)
        return fail(ctx, PB_ERR_ARG, "proposal must be 0 (table), 1 (learned connection) or 2 (and learned proxy)");
    if (!(c->side_in >= 0.0f && c->side_in < 1.0f)) return fail(ctx, PB_ERR_ARG, "side_in must lie in [0, 1)");
    if (c->estimator < 0 || c->estimator > 1) return fail(ctx, PB_ERR_ARG, "estimator must be 0 or 1");
    if (!(c->booth >= 0.0f && c->booth < 3.0e38f)) return fail(ctx, PB_ERR_ARG, "booth must be finite and >= 0");
    if (c->trace < 0 || c->trace > 1) return fail(ctx, PB_ERR_ARG, "trace must be 0 or 1");
    if (c->film < 0 || c->film > 2) return fail(ctx, PB_ERR_ARG, "film must be 0, 1 or 2");
    if (c->booth > 0.0f && c->estimator != 0)
        return fail(ctx, PB_ERR_ARG, "Booth's roulette runs on the wavefront estimator (estimator 0) only");
    return PB_OK;
}

KParams kparams(const pb_ctx *ctx, const pb_config *c) {
    KParams P{};   // every pointer the call does not set stays null (no eye queries, rows or sinks)
    P.seed = c->seed;
    P.max_depth = c->max_depth;
    P.M = c->M;
    P.M_p = std::min(std::max(c->M_p, 0), c->M);
    P.repeats = c->repeats;
    P.proxy = c->proxy ? 1 : 0;
    P.conn = c->conn ? 1 : 0;
    P.trial_cap = c->trial_cap;
    P.L = c->max_depth - 1;
    P.npix = ctx->S.W * ctx->S.H;
    P.count = c->count_traversal ? 1 : 0;
    P.handoff = c->chain_handoff > 0 ? ((c->chain_handoff + 31) / 32) * 32 : 512;
    if (c->pilot_max < 0) {
        P.pilot_min = P.pilot_max = 0;
    } else {
        int lo = c->pilot_min > 0 ? c->pilot_min : 64, hi = c->pilot_max > 0 ? c->pilot_max : 1024;
        lo = std::max(32, ((lo + 31) / 32) * 32);
        hi = std::max(lo, ((hi + 31) / 32) * 32);
        P.pilot_min = lo;
        P.pilot_max = hi;
    }
    P.side_in = c->side_in > 0.0f ? c->side_in : 0.5f;
    P.estimator = c->estimator;
    P.booth = c->booth;
    P.trace = c->trace;
    P.film = c->film;
    P.proposal = c->proposal;
    P.split = c->split_cap == 0 ? (1u << 16) : (c->split_cap < 0 ? 0xFFFFFFFFu : (uint32_t)c->split_cap);
    P.fixed_bound = c->fixed_bound != 0;
    P.acc = LearnAcc{nullptr, nullptr, nullptr, nullptr};
    P.mlp = MlpRows{nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr, 0};
    P.smp = SampleSink{nullptr, nullptr, nullptr, nullptr, nullptr, 0};
    P.mlpp = MlpRows{nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr, 0};
    P.smpp = SampleSink{nullptr, nullptr, nullptr, nullptr, nullptr, 0};
    P.q = EyeQueries{nullptr, nullptr, nullptr, nullptr, 0, nullptr, 0};
    P.iter_dev = nullptr;
    return P;
}

pb_status run_wave(pb_ctx *ctx, const KParams &P, int slots, uint32_t iter_base, bool with_light, bool with_recip,
                   uint32_t *sig) {
    if (with_light) launch_light_pass(ctx->S, P, ctx->B, slots, iter_base, ctx->stream);
    launch_pool_build(ctx->S, ctx->T, P, ctx->B, slots, ctx->stream);
    if (with_recip) launch_recip(ctx->S, ctx->T, P, ctx->B, slots, iter_base, ctx->num_sms, ctx->stream, &ctx->wf);
    CK(cudaGetLastError());
    return pb_eye_stages(ctx, P, slots, iter_base, sig, ctx->stream);
}

// Structural check of a built hierarchy before any kernel walks it: every
// child index in range, every triangle in exactly one leaf, parent/sibling
// links consistent, depth small enough for the 64-bit traversal trail.
bool bvh_valid(const PbBvh &b, int nn, int nt, std::string &why) {
    std::vector<int> seen(nt, 0);
    std::vector<int> depth(nn, -1);
    depth[0] = 0;
    std::vector<int> stack{0};
    int visited = 0;
    while (!stack.empty()) {
        int n = stack.back();
        stack.pop_back();
        ++visited;
        const int32_t *w = reinterpret_cast<const int32_t *>(&b.nodes[(size_t)n * 16]);
        int32_t ch[2] = {w[3], w[7]};
        for (int k = 0; k < 2; ++k) {
            int32_t c = ch[k];
            if (c >= 0) {
                if (c >= nn || c == 0 || depth[c] != -1) { why = "bad child index"; return false; }
                if (b.parent[c] != n) { why = "parent link"; return false; }
                depth[c] = depth[n] + 1;
                if (depth[c] > 62) { why = "hierarchy deeper than 62"; return false; }
                int32_t o = ch[1 - k];
                if (o >= 0 ? b.sibling[c] != o : b.sibling[c] != -1) { why = "sibling link"; return false; }
                stack.push_back(c);
            } else {
                int v = -c - 1, first = v >> 4, cnt = v & 15;
                if (first < 0 || first + cnt > nt) { why = "leaf range"; return false; }
                for (int i = first; i < first + cnt; ++i) {
                    int t = b.order[i];
                    if (t < 0 || t >= nt || seen[t]++) { why = "triangle order"; return false; }
                }
            }
        }
    }
    if (visited != nn) { why = "unreachable nodes"; return false; }
    for (int t = 0; t < nt; ++t)
        if (seen[t] != 1) { why = "triangle missing from leaves"; return false; }
    return true;
}

void read_counters(pb_ctx *ctx, pb_stats *st) {
    unsigned long long c[CNT_N];
    cudaMemcpy(c, ctx->B.counters, sizeof(c), cudaMemcpyDeviceToHost);
    st->n_entries = (int64_t)c[CNT_ENTRIES];
    st->n_truncated = (int64_t)c[CNT_TRUNC];
    st->n_nodes = (int64_t)c[CNT_NODES];
    st->n_conn = (int64_t)c[CNT_CONN];
    st->n_proxy = (int64_t)c[CNT_PROXY];
    st->n_proxy_ok = (int64_t)c[CNT_PROXY_OK];
    st->eye_nodes = (int64_t)c[CNT_EYE_NODES];
    st->eye_tris = (int64_t)c[CNT_EYE_TRIS];
    st->eye_rays = (int64_t)c[CNT_EYE_RAYS];
    st->rec_nodes = (int64_t)c[CNT_REC_NODES];
    st->rec_tris = (int64_t)c[CNT_REC_TRIS];
    st->rec_rays = (int64_t)c[CNT_REC_RAYS];
    st->cam_nodes = (int64_t)c[CNT_CAM_NODES];
    st->cam_tris = (int64_t)c[CNT_CAM_TRIS];
    st->cam_rays = (int64_t)c[CNT_CAM_RAYS];
    st->shd_nodes = (int64_t)c[CNT_SHD_NODES];
    st->shd_tris = (int64_t)c[CNT_SHD_TRIS];
    st->shd_rays = (int64_t)c[CNT_SHD_RAYS];
}

// ---- debug kernels --------------------------------------------------------
__global__ void k_trace(DScene S, const float *rays, int n, float *hits, int count, unsigned long long *counters) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *r = rays + 7 * (size_t)i;
    TravCount tc{0, 0, 0};
    Hit h = count ? closest_hit<true>(S, f3(r[0], r[1], r[2]), f3(r[3], r[4], r[5]), (int)r[6], &tc)
                  : closest_hit<false>(S, f3(r[0], r[1], r[2]), f3(r[3], r[4], r[5]), (int)r[6]);
    hits[4 * (size_t)i] = (float)h.tri;
    hits[4 * (size_t)i + 1] = h.tri >= 0 ? h.t : -1.0f;
    hits[4 * (size_t)i + 2] = h.b1;
    hits[4 * (size_t)i + 3] = h.b2;
    if (count) {
        atomicAdd(&counters[CNT_NFETCH], (unsigned long long)tc.nodes);
        atomicAdd(&counters[CNT_TTEST], (unsigned long long)tc.tris);
    }
}

__global__ void k_occ(DScene S, const float *seg, int n, int32_t *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *r = seg + 8 * (size_t)i;
    out[i] = occluded(S, f3(r[0], r[1], r[2]), f3(r[3], r[4], r[5]), (int)r[6], (int)r[7]) ? 1 : 0;
}

}  // namespace

pb_status pb_ensure_pool(pb_ctx *ctx, int slots, int ML, int repeats) { return ensure_pool(ctx, slots, ML, repeats, 0); }
pb_status pb_fail(pb_ctx *c, pb_status s, const std::string &m) { return fail(c, s, m); }
pb_status pb_run_wave(pb_ctx *ctx, const KParams &P, int slots, uint32_t iter_base, bool with_light, bool with_recip,
                      uint32_t *sig) {
    return run_wave(ctx, P, slots, iter_base, with_light, with_recip, sig);
}
KParams pb_kparams(const pb_ctx *ctx, const pb_config *c) { return kparams(ctx, c); }
pb_status pb_check_cfg(pb_ctx *ctx, const pb_config *c) { return check_cfg(ctx, c); }

void launch_trace(const DScene &S, const float *rays, int n, float *hits, int count, unsigned long long *counters,
                  cudaStream_t st) {
    k_trace<<<(n + 127) / 128, 128, 0, st>>>(S, rays, n, hits, count, counters);
}

void launch_occluded(const DScene &S, const float *seg, int n, int32_t *out, cudaStream_t st) {
    k_occ<<<(n + 127) / 128, 128, 0, st>>>(S, seg, n, out);
}

extern "C" {

pb_status pb_create(pb_ctx **out, int device, void *cuda_stream) {
    if (!out) return PB_ERR_ARG;
    *out = nullptr;
    pb_ctx *ctx = new pb_ctx();
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        delete ctx;
        return PB_ERR_CUDA;
    }
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return PB_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaEventCreate(&ctx->ev0);
    cudaEventCreate(&ctx->ev1);
    pb_noalloc_setup(ctx);
    *out = ctx;
    return PB_OK;
}

void pb_destroy(pb_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_all(ctx->scene_mem);
    free_all(ctx->table_mem);
    free_graphs(ctx);
    free_all(ctx->pool_mem);
    free_all(ctx->wf_mem);
    free_all(ctx->eye_mem);
    mlp_free(ctx);
    if (ctx->d_iter0) cudaFree(ctx->d_iter0);
    if (ctx->film) cudaFree(ctx->film);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *pb_last_error(const pb_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

pb_status pb_scene_upload(pb_ctx *ctx, const pb_scene_desc *d) {
    if (!ctx) return PB_ERR_ARG;
    if (!d || d->nv <= 0 || d->nt <= 0 || d->nm <= 0 || !d->verts || !d->tris || !d->tri_mat || !d->mats || !d->cam)
        return fail(ctx, PB_ERR_ARG, "scene: empty or missing arrays");
    for (int i = 0; i < 3 * d->nt; ++i)
        if (d->tris[i] < 0 || d->tris[i] >= d->nv) return fail(ctx, PB_ERR_ARG, "scene: vertex index out of range");
    for (int i = 0; i < d->nt; ++i)
        if (d->tri_mat[i] < 0 || d->tri_mat[i] >= d->nm) return fail(ctx, PB_ERR_ARG, "scene: material index out of range");
    int W = (int)d->cam[10], H = (int)d->cam[11];
    if (W <= 0 || H <= 0) return fail(ctx, PB_ERR_ARG, "scene: camera resolution must be positive");
    if (d->tex_w > 0 && (!d->tex || d->tex_h <= 0)) return fail(ctx, PB_ERR_ARG, "scene: texture size without data");
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    int nt = d->nt;
    PbBvh bvh;
    int nn = pb_bvh_build(d->verts, d->nv, d->tris, nt, &bvh);
    std::string why;
    if (!bvh_valid(bvh, nn, nt, why)) return fail(ctx, PB_ERR_STATE, "BVH build produced an invalid tree: " + why);
    // leaf-ordered intersection records and per-triangle shading records
    std::vector<float4> itri(3 * (size_t)nt), stri(4 * (size_t)nt);
    std::vector<float> uv(6 * (size_t)nt, 0.0f);
    std::vector<int> tri2e(nt, -1);
    std::vector<float> epw;
    std::vector<int> etri;
    double wsum = 0.0;
    float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
    for (int i = 0; i < d->nv; ++i)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], d->verts[3 * (size_t)i + a]);
            hi[a] = std::max(hi[a], d->verts[3 * (size_t)i + a]);
        }
    for (int t = 0; t < nt; ++t) {
        const float *p0 = d->verts + 3 * (size_t)d->tris[3 * (size_t)t];
        const float *p1 = d->verts + 3 * (size_t)d->tris[3 * (size_t)t + 1];
        const float *p2 = d->verts + 3 * (size_t)d->tris[3 * (size_t)t + 2];
        float e1[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
        float e2[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
        double cx = (double)e1[1] * e2[2] - (double)e1[2] * e2[1];
        double cy = (double)e1[2] * e2[0] - (double)e1[0] * e2[2];
        double cz = (double)e1[0] * e2[1] - (double)e1[1] * e2[0];
        double l = std::sqrt(cx * cx + cy * cy + cz * cz);
        float n[3] = {0, 0, 1};
        if (l > 0) {
            n[0] = (float)(cx / l);
            n[1] = (float)(cy / l);
            n[2] = (float)(cz / l);
        }
        const float *m = d->mats + 12 * (size_t)d->tri_mat[t];
        double le = (double)m[6] + m[7] + m[8];
        if (le > 0 && l > 0) {
            tri2e[t] = (int)etri.size();
            etri.push_back(t);
            double w = 0.5 * l * le;
            wsum += w;
            epw.push_back((float)w);
        }
        stri[4 * (size_t)t] = make_float4(p0[0], p0[1], p0[2], 0.0f);
        int mi = d->tri_mat[t];
        memcpy(&stri[4 * (size_t)t].w, &mi, 4);
        stri[4 * (size_t)t + 1] = make_float4(e1[0], e1[1], e1[2], 0.0f);
        stri[4 * (size_t)t + 2] = make_float4(e2[0], e2[1], e2[2], 0.0f);
        stri[4 * (size_t)t + 3] = make_float4(n[0], n[1], n[2], 0.0f);
        memcpy(&stri[4 * (size_t)t + 3].w, &tri2e[t], 4);
        if (d->uvs)
            for (int k = 0; k < 3; ++k) {
                uv[6 * (size_t)t + 2 * k] = d->uvs[2 * (size_t)d->tris[3 * (size_t)t + k]];
                uv[6 * (size_t)t + 2 * k + 1] = d->uvs[2 * (size_t)d->tris[3 * (size_t)t + k] + 1];
            }
    }
    for (size_t i = 0; i < bvh.order.size(); ++i) {
        int t = bvh.order[i];
        itri[3 * i] = stri[4 * (size_t)t];
        memcpy(&itri[3 * i].w, &t, 4);
        itri[3 * i + 1] = stri[4 * (size_t)t + 1];
        itri[3 * i + 2] = stri[4 * (size_t)t + 2];
    }
    // emitter selection: cumulative power share, last entry exactly 1
    int ne = (int)etri.size();
    std::vector<float> ecdf(std::max(ne, 1)), epmf(std::max(ne, 1));
    double acc = 0.0;
    for (int e = 0; e < ne; ++e) {
        acc += epw[e];
        ecdf[e] = (float)(acc / wsum);
        epmf[e] = (float)(epw[e] / wsum);
    }
    if (ne > 0) ecdf[ne - 1] = 1.0f;
    std::vector<DMat> mats(d->nm);
    for (int i = 0; i < d->nm; ++i) {
        const float *m = d->mats + 12 * (size_t)i;
        DMat M{};
        M.kind = (int)m[0];
        M.cr = m[1]; M.cg = m[2]; M.cb = m[3];
        M.alpha = m[4] * m[4];
        M.rough = m[4];
        M.ior = m[5];
        M.ler = m[6]; M.leg = m[7]; M.leb = m[8];
        M.textured = m[9] != 0.0f;
        M.specular = (M.kind != MK_LAMBERT) && (m[4] < 0.2f);
        M.emitter = ((double)m[6] + m[7] + m[8]) > 0.0;
        M.black = (M.kind == MK_LAMBERT) && !(std::max(m[1], std::max(m[2], m[3])) > 0.0f);
        if (M.kind < 0 || M.kind > 2) return fail(ctx, PB_ERR_ARG, "scene: unknown material kind");
        mats[i] = M;
    }
    DScene S{};
    auto &o = ctx->scene_mem;
    std::vector<int> etv(etri);
    if (etv.empty()) etv.push_back(0);
    const int tw = d->tex_w > 0 ? d->tex_w : 0, th = d->tex_w > 0 ? d->tex_h : 0;
    // A scene with the layout of the current one (same counts and resolution) is copied into the
    // current buffers: the pool, the film and the captured renders stay valid, and are freed only
    // if the scene's own parameters (camera, epsilon) changed. Any other scene replaces them all.
    const bool reuse = ctx->has_scene && ctx->S.nnodes == nn && ctx->S.nt == nt && ctx->S.ne == ne &&
                       ctx->scene_nm == d->nm && ctx->S.tw == tw && ctx->S.th == th && ctx->S.W == W &&
                       ctx->S.H == H;
    float4 *nodes, *it_, *st_;
    int *par, *sib, *etd;
    float *uvd, *texd = nullptr, *ecd, *epd;
    DMat *md;
    if (reuse) {
        const DScene &C = ctx->S;   // the context's own buffers (DScene holds them as const)
        nodes = const_cast<float4 *>(C.nodes);
        par = const_cast<int *>(C.parent);
        sib = const_cast<int *>(C.sibling);
        it_ = const_cast<float4 *>(C.itri);
        st_ = const_cast<float4 *>(C.stri);
        uvd = const_cast<float *>(C.uv);
        md = const_cast<DMat *>(C.mats);
        texd = const_cast<float *>(C.tex);
        ecd = const_cast<float *>(C.ecdf);
        epd = const_cast<float *>(C.epmf);
        etd = const_cast<int *>(C.etri);
        auto put = [&](void *dst, const void *src, size_t bytes) {
            return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream) : cudaSuccess;
        };
        CK(put(nodes, bvh.nodes.data(), 64 * (size_t)nn));
        CK(put(par, bvh.parent.data(), 4 * (size_t)nn));
        CK(put(sib, bvh.sibling.data(), 4 * (size_t)nn));
        CK(put(it_, itri.data(), sizeof(float4) * itri.size()));
        CK(put(st_, stri.data(), sizeof(float4) * stri.size()));
        CK(put(uvd, uv.data(), 4 * uv.size()));
        CK(put(md, mats.data(), sizeof(DMat) * mats.size()));
        if (tw > 0) CK(put(texd, d->tex, 12 * (size_t)tw * th));
        CK(put(ecd, ecdf.data(), 4 * ecdf.size()));
        CK(put(epd, epmf.data(), 4 * epmf.size()));
        CK(put(etd, etv.data(), 4 * etv.size()));
    } else {
        free_graphs(ctx);   // captured renders point into the buffers replaced here
        free_all(ctx->scene_mem);
        free_all(ctx->pool_mem);
        ctx->cap_slots = ctx->cap_ML = 0;
        ctx->Lbuf = nullptr;
        ctx->sigbuf = nullptr;
        ctx->has_scene = false;
        CK(upload(ctx, o, &nodes, reinterpret_cast<const float4 *>(bvh.nodes.data()), 4 * (size_t)nn));
        CK(upload(ctx, o, &par, bvh.parent.data(), (size_t)nn));
        CK(upload(ctx, o, &sib, bvh.sibling.data(), (size_t)nn));
        CK(upload(ctx, o, &it_, itri.data(), itri.size()));
        CK(upload(ctx, o, &st_, stri.data(), stri.size()));
        CK(upload(ctx, o, &uvd, uv.data(), uv.size()));
        CK(upload(ctx, o, &md, mats.data(), mats.size()));
        if (tw > 0) CK(upload(ctx, o, &texd, d->tex, 3 * (size_t)tw * th));
        CK(upload(ctx, o, &ecd, ecdf.data(), ecdf.size()));
        CK(upload(ctx, o, &epd, epmf.data(), epmf.size()));
        CK(upload(ctx, o, &etd, etv.data(), etv.size()));
    }
    S.nodes = nodes;
    S.parent = par;
    S.sibling = sib;
    S.itri = it_;
    S.stri = st_;
    S.uv = uvd;
    S.mats = md;
    S.tex = texd;
    S.ecdf = ecd;
    S.epmf = epd;
    S.etri = etd;
    S.nt = nt;
    S.nnodes = nn;
    S.ne = ne;
    S.tw = tw;
    S.th = th;
    S.W = W;
    S.H = H;
    float ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    ctx->scene_lo = make_float3(lo[0], lo[1], lo[2]);
    ctx->scene_hi = make_float3(hi[0], hi[1], hi[2]);
    S.eps_t = 1e-5f * ext;
    const float *c = d->cam;
    float3 pos = make_float3(c[0], c[1], c[2]);
    double fx = (double)c[3] - c[0], fy = (double)c[4] - c[1], fz = (double)c[5] - c[2];
    double fl = std::sqrt(fx * fx + fy * fy + fz * fz);
    fx /= fl; fy /= fl; fz /= fl;
    double rx = fy * c[8] - fz * c[7], ry = fz * c[6] - fx * c[8], rz = fx * c[7] - fy * c[6];
    double rl = std::sqrt(rx * rx + ry * ry + rz * rz);
    rx /= rl; ry /= rl; rz /= rl;
    double ux = ry * fz - rz * fy, uy = rz * fx - rx * fz, uz = rx * fy - ry * fx;
    S.cpos = pos;
    S.cfwd = make_float3((float)fx, (float)fy, (float)fz);
    S.cright = make_float3((float)rx, (float)ry, (float)rz);
    S.cup = make_float3((float)ux, (float)uy, (float)uz);
    S.tanh_ = (float)std::tan(0.5 * (double)c[9] * M_PI / 180.0);
    S.aspect = (float)W / (float)H;
    if (reuse) {
        // the feature box comes with the tables; keep the current one
        S.lo = ctx->S.lo;
        S.ext = ctx->S.ext;
        if (std::memcmp(&S, &ctx->S, sizeof(DScene)) != 0) free_graphs(ctx);
    } else {
        S.lo = make_float3(0, 0, 0);
        S.ext = make_float3(1, 1, 1);
    }
    ctx->S = S;
    ctx->scene_nm = d->nm;
    CK(cudaStreamSynchronize(ctx->stream));
    if (!reuse || !ctx->film) {
        if (ctx->film) cudaFree(ctx->film);
        ctx->film = nullptr;
        CK(cudaMalloc(&ctx->film, sizeof(float) * 3 * (size_t)W * H));
    }
    CK(cudaMemset(ctx->film, 0, sizeof(float) * 3 * (size_t)W * H));
    ctx->film_iters = 0;
    ctx->has_scene = true;
    return PB_OK;
}

pb_status pb_tables_upload(pb_ctx *ctx, const pb_tables_desc *t) {
    if (!ctx) return PB_ERR_ARG;
    if (!ctx->has_scene) return fail(ctx, PB_ERR_STATE, "upload the scene before the tables");
    if (!t || t->KT <= 0 || t->KS <= 0 || t->KSp <= 0 || t->KC <= 0 || t->KS > 1023 || t->KSp > 1023 ||
        t->KC > 1000 || t->tile <= 0 || !t->cent_T || !t->cent_S || !t->cent_Sp || !t->cent_C || !t->gamma_conn ||
        !t->gamma_proxy || !t->B_tab || !t->mis_tab || !t->pi_grid || !t->bbox_lo || !t->bbox_hi)
        return fail(ctx, PB_ERR_ARG, "tables: bad sizes or missing arrays (KS, KSp <= 1023)");
    int gw = (ctx->S.W + t->tile - 1) / t->tile, gh = (ctx->S.H + t->tile - 1) / t->tile;
    if (t->grid_w != gw || t->grid_h != gh) return fail(ctx, PB_ERR_ARG, "tables: grid size does not match W/H/tile");
    int ncell = 4 * t->KSp * (t->KC + 1);
    for (int i = 0; i < ncell; ++i)
        if (!(t->B_tab[i] > 0.0f)) return fail(ctx, PB_ERR_ARG, "tables: B must be positive");
    CK(cudaStreamSynchronize(ctx->stream));
    // tables of the current sizes are copied into the current buffers (captured renders stay valid
    // unless the feature box or the tile changed); other sizes replace them
    const DTables &C = ctx->T;
    const bool reuse = ctx->has_tables && C.KT == t->KT && C.KS == t->KS && C.KSp == t->KSp && C.KC == t->KC &&
                       C.gw == gw && C.gh == gh;
    DTables T{};
    T.KT = t->KT; T.KS = t->KS; T.KSp = t->KSp; T.KC = t->KC;
    if (reuse) {
        T = C;
        auto put = [&](const float *dst, const float *src, size_t n) {   // the context's own table buffers
            return cudaMemcpyAsync(const_cast<float *>(dst), src, 4 * n, cudaMemcpyHostToDevice, ctx->stream);
        };
        CK(put(T.cT, t->cent_T, (size_t)t->KT * 9));
        CK(put(T.cS, t->cent_S, (size_t)t->KS * 9));
        CK(put(T.cSp, t->cent_Sp, (size_t)t->KSp * 6));
        CK(put(T.cC, t->cent_C, (size_t)t->KC * 3));
        CK(put(T.gC, t->gamma_conn, (size_t)t->KT * t->KS));
        CK(put(T.gP, t->gamma_proxy, (size_t)t->KT * t->KSp));
        CK(put(T.Bt, t->B_tab, (size_t)ncell));
        CK(put(T.mis, t->mis_tab, (size_t)ncell));
        CK(put(T.pi, t->pi_grid, (size_t)gw * gh));
    } else {
        free_graphs(ctx);   // captured renders point into the buffers replaced here
        free_all(ctx->table_mem);
        auto &o = ctx->table_mem;
        float *p;
        CK(upload(ctx, o, &p, t->cent_T, (size_t)t->KT * 9)); T.cT = p;
        CK(upload(ctx, o, &p, t->cent_S, (size_t)t->KS * 9)); T.cS = p;
        CK(upload(ctx, o, &p, t->cent_Sp, (size_t)t->KSp * 6)); T.cSp = p;
        CK(upload(ctx, o, &p, t->cent_C, (size_t)t->KC * 3)); T.cC = p;
        CK(upload(ctx, o, &p, t->gamma_conn, (size_t)t->KT * t->KS)); T.gC = p;
        CK(upload(ctx, o, &p, t->gamma_proxy, (size_t)t->KT * t->KSp)); T.gP = p;
        CK(upload(ctx, o, &p, t->B_tab, (size_t)ncell)); T.Bt = p;
        CK(upload(ctx, o, &p, t->mis_tab, (size_t)ncell)); T.mis = p;
        CK(upload(ctx, o, &p, t->pi_grid, (size_t)gw * gh)); T.pi = p;
    }
    T.tile = t->tile;
    T.gw = gw;
    T.gh = gh;
    float3 lo = make_float3(t->bbox_lo[0], t->bbox_lo[1], t->bbox_lo[2]);
    float ex = t->bbox_hi[0] - t->bbox_lo[0], ey = t->bbox_hi[1] - t->bbox_lo[1], ez = t->bbox_hi[2] - t->bbox_lo[2];
    const float3 ext = make_float3(ex > 0 ? ex : 1.0f, ey > 0 ? ey : 1.0f, ez > 0 ? ez : 1.0f);
    if (reuse && (T.tile != C.tile || std::memcmp(&lo, &ctx->S.lo, sizeof(float3)) != 0 ||
                  std::memcmp(&ext, &ctx->S.ext, sizeof(float3)) != 0))
        free_graphs(ctx);
    ctx->T = T;
    ctx->S.lo = lo;
    ctx->S.ext = ext;
    // pool buffers that depend on the table sizes are re-checked by ensure_pool
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->has_tables = true;
    return PB_OK;
}

}  // extern "C"

pb_status pb_collect_wave(pb_ctx *ctx, const pb_config *cfg, int slots, uint32_t iter_base, const SampleSink &sink,
                          const SampleSink &sink_proxy) {
    KParams P = kparams(ctx, cfg);
    pb_status s = ensure_pool(ctx, slots, P.M * P.L, P.repeats, P.npix);
    if (s != PB_OK) return s;
    if (cfg->estimator == 0 && (s = wf_ensure(ctx)) != PB_OK) return s;
    launch_light_pass(ctx->S, P, ctx->B, slots, iter_base, ctx->stream);
    launch_pool_build(ctx->S, ctx->T, P, ctx->B, slots, ctx->stream);
    launch_recip(ctx->S, ctx->T, P, ctx->B, slots, iter_base, ctx->num_sms, ctx->stream, &ctx->wf);
    if (cfg->proposal) {
        s = mlp_wave(ctx, P, slots, iter_base);
        if (s != PB_OK) return s;
    }
    P.smp = sink;
    P.smpp = sink_proxy;
    s = pb_eye_stages(ctx, P, slots, iter_base, nullptr, ctx->stream);
    if (s != PB_OK) return s;
    if (cfg->proposal) return mlp_check_err(ctx);
    return PB_OK;
}

// ---- wavefront estimator buffers ------------------------------------------------
constexpr int WF_NODE_CAP = 1 << 25;   // nodes per round (about 4 GB of state): long chains rarely wait

pb_status wf_ensure(pb_ctx *ctx) {
    const int chains = ctx->B.chain_cap;
    if (ctx->wf_chain_cap >= chains && ctx->wf.node_cap == WF_NODE_CAP) return PB_OK;
    free_graphs(ctx);
    free_all(ctx->wf_mem);
    WfBufs &W = ctx->wf;
    W = WfBufs{};
    auto &o = ctx->wf_mem;
    const size_t nc = (size_t)std::max(chains, 1), nn = (size_t)WF_NODE_CAP;
    CK(dalloc(o, &W.ch_w, nc));
    CK(dalloc(o, &W.ch_off, nc));
    CK(dalloc(o, &W.ch_win, nc));
    CK(dalloc(o, &W.ch_done, nc));
    CK(dalloc(o, &W.node_chain, nn));
    CK(dalloc(o, &W.node_v, nn));
    CK(dalloc(o, &W.node_nq, nn));
    CK(dalloc(o, &W.node_res, 5 * nn));
    CK(dalloc(o, &W.node_q, nn));
    CK(dalloc(o, &W.node_g, nn));
    CK(dalloc(o, &W.node_n, nn));
    CK(dalloc(o, &W.node_x, nn));
    CK(dalloc(o, &W.node_u, nn));
    CK(dalloc(o, &W.list[0], nn));
    CK(dalloc(o, &W.list[1], nn));
    CK(dalloc(o, &W.ctl, (size_t)16));
    CK(dalloc(o, &W.pil_next, nc));
    CK(dalloc(o, &W.pil_best, nc));
    CK(dalloc(o, &W.pil_sum, nc));
    CK(dalloc(o, &W.pil_draws, nc));
    CK(cudaMemsetAsync(W.ctl, 0, 16 * sizeof(int32_t), ctx->stream));
    W.node_cap = WF_NODE_CAP;
    ctx->wf_chain_cap = chains;
    return PB_OK;
}

// errors of the last wavefront wave (ctl[3]: low byte = error code)
pb_status wf_check(pb_ctx *ctx) {
    if (!ctx->wf.ctl) return PB_OK;
    int32_t e = 0;
    CK(cudaMemcpyAsync(&e, ctx->wf.ctl + 3, sizeof(e), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (e & 0xFF) {
        CK(cudaMemsetAsync(ctx->wf.ctl + 3, 0, sizeof(e), ctx->stream));
        return fail(ctx, PB_ERR_STATE, (e & 0xFF) == 1 ? "wavefront estimator: more estimates in flight than chain slots"
                                                        : "wavefront estimator: a node asked for more queries than u allows");
    }
    return PB_OK;
}

// ---- camera-side wavefront of the eye pass -----------------------------------------
pb_status pb_eye_ensure(pb_ctx *ctx, int slots, int depth) {
    const size_t npix = (size_t)ctx->S.W * ctx->S.H;
    const size_t px = (size_t)slots * depth * npix;           // dense vertices
    const size_t nq = (size_t)slots * npix * (2 * depth + 1);   // at most NEE + connection per vertex, one proxy
    if (px * 4 + 3 > (size_t)INT32_MAX || nq > (size_t)INT32_MAX)
        return fail(ctx, PB_ERR_ARG, "eye pass: too many pixels x iterations in flight x depth");
    if (ctx->eye_cap_px >= px && ctx->eye_cap_q >= nq) return PB_OK;
    free_graphs(ctx);   // captured renders point into the buffers replaced here
    CK(cudaStreamSynchronize(ctx->stream));
    free_all(ctx->eye_mem);
    auto &o = ctx->eye_mem;
    CK(dalloc(o, &ctx->eye_hits, px));
    CK(dalloc(o, &ctx->eye_vis, 3 * px));
    CK(dalloc(o, &ctx->eye_qa, nq));
    CK(dalloc(o, &ctx->eye_qb, nq));
    CK(dalloc(o, &ctx->eye_dst, nq));
    CK(dalloc(o, &ctx->eye_count, (size_t)2));   // queries appended; queries taken by persistent warps
    ctx->eye_cap_px = px;
    ctx->eye_cap_q = nq;
    return PB_OK;
}

pb_status pb_eye_stages(pb_ctx *ctx, const KParams &P0, int slots, uint32_t iter_base, uint32_t *sig,
                        cudaStream_t st, const EyeEvents *ev) {
    pb_status s = pb_eye_ensure(ctx, slots, P0.max_depth);
    if (s != PB_OK) return s;
    KParams P = P0;
    if (!P.mlp.hits) {   // the table proposal: store the hits, no network rows
        P.mlp.hits = ctx->eye_hits;
        P.mlp.rows = nullptr;
        P.mlp.sel = nullptr;
        P.mlp.selq = nullptr;
        launch_eye_feat(ctx->S, ctx->T, P, ctx->B, slots, iter_base, st);
        if (ev && ev->feat_end) CK(cudaEventRecordWithFlags(ev->feat_end, st, ev->flags));
    }
    const size_t npix = (size_t)ctx->S.W * ctx->S.H;
    P.q = EyeQueries{ctx->eye_qa, ctx->eye_qb, ctx->eye_dst, ctx->eye_count,
                     (int)((size_t)slots * npix * (2 * P.max_depth + 1)), ctx->eye_vis,
                     (size_t)slots * P.max_depth * npix};
    CK(cudaMemsetAsync(ctx->eye_count, 0, sizeof(unsigned int), st));
    launch_eye(ctx->S, ctx->T, P, ctx->B, slots, iter_base, ctx->Lbuf, nullptr, st, EYE_EMIT);
    if (ev && ev->emit_end) CK(cudaEventRecordWithFlags(ev->emit_end, st, ev->flags));
    launch_eye_occ(ctx->S, P, ctx->B, ctx->num_sms, st, ctx->eye_count + 1);
    if (ev && ev->occ_end) CK(cudaEventRecordWithFlags(ev->occ_end, st, ev->flags));
    launch_eye(ctx->S, ctx->T, P, ctx->B, slots, iter_base, ctx->Lbuf, sig, st, EYE_READ);
    CK(cudaGetLastError());
    return PB_OK;
}

// ---- render: prepare, enqueue (eager or captured), finish ---------------------
// per wave: light | pool | estimator | proposal | eye | end, then the ends of
// the feature pass, the query pass and the occlusion answers
constexpr int NEV = 9;

static int render_slots(const pb_config *cfg, const KParams &P) {
    // iterations in flight: up to 32, and about 8M eye paths per wave, so that
    // even a 1024^2 image puts 8 iterations' estimates (thousands of chains)
    // in one estimator wavefront; the per-wave eye buffers (about 1.3 GB per
    // 1024^2 iteration) fit HBM with room to spare
    int slots = cfg->batch > 0 ? cfg->batch : std::max(1, std::min(32, (1 << 23) / std::max(1, P.npix)));
    return std::max(1, std::min(slots, std::max(1, cfg->spp)));
}

static pb_status prepare_render(pb_ctx *ctx, const pb_config *cfg, KParams &P, int &slots) {
    pb_status s = check_cfg(ctx, cfg);
    if (s != PB_OK) return s;
    CK(cudaSetDevice(ctx->device));
    P = kparams(ctx, cfg);
    slots = render_slots(cfg, P);
    s = ensure_pool(ctx, slots, P.M * P.L, P.repeats, P.npix);
    if (s != PB_OK) return s;
    if (cfg->proposal) {
        s = mlp_prepare(ctx, slots, P.max_depth, cfg->proposal);
        if (s != PB_OK) return s;
    }
    if (cfg->estimator == 0) {
        s = wf_ensure(ctx);
        if (s != PB_OK) return s;
    }
    s = pb_eye_ensure(ctx, slots, P.max_depth);
    if (s != PB_OK) return s;
    if (!ctx->d_iter0) CK(cudaMalloc(&ctx->d_iter0, sizeof(uint32_t)));
    return PB_OK;
}

// Enqueues the waves of a render on ctx->stream. Iteration numbers are
// iter_off + (iterations already enqueued), plus *P.iter_dev when set
// (graph replay). `ev` holds NEV events per wave; film == false leaves the
// film alone (autotuning trials).
static pb_status enqueue_render(pb_ctx *ctx, const pb_config *cfg, const KParams &P, int slots, uint32_t iter_off,
                                cudaEvent_t *ev, bool film, bool capturing = false) {
    cudaStream_t st = ctx->stream;
    // inside a capture the stage events become event-record nodes of the graph
    const unsigned int evf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    CK(cudaMemsetAsync(ctx->B.counters, 0, sizeof(unsigned long long) * CNT_N, st));
    int w = 0;
    for (int done = 0; done < cfg->spp; ++w) {
        int ns = std::min(slots, cfg->spp - done);
        uint32_t base = iter_off + (uint32_t)done;
        cudaEvent_t *e = ev + NEV * (size_t)w;
        CK(cudaEventRecordWithFlags(e[0], st, evf));
        launch_light_pass(ctx->S, P, ctx->B, ns, base, st);
        CK(cudaEventRecordWithFlags(e[1], st, evf));
        launch_pool_build(ctx->S, ctx->T, P, ctx->B, ns, st);
        CK(cudaEventRecordWithFlags(e[2], st, evf));
        launch_recip(ctx->S, ctx->T, P, ctx->B, ns, base, ctx->num_sms, st, &ctx->wf);
        CK(cudaEventRecordWithFlags(e[3], st, evf));
        KParams Pw = P;
        EyeEvents eev;
        eev.feat_end = e[6];
        eev.emit_end = e[7];
        eev.occ_end = e[8];
        eev.flags = evf;
        if (cfg->proposal) {
            pb_status s = mlp_wave(ctx, Pw, ns, base, &eev);
            if (s != PB_OK) return s;
        }
        CK(cudaEventRecordWithFlags(e[4], st, evf));
        pb_status s = pb_eye_stages(ctx, Pw, ns, base, nullptr, st, &eev);
        if (s != PB_OK) return s;
        CK(cudaEventRecordWithFlags(e[5], st, evf));
        if (film) launch_film_add(P, ns, ctx->Lbuf, ctx->film, st);
        CK(cudaGetLastError());
        done += ns;
    }
    return PB_OK;
}

static pb_status make_events(pb_ctx *ctx, std::vector<cudaEvent_t> &ev, size_t n) {
    ev.resize(n, nullptr);
    for (auto &e : ev)
        if (!e) CK(cudaEventCreate(&e));
    return PB_OK;
}

// stats of a finished render (the caller synchronised)
static pb_status finish_render(pb_ctx *ctx, const pb_config *cfg, const KParams &P, int slots,
                               const std::vector<cudaEvent_t> &ev, cudaEvent_t e0, cudaEvent_t e1, bool film,
                               pb_stats *stats) {
    CK(cudaGetLastError());
    int waves = (cfg->spp + slots - 1) / slots;
    if (film) ctx->film_iters += cfg->spp;
    pb_stats st{};
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    st.ms = ms;
    st.mpaths_per_s = ms > 0 ? (double)P.npix * cfg->spp / (ms * 1e-3) / 1e6 : 0.0;
    for (int i = 0; i < waves; ++i) {
        float a = 0, b = 0, c = 0, d = 0, m = 0;
        const cudaEvent_t *e = ev.data() + NEV * (size_t)i;
        cudaEventElapsedTime(&a, e[0], e[1]);
        cudaEventElapsedTime(&b, e[1], e[2]);
        cudaEventElapsedTime(&c, e[2], e[3]);
        cudaEventElapsedTime(&m, e[3], e[4]);
        cudaEventElapsedTime(&d, e[4], e[5]);
        st.ms_light += a;
        st.ms_pool += b;
        st.ms_recip += c;
        st.ms_mlp += m;
        st.ms_eye += d;
        float f = 0, oc = 0;
        cudaEventElapsedTime(&f, cfg->proposal ? e[3] : e[4], e[6]);   // the feature pass
        cudaEventElapsedTime(&oc, e[7], e[8]);                           // the occlusion answers
        st.ms_eye_feat += f;
        st.ms_eye_occ += oc;
    }
    st.n_waves = waves;
    // per wave: light, pool build, bucket, cdf, eye, film (6); the estimator:
    // warp/block phases = offsets, pilot, two phases, finish (5); wavefront =
    // offsets, pilot (init + rounds x (plan, nodes, steps, traces, reduce), or
    // one kernel without a pilot), init, rounds x (plan, nodes, steps, traces,
    // walk), finisher, finish; the learned proposal adds its feature pass and
    // network
    const int per_round = 3 + 2 * WF_MAXQ + 1;
    const int pr = wf_pilot_rounds(P);
    const int64_t est = cfg->estimator == 1 ? 5
                                            : 4 + (pr > 0 ? 1 + (int64_t)pr * per_round : 1) +
                                                  (int64_t)WF_ROUNDS * per_round;
    // the eye side: feature pass (the network's select kernel too with the
    // learned proposal), query pass, occlusion answers, shading pass
    st.n_launches = (5 + est + 3 + (cfg->proposal ? 2 : 1)) * (int64_t)waves;
    if (cfg->proposal) {
        pb_status s = mlp_check_err(ctx);
        if (s != PB_OK) return s;
    }
    if (cfg->estimator == 0) {
        pb_status s = wf_check(ctx);
        if (s != PB_OK) return s;
    }
    read_counters(ctx, &st);
    if (stats) *stats = st;
    if (st.n_truncated > 0) return fail(ctx, PB_ERR_TRUNCATED, "reciprocal estimate hit the trial cap");
    return PB_OK;
}

static bool same_graph_cfg(const pb_config &a, const pb_config &b) {
    pb_config x = a, y = b;
    x.iter0 = y.iter0 = 0;
    return std::memcmp(&x, &y, sizeof(pb_config)) == 0;
}

// the captured render of `cfg` (any iter0): one graph per configuration,
// iteration numbers offset by *ctx->d_iter0 at replay
static pb_status get_graph(pb_ctx *ctx, const pb_config *cfg, KParams P, int slots, RenderGraph **out) {
    for (RenderGraph *g : ctx->graphs)
        if (same_graph_cfg(g->cfg, *cfg)) {
            *out = g;
            return PB_OK;
        }
    RenderGraph *g = new RenderGraph();
    g->cfg = *cfg;
    g->slots = slots;
    int waves = (cfg->spp + slots - 1) / slots;
    pb_status s = make_events(ctx, g->ev, NEV * (size_t)std::max(waves, 1));
    if (s == PB_OK) s = make_events(ctx, g->ends, 2);
    if (s != PB_OK) {
        delete g;
        return s;
    }
    P.iter_dev = ctx->d_iter0;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    cudaEventRecordWithFlags(g->ends[0], ctx->stream, cudaEventRecordExternal);
    s = enqueue_render(ctx, cfg, P, slots, 0, g->ev.data(), true, true);
    cudaEventRecordWithFlags(g->ends[1], ctx->stream, cudaEventRecordExternal);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (s != PB_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        delete g;
        if (s != PB_OK) return s;
        return fail(ctx, PB_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    g->graph = graph;
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        delete g;
        return fail(ctx, PB_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    ctx->graphs.push_back(g);
    *out = g;
    return PB_OK;
}

void free_graphs(pb_ctx *ctx) {
    for (RenderGraph *g : ctx->graphs) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        for (auto e : g->ev) cudaEventDestroy(e);
        for (auto e : g->ends) cudaEventDestroy(e);
        delete g;
    }
    ctx->graphs.clear();
}

// ---- autotuning: iterations in flight x estimator hand-off per size bucket ----
struct TuneEntry {
    int batch, estimator;
    double ms_per_iter;
};
static std::mutex g_tune_mutex;
static std::map<std::string, TuneEntry> g_tune;

static std::string tune_key(const pb_ctx *ctx, const pb_config *cfg) {
    auto lg = [](long long v) {
        int b = 0;
        while ((1ll << (b + 1)) <= v) ++b;
        return b;
    };
    char buf[192];
    std::snprintf(buf, sizeof(buf), "tris2^%d|pix2^%d|depth%d|M%d|Mp%d|rep%d|prop%d|proxy%d", lg(ctx->S.nt),
                  lg((long long)ctx->S.W * ctx->S.H), cfg->max_depth, cfg->M, cfg->M_p, cfg->repeats, cfg->proposal,
                  cfg->proxy);
    std::string key(buf);
    if (cfg->booth > 0.0f) {   // Booth's roulette has one schedule and its own chain lengths
        std::snprintf(buf, sizeof(buf), "|booth%g", (double)cfg->booth);
        key += buf;
    }
    if (cfg->trace) key += "|trace1";
    if (cfg->fixed_bound) key += "|fixedB";   // longer chains where a bound sits below f/q / 2
    return key;
}

extern "C" {

pb_status pb_render(pb_ctx *ctx, const pb_config *cfg, pb_stats *stats) {
    if (!ctx) return PB_ERR_ARG;
    KParams P;
    int slots;
    pb_status s = prepare_render(ctx, cfg, P, slots);
    if (s != PB_OK) return s;
    if (cfg->graph) {
        RenderGraph *g;
        s = get_graph(ctx, cfg, P, slots, &g);
        if (s != PB_OK) return s;
        uint32_t it0 = (uint32_t)cfg->iter0;   // pageable source: staged before the call returns
        CK(cudaMemcpyAsync(ctx->d_iter0, &it0, sizeof(it0), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaGraphLaunch(g->exec, ctx->stream));
        CK(cudaEventSynchronize(g->ends[1]));
        CK(cudaStreamSynchronize(ctx->stream));
        return finish_render(ctx, cfg, P, slots, g->ev, g->ends[0], g->ends[1], true, stats);
    }
    int waves = (cfg->spp + slots - 1) / slots;
    std::vector<cudaEvent_t> ev;
    if ((s = make_events(ctx, ev, NEV * (size_t)std::max(waves, 1))) != PB_OK) return s;
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    s = enqueue_render(ctx, cfg, P, slots, (uint32_t)cfg->iter0, ev.data(), true);
    if (s == PB_OK) {
        CK(cudaEventRecord(ctx->ev1, ctx->stream));
        CK(cudaEventSynchronize(ctx->ev1));
        s = finish_render(ctx, cfg, P, slots, ev, ctx->ev0, ctx->ev1, true, stats);
    }
    for (auto &e : ev) cudaEventDestroy(e);
    return s;
}

pb_status pb_render_batch(pb_ctx *const *ctxs, const pb_config *cfgs, int n, pb_stats *stats) {
    if (!ctxs || !cfgs || n < 1) return PB_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return PB_ERR_ARG;
    pb_ctx *c0 = ctxs[0];
    for (int i = 0; i < n; ++i) {
        if (ctxs[i]->device != c0->device) return fail(c0, PB_ERR_ARG, "batch: contexts on different devices");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return fail(c0, PB_ERR_ARG, "batch: a context appears twice");
    }
    std::vector<KParams> Ps(n);
    std::vector<int> slots(n);
    std::vector<RenderGraph *> gs(n);
    for (int i = 0; i < n; ++i) {
        pb_config c = cfgs[i];
        c.graph = 1;
        pb_status s = prepare_render(ctxs[i], &c, Ps[i], slots[i]);
        if (s == PB_OK) s = get_graph(ctxs[i], &c, Ps[i], slots[i], &gs[i]);
        if (s != PB_OK) {
            if (ctxs[i] != c0) c0->err = "batch item " + std::to_string(i) + ": " + ctxs[i]->err;
            return s;
        }
    }
    // one graph: per scene, set its iteration base, then its render
    pb_ctx *ctx = c0;
    cudaGraph_t parent = nullptr;
    CK(cudaGraphCreate(&parent, 0));
    pb_status s = PB_OK;
    for (int i = 0; i < n && s == PB_OK; ++i) {
        cudaMemsetParams mp{};
        mp.dst = ctxs[i]->d_iter0;
        mp.value = (unsigned int)cfgs[i].iter0;
        mp.elementSize = 4;
        mp.width = 1;
        mp.height = 1;
        cudaGraphNode_t ms, child;
        cudaError_t e = cudaGraphAddMemsetNode(&ms, parent, nullptr, 0, &mp);
        if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&child, parent, &ms, 1, gs[i]->graph);
        if (e != cudaSuccess) s = fail(ctx, PB_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    if (s == PB_OK) {
        cudaError_t e = cudaGraphInstantiate(&exec, parent, 0);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev0, ctx->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev1, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) s = fail(ctx, PB_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    }
    if (exec) cudaGraphExecDestroy(exec);
    cudaGraphDestroy(parent);
    if (s != PB_OK) return s;
    pb_status worst = PB_OK;
    for (int i = 0; i < n; ++i) {
        pb_config c = cfgs[i];
        c.graph = 1;
        pb_status si = finish_render(ctxs[i], &c, Ps[i], slots[i], gs[i]->ev, gs[i]->ends[0], gs[i]->ends[1], true,
                                     stats ? &stats[i] : nullptr);
        if (si != PB_OK && si != PB_ERR_TRUNCATED) return si;
        if (si == PB_ERR_TRUNCATED) worst = si;
    }
    if (stats) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        stats[0].batch_ms = ms;
    }
    return worst;
}

pb_status pb_autotune(pb_ctx *ctx, const pb_config *cfg, int trial_iters, pb_config *best, int *from_cache) {
    if (!ctx) return PB_ERR_ARG;
    if (!cfg || !best) return fail(ctx, PB_ERR_ARG, "autotune: null config");
    pb_status s = check_cfg(ctx, cfg);
    if (s != PB_OK) return s;
    std::string key = tune_key(ctx, cfg);
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            *best = *cfg;
            best->batch = it->second.batch;
            best->estimator = it->second.estimator;
            if (from_cache) *from_cache = 1;
            return PB_OK;
        }
    }
    if (from_cache) *from_cache = 0;
    int n = trial_iters > 0 ? trial_iters : 32;
    const int batches[] = {4, 8, 16, 32};
    const int schedules[] = {0, 1};   // wavefront, warp/block phases (Booth's roulette: wavefront only)
    const int n_sched = cfg->booth > 0.0f ? 1 : 2;
    TuneEntry bestE{0, 0, 1e300};
    std::vector<cudaEvent_t> ev;
    bool warmed = false;
    for (int b : batches) {
        if (b > n) continue;
        for (int hi = 0; hi < n_sched; ++hi) {
            const int h = schedules[hi];
            pb_config c = *cfg;
            c.batch = b;
            c.estimator = h;
            c.spp = n;
            c.iter0 = (1 << 28) + 7919;   // iterations no render uses
            c.graph = 0;
            KParams P;
            int slots;
            if ((s = prepare_render(ctx, &c, P, slots)) != PB_OK) return s;
            int waves = (n + slots - 1) / slots;
            if ((s = make_events(ctx, ev, NEV * (size_t)waves)) != PB_OK) return s;
            for (int rep = warmed ? 0 : 1; rep >= 0; --rep) {   // the first trial runs twice (warm-up)
                CK(cudaEventRecord(ctx->ev0, ctx->stream));
                if ((s = enqueue_render(ctx, &c, P, slots, (uint32_t)c.iter0, ev.data(), false)) != PB_OK) return s;
                CK(cudaEventRecord(ctx->ev1, ctx->stream));
                CK(cudaEventSynchronize(ctx->ev1));
            }
            warmed = true;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
            if (cfg->proposal) {
                if ((s = mlp_check_err(ctx)) != PB_OK) return s;
            }
            double per = ms / n;
            if (per < bestE.ms_per_iter) bestE = TuneEntry{b, h, per};
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (bestE.batch == 0) return fail(ctx, PB_ERR_ARG, "autotune: no candidate fits trial_iters");
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune[key] = bestE;
    }
    *best = *cfg;
    best->batch = bestE.batch;
    best->estimator = bestE.estimator;
    return PB_OK;
}

pb_status pb_autotune_cache_save(const char *path) {
    if (!path) return PB_ERR_ARG;
    FILE *f = std::fopen(path, "w");
    if (!f) return PB_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    for (auto &kv : g_tune)
        std::fprintf(f, "%s %d %d %.9g\n", kv.first.c_str(), kv.second.batch, kv.second.estimator, kv.second.ms_per_iter);
    std::fclose(f);
    return PB_OK;
}

pb_status pb_autotune_cache_load(const char *path) {
    if (!path) return PB_ERR_ARG;
    FILE *f = std::fopen(path, "r");
    if (!f) return PB_ERR_ARG;
    char key[256];
    TuneEntry e;
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    while (std::fscanf(f, "%255s %d %d %lf", key, &e.batch, &e.estimator, &e.ms_per_iter) == 4)
        if (e.batch > 0 && e.batch <= 64 && (e.estimator == 0 || e.estimator == 1)) g_tune[key] = e;
    std::fclose(f);
    return PB_OK;
}

void pb_autotune_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    g_tune.clear();
}

pb_status pb_film_clear(pb_ctx *ctx) {
    if (!ctx) return PB_ERR_ARG;
    if (!ctx->has_scene) return fail(ctx, PB_ERR_STATE, "no scene");
    CK(cudaMemsetAsync(ctx->film, 0, sizeof(float) * 3 * (size_t)ctx->S.W * ctx->S.H, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->film_iters = 0;
    return PB_OK;
}

pb_status pb_film_readback(pb_ctx *ctx, float *host_rgb, size_t n) {
    if (!ctx) return PB_ERR_ARG;
    if (!ctx->has_scene) return fail(ctx, PB_ERR_STATE, "no scene");
    size_t need = 3 * (size_t)ctx->S.W * ctx->S.H;
    if (!host_rgb || n < need) return fail(ctx, PB_ERR_ARG, "film readback: buffer too small");
    CK(cudaMemcpyAsync(host_rgb, ctx->film, need * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->film_iters > 0) {
        float inv = 1.0f / (float)ctx->film_iters;
        for (size_t i = 0; i < need; ++i) host_rgb[i] *= inv;
    }
    return PB_OK;
}

pb_status pb_film_device(pb_ctx *ctx, float **dev_sum, int64_t *iterations) {
    if (!ctx || !dev_sum || !iterations) return PB_ERR_ARG;
    if (!ctx->has_scene) return fail(ctx, PB_ERR_STATE, "no scene");
    *dev_sum = ctx->film;
    *iterations = ctx->film_iters;
    return PB_OK;
}

pb_status pb_trace(pb_ctx *ctx, const float *host_rays, int n, float *host_hits) {
    if (!ctx) return PB_ERR_ARG;
    if (!ctx->has_scene) return fail(ctx, PB_ERR_STATE, "no scene");
    if (n < 0 || (n > 0 && (!host_rays || !host_hits))) return fail(ctx, PB_ERR_ARG, "trace: bad arguments");
    if (n == 0) return PB_OK;
    CK(cudaSetDevice(ctx->device));
    std::vector<void *> tmp;
    float *dr, *dh;
    unsigned long long *cnt;
    CK(upload(ctx, tmp, &dr, host_rays, 7 * (size_t)n));
    CK(dalloc(tmp, &dh, 4 * (size_t)n));
    CK(dalloc(tmp, &cnt, (size_t)CNT_N));
    launch_trace(ctx->S, dr, n, dh, 0, cnt, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(host_hits, dh, 16 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    free_all(tmp);
    return PB_OK;
}

pb_status pb_occluded(pb_ctx *ctx, const float *host_seg, int n, int32_t *host_out) {
    if (!ctx) return PB_ERR_ARG;
    if (!ctx->has_scene) return fail(ctx, PB_ERR_STATE, "no scene");
    if (n < 0 || (n > 0 && (!host_seg || !host_out))) return fail(ctx, PB_ERR_ARG, "occluded: bad arguments");
    if (n == 0) return PB_OK;
    CK(cudaSetDevice(ctx->device));
    std::vector<void *> tmp;
    float *ds;
    int32_t *dout;
    CK(upload(ctx, tmp, &ds, host_seg, 8 * (size_t)n));
    CK(dalloc(tmp, &dout, (size_t)n));
    launch_occluded(ctx->S, ds, n, dout, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(host_out, dout, 4 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    free_all(tmp);
    return PB_OK;
}

pb_status pb_light_pass(pb_ctx *ctx, const pb_config *cfg, int iteration, int32_t *host_tri, float *host_bary) {
    if (!ctx) return PB_ERR_ARG;
    pb_status s = check_cfg(ctx, cfg);
    if (s != PB_OK) return s;
    if (!host_tri || !host_bary) return fail(ctx, PB_ERR_ARG, "light pass: null output");
    CK(cudaSetDevice(ctx->device));
    KParams P = kparams(ctx, cfg);
    s = ensure_pool(ctx, std::max(1, ctx->cap_slots), P.M * P.L, std::max(P.repeats, ctx->cap_rep), P.npix);
    if (s != PB_OK) return s;
    launch_light_pass(ctx->S, P, ctx->B, 1, (uint32_t)iteration, ctx->stream);
    CK(cudaGetLastError());
    size_t n = (size_t)P.M * P.L;
    CK(cudaMemcpyAsync(host_tri, ctx->B.gtri, 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(host_bary, ctx->B.gbary, 8 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PB_OK;
}

pb_status pb_iteration(pb_ctx *ctx, const pb_config *cfg, int iteration, const int32_t *host_tri,
                       const float *host_bary, const double *host_rhat_override, float *host_pix_rgb,
                       uint32_t *host_pix_sig, int cap, int *n_entries, float *host_entry_rhat,
                       uint32_t *host_entry_sig, float *host_entry_nodes, pb_stats *stats) {
    if (!ctx) return PB_ERR_ARG;
    pb_status s = check_cfg(ctx, cfg);
    if (s != PB_OK) return s;
    if (!host_tri || !host_bary) return fail(ctx, PB_ERR_ARG, "iteration: null geometry");
    CK(cudaSetDevice(ctx->device));
    KParams P = kparams(ctx, cfg);
    for (size_t i = 0; i < (size_t)P.M * P.L; ++i)
        if (host_tri[i] < -1 || host_tri[i] >= ctx->S.nt) return fail(ctx, PB_ERR_ARG, "iteration: triangle index out of range");
    s = ensure_pool(ctx, std::max(1, ctx->cap_slots), P.M * P.L, std::max(P.repeats, ctx->cap_rep), P.npix);
    if (s != PB_OK) return s;
    if (cfg->estimator == 0 && (s = wf_ensure(ctx)) != PB_OK) return s;
    size_t n = (size_t)P.M * P.L;
    CK(cudaMemsetAsync(ctx->B.counters, 0, sizeof(unsigned long long) * CNT_N, ctx->stream));
    CK(cudaMemcpyAsync(ctx->B.gtri, host_tri, 4 * n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->B.gbary, host_bary, 8 * n, cudaMemcpyHostToDevice, ctx->stream));
    launch_pool_build(ctx->S, ctx->T, P, ctx->B, 1, ctx->stream);
    int ne = 0;
    CK(cudaMemcpyAsync(&ne, ctx->B.nent, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (host_rhat_override) {
        std::vector<float> r(std::max(ne, 1));
        for (int i = 0; i < ne; ++i) r[i] = (float)host_rhat_override[i];
        CK(cudaMemcpyAsync(ctx->B.rhat, r.data(), 4 * (size_t)ne, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    } else {
        launch_recip(ctx->S, ctx->T, P, ctx->B, 1, (uint32_t)iteration, ctx->num_sms, ctx->stream, &ctx->wf);
    }
    if (cfg->proposal) {
        s = mlp_wave(ctx, P, 1, (uint32_t)iteration);
        if (s != PB_OK) return s;
    }
    {
        pb_status se = pb_eye_stages(ctx, P, 1, (uint32_t)iteration, ctx->sigbuf, ctx->stream);
        if (se != PB_OK) return se;
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    if (cfg->proposal) {
        s = mlp_check_err(ctx);
        if (s != PB_OK) return s;
    }
    if (n_entries) *n_entries = ne;
    int k = std::min(ne, std::max(cap, 0));
    if (host_pix_rgb) {
        std::vector<float4> Lh(P.npix);
        CK(cudaMemcpy(Lh.data(), ctx->Lbuf, sizeof(float4) * P.npix, cudaMemcpyDeviceToHost));
        for (int i = 0; i < P.npix; ++i) {
            host_pix_rgb[3 * (size_t)i] = Lh[i].x;
            host_pix_rgb[3 * (size_t)i + 1] = Lh[i].y;
            host_pix_rgb[3 * (size_t)i + 2] = Lh[i].z;
        }
    }
    if (host_pix_sig) CK(cudaMemcpy(host_pix_sig, ctx->sigbuf, 4 * (size_t)P.npix, cudaMemcpyDeviceToHost));
    if (k > 0 && host_entry_rhat) CK(cudaMemcpy(host_entry_rhat, ctx->B.rhat, 4 * (size_t)k, cudaMemcpyDeviceToHost));
    if (k > 0 && host_entry_sig && !host_rhat_override)
        CK(cudaMemcpy(host_entry_sig, ctx->B.esig, 4 * (size_t)k, cudaMemcpyDeviceToHost));
    if (k > 0 && host_entry_nodes && !host_rhat_override) {
        std::vector<float> rn((size_t)k * P.repeats);
        CK(cudaMemcpy(rn.data(), ctx->B.repn, 4 * rn.size(), cudaMemcpyDeviceToHost));
        for (int i = 0; i < k; ++i) {
            float a = 0;
            for (int r = 0; r < P.repeats; ++r) a += rn[(size_t)i * P.repeats + r];
            host_entry_nodes[i] = a;
        }
    }
    pb_stats st{};
    read_counters(ctx, &st);
    if (stats) *stats = st;
    return PB_OK;
}

}  // extern "C"
