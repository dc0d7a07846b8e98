// Supporting distribution q of an incomplete light sub-path (Sec. 5.3) and
// the integrand f = p(g | h_c, w_c) p(y_{s-1} | g, h_c) (Sec. 5.2, Eq.
// reciprocalFinal), shared by the estimator and the table-learning kernels.
#pragma once
#include "pb_device.cuh"

__device__ __forceinline__ float3 fwd_cos_over_d2(float3 a, float3 b, float3 nb, float3 &w, float &d2) {
    float3 d = b - a;
    d2 = len2(d);
    w = d * (1.0f / sqrtf(d2));
    return f3(fabsf(dot(nb, w)), 0, 0);
}

// light-tracer area density of ys[j] (Eq. tracingPdf)
__device__ __forceinline__ float fwd_density(const DScene &S, const Vtx *ys, int j) {
    if (j == 0) return light_pdf(S, ys[0].tri);
    float3 d = ys[j].p - ys[j - 1].p;
    float d2 = len2(d);
    float3 w = d * (1.0f / sqrtf(d2));
    float cn = fabsf(dot(ys[j].n, w));
    if (j == 1) {
        float c0 = dot(ys[0].n, w);
        if (c0 <= 0.0f) return 0.0f;
        return (c0 / PB_PI) * cn / d2;
    }
    const DMat &m = S.mats[ys[j - 1].mat];
    return bsdf_pdf(m, ys[j - 1].n, dirto(ys[j - 1].p, ys[j - 2].p), w) * cn / d2;
}

// ---------------------------------------------------------------------------
// Supporting distribution of an incomplete sub-path (Sec. 5.3) and the
// integrand f = p(g | h_c, w_c) p(y_{s-1} | g, h_c) (Sec. 5.2).
struct Entry {
    Vtx Y, H;
    int u, type;
    int back;     // y_{s-2} lies behind Y's normal
    float pin;    // share of the cosine draws at a dielectric Y on the side of y_{s-2}
};

// cosine density at Y: conductors use their front hemisphere, dielectrics
// both, the side of y_{s-2} with probability pin
__device__ __forceinline__ float cosY_pdf(const DScene &S, const Vtx &Y, float3 w, int back, float pin) {
    const DMat &m = S.mats[Y.mat];
    float c = dot(Y.n, w);
    if (m.kind == MK_DIELECTRIC) return (((c < 0.0f) == (back != 0)) ? pin : 1.0f - pin) * fabsf(c) / PB_PI;
    return c > 0.0f ? c / PB_PI : 0.0f;
}

__device__ __forceinline__ float q_from_Y(const DScene &S, const Vtx *gs, int u, int back, float pin) {
    float3 d = gs[1].p - gs[0].p;
    float d2 = len2(d);
    float3 w = d * (1.0f / sqrtf(d2));
    float q = cosY_pdf(S, gs[0], w, back, pin) * fabsf(dot(gs[1].n, w)) / d2;
    for (int r = 1; r < u; ++r) {
        const DMat &m = S.mats[gs[r].mat];
        float3 dd = gs[r + 1].p - gs[r].p;
        float dd2 = len2(dd);
        float3 ww = dd * (1.0f / sqrtf(dd2));
        q *= bsdf_pdf(m, gs[r].n, dirto(gs[r].p, gs[r - 1].p), ww) * fabsf(dot(gs[r + 1].n, ww)) / dd2;
    }
    return q;
}

__device__ __forceinline__ void eval_fq(const DScene &S, const Entry &E, const Vtx *gs, bool compA, bool vis, float &f, float &q) {
    int u = E.u;
    Vtx ys[8];
    int n = 0;
    if (E.type == 1) ys[n++] = E.H;
    for (int r = u; r >= 1; --r) ys[n++] = gs[r];
    ys[n++] = E.Y;
    bool ok = vis;
    for (int j = 1; j < n && ok; ++j) {
        const DMat &m = S.mats[ys[j].mat];
        int want = (j == n - 1) ? 1 : ((E.type == 1 && j == 1) ? 0 : 1);
        if (m.specular != want) ok = false;
        if (absorbing(S, ys[j], dirto(ys[j].p, ys[j - 1].p))) ok = false;
    }
    if (E.type == 0 && !S.mats[ys[0].mat].emitter) ok = false;
    float fv = 0.0f;
    if (ok) {
        fv = 1.0f;
        for (int j = (E.type == 1 ? 1 : 0); j < n; ++j) fv *= fwd_density(S, ys, j);
    }
    float qB = (vis || !compA) ? q_from_Y(S, gs, u, E.back, E.pin) : 0.0f;
    float qv = qB;
    if (u == 1) {
        float qA;
        if (E.type == 0) {
            qA = light_pdf(S, gs[1].tri);
        } else {
            float3 d = gs[1].p - E.H.p;
            float d2 = len2(d);
            float3 w = d * (1.0f / sqrtf(d2));
            float c0 = dot(E.H.n, w);
            bool visHA = compA ? true : vis;
            qA = (c0 > 0.0f && visHA) ? (c0 / PB_PI) * fabsf(dot(gs[1].n, w)) / d2 : 0.0f;
        }
        qv = 0.5f * qA + 0.5f * qB;
    }
    f = fv;
    q = qv;
}

// closest hit as a vertex; `to_emitter` marks a segment that only counts if it
// ends on an emitter (then the emitter-first query is used when it is cheaper)
template <bool COUNT>
__device__ __forceinline__ bool trace_vtx(const DScene &S, float3 o, float3 w, int skip, Vtx &out, TravCount *tc,
                                          bool to_emitter = false) {
    Hit h = (to_emitter && S.ne <= PB_EMITTER_LIST_MAX) ? closest_emitter_hit<COUNT>(S, o, w, skip, tc)
                                                         : closest_hit<COUNT>(S, o, w, skip, tc);
    if (h.tri < 0) return false;
    out = vertex_at(S, h.tri, h.b1, h.b2);
    return true;
}

// Tracer policies of entry_ratio. The inline tracer walks the BVH at once.
// The replay tracer answers a node's first queries from stored results and
// suspends at the next one, recording it for a traversal kernel (wavefront
// evaluation); replaying the same uniforms and results reaches the same
// decisions, so both give the same f/q.
template <bool COUNT>
struct InlineTracer {
    TravCount *tc;
    static constexpr bool can_suspend = false;
    __device__ __forceinline__ bool suspended() const { return false; }
    __device__ __forceinline__ bool closest(const DScene &S, float3 o, float3 w, int skip, bool to_emitter, Vtx &out) {
        return trace_vtx<COUNT>(S, o, w, skip, out, tc, to_emitter);
    }
    __device__ __forceinline__ bool occluded_seg(const DScene &S, float3 a, float3 b, int s1, int s2) {
        return occluded<COUNT>(S, a, b, s1, s2, tc);
    }
};

struct ReplayTracer {
    const WfResult *res;
    int nres;
    int next;
    bool susp;
    WfQuery q;
    static constexpr bool can_suspend = true;
    __device__ __forceinline__ bool suspended() const { return susp; }
    __device__ __forceinline__ bool closest(const DScene &S, float3 o, float3 w, int skip, bool to_emitter, Vtx &out) {
        if (next < nres) {
            WfResult r = res[next++];
            if (r.tri < 0) return false;
            out = vertex_at(S, r.tri, r.b1, r.b2);
            return true;
        }
        q.o = o;
        q.d = w;
        q.skip = skip;
        q.skip2 = -1;
        q.kind = to_emitter ? 1 : 0;
        susp = true;
        return false;
    }
    __device__ __forceinline__ bool occluded_seg(const DScene &S, float3 a, float3 b, int s1, int s2) {
        if (next < nres) return res[next++].tri != 0;
        q.o = a;
        q.d = b;
        q.skip = s1;
        q.skip2 = s2;
        q.kind = 2;
        susp = true;
        return true;
    }
};

// one draw from q; returns f/q (0 also when the tracer suspended). Dims:
// 0 component, 1-3 light sample, 4-5 cosine direction, 6+3(r-1) BSDF at the
// r-th specular vertex, 18 RRS uniform, 19 hemisphere side.
template <bool COUNT, class Tr>
__device__ __forceinline__ float entry_ratio_t(const DScene &S, const Entry &E, Rng &R, Tr &T) {
    int u = E.u;
    Vtx gs[6];
    gs[0] = E.Y;
    bool compA = (u == 1) && (R.u(0) < 0.5f);
    float f, q;
    if (compA && E.type == 0) {
        int tri;
        float b1, b2;
        if (!sample_light(S, R.u(1), R.u(2), R.u(3), tri, b1, b2)) return 0.0f;
        gs[1] = vertex_at(S, tri, b1, b2);
        bool occ = T.occluded_seg(S, gs[1].p, E.Y.p, gs[1].tri, E.Y.tri);
        if (Tr::can_suspend && T.suspended()) return 0.0f;
        eval_fq(S, E, gs, true, !occ, f, q);
        return q > 0.0f ? f / q : 0.0f;
    }
    if (compA && E.type == 1) {
        float3 w = cosine_dir(E.H.n, R.u(4), R.u(5));
        bool hit = T.closest(S, E.H.p, w, E.H.tri, false, gs[1]);
        if ((Tr::can_suspend && T.suspended()) || !hit) return 0.0f;
        bool occ = T.occluded_seg(S, gs[1].p, E.Y.p, gs[1].tri, E.Y.tri);
        if (Tr::can_suspend && T.suspended()) return 0.0f;
        eval_fq(S, E, gs, true, !occ, f, q);
        return q > 0.0f ? f / q : 0.0f;
    }
    const DMat &mY = S.mats[E.Y.mat];
    float3 nside = E.Y.n;
    if (mY.kind == MK_DIELECTRIC) {
        float3 nin = E.back ? -E.Y.n : E.Y.n;   // toward y_{s-2}
        nside = R.u(19) < E.pin ? nin : -nin;
    }
    float3 w = cosine_dir(nside, R.u(4), R.u(5));
    bool hit = T.closest(S, E.Y.p, w, E.Y.tri, E.type == 0 && u == 1, gs[1]);
    if ((Tr::can_suspend && T.suspended()) || !hit) return 0.0f;
    for (int r = 1; r < u; ++r) {
        const DMat &m = S.mats[gs[r].mat];
        float3 wg = dirto(gs[r].p, gs[r - 1].p);
        if (!m.specular || absorbing(S, gs[r], wg)) return 0.0f;
        float3 ws;
        int d0 = 6 + 3 * (r - 1);
        if (!bsdf_sample(m, gs[r].n, wg, R.u(d0), R.u(d0 + 1), R.u(d0 + 2), ws)) return 0.0f;
        hit = T.closest(S, gs[r].p, ws, gs[r].tri, E.type == 0 && r + 1 == u, gs[r + 1]);
        if ((Tr::can_suspend && T.suspended()) || !hit) return 0.0f;
    }
    bool vis = true;
    if (E.type == 1) {
        bool occ = T.occluded_seg(S, gs[u].p, E.H.p, gs[u].tri, E.H.tri);
        if (Tr::can_suspend && T.suspended()) return 0.0f;
        vis = !occ;
    }
    eval_fq(S, E, gs, false, vis, f, q);
    return q > 0.0f ? f / q : 0.0f;
}

template <bool COUNT = false>
__device__ __forceinline__ float entry_ratio(const DScene &S, const Entry &E, Rng &R, TravCount *tc = nullptr) {
    InlineTracer<COUNT> T{tc};
    return entry_ratio_t<COUNT>(S, E, R, T);
}
