// Device-side building blocks of the proxy-tracing BDPT renderer (sm_103a).
//
// Everything a kernel needs per ray or per vertex: the counter-based
// random stream, scene access, materials, emitters, camera and the
// stackless BVH traversal. FP32 throughout; the GGX terms use |n x h|^2
// for sin^2 so narrow lobes (alpha ~ 1e-2..1e-4) keep full relative
// precision.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#ifndef PB_PI
#define PB_PI 3.14159265358979323846f
#endif

// ---------------------------------------------------------------------------
// float3 helpers
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 mul(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float len2(float3 a) { return dot(a, a); }
__device__ __forceinline__ float3 normalize(float3 a) { return a * (1.0f / sqrtf(dot(a, a))); }
__device__ __forceinline__ float maxc(float3 a) { return fmaxf(a.x, fmaxf(a.y, a.z)); }
__device__ __forceinline__ float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 dirto(float3 a, float3 b) { return normalize(b - a); }

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon et al., SC'11): counter (a, b, c, d>>2), key (seed, kind).
enum : uint32_t { K_CAMERA = 1, K_LIGHT = 2, K_RECIP = 3, K_TRAIN = 4, K_PILOT = 6 };

__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ float u24(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// A stream position (seed, kind, a, b, c); dims d are read in blocks of four.
struct Rng {
    uint32_t seed, kind, a, b, c;
    int blk;
    uint4 v;
    __device__ void init(uint32_t seed_, uint32_t kind_, uint32_t a_, uint32_t b_, uint32_t c_) {
        seed = seed_; kind = kind_; a = a_; b = b_; c = c_;
        blk = -1;
    }
    __device__ float u(int d) {
        int bk = d >> 2;
        if (bk != blk) {
            v = philox(make_uint4(a, b, c, (uint32_t)bk), seed, kind);
            blk = bk;
        }
        int w = d & 3;
        uint32_t x = w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
        return u24(x);
    }
};

// ---------------------------------------------------------------------------
// Scene, materials, tables
enum { MK_LAMBERT = 0, MK_CONDUCTOR = 1, MK_DIELECTRIC = 2 };

struct DMat {
    int kind;
    float cr, cg, cb;
    float alpha, ior;
    float ler, leg, leb;
    int textured, specular, emitter, black;
    float rough;             // roughness (alpha = rough^2)
    float pad[2];
};

struct DScene {
    const float4 *nodes;     // 4 per node
    const int *parent;
    const int *sibling;
    const float4 *itri;      // 3 per leaf-ordered triangle: v0 (w: original id), e1, e2
    const float4 *stri;      // 4 per triangle: v0 (w: material), e1, e2, n (w: emitter slot or -1)
    const float *uv;         // 6 per triangle
    const DMat *mats;
    const float *tex;
    const float *ecdf;       // per emitter slot
    const float *epmf;
    const int *etri;
    int nt, nnodes, ne, tw, th, W, H;
    float eps_t;
    float3 cpos, cfwd, cright, cup;
    float tanh_, aspect;
    float3 lo, ext;          // feature normalisation box (tables)
};

struct DTables {
    int KT, KS, KSp, KC;
    const float *cT, *cS, *cSp, *cC;
    const float *gC, *gP;    // selection matrices
    const float *Bt, *mis;
    const float *pi;
    int tile, gw, gh;
};

struct Vtx {
    float3 p, n;
    int tri, mat;
    float b1, b2;
};

__device__ __forceinline__ Vtx vertex_at(const DScene &S, int tri, float b1, float b2) {
    const float4 *t = S.stri + 4 * (size_t)tri;
    float4 v0 = t[0], e1 = t[1], e2 = t[2], nn = t[3];
    Vtx v;
    v.p = xyz(v0) + xyz(e1) * b1 + xyz(e2) * b2;
    v.n = xyz(nn);
    v.tri = tri;
    v.mat = __float_as_int(v0.w);
    v.b1 = b1;
    v.b2 = b2;
    return v;
}

__device__ __forceinline__ const DMat &mat_of(const DScene &S, int m) { return S.mats[m]; }

// black Lambert, or a conductor seen from its back: ends a sub-path
__device__ __forceinline__ bool absorbing(const DScene &S, const Vtx &v, float3 w_in) {
    const DMat &m = S.mats[v.mat];
    if (m.kind == MK_LAMBERT) return m.black;
    if (m.kind == MK_CONDUCTOR) return dot(v.n, w_in) <= 0.0f;
    return false;
}

// ---------------------------------------------------------------------------
// Orthonormal basis (Duff et al., JCGT 2017) and cosine sampling
__device__ __forceinline__ void onb(float3 n, float3 &t, float3 &b) {
    float sign = copysignf(1.0f, n.z);
    float a = -1.0f / (sign + n.z);
    float bb = n.x * n.y * a;
    t = f3(1.0f + sign * n.x * n.x * a, sign * bb, -sign * n.x);
    b = f3(bb, sign + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ float3 cosine_dir(float3 n, float u1, float u2) {
    float r = sqrtf(u1), ph = 2.0f * PB_PI * u2;
    float s, c;
    sincosf(ph, &s, &c);
    float z = sqrtf(fmaxf(0.0f, 1.0f - u1));
    float3 t, b;
    onb(n, t, b);
    return t * (r * c) + b * (r * s) + n * z;
}

// ---------------------------------------------------------------------------
// Materials (GGX after Walter et al., EGSR 2007). rho(w_light -> w_eye) is
// the radiance BSDF; pdf(w_g, w_s) the density of sampling w_s given w_g.
__device__ __forceinline__ float ggx_D(float a2, float3 n, float3 h) {
    float c = dot(n, h);
    if (c <= 0.0f) return 0.0f;
    float s2 = len2(cross(n, h));
    float den = c * c * a2 + s2;
    return a2 / (PB_PI * den * den);
}

__device__ __forceinline__ float ggx_G1(float a2, float3 n, float3 v, float3 h) {
    float vn = dot(v, n), vh = dot(v, h);
    if (vh * vn <= 0.0f) return 0.0f;
    float t2 = len2(cross(n, v)) / (vn * vn);
    return 2.0f / (1.0f + sqrtf(1.0f + a2 * t2));
}

__device__ __forceinline__ float3 ggx_sample_h(float a2, float3 n, float u1, float u2) {
    float t = 1.0f + (a2 - 1.0f) * u1;
    float c = sqrtf((1.0f - u1) / t);
    float sn = sqrtf(a2 * u1 / t);
    float s, co;
    sincosf(2.0f * PB_PI * u2, &s, &co);
    float3 tt, bb;
    onb(n, tt, bb);
    return tt * (sn * co) + bb * (sn * s) + n * c;
}

__device__ __forceinline__ float fresnel_dielectric(float cos_i, float eta_i, float eta_t) {
    cos_i = fabsf(cos_i);
    float r = eta_i / eta_t;
    float s2 = r * r * (1.0f - cos_i * cos_i);
    if (s2 >= 1.0f) return 1.0f;
    float cos_t = sqrtf(1.0f - s2);
    float rs = (eta_i * cos_i - eta_t * cos_t) / (eta_i * cos_i + eta_t * cos_t);
    float rp = (eta_t * cos_i - eta_i * cos_t) / (eta_t * cos_i + eta_i * cos_t);
    return 0.5f * (rs * rs + rp * rp);
}

#ifdef PB_BSDF_NOINLINE
#define PB_BSDF_FN static __noinline__
#else
#define PB_BSDF_FN __forceinline__
#endif

__device__ PB_BSDF_FN float3 bsdf_eval(const DMat &m, float3 n, float3 wl, float3 we) {
    float cl = dot(n, wl), ce = dot(n, we);
    if (m.kind == MK_LAMBERT) {
        if (cl * ce <= 0.0f) return f3(0, 0, 0);
        return f3(m.cr, m.cg, m.cb) * (1.0f / PB_PI);
    }
    float a2 = m.alpha * m.alpha;
    if (m.kind == MK_CONDUCTOR) {
        if (cl <= 0.0f || ce <= 0.0f) return f3(0, 0, 0);
        float3 h = normalize(wl + we);
        float D = ggx_D(a2, n, h);
        float G = ggx_G1(a2, n, wl, h) * ggx_G1(a2, n, we, h);
        float x = 1.0f - fmaxf(0.0f, dot(we, h));
        float s = x * x * x * x * x;
        float k = D * G / (4.0f * cl * ce);
        return f3((m.cr + (1.0f - m.cr) * s) * k, (m.cg + (1.0f - m.cg) * s) * k, (m.cb + (1.0f - m.cb) * s) * k);
    }
    if (cl == 0.0f || ce == 0.0f) return f3(0, 0, 0);
    float eta_l = cl > 0.0f ? 1.0f : m.ior, eta_e = ce > 0.0f ? 1.0f : m.ior;
    if (cl * ce > 0.0f) {
        float3 h = normalize(wl + we);
        if (dot(n, h) < 0.0f) h = -h;
        float D = ggx_D(a2, n, h);
        float G = ggx_G1(a2, n, wl, h) * ggx_G1(a2, n, we, h);
        float F = fresnel_dielectric(dot(wl, h), eta_l, eta_l == 1.0f ? m.ior : 1.0f);
        float f = F * D * G / (4.0f * fabsf(cl) * fabsf(ce));
        return f3(f, f, f);
    }
    float3 hv = -(wl * eta_l + we * eta_e);
    float hl = sqrtf(len2(hv));
    if (hl == 0.0f) return f3(0, 0, 0);
    float3 h = hv * (1.0f / hl);
    if (dot(n, h) < 0.0f) h = -h;
    float lh = dot(wl, h), eh = dot(we, h);
    float den = eta_l * lh + eta_e * eh;
    if (den == 0.0f) return f3(0, 0, 0);
    float D = ggx_D(a2, n, h);
    float G = ggx_G1(a2, n, wl, h) * ggx_G1(a2, n, we, h);
    float F = fresnel_dielectric(lh, eta_l, eta_e);
    float f = fabsf(lh) * fabsf(eh) * eta_e * eta_e * (1.0f - F) * D * G / (fabsf(cl) * fabsf(ce) * den * den);
    return f3(f, f, f);
}

__device__ PB_BSDF_FN float bsdf_pdf(const DMat &m, float3 n, float3 wg, float3 ws) {
    float cg = dot(n, wg), cs = dot(n, ws);
    if (m.kind == MK_LAMBERT) {
        if (cg * cs <= 0.0f) return 0.0f;
        return fabsf(cs) / PB_PI;
    }
    float a2 = m.alpha * m.alpha;
    if (m.kind == MK_CONDUCTOR) {
        if (cg <= 0.0f || cs <= 0.0f) return 0.0f;
        float3 h = normalize(wg + ws);
        float sh = dot(ws, h);
        if (sh <= 0.0f) return 0.0f;
        return ggx_D(a2, n, h) * dot(n, h) / (4.0f * sh);
    }
    if (cg == 0.0f || cs == 0.0f) return 0.0f;
    float eta_g = cg > 0.0f ? 1.0f : m.ior, eta_s = cs > 0.0f ? 1.0f : m.ior;
    if (cg * cs > 0.0f) {
        float3 h = normalize(wg + ws);
        if (dot(n, h) < 0.0f) h = -h;
        if (dot(wg, h) * cg <= 0.0f || dot(ws, h) * cs <= 0.0f) return 0.0f;
        float F = fresnel_dielectric(dot(wg, h), eta_g, eta_g == 1.0f ? m.ior : 1.0f);
        return F * ggx_D(a2, n, h) * dot(n, h) / (4.0f * fabsf(dot(ws, h)));
    }
    float3 hv = -(wg * eta_g + ws * eta_s);
    float hl = sqrtf(len2(hv));
    if (hl == 0.0f) return 0.0f;
    float3 h = hv * (1.0f / hl);
    if (dot(n, h) < 0.0f) h = -h;
    float gh = dot(wg, h), sh = dot(ws, h);
    if (gh * cg <= 0.0f || sh * cs <= 0.0f) return 0.0f;
    float den = eta_g * gh + eta_s * sh;
    if (den == 0.0f) return 0.0f;
    float F = fresnel_dielectric(gh, eta_g, eta_s);
    return (1.0f - F) * ggx_D(a2, n, h) * dot(n, h) * eta_s * eta_s * fabsf(sh) / (den * den);
}

__device__ PB_BSDF_FN bool bsdf_sample(const DMat &m, float3 n, float3 wg, float u0, float u1, float u2,
                                       float3 &ws) {
    float cg = dot(n, wg);
    if (m.kind == MK_LAMBERT) {
        if (cg == 0.0f) return false;
        float3 nn = cg > 0.0f ? n : -n;
        ws = cosine_dir(nn, u1, u2);
        return dot(n, ws) * cg > 0.0f;
    }
    float a2 = m.alpha * m.alpha;
    if (m.kind == MK_CONDUCTOR) {
        if (cg <= 0.0f) return false;
        float3 h = ggx_sample_h(a2, n, u1, u2);
        float c = dot(wg, h);
        if (c <= 0.0f) return false;
        ws = h * (2.0f * c) - wg;
        return dot(n, ws) > 0.0f;
    }
    if (cg == 0.0f) return false;
    float3 h = ggx_sample_h(a2, n, u1, u2);
    float3 hh = cg > 0.0f ? h : -h;
    float c = dot(wg, hh);
    if (c <= 0.0f) return false;
    float eta_g = cg > 0.0f ? 1.0f : m.ior, eta_o = cg > 0.0f ? m.ior : 1.0f;
    float F = fresnel_dielectric(c, eta_g, eta_o);
    if (u0 < F) {
        ws = hh * (2.0f * c) - wg;
        return dot(n, ws) * cg > 0.0f;
    }
    float eta = eta_g / eta_o;
    float s2 = eta * eta * (1.0f - c * c);
    if (s2 >= 1.0f) return false;
    float ct = sqrtf(1.0f - s2);
    ws = normalize(wg * (-eta) + hh * (eta * c - ct));
    return dot(n, ws) * cg < 0.0f;
}

// ---------------------------------------------------------------------------
// Emitters
__device__ __forceinline__ float3 tex_lookup(const DScene &S, float u, float v) {
    if (S.tw <= 0) return f3(1, 1, 1);
    float x = u * S.tw - 0.5f, y = v * S.th - 0.5f;
    float x0 = floorf(x), y0 = floorf(y);
    float fx = x - x0, fy = y - y0;
    int ix0 = min(max((int)x0, 0), S.tw - 1), ix1 = min(max((int)x0 + 1, 0), S.tw - 1);
    int iy0 = min(max((int)y0, 0), S.th - 1), iy1 = min(max((int)y0 + 1, 0), S.th - 1);
    const float *t = S.tex;
    float3 a = f3(t[((size_t)iy0 * S.tw + ix0) * 3], t[((size_t)iy0 * S.tw + ix0) * 3 + 1], t[((size_t)iy0 * S.tw + ix0) * 3 + 2]);
    float3 b = f3(t[((size_t)iy0 * S.tw + ix1) * 3], t[((size_t)iy0 * S.tw + ix1) * 3 + 1], t[((size_t)iy0 * S.tw + ix1) * 3 + 2]);
    float3 c = f3(t[((size_t)iy1 * S.tw + ix0) * 3], t[((size_t)iy1 * S.tw + ix0) * 3 + 1], t[((size_t)iy1 * S.tw + ix0) * 3 + 2]);
    float3 e = f3(t[((size_t)iy1 * S.tw + ix1) * 3], t[((size_t)iy1 * S.tw + ix1) * 3 + 1], t[((size_t)iy1 * S.tw + ix1) * 3 + 2]);
    return (a * (1 - fx) + b * fx) * (1 - fy) + (c * (1 - fx) + e * fx) * fy;
}

// radiance emitted from v toward w (front side only)
__device__ __forceinline__ float3 emitted(const DScene &S, const Vtx &v, float3 w) {
    const DMat &m = S.mats[v.mat];
    if (!m.emitter || dot(v.n, w) <= 0.0f) return f3(0, 0, 0);
    float3 Le = f3(m.ler, m.leg, m.leb);
    if (!m.textured) return Le;
    const float *uv = S.uv + 6 * (size_t)v.tri;
    float b0 = 1.0f - v.b1 - v.b2;
    float u = b0 * uv[0] + v.b1 * uv[2] + v.b2 * uv[4];
    float vv = b0 * uv[1] + v.b1 * uv[3] + v.b2 * uv[5];
    return mul(Le, tex_lookup(S, u, vv));
}

__device__ __forceinline__ float light_pdf(const DScene &S, int tri) {
    if (tri < 0) return 0.0f;
    int e = __float_as_int(S.stri[4 * (size_t)tri + 3].w);
    if (e < 0) return 0.0f;
    float4 e1 = S.stri[4 * (size_t)tri + 1], e2 = S.stri[4 * (size_t)tri + 2];
    float area = 0.5f * sqrtf(len2(cross(xyz(e1), xyz(e2))));
    return S.epmf[e] / area;
}

// emitter triangle: first slot with u0 < cdf; point uniform on it
__device__ __forceinline__ bool sample_light(const DScene &S, float u0, float u1, float u2, int &tri, float &b1,
                                             float &b2) {
    if (S.ne <= 0) return false;
    int lo = 0, hi = S.ne - 1;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (u0 < S.ecdf[mid]) hi = mid;
        else lo = mid + 1;
    }
    tri = S.etri[lo];
    float su = sqrtf(u1);
    b1 = su * (1.0f - u2);
    b2 = su * u2;
    return true;
}

// ---------------------------------------------------------------------------
// Stackless BVH traversal. State: current internal node and a 64-bit trail
// with one bit per level on the path from the root (1 = the far child of that
// level is still to visit). Leaf children are intersected when their parent
// is visited; only internal children are descended into. Backtracking pops
// trail bits through parent[] and resumes at sibling[] of the level whose bit
// is set.
struct Hit {
    int tri;      // original triangle index, -1 for none
    float t, b1, b2;
};

// traversal work counters (node visits of 64 B, triangle tests of 48 B, rays)
struct TravCount {
    uint32_t nodes, tris, rays;
};

template <class SV>
__device__ __forceinline__ void tri_test(const SV &S, int slot, float3 o, float3 d, int skip, Hit &h) {
    const float4 *T = S.itri + 3 * (size_t)slot;
    float4 v0 = __ldg(T), e1 = __ldg(T + 1), e2 = __ldg(T + 2);
    int id = __float_as_int(v0.w);
    if (id == skip) return;
    float3 E1 = xyz(e1), E2 = xyz(e2);
    float3 pv = cross(d, E2);
    float det = dot(E1, pv);
    if (det == 0.0f) return;
    float inv = 1.0f / det;
    float3 tv = o - xyz(v0);
    float u = dot(tv, pv) * inv;
    if (u < 0.0f || u > 1.0f) return;
    float3 qv = cross(tv, E1);
    float v = dot(d, qv) * inv;
    if (v < 0.0f || u + v > 1.0f) return;
    float t = dot(E2, qv) * inv;
    if (!(t > S.eps_t)) return;
    if (t < h.t || (t == h.t && id < h.tri)) {
        h.tri = id;
        h.t = t;
        h.b1 = u;
        h.b2 = v;
    }
}

template <class SV>
__device__ __forceinline__ bool seg_test(const SV &S, int slot, float3 o, float3 d, int s1, int s2) {
    const float4 *T = S.itri + 3 * (size_t)slot;
    float4 v0 = __ldg(T), e1 = __ldg(T + 1), e2 = __ldg(T + 2);
    int id = __float_as_int(v0.w);
    if (id == s1 || id == s2) return false;
    float3 E1 = xyz(e1), E2 = xyz(e2);
    float3 pv = cross(d, E2);
    float det = dot(E1, pv);
    if (det == 0.0f) return false;
    float inv = 1.0f / det;
    float3 tv = o - xyz(v0);
    float u = dot(tv, pv) * inv;
    if (u < 0.0f || u > 1.0f) return false;
    float3 qv = cross(tv, E1);
    float v = dot(d, qv) * inv;
    if (v < 0.0f || u + v > 1.0f) return false;
    float t = dot(E2, qv) * inv;
    return t > 1e-4f && t < 1.0f - 1e-4f;
}

// slab test of two child boxes of a node; returns entry distances
template <class SV>
__device__ __forceinline__ void child_boxes(const SV &S, int node, float3 o, float3 inv, float tmax,
                                            bool &hitL, bool &hitR, float &tl, float &tr, int &cl, int &cr) {
    const float4 *N = S.nodes + 4 * (size_t)node;
    float4 a = __ldg(N), b = __ldg(N + 1), c = __ldg(N + 2), d = __ldg(N + 3);
    cl = __float_as_int(a.w);
    cr = __float_as_int(b.w);
    // robust slab (Ize 2013): widen the far distance by 2 gamma(3)
    const float grow = 1.0f + 2.0f * 3.0f * 5.96046448e-08f;
    float t0x = (a.x - o.x) * inv.x, t1x = (b.x - o.x) * inv.x;
    float t0y = (a.y - o.y) * inv.y, t1y = (b.y - o.y) * inv.y;
    float t0z = (a.z - o.z) * inv.z, t1z = (b.z - o.z) * inv.z;
    float ln = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), 0.0f));
    float lf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fminf(fmaxf(t0z, t1z), tmax)) * grow;
    float s0x = (c.x - o.x) * inv.x, s1x = (d.x - o.x) * inv.x;
    float s0y = (c.y - o.y) * inv.y, s1y = (d.y - o.y) * inv.y;
    float s0z = (c.z - o.z) * inv.z, s1z = (d.z - o.z) * inv.z;
    float rn = fmaxf(fmaxf(fminf(s0x, s1x), fminf(s0y, s1y)), fmaxf(fminf(s0z, s1z), 0.0f));
    float rf = fminf(fminf(fmaxf(s0x, s1x), fmaxf(s0y, s1y)), fminf(fmaxf(s0z, s1z), tmax)) * grow;
    hitL = ln <= lf;
    hitR = rn <= rf;
    tl = ln;
    tr = rn;
}

__device__ __forceinline__ float3 safe_inv(float3 d) {
    // 1/0 = inf keeps the slab test correct; avoid -0 -> -inf surprises by sign
    return f3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
}

// The traversal cores take a compact by-value view of the scene and are
// shared out-of-line functions: kernels with many ray queries stay small
// enough for the instruction cache (measured 1.4-1.9x faster than inlining
// every query). Define PB_TRAV_INLINE to inline them instead.
struct TravView {
    const float4 *nodes;
    const int *parent, *sibling;
    const float4 *itri;
    float eps_t;
};
#ifdef PB_TRAV_INLINE
#define PB_TRAV_FN __forceinline__
#else
#define PB_TRAV_FN __noinline__
#endif

__device__ __forceinline__ TravView trav_view(const DScene &S) {
    TravView v;
    v.nodes = S.nodes;
    v.parent = S.parent;
    v.sibling = S.sibling;
    v.itri = S.itri;
    v.eps_t = S.eps_t;
    return v;
}

template <bool COUNT>
__device__ PB_TRAV_FN Hit trav_closest(TravView S, float3 o, float3 d, int skip, Hit h, TravCount *cnt);
template <bool COUNT>
__device__ PB_TRAV_FN bool trav_occluded(TravView S, float3 a, float3 b, int s1, int s2, TravCount *cnt);

// closest hit starting from a known candidate `h` (h.tri = -1, h.t = inf for
// a plain query): only triangles with a smaller t (or the same t and a lower
// index) replace it, so the result equals the unrestricted closest hit
template <bool COUNT>
__device__ __forceinline__ Hit closest_hit_from(const DScene &S, float3 o, float3 d, int skip, Hit h,
                                                TravCount *cnt = nullptr) {
    return trav_closest<COUNT>(trav_view(S), o, d, skip, h, cnt);
}

template <bool COUNT>
__device__ PB_TRAV_FN Hit trav_closest(TravView S, float3 o, float3 d, int skip, Hit h, TravCount *cnt) {
    if (COUNT) cnt->rays++;
    float3 inv = safe_inv(d);
    int node = 0;
    uint64_t trail = 0;
    for (int guard = 0; guard < (1 << 22); ++guard) {
        bool hL, hR;
        float tl, tr;
        int cl, cr;
        child_boxes(S, node, o, inv, h.t, hL, hR, tl, tr, cl, cr);
        if (COUNT) cnt->nodes++;
        if (hL && cl < 0) {
            int v = -cl - 1, first = v >> 4, n = v & 15;
            for (int i = 0; i < n; ++i) tri_test(S, first + i, o, d, skip, h);
            if (COUNT) cnt->tris += n;
            hL = false;
        }
        if (hR && cr < 0) {
            int v = -cr - 1, first = v >> 4, n = v & 15;
            for (int i = 0; i < n; ++i) tri_test(S, first + i, o, d, skip, h);
            if (COUNT) cnt->tris += n;
            hR = false;
        }
        hL = hL && tl <= h.t;
        hR = hR && tr <= h.t;
        if (hL && hR) {
            trail = (trail << 1) | 1ull;
            node = tl <= tr ? cl : cr;
            continue;
        }
        if (hL || hR) {
            trail <<= 1;
            node = hL ? cl : cr;
            continue;
        }
        // backtrack
        while ((trail & 1ull) == 0ull) {
            if (trail == 0ull) return h;
            trail >>= 1;
            node = __ldg(S.parent + node);
        }
        trail ^= 1ull;
        node = __ldg(S.sibling + node);
    }
    return h;
}

template <bool COUNT>
__device__ __forceinline__ Hit closest_hit(const DScene &S, float3 o, float3 d, int skip, TravCount *cnt = nullptr) {
    Hit h;
    h.tri = -1;
    h.t = INFINITY;
    h.b1 = h.b2 = 0.0f;
    return closest_hit_from<COUNT>(S, o, d, skip, h, cnt);
}

// the nearest emitter triangle the ray meets (tri = -1 if none), with the
// traversal's triangle predicate: the start candidate of closest_emitter_hit
__device__ __forceinline__ Hit emitter_candidate(const DScene &S, float3 o, float3 d, int skip) {
    Hit e;
    e.tri = -1;
    e.t = INFINITY;
    e.b1 = e.b2 = 0.0f;
    for (int i = 0; i < S.ne; ++i) {
        int id = S.etri[i];
        if (id == skip) continue;
        const float4 *T = S.stri + 4 * (size_t)id;
        float3 v0 = xyz(T[0]), E1 = xyz(T[1]), E2 = xyz(T[2]);
        float3 pv = cross(d, E2);
        float det = dot(E1, pv);
        if (det == 0.0f) continue;
        float inv = 1.0f / det;
        float3 tv = o - v0;
        float u = dot(tv, pv) * inv;
        if (u < 0.0f || u > 1.0f) continue;
        float3 qv = cross(tv, E1);
        float v = dot(d, qv) * inv;
        if (v < 0.0f || u + v > 1.0f) continue;
        float t = dot(E2, qv) * inv;
        if (!(t > S.eps_t)) continue;
        if (t < e.t || (t == e.t && id < e.tri)) {
            e.tri = id;
            e.t = t;
            e.b1 = u;
            e.b2 = v;
        }
    }
    return e;
}

// Closest hit of a ray that only matters if it ends on an emitter: the
// emitter triangles are tested first (same predicate as the traversal); if
// none is hit the answer "no emitter is the closest hit" needs no traversal,
// else the traversal is bounded by the nearest emitter hit. Returns the
// closest hit when it lies on an emitter, otherwise tri = -1.
template <bool COUNT>
__device__ __forceinline__ Hit closest_emitter_hit(const DScene &S, float3 o, float3 d, int skip,
                                                   TravCount *cnt = nullptr) {
    Hit e = emitter_candidate(S, o, d, skip);
    if (e.tri < 0) return e;
    Hit h = closest_hit_from<COUNT>(S, o, d, skip, e, cnt);
    int em = __float_as_int(S.stri[4 * (size_t)h.tri + 3].w);
    if (em < 0) h.tri = -1;
    return h;
}

// emitter lists longer than this use the plain closest hit
#define PB_EMITTER_LIST_MAX 64

// any hit strictly inside the open segment a -> b (parameter in (1e-4, 1-1e-4))
template <bool COUNT = false>
__device__ __forceinline__ bool occluded(const DScene &S, float3 a, float3 b, int s1, int s2, TravCount *cnt = nullptr) {
    return trav_occluded<COUNT>(trav_view(S), a, b, s1, s2, cnt);
}

template <bool COUNT>
__device__ PB_TRAV_FN bool trav_occluded(TravView S, float3 a, float3 b, int s1, int s2, TravCount *cnt) {
    float3 d = b - a;
    float3 inv = safe_inv(d);
    if (COUNT) cnt->rays++;
    int node = 0;
    uint64_t trail = 0;
    for (int guard = 0; guard < (1 << 22); ++guard) {
        bool hL, hR;
        float tl, tr;
        int cl, cr;
        child_boxes(S, node, a, inv, 1.0f, hL, hR, tl, tr, cl, cr);
        if (COUNT) cnt->nodes++;
        if (hL && cl < 0) {
            int v = -cl - 1, first = v >> 4, n = v & 15;
            for (int i = 0; i < n; ++i) {
                if (COUNT) cnt->tris++;
                if (seg_test(S, first + i, a, d, s1, s2)) return true;
            }
            hL = false;
        }
        if (hR && cr < 0) {
            int v = -cr - 1, first = v >> 4, n = v & 15;
            for (int i = 0; i < n; ++i) {
                if (COUNT) cnt->tris++;
                if (seg_test(S, first + i, a, d, s1, s2)) return true;
            }
            hR = false;
        }
        if (hL && hR) {
            trail = (trail << 1) | 1ull;
            node = tl <= tr ? cl : cr;
            continue;
        }
        if (hL || hR) {
            trail <<= 1;
            node = hL ? cl : cr;
            continue;
        }
        while ((trail & 1ull) == 0ull) {
            if (trail == 0ull) return false;
            trail >>= 1;
            node = __ldg(S.parent + node);
        }
        trail ^= 1ull;
        node = __ldg(S.sibling + node);
    }
    return false;
}

// ---------------------------------------------------------------------------
// Traversal one node visit at a time, for persistent warps that refill idle
// lanes: a lane's ray state lives in a PtRay, and pt_step runs the loop body of
// trav_closest / trav_occluded once, so a query answered in steps is answered
// node for node as the one-call traversal answers it.
constexpr int PT_STEPS = 8;   // node visits per lane between refills

struct PtRay {
    float3 o, d, inv;   // occlusion: d = b - a
    Hit h;              // closest: best so far; occlusion: tri = 1 once blocked
    uint64_t trail;
    int node, kind, s1, s2, steps;   // kind 0 closest, 2 occlusion, 3 closest that must end on an emitter
};

// one node visit of r's traversal (the loop body of trav_closest or
// trav_occluded); true when the traversal has ended
template <bool COUNT>
__device__ __forceinline__ bool pt_step(const TravView &S, PtRay &r, TravCount *tc) {
    if (r.steps++ >= (1 << 22)) return true;
    const bool occl = r.kind == 2;
    bool hL, hR;
    float tl, tr;
    int cl, cr;
    child_boxes(S, r.node, r.o, r.inv, occl ? 1.0f : r.h.t, hL, hR, tl, tr, cl, cr);
    if (COUNT) tc->nodes++;
    if (hL && cl < 0) {
        int v = -cl - 1, first = v >> 4, n = v & 15;
        if (occl) {
            for (int i = 0; i < n; ++i) {
                if (COUNT) tc->tris++;
                if (seg_test(S, first + i, r.o, r.d, r.s1, r.s2)) {
                    r.h.tri = 1;
                    return true;
                }
            }
        } else {
            for (int i = 0; i < n; ++i) tri_test(S, first + i, r.o, r.d, r.s1, r.h);
            if (COUNT) tc->tris += n;
        }
        hL = false;
    }
    if (hR && cr < 0) {
        int v = -cr - 1, first = v >> 4, n = v & 15;
        if (occl) {
            for (int i = 0; i < n; ++i) {
                if (COUNT) tc->tris++;
                if (seg_test(S, first + i, r.o, r.d, r.s1, r.s2)) {
                    r.h.tri = 1;
                    return true;
                }
            }
        } else {
            for (int i = 0; i < n; ++i) tri_test(S, first + i, r.o, r.d, r.s1, r.h);
            if (COUNT) tc->tris += n;
        }
        hR = false;
    }
    if (!occl) {
        hL = hL && tl <= r.h.t;
        hR = hR && tr <= r.h.t;
    }
    if (hL && hR) {
        r.trail = (r.trail << 1) | 1ull;
        r.node = tl <= tr ? cl : cr;
        return false;
    }
    if (hL || hR) {
        r.trail <<= 1;
        r.node = hL ? cl : cr;
        return false;
    }
    while ((r.trail & 1ull) == 0ull) {
        if (r.trail == 0ull) return true;
        r.trail >>= 1;
        r.node = __ldg(S.parent + r.node);
    }
    r.trail ^= 1ull;
    r.node = __ldg(S.sibling + r.node);
    return false;
}

// ---------------------------------------------------------------------------
// Subspace labels: nearest centroid in bbox-normalised feature space, ties to
// the lowest index (Sec. 3.2: subspaces by position, normal and direction).
__device__ __forceinline__ int nearest(const float *f, int dim, int K, const float *cent) {
    int best = 0;
    float bd = INFINITY;
    for (int k = 0; k < K; ++k) {
        float d = 0.0f;
        for (int i = 0; i < dim; ++i) {
            float e = f[i] - __ldg(cent + k * dim + i);
            d += e * e;
        }
        if (d < bd) {
            bd = d;
            best = k;
        }
    }
    return best;
}

__device__ __forceinline__ void feat_pos(const DScene &S, float3 p, float *f) {
    f[0] = (p.x - S.lo.x) / S.ext.x;
    f[1] = (p.y - S.lo.y) / S.ext.y;
    f[2] = (p.z - S.lo.z) / S.ext.z;
}

__device__ __forceinline__ int label_dir(const DScene &S, const Vtx &v, float3 w, int K, const float *cent) {
    float f[9];
    feat_pos(S, v.p, f);
    float3 n = dot(v.n, w) >= 0.0f ? v.n : -v.n;
    f[3] = n.x; f[4] = n.y; f[5] = n.z;
    f[6] = w.x; f[7] = w.y; f[8] = w.z;
    return nearest(f, 9, K, cent);
}

__device__ __forceinline__ int label_spec(const DScene &S, const DTables &T, const Vtx &v) {
    float f[6];
    feat_pos(S, v.p, f);
    f[3] = v.n.x; f[4] = v.n.y; f[5] = v.n.z;
    return nearest(f, 6, T.KSp, T.cSp);
}

__device__ __forceinline__ int label_ctrl(const DScene &S, const DTables &T, const Vtx &v) {
    float f[3];
    feat_pos(S, v.p, f);
    return nearest(f, 3, T.KC, T.cC);
}

__device__ __forceinline__ bool spec_v(const DScene &S, const Vtx &v) { return S.mats[v.mat].specular; }

