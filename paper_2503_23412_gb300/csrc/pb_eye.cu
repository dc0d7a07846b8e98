// Eye side of an iteration: one thread per (iteration slot, pixel).
//
// The camera sub-path is traced by BSDF sampling (Sec. 3.1). At every
// vertex z_a:
//   s = 0  an emitter hit adds beta * Le with its MIS weight;
//   s = 1  next-event estimation at non-specular vertices;
//   s >= 2 one probabilistic connection (Sec. 3.2): eye subspace T of z_a,
//          light subspace S ~ Gamma[T, .] over non-empty subspaces, then a
//          uniform stored light vertex of S (SPCBPT, Sec. 5.5); the estimate
//          divides by M * Q_j;
//   proxy  at the first non-specular vertex, with the tile probability pi:
//          select an incomplete light sub-path (Gamma'[T, .] then uniform),
//          retrace the dropped vertices by BSDF sampling from y_{s-1} with
//          z_a as the incoming side (Sec. 5.1), reject specular/diffuse
//          mismatches, and weight by the stored reciprocal estimate of
//          1/P(u, h_c, y_{s-1}, w_c) (Sec. 5.2, Eq. reciprocalFinal).
// MIS weights (Sec. 5.4, Eq. MIS_1) are formed from recursive sums of
// density ratios: the light side's partial sum is stored per pool vertex,
// the eye side's is carried here (E_a = r_a (avail_{a-1} + E_{a-1}),
// r_c = fwd(z_c)/rev(z_c)); the last two ratios on each side depend on the
// connection and are finished at connection time. The proxy term enters PT
// and NEE weights of paths with the proxy shape; connections (s >= 2) can
// never produce such paths (both joined vertices must be non-specular).
//
// Camera-side wavefront: the feature pass traces every camera sub-path and
// stores its hits; an EYE_EMIT pass replays them with exactly the control
// flow of the shading pass and appends each NEE, connection and proxy-entry
// occlusion query to a queue (warp-aggregated appends); k_eye_occ answers
// the queue with a traversal-only kernel; the EYE_READ pass replays again,
// reads the answers and shades. Each query is the same segment the inline
// pass would test, so the images are identical; the traversal runs at the
// occupancy of a small kernel instead of the shading kernel's.
#include <algorithm>
#include <cooperative_groups.h>

#include "pb_kernels.h"
#include "pb_mlp.cuh"

namespace cg = cooperative_groups;

namespace {

struct EV {            // eye vertex history
    float3 p, n, we;   // position, normal, direction toward the previous eye vertex
    int mat;
    bool nonS;
    float rev;         // eye-tracer area density of this vertex (1 for z_1)
    float cos_out, d2_out;   // |cos| toward the next vertex and squared distance to it
};

__device__ __forceinline__ uint32_t sig_upd(uint32_t h, uint32_t x) { return (h ^ x) * 16777619u; }

__device__ __forceinline__ int select_cdf(const float *cdf, int K, float u) {
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (u < cdf[mid]) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ float lum(float3 c) { return (c.x + c.y + c.z) * (1.0f / 3.0f); }

// hit of eye vertex a stored by the feature pass
__device__ __forceinline__ Hit stored_hit(const KParams &P, int slot, int a, int pix) {
    int4 v = P.mlp.hits[((size_t)slot * P.max_depth + (a - 1)) * P.npix + pix];
    Hit h;
    h.tri = v.x;
    h.t = __int_as_float(v.y);
    h.b1 = __int_as_float(v.z);
    h.b2 = __int_as_float(v.w);
    return h;
}

__device__ __forceinline__ float mis_cell(const DTables &T, int u, int Sp, int C) {
    return T.mis[((u - 1) * T.KSp + Sp) * (T.KC + 1) + C];
}

// visibility of the segment a -> b (kind 0 NEE, 1 connection, 2 the proxy's
// first segment) at dense vertex index `dv`: traced here, appended to the
// query queue (answer unknown yet: false), or read from the answers
template <bool COUNT, int MODE>
__device__ __forceinline__ bool eye_visible(const DScene &S, const KParams &P, size_t dv, int kind, float3 a,
                                            float3 b, int sa, int sb, TravCount *tc) {
    if (MODE == EYE_INLINE) return !occluded<COUNT>(S, a, b, sa, sb, tc);
    if (MODE == EYE_READ) return P.q.vis[(size_t)kind * P.q.plane + dv] != 0;
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned int base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(P.q.count, (unsigned int)g.size());
    const unsigned int idx = g.shfl(base, 0) + g.thread_rank();
    if (idx < (unsigned int)P.q.cap) {   // the capacity covers every vertex's queries
        P.q.qa[idx] = make_float4(a.x, a.y, a.z, __int_as_float(sa));
        P.q.qb[idx] = make_float4(b.x, b.y, b.z, __int_as_float(sb));
        P.q.dst[idx] = (int32_t)(dv * 4 + (size_t)kind);
    }
    return false;
}

template <bool COUNT, int MODE>
__global__ void __launch_bounds__(128, 4) k_eye(DScene S, DTables T, KParams P, Pool B, uint32_t iter_base,
                                             float4 *Lbuf, uint32_t *sigbuf) {
    constexpr bool SHADE = MODE != EYE_EMIT;   // the emit pass only walks the paths and appends queries
    iter_base = eff_iter(P, iter_base);
    TravCount tc{0, 0, 0};
    int pix = blockIdx.x * blockDim.x + threadIdx.x;
    int slot = blockIdx.y;
    if (pix >= P.npix) return;
    uint32_t it = iter_base + (uint32_t)slot;
    size_t so = (size_t)slot * B.ML;
    int npool = B.npool[slot], nent = B.nent[slot];
    int px = pix % S.W, py = pix / S.W;
    Rng r0;
    r0.init(P.seed, K_CAMERA, it, (uint32_t)pix, 0);
    float j0 = r0.u(0), j1 = r0.u(1);
    float sx = 2.0f * ((float)px + j0) / (float)S.W - 1.0f, sy = 1.0f - 2.0f * ((float)py + j1) / (float)S.H;
    float3 d = normalize(S.cfwd + (S.cright * (sx * S.tanh_ * S.aspect) + S.cup * (sy * S.tanh_)));
    float3 L = f3(0, 0, 0);
    uint32_t sig = 2166136261u;
    float3 beta = f3(1, 1, 1);
    int tile = (py / T.tile) * T.gw + (px / T.tile);
    float pi_pix = T.pi[tile];
    EV zp, zpp;               // z_{a-1}, z_{a-2}
    zp.p = S.cpos;
    zp.nonS = true;
    zpp.nonS = true;
    bool nonS_ppp = true;     // z_{a-3}
    float Ef = 0.0f;          // E_{a-2}
    int pstate = 0, f_idx = 0, Sp_f1 = 0;
    float rev_f1 = 1.0f;
    unsigned long long n_conn = 0, n_proxy = 0, n_proxy_ok = 0;
    const bool replay = P.mlp.hits != nullptr;   // eye rays were traced by the feature pass
    Hit h = replay ? stored_hit(P, slot, 1, pix) : closest_hit<COUNT>(S, S.cpos, d, -1, &tc);
    int a = 1;
    while (h.tri >= 0) {
        Vtx z = vertex_at(S, h.tri, h.b1, h.b2);
        const DMat &mz = S.mats[z.mat];
        float3 we = -d;
        sig = sig_upd(sig, (uint32_t)z.tri);
        float d2_in = len2(z.p - zp.p);
        float cos_in = fabsf(dot(z.n, d));
        float rev_a = 1.0f;
        if (a >= 2) {
            zp.cos_out = fabsf(dot(zp.n, d));
            zp.d2_out = d2_in;
            rev_a = bsdf_pdf(S.mats[zp.mat], zp.n, zp.we, d) * cos_in / d2_in;
        }
        if (a >= 4) {
            // finish E_{a-2}: r_{a-2} = fwd(z_{a-2}) / rev(z_{a-2})
            float fwd_pp = bsdf_pdf(S.mats[zp.mat], zp.n, d, zp.we) * zpp.cos_out / zpp.d2_out;
            float av = (nonS_ppp && zpp.nonS && P.conn) ? 1.0f : 0.0f;
            Ef = zpp.rev > 0.0f ? (fwd_pp / zpp.rev) * (av + Ef) : 0.0f;
        }
        bool nonS = !mz.specular;
        Rng R;
        R.init(P.seed, K_CAMERA, it, (uint32_t)pix, (uint32_t)a);
        const size_t dv = ((size_t)slot * P.max_depth + (a - 1)) * P.npix + pix;

        // ---- (s = 0) emitter hit
        if (SHADE && mz.emitter && dot(z.n, we) > 0.0f) {
            float3 Le = emitted(S, z, we);
            if (maxc(Le) > 0.0f) {
                float w = 1.0f;
                if (a >= 2) {
                    float fz = light_pdf(S, z.tri);
                    float fz1 = (dot(z.n, we) / PB_PI) * zp.cos_out / zp.d2_out;
                    float Em1 = 0.0f;
                    if (a - 1 >= 2) {
                        float av = (zpp.nonS && zp.nonS && P.conn) ? 1.0f : 0.0f;
                        Em1 = zp.rev > 0.0f ? (fz1 / zp.rev) * (av + Ef) : 0.0f;
                    }
                    float Epr = rev_a > 0.0f ? (fz / rev_a) * ((zp.nonS ? 1.0f : 0.0f) + Em1) : 0.0f;
                    float pt = 0.0f;
                    if (P.proxy) {
                        if (pstate == 1) {
                            int u = a - f_idx - 1;
                            if (u >= 1 && u <= 4) pt = pi_pix * mis_cell(T, u, Sp_f1, T.KC) / rev_f1;
                        } else if (pstate == 2) {
                            int u = (a - 1) - f_idx - 1;
                            if (u >= 1 && u <= 4 && rev_a > 0.0f) {
                                int C = label_ctrl(S, T, z);
                                pt = fz * pi_pix * mis_cell(T, u, Sp_f1, C) / (rev_f1 * rev_a);
                            }
                        }
                    }
                    w = 1.0f / (1.0f + Epr + pt);
                }
                if (P.film != 1) L = L + mul(beta, Le) * w;
                if (P.acc.tile_all) atomicAdd(&P.acc.tile_all[tile], lum(mul(beta, Le)) * w);
            }
        }
        if (absorbing(S, z, we)) break;
        int Tl = -1;
        if (nonS) {
            // ---- (s = 1) next-event estimation
            if (a + 1 <= P.max_depth && S.ne > 0) {
                int lt;
                float b1, b2;
                sample_light(S, R.u(3), R.u(4), R.u(5), lt, b1, b2);
                Vtx y = vertex_at(S, lt, b1, b2);
                bool vis = eye_visible<COUNT, MODE>(S, P, dv, 0, z.p, y.p, z.tri, y.tri, &tc);
                sig = sig_upd(sig, 0xA0000000u | (uint32_t)lt);
                sig = sig_upd(sig, vis ? 1u : 0u);
                if (vis) {
                    float3 dd = y.p - z.p;
                    float d2 = len2(dd);
                    float3 wy = dd * (1.0f / sqrtf(d2));
                    float3 Le = emitted(S, y, -wy);
                    float3 rz = bsdf_eval(mz, z.n, wy, we);
                    if (maxc(Le) > 0.0f && maxc(rz) > 0.0f) {
                        float cz = fabsf(dot(z.n, wy)), cy = fabsf(dot(y.n, wy));
                        float pL = light_pdf(S, lt);
                        float3 c = mul(mul(beta, rz), Le) * (cz * cy / (d2 * pL));
                        float rev0 = bsdf_pdf(mz, z.n, we, wy) * cy / d2;
                        float Lsum0 = rev0 / pL;
                        float Ea = 0.0f;
                        if (a >= 2) {
                            float fz = (dot(y.n, -wy) / PB_PI) * cz / d2;
                            float fz1 = bsdf_pdf(mz, z.n, wy, we) * zp.cos_out / zp.d2_out;
                            float Em1 = 0.0f;
                            if (a - 1 >= 2) {
                                float av = (zpp.nonS && zp.nonS && P.conn) ? 1.0f : 0.0f;
                                Em1 = zp.rev > 0.0f ? (fz1 / zp.rev) * (av + Ef) : 0.0f;
                            }
                            float av1 = (zp.nonS && P.conn) ? 1.0f : 0.0f;
                            Ea = rev_a > 0.0f ? (fz / rev_a) * (av1 + Em1) : 0.0f;
                        }
                        float pt = 0.0f;
                        if (P.proxy && pstate == 1) {
                            int u = a - f_idx - 1;
                            if (u >= 1 && u <= 4) {
                                int C = label_ctrl(S, T, y);
                                pt = pi_pix * mis_cell(T, u, Sp_f1, C) / rev_f1;
                            }
                        }
                        float w = 1.0f / (1.0f + Lsum0 + Ea + pt);
                        if (P.film != 1) L = L + c * w;
                        if (P.acc.tile_all) atomicAdd(&P.acc.tile_all[tile], lum(c) * w);
                    }
                }
            }
            // ---- (s >= 2) subspace probabilistic connection
            if (P.conn && a + 2 <= P.max_depth && npool > 0) {
                Tl = label_dir(S, z, we, T.KT, T.cT);
                int Ssel;
                float QS;   // probability of the subspace
                if (P.mlp.sel) {
                    // learned proposal: drawn by the network kernel from this vertex's row
                    size_t row = ((size_t)slot * P.mlp.A + (a - 1)) * P.npix + pix;
                    Ssel = P.mlp.sel[row];
                    QS = P.mlp.selq[row];
                } else {
                    const float *cdf = B.cdfC + (size_t)slot * T.KT * T.KS + (size_t)Tl * T.KS;
                    Ssel = select_cdf(cdf, T.KS, R.u(6));
                    QS = T.gC[(size_t)Tl * T.KS + Ssel] / B.ZC[(size_t)slot * T.KT + Tl];
                }
                const int32_t *bst = B.bstart + (size_t)slot * (T.KS + 1);
                int nS = Ssel >= 0 ? bst[Ssel + 1] - bst[Ssel] : 0;
                if (nS > 0) {
                    int jj = min((int)(R.u(7) * (float)nS), nS - 1);
                    int jp = B.bitems[so + bst[Ssel] + jj];
                    int fixed = B.pool_idx[so + jp];
                    int e = fixed % P.L;
                    float Q = QS / (float)nS;
                    sig = sig_upd(sig, 0xB0000000u | (uint32_t)jp);
                    n_conn++;
                    int sl = e + 1;
                    if (sl + a > P.max_depth) {
                        sig = sig_upd(sig, 2u);
                    } else {
                        float4 vp = B.vpos[so + fixed], vn = B.vnrm[so + fixed], vw = B.vwl[so + fixed];
                        float4 va = B.valpha[so + fixed], vm = B.vmis[so + fixed];
                        float3 yp = xyz(vp), yn = xyz(vn), ywl = xyz(vw);
                        int ymat = __float_as_int(vp.w), ytri = __float_as_int(vn.w);
                        bool vis = eye_visible<COUNT, MODE>(S, P, dv, 1, z.p, yp, z.tri, ytri, &tc);
                        sig = sig_upd(sig, vis ? 1u : 0u);
                        if (vis) {
                            float3 dd = yp - z.p;
                            float d2 = len2(dd);
                            float3 wy = dd * (1.0f / sqrtf(d2));
                            const DMat &my = S.mats[ymat];
                            float3 rz = bsdf_eval(mz, z.n, wy, we);
                            float3 ry = bsdf_eval(my, yn, ywl, -wy);
                            float cz = fabsf(dot(z.n, wy)), cy = fabsf(dot(yn, wy));
                            float3 c = mul(mul(mul(beta, rz), ry), xyz(va)) * (cz * cy / (d2 * (float)P.M * Q));
                            if (maxc(c) > 0.0f) {
                                int flags = __float_as_int(vm.w);
                                float fwd_em1 = vm.x, fwd_e = vw.w;
                                float rev_em1 = bsdf_pdf(my, yn, -wy, ywl) * vm.y / vm.z;
                                float Ls1 = fwd_em1 > 0.0f ? (rev_em1 / fwd_em1) * ((float)(flags & 1) + va.w) : 0.0f;
                                float rev_e = bsdf_pdf(mz, z.n, we, wy) * cy / d2;
                                float Ls = fwd_e > 0.0f ? (rev_e / fwd_e) * ((float)((flags >> 1) & 1) + Ls1) : 0.0f;
                                float Ea = 0.0f;
                                if (a >= 2) {
                                    float fz = bsdf_pdf(my, yn, ywl, -wy) * cz / d2;
                                    float fz1 = bsdf_pdf(mz, z.n, wy, we) * zp.cos_out / zp.d2_out;
                                    float Em1 = 0.0f;
                                    if (a - 1 >= 2) {
                                        float av = (zpp.nonS && zp.nonS) ? 1.0f : 0.0f;
                                        Em1 = zp.rev > 0.0f ? (fz1 / zp.rev) * (av + Ef) : 0.0f;
                                    }
                                    float av1 = zp.nonS ? 1.0f : 0.0f;
                                    Ea = rev_a > 0.0f ? (fz / rev_a) * (av1 + Em1) : 0.0f;
                                }
                                float w = 1.0f / (1.0f + Ls + Ea);
                                if (P.film != 1) L = L + c * w;
                                if (P.smp.raw) {
                                    unsigned int idx = atomicAdd(P.smp.count, 1u);
                                    if (idx < (unsigned int)P.smp.cap) {
                                        mlp_raw(S, z, we, P.smp.raw + (size_t)MLP_NRAW * idx);
                                        P.smp.T[idx] = Tl;
                                        P.smp.S[idx] = Ssel;
                                        P.smp.w[idx] = lum(c);
                                    }
                                }
                                if (P.acc.conn) {
                                    atomicAdd(&P.acc.tile_all[tile], lum(c) * w);
                                    atomicAdd(&P.acc.conn[(size_t)Tl * T.KS + Ssel], lum(c));
                                }
                            }
                        }
                    }
                }
            }
            // ---- proxy at the first non-specular eye vertex (Sec. 6.1.1)
            if (P.proxy && pstate == 0 && nent > 0 && pi_pix > 0.0f) {
                bool coin = R.u(8) < pi_pix;
                sig = sig_upd(sig, 0xC0000000u | (coin ? 1u : 0u));
                if (coin) {
                    if (Tl < 0) Tl = label_dir(S, z, we, T.KT, T.cT);
                    int Ssel;
                    float QS;   // probability of the specular subspace
                    if (P.mlpp.sel && a + 2 <= P.max_depth) {
                        // learned proposal of the proxy: drawn by the proxy network's kernel
                        const size_t row = ((size_t)slot * P.mlpp.A + (a - 1)) * P.npix + pix;
                        Ssel = P.mlpp.sel[row];
                        QS = P.mlpp.selq[row];
                    } else {
                        const float *cdf = B.cdfP + (size_t)slot * T.KT * T.KSp + (size_t)Tl * T.KSp;
                        Ssel = select_cdf(cdf, T.KSp, R.u(9));
                        QS = T.gP[(size_t)Tl * T.KSp + Ssel] / B.ZP[(size_t)slot * T.KT + Tl];
                    }
                    const int32_t *est = B.estart + (size_t)slot * (T.KSp + 1);
                    int nS = Ssel >= 0 ? est[Ssel + 1] - est[Ssel] : 0;
                    if (nS > 0) {
                        int jj = min((int)(R.u(10) * (float)nS), nS - 1);
                        int k = B.eitems[so + est[Ssel] + jj];
                        float Q = QS / (float)nS;
                        sig = sig_upd(sig, (uint32_t)k);
                        n_proxy++;
                        int fixed = B.ent_idx[so + k];
                        int l = fixed / P.L, e = fixed % P.L;
                        size_t gb = so + (size_t)l * P.L;
                        Vtx gs[6], H;
                        gs[0] = vertex_at(S, B.gtri[gb + e], B.gbary[gb + e].x, B.gbary[gb + e].y);
                        H = vertex_at(S, B.gtri[gb], B.gbary[gb].x, B.gbary[gb].y);
                        int info = B.einfo[so + fixed];
                        int u = info & 7, type = (info >> 3) & 1, C = info >> 4;
                        int Sp = B.elabel[so + fixed];
                        int sl = u + (type ? 2 : 1);
                        int status = 0;
                        if (sl + a > P.max_depth) status = 1;
                        else if (!eye_visible<COUNT, MODE>(S, P, dv, 2, z.p, gs[0].p, z.tri, gs[0].tri, &tc)) status = 2;
                        else {
                            float3 prev = z.p;
                            for (int r = 1; r <= u && !status; ++r) {
                                const Vtx &g = gs[r - 1];
                                const DMat &mg = S.mats[g.mat];
                                float3 wg = dirto(g.p, prev);
                                float3 ws;
                                int d0 = 11 + 3 * (r - 1);
                                if (absorbing(S, g, wg) || !bsdf_sample(mg, g.n, wg, R.u(d0), R.u(d0 + 1), R.u(d0 + 2), ws)) {
                                    status = 3;
                                    break;
                                }
                                Hit hh = closest_hit<COUNT>(S, g.p, ws, g.tri, &tc);
                                sig = sig_upd(sig, hh.tri >= 0 ? (uint32_t)hh.tri : 0x0FFFFFFFu);
                                if (hh.tri < 0) {
                                    status = 4;
                                    break;
                                }
                                gs[r] = vertex_at(S, hh.tri, hh.b1, hh.b2);
                                const DMat &mr = S.mats[gs[r].mat];
                                float3 back = -ws;
                                if (r < u) {
                                    if (!mr.specular || absorbing(S, gs[r], back)) status = 5;
                                } else if (type == 0) {
                                    if (!mr.emitter || dot(gs[r].n, back) <= 0.0f) status = 5;
                                } else {
                                    if (mr.specular || absorbing(S, gs[r], back)) status = 5;
                                }
                                prev = g.p;
                            }
                            if (!status && type && occluded<COUNT>(S, gs[u].p, H.p, gs[u].tri, H.tri, &tc)) status = 6;
                        }
                        sig = sig_upd(sig, 0xD0000000u | (uint32_t)status);
                        if (!status) {
                            const Vtx &Y = gs[0];
                            float3 dd = Y.p - z.p;
                            float d2 = len2(dd);
                            float3 wY = dd * (1.0f / sqrtf(d2));
                            float3 rz = bsdf_eval(mz, z.n, wY, we);
                            float cz = fabsf(dot(z.n, wY)), cY = fabsf(dot(Y.n, wY));
                            float3 tp = rz * (cz * cY / d2);
                            // retraced segments: rho |cos| / pdf at Y, g_1 .. g_{u-1}
                            float3 nextw = -wY;   // direction from the current vertex toward the eye side
                            for (int r = 0; r < u; ++r) {
                                const Vtx &g = gs[r];
                                const DMat &mg = S.mats[g.mat];
                                float3 wl = dirto(g.p, gs[r + 1].p);
                                float3 wv = (r == 0) ? nextw : dirto(g.p, gs[r - 1].p);
                                float pw = bsdf_pdf(mg, g.n, wv, wl);
                                tp = pw > 0.0f ? mul(tp, bsdf_eval(mg, g.n, wl, wv)) * (fabsf(dot(g.n, wl)) / pw) : f3(0, 0, 0);
                            }
                            float3 Le;
                            float ph = 1.0f, rev0 = 0.0f;
                            const Vtx &gu = gs[u];
                            if (type == 0) {
                                Le = emitted(S, gu, dirto(gu.p, gs[u - 1].p));
                            } else {
                                float3 hd = H.p - gu.p;
                                float hd2 = len2(hd);
                                float3 wh = hd * (1.0f / sqrtf(hd2));
                                float3 wv = dirto(gu.p, gs[u - 1].p);
                                const DMat &mu = S.mats[gu.mat];
                                float chu = fabsf(dot(gu.n, wh)), chH = fabsf(dot(H.n, wh));
                                tp = mul(tp, bsdf_eval(mu, gu.n, wh, wv)) * (chu * chH / hd2);
                                Le = emitted(S, H, -wh);
                                ph = light_pdf(S, H.tri);
                                rev0 = bsdf_pdf(mu, gu.n, wv, wh) * chH / hd2;
                            }
                            float Rh = B.rhat[so + k];
                            float3 c = mul(mul(beta, tp), Le) * (Rh / (ph * (float)P.M_p * Q * pi_pix));
                            if (maxc(c) > 0.0f) {
                                float revm1 = bsdf_pdf(mz, z.n, we, wY) * cY / d2;
                                float ms = mis_cell(T, u, Sp, C);
                                float w = 0.0f;
                                if (ms > 0.0f) {
                                    float p0r, p1r = 0.0f;   // p_0 / p^ and p_1 / p^
                                    if (type == 0) {
                                        p0r = revm1 / (pi_pix * ms);
                                    } else {
                                        p0r = revm1 * rev0 / (ph * pi_pix * ms);
                                        p1r = revm1 / (pi_pix * ms);
                                    }
                                    w = 1.0f / (1.0f + p0r + p1r);
                                }
                                if (P.film != 2) L = L + c * w;
                                n_proxy_ok++;
                                if (P.smpp.raw) {   // a training sample of the proxy network
                                    unsigned int idx = atomicAdd(P.smpp.count, 1u);
                                    if (idx < (unsigned int)P.smpp.cap) {
                                        mlp_raw(S, z, we, P.smpp.raw + (size_t)MLP_NRAW * idx);
                                        P.smpp.T[idx] = Tl;
                                        P.smpp.S[idx] = Ssel;
                                        // the estimate R is signed; the proposal's training target is not
                                        P.smpp.w[idx] = fmaxf(lum(c), 0.0f);
                                    }
                                }
                                if (P.acc.proxy) {
                                    atomicAdd(&P.acc.tile_all[tile], lum(c) * w);
                                    atomicAdd(&P.acc.tile_proxy[tile], lum(c) * w);
                                    atomicAdd(&P.acc.proxy[(size_t)Tl * T.KSp + Ssel], lum(c));
                                }
                            }
                        }
                    }
                }
            }
        }
        // ---- proxy-shape tracking for later PT / NEE weights
        if (pstate == 0) {
            if (nonS) {
                pstate = 1;
                f_idx = a;
            }
        } else if (pstate == 1) {
            if (!nonS) {
                if (a == f_idx + 1) {
                    rev_f1 = rev_a;
                    Sp_f1 = P.proxy ? label_spec(S, T, z) : 0;
                }
            } else {
                pstate = (a - f_idx - 1 >= 1) ? 2 : 3;
            }
        } else if (pstate == 2) {
            pstate = 3;
        }
        // ---- continue the eye sub-path
        if (a + 1 > P.max_depth) break;
        float3 wl;
        if (!bsdf_sample(mz, z.n, we, R.u(0), R.u(1), R.u(2), wl)) break;
        float pw = bsdf_pdf(mz, z.n, we, wl);
        if (!(pw > 0.0f)) break;
        beta = mul(beta, bsdf_eval(mz, z.n, wl, we)) * (fabsf(dot(z.n, wl)) / pw);
        // shift history
        nonS_ppp = zpp.nonS;
        zpp = zp;
        zp.p = z.p;
        zp.n = z.n;
        zp.we = we;
        zp.mat = z.mat;
        zp.nonS = nonS;
        zp.rev = rev_a;
        d = wl;
        h = replay ? stored_hit(P, slot, a + 1, pix) : closest_hit<COUNT>(S, z.p, d, z.tri, &tc);
        ++a;
    }
    if (!SHADE) return;
    size_t o = (size_t)slot * P.npix + pix;
    Lbuf[o] = make_float4(L.x, L.y, L.z, 0.0f);
    if (sigbuf) sigbuf[o] = sig;
    if (n_conn) atomicAdd(&B.counters[CNT_CONN], n_conn);
    if (n_proxy) atomicAdd(&B.counters[CNT_PROXY], n_proxy);
    if (n_proxy_ok) atomicAdd(&B.counters[CNT_PROXY_OK], n_proxy_ok);
    if (COUNT) {
        atomicAdd(&B.counters[CNT_EYE_NODES], (unsigned long long)tc.nodes);
        atomicAdd(&B.counters[CNT_EYE_TRIS], (unsigned long long)tc.tris);
        atomicAdd(&B.counters[CNT_EYE_RAYS], (unsigned long long)tc.rays);
    }
}

// Feature pass of the learned proposal: the same camera sub-paths as k_eye
// (the walk uses only the BSDF dimensions 0-2, never a connection's
// choice). Stores every vertex's hit for k_eye to replay, and appends the
// network's input row, eye subspace and dense index of every vertex where
// k_eye makes a subspace connection (row order is arbitrary; each row's
// result depends on its own content only).
template <bool COUNT>
__global__ void __launch_bounds__(128, 8) k_eye_feat(DScene S, DTables T, KParams P, Pool B, uint32_t iter_base) {
    iter_base = eff_iter(P, iter_base);
    TravCount tc{0, 0, 0};
    int pix = blockIdx.x * blockDim.x + threadIdx.x;
    int slot = blockIdx.y;
    if (pix >= P.npix) return;
    uint32_t it = iter_base + (uint32_t)slot;
    int px = pix % S.W, py = pix / S.W;
    Rng r0;
    r0.init(P.seed, K_CAMERA, it, (uint32_t)pix, 0);
    float j0 = r0.u(0), j1 = r0.u(1);
    float sx = 2.0f * ((float)px + j0) / (float)S.W - 1.0f, sy = 1.0f - 2.0f * ((float)py + j1) / (float)S.H;
    float3 d = normalize(S.cfwd + (S.cright * (sx * S.tanh_ * S.aspect) + S.cup * (sy * S.tanh_)));
    Hit h = closest_hit<COUNT>(S, S.cpos, d, -1, &tc);
    int a = 1;
    bool conn = P.conn && B.npool[slot] > 0;
    // a row of the proxy network at the first non-specular vertex where the eye
    // pass draws a proxy (the tile's coin, camera dimension 8)
    bool proxy_row = P.mlpp.rows && P.proxy && B.nent[slot] > 0;
    const float pi_pix = T.pi[(py / T.tile) * T.gw + (px / T.tile)];
    while (true) {
        P.mlp.hits[((size_t)slot * P.max_depth + (a - 1)) * P.npix + pix] =
            make_int4(h.tri, __float_as_int(h.t), __float_as_int(h.b1), __float_as_int(h.b2));
        if (h.tri < 0) break;
        Vtx z = vertex_at(S, h.tri, h.b1, h.b2);
        const DMat &mz = S.mats[z.mat];
        float3 we = -d;
        if (absorbing(S, z, we)) break;
        if (proxy_row && !mz.specular) {
            proxy_row = false;   // only the first non-specular vertex
            Rng Rc;
            Rc.init(P.seed, K_CAMERA, it, (uint32_t)pix, (uint32_t)a);
            if (pi_pix > 0.0f && a + 2 <= P.max_depth && Rc.u(8) < pi_pix) {
                int Tl = label_dir(S, z, we, T.KT, T.cT);
                cg::coalesced_group g = cg::coalesced_threads();
                unsigned int base = 0;
                if (g.thread_rank() == 0) base = atomicAdd(P.mlpp.count, (unsigned int)g.size());
                unsigned int idx = g.shfl(base, 0) + g.thread_rank();
                if (idx < (unsigned int)P.mlpp.cap) {
                    float raw[MLP_NRAW];
                    mlp_raw(S, z, we, raw);
                    mlp_pack_row(raw, Tl, P.mlpp.emb, P.mlpp.rows + (size_t)MLP_NX * idx);
                    P.mlpp.rowT[idx] = Tl;
                    P.mlpp.rowPos[idx] = (int32_t)(((size_t)slot * P.mlpp.A + (a - 1)) * P.npix + pix);
                }
            }
        }
        if (conn && P.mlp.rows && !mz.specular && a + 2 <= P.max_depth) {
            int Tl = label_dir(S, z, we, T.KT, T.cT);
            cg::coalesced_group g = cg::coalesced_threads();
            unsigned int base = 0;
            if (g.thread_rank() == 0) base = atomicAdd(P.mlp.count, (unsigned int)g.size());
            unsigned int idx = g.shfl(base, 0) + g.thread_rank();
            if (idx < (unsigned int)P.mlp.cap) {
                float raw[MLP_NRAW];
                mlp_raw(S, z, we, raw);
                mlp_pack_row(raw, Tl, P.mlp.emb, P.mlp.rows + (size_t)MLP_NX * idx);
                P.mlp.rowT[idx] = Tl;
                P.mlp.rowPos[idx] = (int32_t)(((size_t)slot * P.mlp.A + (a - 1)) * P.npix + pix);
            }
        }
        if (a + 1 > P.max_depth) break;
        Rng R;
        R.init(P.seed, K_CAMERA, it, (uint32_t)pix, (uint32_t)a);
        float3 wl;
        if (!bsdf_sample(mz, z.n, we, R.u(0), R.u(1), R.u(2), wl)) break;
        float pw = bsdf_pdf(mz, z.n, we, wl);
        if (!(pw > 0.0f)) break;
        d = wl;
        h = closest_hit<COUNT>(S, z.p, d, z.tri, &tc);
        ++a;
    }
    if (COUNT) {
        atomicAdd(&B.counters[CNT_CAM_NODES], (unsigned long long)tc.nodes);
        atomicAdd(&B.counters[CNT_CAM_TRIS], (unsigned long long)tc.tris);
        atomicAdd(&B.counters[CNT_CAM_RAYS], (unsigned long long)tc.rays);
    }
}

// answers of the eye pass's occlusion queries: one query per thread, the
// same traversal as the inline test, nothing else in the kernel
template <bool COUNT>
__global__ void __launch_bounds__(128) k_eye_occ(DScene S, KParams P, unsigned long long *counters) {
    const unsigned int n = min(*P.q.count, (unsigned int)P.q.cap);
    TravCount tc{0, 0, 0};
    for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 a = P.q.qa[i], b = P.q.qb[i];
        const bool occ = occluded<COUNT>(S, xyz(a), xyz(b), __float_as_int(a.w), __float_as_int(b.w), &tc);
        const int32_t d = P.q.dst[i];
        P.q.vis[(size_t)(d & 3) * P.q.plane + (size_t)(d >> 2)] = occ ? 0 : 1;
    }
    if (COUNT) {
        atomicAdd(&counters[CNT_SHD_NODES], (unsigned long long)tc.nodes);
        atomicAdd(&counters[CNT_SHD_TRIS], (unsigned long long)tc.tris);
        atomicAdd(&counters[CNT_SHD_RAYS], (unsigned long long)tc.rays);
    }
}

// The occlusion answers on persistent warps (KParams.trace = 1): a lane whose
// traversal ends takes the next query from a counter, and every trip advances
// each busy lane by up to PT_STEPS node visits. Each query is traversed node
// for node as in k_eye_occ, so the answers are identical.
template <bool COUNT>
__global__ void __launch_bounds__(128) k_eye_occ_pt(DScene S, KParams P, unsigned long long *counters,
                                                    unsigned int *fetch) {
    const unsigned FULL = 0xffffffffu;
    const unsigned int n = min(*P.q.count, (unsigned int)P.q.cap);
    TravCount tc{0, 0, 0};
    const TravView V = trav_view(S);
    const int lane = threadIdx.x & 31;
    int q = -1;
    bool drained = false;
    PtRay r;
    for (;;) {
        const bool need = q < 0 && !drained;
        const unsigned m = __ballot_sync(FULL, need);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned int base = 0;
            if (lane == leader) base = atomicAdd(fetch, (unsigned int)__popc(m));
            base = __shfl_sync(FULL, base, leader);
            if (need) {
                const unsigned int k = base + (unsigned int)__popc(m & ((1u << lane) - 1u));
                if (k < n) {
                    q = (int)k;
                    const float4 a = P.q.qa[k], b = P.q.qb[k];
                    r.o = xyz(a);
                    r.d = xyz(b) - r.o;
                    r.inv = safe_inv(r.d);
                    r.s1 = __float_as_int(a.w);
                    r.s2 = __float_as_int(b.w);
                    r.kind = 2;
                    r.node = 0;
                    r.trail = 0ull;
                    r.steps = 0;
                    r.h.tri = -1;
                    r.h.t = INFINITY;
                    r.h.b1 = r.h.b2 = 0.0f;
                    if (COUNT) tc.rays++;
                } else {
                    drained = true;
                }
            }
        }
        if (!__any_sync(FULL, q >= 0)) {
            if (__all_sync(FULL, drained)) break;
            continue;
        }
        if (q >= 0) {
            for (int st = 0; st < PT_STEPS; ++st) {
                if (pt_step<COUNT>(V, r, &tc)) {
                    const int32_t d = P.q.dst[q];
                    P.q.vis[(size_t)(d & 3) * P.q.plane + (size_t)(d >> 2)] = r.h.tri >= 0 ? 0 : 1;
                    q = -1;
                    break;
                }
            }
        }
    }
    if (COUNT) {
        atomicAdd(&counters[CNT_SHD_NODES], (unsigned long long)tc.nodes);
        atomicAdd(&counters[CNT_SHD_TRIS], (unsigned long long)tc.tris);
        atomicAdd(&counters[CNT_SHD_RAYS], (unsigned long long)tc.rays);
    }
}

__global__ void k_film_add(KParams P, int slots, const float4 *Lbuf, float *film) {
    int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= P.npix) return;
    float r = film[3 * (size_t)pix], g = film[3 * (size_t)pix + 1], b = film[3 * (size_t)pix + 2];
    for (int s = 0; s < slots; ++s) {
        float4 v = Lbuf[(size_t)s * P.npix + pix];
        r += v.x;
        g += v.y;
        b += v.z;
    }
    film[3 * (size_t)pix] = r;
    film[3 * (size_t)pix + 1] = g;
    film[3 * (size_t)pix + 2] = b;
}

}  // namespace

void launch_eye(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots, uint32_t iter_base,
                float4 *Lbuf, uint32_t *sigbuf, cudaStream_t st, int mode) {
    dim3 grid((P.npix + 127) / 128, slots);
    if (mode == EYE_EMIT) {   // traversal counts come from k_eye_occ
        k_eye<false, EYE_EMIT><<<grid, 128, 0, st>>>(S, T, P, B, iter_base, Lbuf, sigbuf);
    } else if (mode == EYE_READ) {
        if (P.count) k_eye<true, EYE_READ><<<grid, 128, 0, st>>>(S, T, P, B, iter_base, Lbuf, sigbuf);
        else k_eye<false, EYE_READ><<<grid, 128, 0, st>>>(S, T, P, B, iter_base, Lbuf, sigbuf);
    } else {
        if (P.count) k_eye<true, EYE_INLINE><<<grid, 128, 0, st>>>(S, T, P, B, iter_base, Lbuf, sigbuf);
        else k_eye<false, EYE_INLINE><<<grid, 128, 0, st>>>(S, T, P, B, iter_base, Lbuf, sigbuf);
    }
}

void launch_eye_occ(const DScene &S, const KParams &P, const Pool &B, int num_sms, cudaStream_t st,
                    unsigned int *fetch) {
    if (P.trace && fetch) {
        cudaMemsetAsync(fetch, 0, sizeof(unsigned int), st);
        if (P.count) k_eye_occ_pt<true><<<num_sms * 8, 128, 0, st>>>(S, P, B.counters, fetch);
        else k_eye_occ_pt<false><<<num_sms * 8, 128, 0, st>>>(S, P, B.counters, fetch);
        return;
    }
    const int blocks = std::max(1, std::min(num_sms * 16, (P.q.cap + 127) / 128));
    if (P.count) k_eye_occ<true><<<blocks, 128, 0, st>>>(S, P, B.counters);
    else k_eye_occ<false><<<blocks, 128, 0, st>>>(S, P, B.counters);
}

// The feature pass stays one camera path per thread for either trace mode: a
// persistent variant that refilled lanes with new paths (and batched their
// vertex steps) measured 167 ms against 140 ms on the 1024^2 glossy step, as
// refilled lanes lose the coherence of neighbouring camera paths.
void launch_eye_feat(const DScene &S, const DTables &T, const KParams &P, const Pool &B, int slots, uint32_t iter_base,
                     cudaStream_t st) {
    dim3 grid((P.npix + 127) / 128, slots);
    if (P.count) k_eye_feat<true><<<grid, 128, 0, st>>>(S, T, P, B, iter_base);
    else k_eye_feat<false><<<grid, 128, 0, st>>>(S, T, P, B, iter_base);
}

void launch_film_add(const KParams &P, int slots, const float4 *Lbuf, float *film, cudaStream_t st) {
    k_film_add<<<(P.npix + 255) / 256, 256, 0, st>>>(P, slots, Lbuf, film);
}
