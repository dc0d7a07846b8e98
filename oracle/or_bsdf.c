/* CPU oracle (test infrastructure only): materials.
 *
 * The paper renders its specular class with the Disney principled BSDF at
 * roughness 0.01 and calls a conductor or dielectric with roughness < 0.2
 * specular (Sec. 1 footnote, Sec. 6.1.1). Here: two-sided Lambert, a
 * one-sided GGX conductor (Schlick Fresnel), and a two-sided GGX rough
 * dielectric (Walter, Marschner, Li, Torrance, EGSR 2007: D, separable
 * Smith G1, exact unpolarised Fresnel, the refraction half vector and
 * Jacobian of their Eqs. 16-17 and 20-21). alpha = roughness^2.
 *
 * eval(w_light, w_eye) is the radiance BSDF rho(x_{i-1}, x_i, x_{i+1}) of the
 * path integral (Sec. 3.1): light arrives from w_light and leaves toward
 * w_eye. pdf(w_g, w_s) is the solid-angle density of the sampling routine
 * that draws w_s given w_g; the same routine serves light tracing (given
 * w_light) and eye tracing (given w_eye). */
#include "or_internal.h"

static double ggx_D(double alpha, double cos_h) {
    if (cos_h <= 0.0) return 0.0;
    double a2 = alpha * alpha;
    double c2 = cos_h * cos_h;
    double den = c2 * (a2 - 1.0) + 1.0;
    return a2 / (M_PI * den * den);
}

static double ggx_G1(double alpha, v3 n, v3 v, v3 h) {
    double vn = vdot(v, n), vh = vdot(v, h);
    if (vh * vn <= 0.0) return 0.0;
    double c2 = vn * vn;
    double t2 = (1.0 - c2) / c2;
    return 2.0 / (1.0 + sqrt(1.0 + alpha * alpha * t2));
}

/* microfacet normal drawn with density D(h) cos(theta_h) about n */
static v3 ggx_sample_h(double alpha, v3 n, double u1, double u2) {
    double a2 = alpha * alpha;
    double c2 = (1.0 - u1) / (1.0 + (a2 - 1.0) * u1);
    double c = sqrt(c2), sn = sqrt(fmax(0.0, 1.0 - c2));
    double ph = 2.0 * M_PI * u2;
    v3 t, b;
    or_onb(n, &t, &b);
    return vadd(vadd(vscale(t, sn * cos(ph)), vscale(b, sn * sin(ph))), vscale(n, c));
}

static double fresnel_dielectric(double cos_i, double eta_i, double eta_t) {
    cos_i = fabs(cos_i);
    double s2 = (eta_i / eta_t) * (eta_i / eta_t) * (1.0 - cos_i * cos_i);
    if (s2 >= 1.0) return 1.0;
    double cos_t = sqrt(1.0 - s2);
    double rs = (eta_i * cos_i - eta_t * cos_t) / (eta_i * cos_i + eta_t * cos_t);
    double rp = (eta_t * cos_i - eta_i * cos_t) / (eta_t * cos_i + eta_i * cos_t);
    return 0.5 * (rs * rs + rp * rp);
}

static double side_eta(const or_mat *m, v3 n, v3 w) { return vdot(n, w) > 0.0 ? 1.0 : m->ior; }

v3 or_bsdf_eval(const or_mat *m, v3 n, v3 wl, v3 we) {
    double cl = vdot(n, wl), ce = vdot(n, we);
    v3 zero = v3m(0, 0, 0);
    if (m->kind == MK_LAMBERT) {
        if (cl * ce <= 0.0) return zero;
        return vscale(m->color, 1.0 / M_PI);
    }
    if (m->kind == MK_CONDUCTOR) {
        if (cl <= 0.0 || ce <= 0.0) return zero;
        v3 h = vnorm(vadd(wl, we));
        double D = ggx_D(m->alpha, vdot(n, h));
        double G = ggx_G1(m->alpha, n, wl, h) * ggx_G1(m->alpha, n, we, h);
        double s = pow(1.0 - fmax(0.0, vdot(we, h)), 5.0);
        v3 F = v3m(m->color.x + (1 - m->color.x) * s, m->color.y + (1 - m->color.y) * s,
                   m->color.z + (1 - m->color.z) * s);
        return vscale(F, D * G / (4.0 * cl * ce));
    }
    /* rough dielectric */
    if (cl == 0.0 || ce == 0.0) return zero;
    double eta_l = side_eta(m, n, wl), eta_e = side_eta(m, n, we);
    if (cl * ce > 0.0) {
        v3 h = vnorm(vadd(wl, we));
        if (vdot(n, h) < 0.0) h = vneg(h);
        double D = ggx_D(m->alpha, vdot(n, h));
        double G = ggx_G1(m->alpha, n, wl, h) * ggx_G1(m->alpha, n, we, h);
        double F = fresnel_dielectric(vdot(wl, h), eta_l, eta_l == 1.0 ? m->ior : 1.0);
        double f = F * D * G / (4.0 * fabs(cl) * fabs(ce));
        return v3m(f, f, f);
    }
    v3 h = vneg(vadd(vscale(wl, eta_l), vscale(we, eta_e)));
    double hl = vlen(h);
    if (hl == 0.0) return zero;
    h = vscale(h, 1.0 / hl);
    if (vdot(n, h) < 0.0) h = vneg(h);
    double lh = vdot(wl, h), eh = vdot(we, h);
    double den = eta_l * lh + eta_e * eh;
    if (den == 0.0) return zero;
    double D = ggx_D(m->alpha, vdot(n, h));
    double G = ggx_G1(m->alpha, n, wl, h) * ggx_G1(m->alpha, n, we, h);
    double F = fresnel_dielectric(lh, eta_l, eta_e);
    double f = fabs(lh) * fabs(eh) * eta_e * eta_e * (1.0 - F) * D * G /
               (fabs(cl) * fabs(ce) * den * den);
    return v3m(f, f, f);
}

double or_bsdf_pdf(const or_mat *m, v3 n, v3 wg, v3 ws) {
    double cg = vdot(n, wg), cs = vdot(n, ws);
    if (m->kind == MK_LAMBERT) {
        if (cg * cs <= 0.0) return 0.0;
        return fabs(cs) / M_PI;
    }
    if (m->kind == MK_CONDUCTOR) {
        if (cg <= 0.0 || cs <= 0.0) return 0.0;
        v3 h = vnorm(vadd(wg, ws));
        double sh = vdot(ws, h);
        if (sh <= 0.0) return 0.0;
        return ggx_D(m->alpha, vdot(n, h)) * vdot(n, h) / (4.0 * sh);
    }
    if (cg == 0.0 || cs == 0.0) return 0.0;
    double eta_g = side_eta(m, n, wg), eta_s = side_eta(m, n, ws);
    if (cg * cs > 0.0) {
        v3 h = vnorm(vadd(wg, ws));
        if (vdot(n, h) < 0.0) h = vneg(h);
        if (vdot(wg, h) * cg <= 0.0 || vdot(ws, h) * cs <= 0.0) return 0.0;
        double F = fresnel_dielectric(vdot(wg, h), eta_g, eta_g == 1.0 ? m->ior : 1.0);
        return F * ggx_D(m->alpha, vdot(n, h)) * vdot(n, h) / (4.0 * fabs(vdot(ws, h)));
    }
    v3 h = vneg(vadd(vscale(wg, eta_g), vscale(ws, eta_s)));
    double hl = vlen(h);
    if (hl == 0.0) return 0.0;
    h = vscale(h, 1.0 / hl);
    if (vdot(n, h) < 0.0) h = vneg(h);
    double gh = vdot(wg, h), sh = vdot(ws, h);
    if (gh * cg <= 0.0 || sh * cs <= 0.0) return 0.0;
    double den = eta_g * gh + eta_s * sh;
    if (den == 0.0) return 0.0;
    double F = fresnel_dielectric(gh, eta_g, eta_s);
    return (1.0 - F) * ggx_D(m->alpha, vdot(n, h)) * vdot(n, h) * eta_s * eta_s * fabs(sh) /
           (den * den);
}

int or_bsdf_sample(const or_mat *m, v3 n, v3 wg, double u0, double u1, double u2, v3 *ws) {
    double cg = vdot(n, wg);
    if (m->kind == MK_LAMBERT) {
        if (cg == 0.0) return 0;
        v3 nn = cg > 0.0 ? n : vneg(n);
        *ws = or_cosine_dir(nn, u1, u2);
        return vdot(n, *ws) * cg > 0.0;
    }
    if (m->kind == MK_CONDUCTOR) {
        if (cg <= 0.0) return 0;
        v3 h = ggx_sample_h(m->alpha, n, u1, u2);
        double c = vdot(wg, h);
        if (c <= 0.0) return 0;
        *ws = vsub(vscale(h, 2.0 * c), wg);
        return vdot(n, *ws) > 0.0;
    }
    if (cg == 0.0) return 0;
    v3 h = ggx_sample_h(m->alpha, n, u1, u2);
    v3 hh = cg > 0.0 ? h : vneg(h);
    double c = vdot(wg, hh);
    if (c <= 0.0) return 0;
    double eta_g = cg > 0.0 ? 1.0 : m->ior, eta_o = cg > 0.0 ? m->ior : 1.0;
    double F = fresnel_dielectric(c, eta_g, eta_o);
    if (u0 < F) {
        *ws = vsub(vscale(hh, 2.0 * c), wg);
        return vdot(n, *ws) * cg > 0.0;
    }
    double eta = eta_g / eta_o;
    double s2 = eta * eta * (1.0 - c * c);
    if (s2 >= 1.0) return 0;
    double ct = sqrt(1.0 - s2);
    *ws = vnorm(vadd(vscale(wg, -eta), vscale(hh, eta * c - ct)));
    return vdot(n, *ws) * cg < 0.0;
}

/* exported wrappers for the BSDF pins */
static or_mat mat_from(const float *r) {
    or_mat M;
    M.kind = (int)r[0];
    M.color = v3m(r[1], r[2], r[3]);
    M.rough = r[4];
    M.alpha = (double)r[4] * (double)r[4];
    M.ior = r[5];
    M.Le = v3m(r[6], r[7], r[8]);
    M.textured = r[9] != 0.0f;
    M.specular = M.kind != MK_LAMBERT && r[4] < 0.2f;
    M.emitter = vsumc(M.Le) > 0.0;
    return M;
}

void or_bsdf_eval_x(const float *mat, const double *n, const double *wl, const double *we,
                    double *out3) {
    or_mat M = mat_from(mat);
    v3 f = or_bsdf_eval(&M, v3m(n[0], n[1], n[2]), v3m(wl[0], wl[1], wl[2]), v3m(we[0], we[1], we[2]));
    out3[0] = f.x; out3[1] = f.y; out3[2] = f.z;
}

double or_bsdf_pdf_x(const float *mat, const double *n, const double *wg, const double *ws) {
    or_mat M = mat_from(mat);
    return or_bsdf_pdf(&M, v3m(n[0], n[1], n[2]), v3m(wg[0], wg[1], wg[2]), v3m(ws[0], ws[1], ws[2]));
}

int or_bsdf_sample_x(const float *mat, const double *n, const double *wg, double u0, double u1,
                     double u2, double *ws) {
    or_mat M = mat_from(mat);
    v3 w;
    int ok = or_bsdf_sample(&M, v3m(n[0], n[1], n[2]), v3m(wg[0], wg[1], wg[2]), u0, u1, u2, &w);
    ws[0] = w.x; ws[1] = w.y; ws[2] = w.z;
    return ok;
}
