/* CPU oracle (test infrastructure only): scene, brute-force ray queries,
 * emitters and the pinhole camera. Closest hit is the plain definition:
 * the smallest t over every triangle (Moller-Trumbore in double), ties to
 * the lower triangle index. */
#include <stdio.h>

#include "or_internal.h"

static double clampd(double x, double a, double b) { return x < a ? a : (x > b ? b : x); }
static void bvh_init(or_scene_t *s);

int or_scene_init(or_scene_t *s, const or_scene_desc *d) {
    memset(s, 0, sizeof(*s));
    s->nv = d->nv;
    s->nt = d->nt;
    s->nm = d->nm;
    s->P = (v3 *)malloc(sizeof(v3) * (size_t)d->nv);
    s->UV = (double *)malloc(sizeof(double) * 2 * (size_t)d->nv);
    s->T = (int *)malloc(sizeof(int) * 3 * (size_t)d->nt);
    s->tm = (int *)malloc(sizeof(int) * (size_t)d->nt);
    s->N = (v3 *)malloc(sizeof(v3) * (size_t)d->nt);
    s->area = (double *)malloc(sizeof(double) * (size_t)d->nt);
    s->mats = (or_mat *)malloc(sizeof(or_mat) * (size_t)d->nm);
    s->tri2e = (int *)malloc(sizeof(int) * (size_t)d->nt);
    for (int i = 0; i < d->nv; ++i) {
        s->P[i] = v3m(d->verts[3 * i], d->verts[3 * i + 1], d->verts[3 * i + 2]);
        s->UV[2 * i] = d->uvs ? d->uvs[2 * i] : 0.0;
        s->UV[2 * i + 1] = d->uvs ? d->uvs[2 * i + 1] : 0.0;
    }
    for (int m = 0; m < d->nm; ++m) {
        const float *r = d->mats + 12 * m;
        or_mat *M = &s->mats[m];
        M->kind = (int)r[0];
        M->color = v3m(r[1], r[2], r[3]);
        M->rough = r[4];
        M->alpha = (double)r[4] * (double)r[4];
        M->ior = r[5];
        M->Le = v3m(r[6], r[7], r[8]);
        M->textured = r[9] != 0.0f;
        M->specular = (M->kind != MK_LAMBERT) && (r[4] < 0.2f);
        M->emitter = vsumc(M->Le) > 0.0;
    }
    s->lo = v3m(1e300, 1e300, 1e300);
    s->hi = v3m(-1e300, -1e300, -1e300);
    for (int i = 0; i < d->nv; ++i) {
        v3 p = s->P[i];
        s->lo = v3m(fmin(s->lo.x, p.x), fmin(s->lo.y, p.y), fmin(s->lo.z, p.z));
        s->hi = v3m(fmax(s->hi.x, p.x), fmax(s->hi.y, p.y), fmax(s->hi.z, p.z));
    }
    v3 ext = vsub(s->hi, s->lo);
    s->extent = vmaxc(ext);
    s->eps_t = 1e-5 * s->extent;
    double wsum = 0.0;
    s->ne = 0;
    for (int t = 0; t < d->nt; ++t) {
        for (int k = 0; k < 3; ++k) s->T[3 * t + k] = d->tris[3 * t + k];
        s->tm[t] = d->tri_mat[t];
        v3 p0 = s->P[s->T[3 * t]], p1 = s->P[s->T[3 * t + 1]], p2 = s->P[s->T[3 * t + 2]];
        v3 c = vcross(vsub(p1, p0), vsub(p2, p0));
        double l = vlen(c);
        s->area[t] = 0.5 * l;
        s->N[t] = l > 0 ? vscale(c, 1.0 / l) : v3m(0, 0, 1);
        s->tri2e[t] = -1;
        if (s->mats[s->tm[t]].emitter && s->area[t] > 0) s->ne++;
    }
    s->etri = (int *)malloc(sizeof(int) * (size_t)(s->ne + 1));
    s->ecdf = (double *)malloc(sizeof(double) * (size_t)(s->ne + 1));
    s->epmf = (double *)malloc(sizeof(double) * (size_t)(s->ne + 1));
    int e = 0;
    for (int t = 0; t < d->nt; ++t) {
        const or_mat *M = &s->mats[s->tm[t]];
        if (!(M->emitter && s->area[t] > 0)) continue;
        s->etri[e] = t;
        s->tri2e[t] = e;
        double w = s->area[t] * vsumc(M->Le);
        wsum += w;
        s->ecdf[e] = wsum;
        s->epmf[e] = w;
        ++e;
    }
    for (e = 0; e < s->ne; ++e) {
        s->ecdf[e] /= wsum;
        s->epmf[e] /= wsum;
    }
    if (s->ne > 0) s->ecdf[s->ne - 1] = 1.0;
    s->tw = d->tex_w;
    s->th = d->tex_h;
    s->tex = d->tex;
    const float *c = d->cam;
    s->cpos = v3m(c[0], c[1], c[2]);
    s->cfwd = vnorm(vsub(v3m(c[3], c[4], c[5]), s->cpos));
    s->cright = vnorm(vcross(s->cfwd, v3m(c[6], c[7], c[8])));
    s->cup = vcross(s->cright, s->cfwd);
    s->tanh_ = tan(0.5 * (double)c[9] * M_PI / 180.0);
    s->W = (int)c[10];
    s->H = (int)c[11];
    s->aspect = (double)s->W / (double)s->H;
    bvh_init(s);
    return 0;
}

void or_scene_free(or_scene_t *s) {
    free(s->P); free(s->UV); free(s->T); free(s->tm); free(s->N); free(s->area);
    free(s->mats); free(s->tri2e); free(s->etri); free(s->ecdf); free(s->epmf);
    free(s->blo); free(s->bhi); free(s->bl); free(s->br); free(s->bfirst); free(s->bcount); free(s->order);
}

void or_set_brute(void *h, int brute) { ((or_scene_t *)h)->brute = brute; }

/* Moller-Trumbore; returns 1 and (t, b1, b2) if the line o + t d meets the
 * closed triangle. */
static int tri_hit(const or_scene_t *s, int t, v3 o, v3 d, double *tt, double *b1, double *b2) {
    v3 p0 = s->P[s->T[3 * t]], p1 = s->P[s->T[3 * t + 1]], p2 = s->P[s->T[3 * t + 2]];
    v3 e1 = vsub(p1, p0), e2 = vsub(p2, p0);
    v3 pv = vcross(d, e2);
    double det = vdot(e1, pv);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    v3 tv = vsub(o, p0);
    double u = vdot(tv, pv) * inv;
    if (u < 0.0 || u > 1.0) return 0;
    v3 qv = vcross(tv, e1);
    double v = vdot(d, qv) * inv;
    if (v < 0.0 || u + v > 1.0) return 0;
    *tt = vdot(e2, qv) * inv;
    *b1 = u;
    *b2 = v;
    return 1;
}


/* ---- bounding-volume hierarchy (acceleration only) ------------------------ */
static const or_scene_t *g_sort_scene;
static int g_sort_axis;
static double centroid_axis(const or_scene_t *s, int t, int ax) {
    double c = 0.0;
    for (int k = 0; k < 3; ++k) {
        v3 p = s->P[s->T[3 * t + k]];
        c += ax == 0 ? p.x : (ax == 1 ? p.y : p.z);
    }
    return c;
}
static int cmp_centroid(const void *a, const void *b) {
    int ta = *(const int *)a, tb = *(const int *)b;
    double ca = centroid_axis(g_sort_scene, ta, g_sort_axis), cb = centroid_axis(g_sort_scene, tb, g_sort_axis);
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return ta - tb;
}
static int bvh_build(or_scene_t *s, int first, int count) {
    int id = s->nnodes++;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    double clo[3] = {1e300, 1e300, 1e300}, chi[3] = {-1e300, -1e300, -1e300};
    for (int i = first; i < first + count; ++i) {
        int t = s->order[i];
        for (int k = 0; k < 3; ++k) {
            v3 p = s->P[s->T[3 * t + k]];
            double c[3] = {p.x, p.y, p.z};
            for (int a = 0; a < 3; ++a) { lo[a] = fmin(lo[a], c[a]); hi[a] = fmax(hi[a], c[a]); }
        }
        for (int a = 0; a < 3; ++a) {
            double c = centroid_axis(s, t, a);
            clo[a] = fmin(clo[a], c); chi[a] = fmax(chi[a], c);
        }
    }
    double pad = 1e-9 * (s->extent > 0 ? s->extent : 1.0);
    for (int a = 0; a < 3; ++a) { s->blo[3 * id + a] = lo[a] - pad; s->bhi[3 * id + a] = hi[a] + pad; }
    s->bl[id] = s->br[id] = -1;
    s->bfirst[id] = first;
    s->bcount[id] = count;
    if (count <= 4) return id;
    int ax = 0;
    for (int a = 1; a < 3; ++a) if (chi[a] - clo[a] > chi[ax] - clo[ax]) ax = a;
    g_sort_scene = s;
    g_sort_axis = ax;
    qsort(s->order + first, (size_t)count, sizeof(int), cmp_centroid);
    int half = count / 2;
    s->bcount[id] = 0;
    int l = bvh_build(s, first, half);
    int r = bvh_build(s, first + half, count - half);
    s->bl[id] = l;
    s->br[id] = r;
    return id;
}
static void bvh_init(or_scene_t *s) {
    int cap = 2 * (s->nt > 0 ? s->nt : 1);
    s->blo = (double *)malloc(sizeof(double) * 3 * (size_t)cap);
    s->bhi = (double *)malloc(sizeof(double) * 3 * (size_t)cap);
    s->bl = (int *)malloc(sizeof(int) * (size_t)cap);
    s->br = (int *)malloc(sizeof(int) * (size_t)cap);
    s->bfirst = (int *)malloc(sizeof(int) * (size_t)cap);
    s->bcount = (int *)malloc(sizeof(int) * (size_t)cap);
    s->order = (int *)malloc(sizeof(int) * (size_t)(s->nt > 0 ? s->nt : 1));
    for (int t = 0; t < s->nt; ++t) s->order[t] = t;
    s->nnodes = 0;
    if (s->nt > 0) bvh_build(s, 0, s->nt);
}
/* does o + t d, t in [t0, t1], meet box id? (conservative slab test) */
static int box_hit(const or_scene_t *s, int id, v3 o, v3 d, double t0, double t1) {
    double oc[3] = {o.x, o.y, o.z}, dc[3] = {d.x, d.y, d.z};
    for (int a = 0; a < 3; ++a) {
        double lo = s->blo[3 * id + a], hi = s->bhi[3 * id + a];
        if (dc[a] == 0.0) {
            if (oc[a] < lo || oc[a] > hi) return 0;
            continue;
        }
        double ta = (lo - oc[a]) / dc[a], tb = (hi - oc[a]) / dc[a];
        if (ta > tb) { double x = ta; ta = tb; tb = x; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1 * (1.0 + 1e-12) + 1e-300) return 0;
    }
    return 1;
}

static void consider(const or_scene_t *s, int t, v3 o, v3 d, or_hit *h) {
    double tt, b1, b2;
    if (!tri_hit(s, t, o, d, &tt, &b1, &b2)) return;
    if (!(tt > s->eps_t)) return;
    if (tt < h->t || (tt == h->t && t < h->tri)) {
        h->tri = t; h->t = tt; h->b1 = b1; h->b2 = b2;
    }
}

or_hit or_closest(const or_scene_t *s, v3 o, v3 d, int skip) {
    if (!s->brute && s->nnodes > 0) {
        or_hit h = {-1, INFINITY, 0, 0};
        int stack[128], sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            int id = stack[--sp];
            if (!box_hit(s, id, o, d, 0.0, h.t)) continue;
            if (s->bl[id] < 0) {
                for (int i = s->bfirst[id]; i < s->bfirst[id] + s->bcount[id]; ++i)
                    if (s->order[i] != skip) consider(s, s->order[i], o, d, &h);
            } else {
                stack[sp++] = s->bl[id];
                stack[sp++] = s->br[id];
            }
        }
        return h;
    }
    return or_closest_brute(s, o, d, skip);
}

or_hit or_closest_brute(const or_scene_t *s, v3 o, v3 d, int skip) {
    or_hit h = {-1, INFINITY, 0, 0};
    for (int t = 0; t < s->nt; ++t) {
        if (t == skip) continue;
        double tt, b1, b2;
        if (!tri_hit(s, t, o, d, &tt, &b1, &b2)) continue;
        if (!(tt > s->eps_t)) continue;
        if (tt < h.t || (tt == h.t && t < h.tri)) {
            h.tri = t; h.t = tt; h.b1 = b1; h.b2 = b2;
        }
    }
    return h;
}

int or_occluded(const or_scene_t *s, v3 a, v3 b, int skip_a, int skip_b) {
    v3 d = vsub(b, a);
    if (!s->brute && s->nnodes > 0) {
        int stack[128], sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            int id = stack[--sp];
            if (!box_hit(s, id, a, d, 0.0, 1.0)) continue;
            if (s->bl[id] < 0) {
                for (int i = s->bfirst[id]; i < s->bfirst[id] + s->bcount[id]; ++i) {
                    int t = s->order[i];
                    if (t == skip_a || t == skip_b) continue;
                    double tt, b1, b2;
                    if (tri_hit(s, t, a, d, &tt, &b1, &b2) && tt > 1e-4 && tt < 1.0 - 1e-4) return 1;
                }
            } else {
                stack[sp++] = s->bl[id];
                stack[sp++] = s->br[id];
            }
        }
        return 0;
    }
    for (int t = 0; t < s->nt; ++t) {
        if (t == skip_a || t == skip_b) continue;
        double tt, b1, b2;
        if (!tri_hit(s, t, a, d, &tt, &b1, &b2)) continue;
        if (tt > 1e-4 && tt < 1.0 - 1e-4) return 1;
    }
    return 0;
}

or_vtx or_vertex_at(const or_scene_t *s, int tri, double b1, double b2) {
    or_vtx v;
    v3 p0 = s->P[s->T[3 * tri]], p1 = s->P[s->T[3 * tri + 1]], p2 = s->P[s->T[3 * tri + 2]];
    v.p = vadd(p0, vadd(vscale(vsub(p1, p0), b1), vscale(vsub(p2, p0), b2)));
    v.n = s->N[tri];
    v.tri = tri;
    v.mat = s->tm[tri];
    v.is_light = 0;
    v.b1 = b1;
    v.b2 = b2;
    return v;
}

static v3 tex_lookup(const or_scene_t *s, double u, double v) {
    if (!s->tex || s->tw <= 0) return v3m(1, 1, 1);
    double x = u * s->tw - 0.5, y = v * s->th - 0.5;
    double x0 = floor(x), y0 = floor(y);
    double fx = x - x0, fy = y - y0;
    int ix0 = (int)clampd(x0, 0, s->tw - 1), ix1 = (int)clampd(x0 + 1, 0, s->tw - 1);
    int iy0 = (int)clampd(y0, 0, s->th - 1), iy1 = (int)clampd(y0 + 1, 0, s->th - 1);
    double r[3];
    for (int k = 0; k < 3; ++k) {
        double a = s->tex[((size_t)iy0 * s->tw + ix0) * 3 + k];
        double b = s->tex[((size_t)iy0 * s->tw + ix1) * 3 + k];
        double c = s->tex[((size_t)iy1 * s->tw + ix0) * 3 + k];
        double e = s->tex[((size_t)iy1 * s->tw + ix1) * 3 + k];
        r[k] = (a * (1 - fx) + b * fx) * (1 - fy) + (c * (1 - fx) + e * fx) * fy;
    }
    return v3m(r[0], r[1], r[2]);
}

v3 or_emitted(const or_scene_t *s, const or_vtx *v, v3 w) {
    const or_mat *M = &s->mats[v->mat];
    if (!M->emitter || vdot(v->n, w) <= 0.0) return v3m(0, 0, 0);
    if (!M->textured) return M->Le;
    int i0 = s->T[3 * v->tri], i1 = s->T[3 * v->tri + 1], i2 = s->T[3 * v->tri + 2];
    double b0 = 1.0 - v->b1 - v->b2;
    double u = b0 * s->UV[2 * i0] + v->b1 * s->UV[2 * i1] + v->b2 * s->UV[2 * i2];
    double vv = b0 * s->UV[2 * i0 + 1] + v->b1 * s->UV[2 * i1 + 1] + v->b2 * s->UV[2 * i2 + 1];
    return vmul(M->Le, tex_lookup(s, u, vv));
}

double or_light_pdf(const or_scene_t *s, int tri) {
    int e = (tri >= 0) ? s->tri2e[tri] : -1;
    if (e < 0) return 0.0;
    return s->epmf[e] / s->area[tri];
}

int or_sample_light(const or_scene_t *s, double u0, double u1, double u2, int *tri, double *b1,
                    double *b2) {
    if (s->ne == 0) return 0;
    int e = 0;
    while (e < s->ne - 1 && !(u0 < s->ecdf[e])) ++e;
    *tri = s->etri[e];
    double su = sqrt(u1);
    *b1 = su * (1.0 - u2);
    *b2 = su * u2;
    return 1;
}

/* Orthonormal basis around unit n (Duff et al., JCGT 2017). */
void or_onb(v3 n, v3 *t, v3 *b) {
    double sign = copysign(1.0, n.z);
    double a = -1.0 / (sign + n.z);
    double bb = n.x * n.y * a;
    *t = v3m(1.0 + sign * n.x * n.x * a, sign * bb, -sign * n.x);
    *b = v3m(bb, sign + n.y * n.y * a, -n.y);
}

/* cosine-weighted direction about unit n: pdf cos/pi */
v3 or_cosine_dir(v3 n, double u1, double u2) {
    double r = sqrt(u1), ph = 2.0 * M_PI * u2;
    double z = sqrt(fmax(0.0, 1.0 - u1));
    v3 t, b;
    or_onb(n, &t, &b);
    return vadd(vadd(vscale(t, r * cos(ph)), vscale(b, r * sin(ph))), vscale(n, z));
}

int or_is_specular(const or_scene_t *s, int tri) { return s->mats[s->tm[tri]].specular; }

/* A vertex that ends every light or eye sub-path reaching it: a black
 * Lambert surface, or a conductor seen from its back side. w_in points from
 * the vertex toward where the path came from. */
int or_absorbing(const or_scene_t *s, const or_vtx *v, v3 w_in) {
    const or_mat *M = &s->mats[v->mat];
    if (M->kind == MK_LAMBERT) return vmaxc(M->color) <= 0.0;
    if (M->kind == MK_CONDUCTOR) return vdot(v->n, w_in) <= 0.0;
    return 0;
}

void or_closest_batch(void *h, int n, const double *rays, double *out) {
    const or_scene_t *s = (const or_scene_t *)h;
    for (int i = 0; i < n; ++i) {
        const double *r = rays + 7 * i;
        or_hit hh = or_closest(s, v3m(r[0], r[1], r[2]), v3m(r[3], r[4], r[5]), (int)r[6]);
        out[4 * i] = hh.tri;
        out[4 * i + 1] = hh.tri >= 0 ? hh.t : -1.0;
        out[4 * i + 2] = hh.b1;
        out[4 * i + 3] = hh.b2;
    }
}

void or_occluded_batch(void *h, int n, const double *seg, int *out) {
    const or_scene_t *s = (const or_scene_t *)h;
    for (int i = 0; i < n; ++i) {
        const double *r = seg + 8 * i;
        out[i] = or_occluded(s, v3m(r[0], r[1], r[2]), v3m(r[3], r[4], r[5]), (int)r[6], (int)r[7]);
    }
}
