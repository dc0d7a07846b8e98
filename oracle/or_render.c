/* CPU oracle (test infrastructure only): the render loop.
 *
 * Every contribution is evaluated from its definition. A full path
 * x_0..x_k (x_0 on a light, x_k the camera) is assembled as a vertex list;
 * f(x) is the measurement contribution of Sec. 3.1 (Eq. path intergral):
 * Le(x_0->x_1) * prod rho(x_{j-1}, x_j, x_{j+1}) * prod G(x_j, x_{j+1}), with
 * the camera's W_e G / p(z_1) factor equal to 1 (box-filtered pinhole, the
 * pixel value is mean radiance). Vertex densities follow Eq. tracingPdf:
 *   fwd_j  light-tracer density of x_j (fwd_0 = p_L, fwd_1 = cosine
 *          emission, fwd_j = BSDF pdf at x_{j-1} given x_{j-2}) in area measure;
 *   rev_j  eye-tracer density of x_j (BSDF pdf at x_{j+1} given x_{j+2}),
 *          rev_{k-1} = 1 (shared by every strategy, t >= 2 always).
 * Strategy s (s light vertices, t = k+1-s >= 2 eye vertices) has density
 * p_s = prod_{j<s} fwd_j * prod_{j>=s} rev_j: s=0 eye path hits an emitter,
 * s=1 next-event estimation, s>=2 a subspace connection to a stored light
 * vertex (Sec. 3.2: PCBPT resampling with the SPCBPT two-stage selection,
 * Sec. 5.5). Connections and NEE are made only where both joined vertices
 * are non-specular. The proxy strategy (Sec. 5.1-5.2) applies at the eye
 * path's first non-specular vertex to incomplete light sub-paths of type
 * L S^u or L D S^u, 1 <= u <= 4 (Sec. 6.1.1).
 *
 * MIS (Sec. 5.4, Eq. MIS_1): w_t = (1/(E[1/p~_t^2] p_t)) / sum_i (...). For
 * exact densities this is the balance heuristic on p_s. For the proxy,
 * 1/(E[1/p~^2] p) = p(h*) p_ret p(z) pi / (E[R^2] P), approximated from the
 * frozen per-cell table mis(u,S',C) = 1/(E[R^2] Pbar) (Sec. 5.4-5.5,
 * Eq. subspaceApproximate). Resampled strategies enter the weights with
 * their un-resampled densities (selection factor 1), so every weight is a
 * deterministic function of the path and of frozen tables. */
#include <stdio.h>

#include "or_internal.h"

double or_fwd_density(const or_scene_t *s, const or_vtx *ys, int j);
double or_entry_rhat(const or_scene_t *s, const or_entry *en, double B, double booth, uint32_t seed,
                     uint32_t iteration, uint32_t entry, int repeats, int cap, int split, int fixed,
                     double *nodes, int *trunc, uint32_t *sig);
double or_pilot_B(const or_scene_t *s, const or_entry *en, uint32_t seed, uint32_t iteration, uint32_t entry,
                  int min_draws, int max_draws);

#define MAXV 40
/* B is the largest f/q observed during learning (App. "Optimal value for B":
 * B = max f/q) times this factor. Where the observed maximum falls short of
 * the true one the estimator splits (still unbiased). */
#define B_SAFETY 1.0

typedef struct { or_vtx v[MAXV]; int n; } or_path;

typedef struct {
    int KT, KS, KSp, KC;
    double lo[3], ext[3];
    const float *cT, *cS, *cSp, *cC, *gC, *gP, *Bt, *mis, *pi;
    const double *mlp, *mlp_p;
    int tile, gw, gh;
} or_tab;

typedef struct {
    int n;
    or_vtx v[MAXV];
} or_lpath;

typedef struct {
    int M, M_p;
    or_lpath *lp;
    int npool;
    int *pool_l, *pool_e, *pool_S;
    int *bstart, *bitems;   /* buckets by light subspace */
    int nent;
    or_entry *ent;
    int *ent_l, *ent_e, *ent_Sp, *ent_C;
    double *rhat;
    int *estart, *eitems;   /* buckets by specular subspace */
} or_iter;

typedef struct {
    double *conn, *proxy;          /* KT*KS, KT*KSp: unweighted contribution luminance */
    double *tile_proxy, *tile_all; /* weighted proxy / all contribution luminance */
} learn_acc;

static void tab_init(or_tab *T, const or_tables_desc *t) {
    T->KT = t->KT; T->KS = t->KS; T->KSp = t->KSp; T->KC = t->KC;
    for (int k = 0; k < 3; ++k) {
        T->lo[k] = t->bbox_lo[k];
        double e = (double)t->bbox_hi[k] - (double)t->bbox_lo[k];
        T->ext[k] = e > 0 ? e : 1.0;
    }
    T->cT = t->cent_T; T->cS = t->cent_S; T->cSp = t->cent_Sp; T->cC = t->cent_C;
    T->gC = t->gamma_conn; T->gP = t->gamma_proxy; T->Bt = t->B_tab; T->mis = t->mis_tab;
    T->pi = t->pi_grid; T->tile = t->tile; T->gw = t->grid_w; T->gh = t->grid_h;
    T->mlp = t->mlp_w;
    T->mlp_p = t->mlp_wp;
}

static int nearest(const double *f, int dim, int K, const float *cent) {
    int best = 0;
    double bd = INFINITY;
    for (int k = 0; k < K; ++k) {
        double d = 0.0;
        for (int i = 0; i < dim; ++i) {
            double e = f[i] - (double)cent[k * dim + i];
            d += e * e;
        }
        if (d < bd) {
            bd = d;
            best = k;
        }
    }
    return best;
}

int or_label_9(const or_tables_desc *t, const double *feat9, int K, const float *cent) {
    (void)t;
    return nearest(feat9, 9, K, cent);
}

static void feat_pos(const or_tab *T, v3 p, double *f) {
    f[0] = (p.x - T->lo[0]) / T->ext[0];
    f[1] = (p.y - T->lo[1]) / T->ext[1];
    f[2] = (p.z - T->lo[2]) / T->ext[2];
}

/* subspace label from position, normal flipped toward w, and w */
static int label_dir(const or_tab *T, const or_vtx *v, v3 w, int K, const float *cent) {
    double f[9];
    feat_pos(T, v->p, f);
    v3 n = vdot(v->n, w) >= 0.0 ? v->n : vneg(v->n);
    f[3] = n.x; f[4] = n.y; f[5] = n.z;
    f[6] = w.x; f[7] = w.y; f[8] = w.z;
    return nearest(f, 9, K, cent);
}

/* raw features of an eye vertex for the learned proposal: normalised
 * position, normal facing w, w, roughness */
static void feat_raw(const or_scene_t *s, const or_tab *T, const or_vtx *v, v3 w, double *f) {
    feat_pos(T, v->p, f);
    v3 n = vdot(v->n, w) >= 0.0 ? v->n : vneg(v->n);
    f[3] = n.x; f[4] = n.y; f[5] = n.z;
    f[6] = w.x; f[7] = w.y; f[8] = w.z;
    f[9] = s->mats[v->mat].rough;
}

static int label_spec(const or_tab *T, const or_vtx *v) {
    double f[6];
    feat_pos(T, v->p, f);
    f[3] = v->n.x; f[4] = v->n.y; f[5] = v->n.z;
    return nearest(f, 6, T->KSp, T->cSp);
}

static int label_ctrl(const or_tab *T, const or_vtx *v) {
    double f[3];
    feat_pos(T, v->p, f);
    return nearest(f, 3, T->KC, T->cC);
}

static v3 dirto(v3 a, v3 b) { return vnorm(vsub(b, a)); }

static inline uint32_t sig_upd(uint32_t h, uint32_t x) { return (h ^ x) * 16777619u; }

/* ---- light pass (Sec. 3.2: M light sub-paths cached per iteration) ------ */
void or_light_pass(void *hs, const or_params *p, int iteration, int *tri, float *bary) {
    const or_scene_t *s = (const or_scene_t *)hs;
    int L = p->max_depth - 1;   /* vertex indices 0 .. max_depth-2 */
    for (int l = 0; l < p->M; ++l) {
        int *tr = tri + (size_t)l * L;
        float *ba = bary + (size_t)l * L * 2;
        for (int e = 0; e < L; ++e) { tr[e] = -1; ba[2 * e] = 0; ba[2 * e + 1] = 0; }
        if (L < 1) continue;
        uint32_t it = (uint32_t)iteration, li = (uint32_t)l;
        int t0;
        double b1, b2;
        if (!or_sample_light(s, or_rnd(p->seed, K_LIGHT, it, li, 0, 0), or_rnd(p->seed, K_LIGHT, it, li, 0, 1),
                             or_rnd(p->seed, K_LIGHT, it, li, 0, 2), &t0, &b1, &b2))
            continue;
        tr[0] = t0; ba[0] = (float)b1; ba[1] = (float)b2;
        or_vtx cur = or_vertex_at(s, t0, b1, b2);
        v3 w = or_cosine_dir(cur.n, or_rnd(p->seed, K_LIGHT, it, li, 0, 3), or_rnd(p->seed, K_LIGHT, it, li, 0, 4));
        for (int e = 1; e < L; ++e) {
            or_hit h = or_closest(s, cur.p, w, cur.tri);
            if (h.tri < 0) break;
            or_vtx nx = or_vertex_at(s, h.tri, h.b1, h.b2);
            v3 wl = vneg(w);
            if (or_absorbing(s, &nx, wl)) break;
            tr[e] = h.tri; ba[2 * e] = (float)h.b1; ba[2 * e + 1] = (float)h.b2;
            if (e + 1 >= L) break;
            const or_mat *m = &s->mats[nx.mat];
            v3 ws;
            if (!or_bsdf_sample(m, nx.n, wl, or_rnd(p->seed, K_LIGHT, it, li, (uint32_t)e, 0),
                                or_rnd(p->seed, K_LIGHT, it, li, (uint32_t)e, 1),
                                or_rnd(p->seed, K_LIGHT, it, li, (uint32_t)e, 2), &ws))
                break;
            cur = nx;
            w = ws;
        }
    }
}

/* ---- pool and incomplete sub-paths --------------------------------------- */
static void build_lpaths(const or_scene_t *s, const or_params *p, const int *tri, const float *bary,
                         or_iter *it) {
    int L = p->max_depth - 1;
    it->M = p->M;
    it->lp = (or_lpath *)calloc((size_t)p->M, sizeof(or_lpath));
    for (int l = 0; l < p->M; ++l) {
        or_lpath *lp = &it->lp[l];
        for (int e = 0; e < L; ++e) {
            int t = tri[(size_t)l * L + e];
            if (t < 0) break;
            lp->v[e] = or_vertex_at(s, t, bary[((size_t)l * L + e) * 2], bary[((size_t)l * L + e) * 2 + 1]);
            lp->n = e + 1;
        }
        if (lp->n > 0) lp->v[0].is_light = 1;
    }
}

static void bucketize(int n, const int *label, int K, int **start, int **items) {
    *start = (int *)calloc((size_t)K + 1, sizeof(int));
    *items = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) (*start)[label[i] + 1]++;
    for (int k = 0; k < K; ++k) (*start)[k + 1] += (*start)[k];
    int *fill = (int *)calloc((size_t)K, sizeof(int));
    for (int i = 0; i < n; ++i) (*items)[(*start)[label[i]] + fill[label[i]]++] = i;
    free(fill);
}

static int spec(const or_scene_t *s, const or_vtx *v) { return s->mats[v->mat].specular; }

static int collect_entries(const or_scene_t *s, const or_params *p, const or_lpath *lp, int cap,
                           or_entry *out, int *ol, int *oe) {
    int n = 0;
    int Mp = p->M_p < p->M ? p->M_p : p->M;
    for (int l = 0; l < Mp; ++l) {
        for (int e = 1; e < lp[l].n; ++e) {
            if (!spec(s, &lp[l].v[e])) continue;
            int u = 0, j = e;
            while (j >= 1 && spec(s, &lp[l].v[j])) { ++u; --j; }
            if (u < 1 || u > 4 || j > 1) continue;
            if (n < cap) {
                or_entry *E = &out[n];
                E->y_tri = lp[l].v[e].tri; E->y_b1 = lp[l].v[e].b1; E->y_b2 = lp[l].v[e].b2;
                E->u = u;
                E->type = (j == 1);
                E->h_tri = lp[l].v[0].tri; E->h_b1 = lp[l].v[0].b1; E->h_b2 = lp[l].v[0].b2;
                E->back = vdot(lp[l].v[e].n, vsub(lp[l].v[e - 1].p, lp[l].v[e].p)) < 0.0;
                E->side_in = p->side_in;
                if (ol) ol[n] = l;
                if (oe) oe[n] = e;
            }
            ++n;
        }
    }
    return n;
}

static int table_cell(const or_tab *T, int u, int Sp, int C) {
    return ((u - 1) * T->KSp + Sp) * (T->KC + 1) + C;
}

/* The reciprocal estimate of entry k of an iteration whose entries are
 * labelled. B is the entry's pilot maximum of f/q, or the learned cell value
 * when the pilot is off or saw only f = 0. */
static double entry_estimate(const or_scene_t *s, const or_params *p, const or_tab *T, const or_iter *it,
                             uint32_t iteration, int k, double *nodes, int *trunc, uint32_t *sig) {
    double B = T->Bt[table_cell(T, it->ent[k].u, it->ent_Sp[k], it->ent_C[k])];
    if (p->pilot_max > 0) {
        double Bp = or_pilot_B(s, &it->ent[k], p->seed, iteration, (uint32_t)k, p->pilot_min, p->pilot_max);
        if (Bp > 0.0) B = Bp;
    }
    return or_entry_rhat(s, &it->ent[k], B, p->booth, p->seed, iteration, (uint32_t)k, p->repeats, p->trial_cap,
                         p->split_cap, p->fixed_bound, nodes, trunc, sig);
}

static void build_iter(const or_scene_t *s, const or_params *p, const or_tab *T, uint32_t iteration,
                       const int *tri, const float *bary, const double *rhat_override, or_iter *it,
                       double *entry_nodes, uint32_t *entry_sig, or_stats *st) {
    memset(it, 0, sizeof(*it));
    build_lpaths(s, p, tri, bary, it);
    it->M_p = p->M_p < p->M ? p->M_p : p->M;
    /* connection pool: non-specular light vertices y_e, e >= 1 */
    int cap = 0;
    for (int l = 0; l < p->M; ++l) cap += it->lp[l].n;
    it->pool_l = (int *)malloc(sizeof(int) * (size_t)(cap + 1));
    it->pool_e = (int *)malloc(sizeof(int) * (size_t)(cap + 1));
    it->pool_S = (int *)malloc(sizeof(int) * (size_t)(cap + 1));
    for (int l = 0; l < p->M; ++l) {
        const or_lpath *lp = &it->lp[l];
        for (int e = 1; e < lp->n; ++e) {
            if (spec(s, &lp->v[e])) continue;
            int k = it->npool++;
            it->pool_l[k] = l;
            it->pool_e[k] = e;
            it->pool_S[k] = label_dir(T, &lp->v[e], dirto(lp->v[e].p, lp->v[e - 1].p), T->KS, T->cS);
        }
    }
    bucketize(it->npool, it->pool_S, T->KS, &it->bstart, &it->bitems);
    /* incomplete light sub-paths */
    int ne = collect_entries(s, p, it->lp, 0, NULL, NULL, NULL);
    it->nent = ne;
    it->ent = (or_entry *)malloc(sizeof(or_entry) * (size_t)(ne + 1));
    it->ent_l = (int *)malloc(sizeof(int) * (size_t)(ne + 1));
    it->ent_e = (int *)malloc(sizeof(int) * (size_t)(ne + 1));
    it->ent_Sp = (int *)malloc(sizeof(int) * (size_t)(ne + 1));
    it->ent_C = (int *)malloc(sizeof(int) * (size_t)(ne + 1));
    it->rhat = (double *)malloc(sizeof(double) * (size_t)(ne + 1));
    collect_entries(s, p, it->lp, ne, it->ent, it->ent_l, it->ent_e);
    /* labels; entries of cells whose MIS scale is 0 (left to the other
     * strategies by the learned cost rule) leave the pool, order kept */
    int kept = 0;
    for (int k = 0; k < ne; ++k) {
        const or_lpath *lp = &it->lp[it->ent_l[k]];
        int Sp = label_spec(T, &lp->v[it->ent_e[k]]);
        int C = it->ent[k].type ? label_ctrl(T, &lp->v[0]) : T->KC;
        if (!(T->mis[table_cell(T, it->ent[k].u, Sp, C)] > 0.0f)) continue;
        it->ent[kept] = it->ent[k];
        it->ent_l[kept] = it->ent_l[k];
        it->ent_e[kept] = it->ent_e[k];
        it->ent_Sp[kept] = Sp;
        it->ent_C[kept] = C;
        ++kept;
    }
    ne = kept;
    it->nent = ne;
    for (int k = 0; k < ne; ++k) {
        if (rhat_override) {
            it->rhat[k] = rhat_override[k];
            continue;
        }
        double nodes;
        int trunc;
        uint32_t sg;
        it->rhat[k] = entry_estimate(s, p, T, it, iteration, k, &nodes, &trunc, &sg);
        if (st) {
            st->n_nodes += (int64_t)nodes;
            st->n_truncated += trunc;
        }
        if (entry_nodes) entry_nodes[k] = nodes;
        if (entry_sig) entry_sig[k] = sg;
    }
    bucketize(ne, it->ent_Sp, T->KSp, &it->estart, &it->eitems);
    if (st) st->n_entries += ne;
}

static void free_iter(or_iter *it) {
    free(it->lp); free(it->pool_l); free(it->pool_e); free(it->pool_S); free(it->bstart);
    free(it->bitems); free(it->ent); free(it->ent_l); free(it->ent_e); free(it->ent_Sp);
    free(it->ent_C); free(it->rhat); free(it->estart); free(it->eitems);
}

/* ---- path evaluation ------------------------------------------------------ */
static v3 path_f(const or_scene_t *s, const or_path *x) {
    int k = x->n - 1;
    v3 f = or_emitted(s, &x->v[0], dirto(x->v[0].p, x->v[1].p));
    for (int j = 1; j <= k - 1; ++j) {
        const or_vtx *v = &x->v[j];
        v3 rho = or_bsdf_eval(&s->mats[v->mat], v->n, dirto(v->p, x->v[j - 1].p), dirto(v->p, x->v[j + 1].p));
        f = vmul(f, rho);
    }
    for (int j = 0; j <= k - 2; ++j) {
        v3 d = vsub(x->v[j + 1].p, x->v[j].p);
        double d2 = vdot(d, d);
        v3 w = vscale(d, 1.0 / sqrt(d2));
        f = vscale(f, fabs(vdot(x->v[j].n, w)) * fabs(vdot(x->v[j + 1].n, w)) / d2);
    }
    return f;
}

static void path_densities(const or_scene_t *s, const or_path *x, double *fwd, double *rev) {
    int k = x->n - 1;
    for (int j = 0; j <= k - 1; ++j) fwd[j] = or_fwd_density(s, x->v, j);
    for (int j = 0; j <= k - 2; ++j) {
        const or_vtx *a = &x->v[j + 1];
        v3 d = vsub(x->v[j].p, a->p);
        double d2 = vdot(d, d);
        v3 w = vscale(d, 1.0 / sqrt(d2));
        double pw = or_bsdf_pdf(&s->mats[a->mat], a->n, dirto(a->p, x->v[j + 2].p), w);
        rev[j] = pw * fabs(vdot(x->v[j].n, w)) / d2;
    }
    rev[k - 1] = 1.0;
}

static int nonS_at(const or_scene_t *s, const or_path *x, int j) {
    return j == 0 ? 1 : !s->mats[x->v[j].mat].specular;
}

static double strat_pdf(const double *fwd, const double *rev, int k, int sidx) {
    double p = 1.0;
    for (int j = 0; j < sidx; ++j) p *= fwd[j];
    for (int j = sidx; j <= k - 1; ++j) p *= rev[j];
    return p;
}

static int strat_avail(const or_scene_t *s, const or_params *p, const or_path *x, int sidx) {
    if (sidx == 0) return 1;
    if (sidx >= 2 && !p->conn) return 0;
    return nonS_at(s, x, sidx - 1) && nonS_at(s, x, sidx);
}

/* proxy decomposition of x: first non-specular eye vertex m, trailing
 * specular count u, type; returns 1 if x is a proxy path (Sec. 6.1.1). */
static int proxy_shape(const or_scene_t *s, const or_path *x, int *m, int *u, int *type) {
    int k = x->n - 1, mm = 0;
    for (int j = k - 1; j >= 1; --j)
        if (nonS_at(s, x, j)) { mm = j; break; }
    if (mm == 0) return 0;
    int uu = 0, j = mm - 1;
    while (j >= 1 && !nonS_at(s, x, j)) { ++uu; --j; }
    if (uu < 1 || uu > 4 || j > 1) return 0;
    *m = mm; *u = uu; *type = (j == 1);
    return 1;
}

static double pi_of(const or_tab *T, const or_scene_t *s, int pix) {
    int px = pix % s->W, py = pix / s->W;
    return (double)T->pi[(py / T->tile) * T->gw + (px / T->tile)];
}

/* proxy-strategy MIS density p^_proxy(x) (zero when x is not a proxy path) */
static double proxy_mis_pdf(const or_scene_t *s, const or_tab *T, const or_params *p, const or_path *x,
                            const double *fwd, const double *rev, int pix, int *cell_out) {
    int m, u, type;
    if (!p->proxy || !proxy_shape(s, x, &m, &u, &type)) return 0.0;
    int k = x->n - 1;
    int Sp = label_spec(T, &x->v[m - 1]);
    int C = type ? label_ctrl(T, &x->v[0]) : T->KC;
    int cell = table_cell(T, u, Sp, C);
    if (cell_out) *cell_out = cell;
    double pr = (type ? fwd[0] : 1.0) * pi_of(T, s, pix) * (double)T->mis[cell];
    for (int j = m - u - 1; j <= m - 2; ++j) pr *= rev[j];
    for (int j = m; j <= k - 1; ++j) pr *= rev[j];
    return pr;
}

enum { ST_PT = 0, ST_NEE = 1, ST_CONN = 2, ST_PROXY = 3 };

/* MIS weight of strategy `kind` (s index for PT/NEE/CONN) for path x */
static double mis_weight(const or_scene_t *s, const or_tab *T, const or_params *p, const or_path *x,
                         int kind, int sidx, int pix) {
    double fwd[MAXV], rev[MAXV];
    int k = x->n - 1;
    path_densities(s, x, fwd, rev);
    double sum = 0.0;
    for (int i = 0; i <= k - 1; ++i)
        if (strat_avail(s, p, x, i)) sum += strat_pdf(fwd, rev, k, i);
    double pp = proxy_mis_pdf(s, T, p, x, fwd, rev, pix, NULL);
    sum += pp;
    double num = (kind == ST_PROXY) ? pp : strat_pdf(fwd, rev, k, sidx);
    return sum > 0.0 ? num / sum : 0.0;
}

static void path_from_eye(or_path *x, const or_vtx *zs, int i) {
    /* appends z_i .. z_0 after the current x->n vertices */
    for (int j = i; j >= 0; --j) x->v[x->n++] = zs[j];
}

/* selection: subspace by the row `g` over non-empty buckets, then uniform */
static int select_item(const float *g, int K, const int *start, double u_s, double u_j, double *Q) {
    double Z = 0.0;
    int last = -1;
    for (int k = 0; k < K; ++k)
        if (start[k + 1] > start[k]) { Z += g[k]; last = k; }
    if (last < 0 || Z <= 0.0) return -1;
    double cum = 0.0;
    int pick = last;
    for (int k = 0; k < K; ++k) {
        if (start[k + 1] == start[k]) continue;
        cum += g[k] / Z;
        if (u_s < cum) { pick = k; break; }
    }
    int nS = start[pick + 1] - start[pick];
    int jj = (int)floor(u_j * nS);
    if (jj > nS - 1) jj = nS - 1;
    *Q = (g[pick] / Z) / nS;
    return start[pick] + jj;
}

typedef struct {
    double lum_unweighted;
} contrib_info;

static double lum(v3 c) { return (c.x + c.y + c.z) / 3.0; }

/* one camera sample: returns its radiance estimate and signature */
static v3 eye_path(const or_scene_t *s, const or_tab *T, const or_params *p, const or_iter *it,
                   uint32_t iteration, int pix, uint32_t *sig_out, or_stats *st, learn_acc *acc) {
    v3 L = v3m(0, 0, 0);
    uint32_t sig = 2166136261u;
    or_vtx zs[MAXV];
    int px = pix % s->W, py = pix / s->W;
    uint32_t pu = (uint32_t)pix;
    double j0 = or_rnd(p->seed, K_CAMERA, iteration, pu, 0, 0);
    double j1 = or_rnd(p->seed, K_CAMERA, iteration, pu, 0, 1);
    double sx = 2.0 * (px + j0) / s->W - 1.0, sy = 1.0 - 2.0 * (py + j1) / s->H;
    v3 d = vnorm(vadd(s->cfwd, vadd(vscale(s->cright, sx * s->tanh_ * s->aspect), vscale(s->cup, sy * s->tanh_))));
    memset(&zs[0], 0, sizeof(or_vtx));
    zs[0].p = s->cpos;
    zs[0].tri = -1;
    int tile = (py / T->tile) * T->gw + (px / T->tile);
    double pi_pix = pi_of(T, s, pix);
    int seen_nonS = 0;
    or_hit h = or_closest(s, s->cpos, d, -1);
    int i = 1;
    while (h.tri >= 0) {
        zs[i] = or_vertex_at(s, h.tri, h.b1, h.b2);
        const or_vtx *z = &zs[i];
        const or_mat *mz = &s->mats[z->mat];
        v3 we = vneg(d);
        sig = sig_upd(sig, (uint32_t)z->tri);
        uint32_t ci = (uint32_t)i;
        /* (s = 0) the eye path hits an emitter */
        if (mz->emitter && vdot(z->n, we) > 0.0) {
            or_path x;
            x.n = 0;
            path_from_eye(&x, zs, i);
            x.v[0].is_light = 1;
            v3 f = path_f(s, &x);
            if (vmaxc(f) > 0.0) {
                double fwd[MAXV], rev[MAXV];
                path_densities(s, &x, fwd, rev);
                double pa = strat_pdf(fwd, rev, x.n - 1, 0);
                double w = mis_weight(s, T, p, &x, ST_PT, 0, pix);
                v3 c = vscale(f, w / pa);
                if (p->film != 1) L = vadd(L, c);
                if (acc) acc->tile_all[tile] += lum(c);
            }
        }
        if (or_absorbing(s, z, we)) break;
        int nonS = !mz->specular;
        if (nonS) {
            /* (s = 1) next-event estimation */
            if (i + 1 <= p->max_depth && s->ne > 0) {
                int lt;
                double b1, b2;
                or_sample_light(s, or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 3),
                                or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 4),
                                or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 5), &lt, &b1, &b2);
                or_vtx y = or_vertex_at(s, lt, b1, b2);
                y.is_light = 1;
                int vis = !or_occluded(s, z->p, y.p, z->tri, y.tri);
                sig = sig_upd(sig, 0xA0000000u | (uint32_t)lt);
                sig = sig_upd(sig, (uint32_t)vis);
                if (vis) {
                    or_path x;
                    x.n = 0;
                    x.v[x.n++] = y;
                    path_from_eye(&x, zs, i);
                    v3 f = path_f(s, &x);
                    if (vmaxc(f) > 0.0) {
                        double fwd[MAXV], rev[MAXV];
                        path_densities(s, &x, fwd, rev);
                        double pa = strat_pdf(fwd, rev, x.n - 1, 1);
                        double w = mis_weight(s, T, p, &x, ST_NEE, 1, pix);
                        v3 c = vscale(f, w / pa);
                        if (p->film != 1) L = vadd(L, c);
                        if (acc) acc->tile_all[tile] += lum(c);
                    }
                }
            }
            int Tl = -1;
            /* (s >= 2) subspace probabilistic connection */
            if (p->conn && i + 2 <= p->max_depth && it->npool > 0) {
                Tl = label_dir(T, z, we, T->KT, T->cT);
                double Q;
                int slot;
                if (T->mlp) {
                    /* learned proposal: S ~ Q(. | x), then a uniform vertex of S */
                    double raw[10], QS;
                    feat_raw(s, T, z, we, raw);
                    int Sel = or_mlp_select(T->mlp, T->KS, raw, Tl, T->gC + (size_t)Tl * T->KS, it->bstart,
                                            or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 6), &QS);
                    slot = -1;
                    if (Sel >= 0) {
                        int nS = it->bstart[Sel + 1] - it->bstart[Sel];
                        int jj = (int)floor(or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 7) * nS);
                        if (jj > nS - 1) jj = nS - 1;
                        slot = it->bstart[Sel] + jj;
                        Q = QS / nS;
                    }
                } else {
                    slot = select_item(T->gC + (size_t)Tl * T->KS, T->KS, it->bstart,
                                       or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 6),
                                       or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 7), &Q);
                }
                if (slot >= 0) {
                    int jp = it->bitems[slot];
                    int l = it->pool_l[jp], e = it->pool_e[jp];
                    int sl = e + 1;
                    sig = sig_upd(sig, 0xB0000000u | (uint32_t)jp);
                    if (st) st->n_conn++;
                    if (sl + i > p->max_depth) {
                        sig = sig_upd(sig, 2u);
                    } else {
                        const or_vtx *y = &it->lp[l].v[e];
                        int vis = !or_occluded(s, z->p, y->p, z->tri, y->tri);
                        sig = sig_upd(sig, (uint32_t)vis);
                        if (vis) {
                            or_path x;
                            x.n = 0;
                            for (int q = 0; q <= e; ++q) x.v[x.n++] = it->lp[l].v[q];
                            path_from_eye(&x, zs, i);
                            v3 f = path_f(s, &x);
                            if (vmaxc(f) > 0.0) {
                                double fwd[MAXV], rev[MAXV];
                                path_densities(s, &x, fwd, rev);
                                double pa = strat_pdf(fwd, rev, x.n - 1, sl) * (double)it->M * Q;
                                double w = mis_weight(s, T, p, &x, ST_CONN, sl, pix);
                                v3 c = vscale(f, w / pa);
                                if (p->film != 1) L = vadd(L, c);
                                if (acc) {
                                    acc->tile_all[tile] += lum(c);
                                    acc->conn[(size_t)Tl * T->KS + it->pool_S[jp]] += lum(vscale(f, 1.0 / pa));
                                }
                            }
                        }
                    }
                }
            }
            /* proxy sampling at the first non-specular eye vertex (Sec. 6.1.1) */
            if (p->proxy && !seen_nonS && it->nent > 0 && pi_pix > 0.0) {
                int coin = or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 8) < pi_pix;
                sig = sig_upd(sig, 0xC0000000u | (uint32_t)coin);
                if (coin) {
                    if (Tl < 0) Tl = label_dir(T, z, we, T->KT, T->cT);
                    double Q;
                    int slot;
                    if (T->mlp_p && i + 2 <= p->max_depth) {
                        /* learned proposal of the proxy: S' ~ Q'(. | x) (the network mixed with the row
                         * Gamma'[T, .]), then a uniform incomplete sub-path of S'; deeper than
                         * max_depth - 2 no proxy can fit, and the table row is drawn */
                        double raw[10], QS;
                        feat_raw(s, T, z, we, raw);
                        int Sel = or_mlp_select(T->mlp_p, T->KSp, raw, Tl, T->gP + (size_t)Tl * T->KSp, it->estart,
                                                or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 9), &QS);
                        int nS = it->estart[Sel + 1] - it->estart[Sel];
                        int jq = (int)floor(or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 10) * nS);
                        if (jq > nS - 1) jq = nS - 1;
                        slot = it->estart[Sel] + jq;
                        Q = QS / nS;
                    } else {
                        slot = select_item(T->gP + (size_t)Tl * T->KSp, T->KSp, it->estart,
                                           or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 9),
                                           or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 10), &Q);
                    }
                    int jj = it->eitems[slot];
                    const or_entry *E = &it->ent[jj];
                    sig = sig_upd(sig, (uint32_t)jj);
                    if (st) st->n_proxy++;
                    int u = E->u, sl = u + (E->type ? 2 : 1);
                    int status = 0;
                    or_vtx gs[6], H;
                    gs[0] = or_vertex_at(s, E->y_tri, E->y_b1, E->y_b2);
                    if (E->type) {
                        H = or_vertex_at(s, E->h_tri, E->h_b1, E->h_b2);
                        H.is_light = 1;
                    }
                    if (sl + i > p->max_depth) status = 1;
                    else if (or_occluded(s, z->p, gs[0].p, z->tri, gs[0].tri)) status = 2;
                    else {
                        v3 prev = z->p;
                        for (int r = 1; r <= u && !status; ++r) {
                            const or_vtx *g = &gs[r - 1];
                            const or_mat *mg = &s->mats[g->mat];
                            v3 wg = dirto(g->p, prev);
                            v3 ws;
                            uint32_t d0 = 11 + 3 * (uint32_t)(r - 1);
                            if (or_absorbing(s, g, wg) ||
                                !or_bsdf_sample(mg, g->n, wg, or_rnd(p->seed, K_CAMERA, iteration, pu, ci, d0),
                                                or_rnd(p->seed, K_CAMERA, iteration, pu, ci, d0 + 1),
                                                or_rnd(p->seed, K_CAMERA, iteration, pu, ci, d0 + 2), &ws)) {
                                status = 3;
                                break;
                            }
                            or_hit hh = or_closest(s, g->p, ws, g->tri);
                            sig = sig_upd(sig, hh.tri >= 0 ? (uint32_t)hh.tri : 0x0FFFFFFFu);
                            if (hh.tri < 0) { status = 4; break; }
                            gs[r] = or_vertex_at(s, hh.tri, hh.b1, hh.b2);
                            const or_mat *mr = &s->mats[gs[r].mat];
                            v3 back = vneg(ws);
                            if (r < u) {
                                if (!mr->specular || or_absorbing(s, &gs[r], back)) status = 5;
                            } else if (E->type == 0) {
                                if (!mr->emitter || vdot(gs[r].n, back) <= 0.0) status = 5;
                            } else {
                                if (mr->specular || or_absorbing(s, &gs[r], back)) status = 5;
                            }
                            prev = g->p;
                        }
                        if (!status && E->type && or_occluded(s, gs[u].p, H.p, gs[u].tri, H.tri)) status = 6;
                    }
                    sig = sig_upd(sig, 0xD0000000u | (uint32_t)status);
                    if (!status) {
                        or_path x;
                        x.n = 0;
                        if (E->type) x.v[x.n++] = H;
                        for (int r = u; r >= 1; --r) x.v[x.n++] = gs[r];
                        x.v[0].is_light = 1;
                        x.v[x.n++] = gs[0];
                        path_from_eye(&x, zs, i);
                        v3 f = path_f(s, &x);
                        if (vmaxc(f) > 0.0) {
                            double fwd[MAXV], rev[MAXV];
                            path_densities(s, &x, fwd, rev);
                            int k = x.n - 1, m = sl;
                            double pa = (E->type ? fwd[0] : 1.0) / it->rhat[jj];
                            for (int j = m - u - 1; j <= m - 2; ++j) pa *= rev[j];
                            for (int j = m; j <= k - 1; ++j) pa *= rev[j];
                            pa *= (double)it->M_p * Q * pi_pix;
                            double w = mis_weight(s, T, p, &x, ST_PROXY, 0, pix);
                            v3 c = vscale(f, w / pa);
                            if (p->film != 2) L = vadd(L, c);
                            if (st) st->n_proxy_ok++;
                            if (acc) {
                                acc->tile_all[tile] += lum(c);
                                acc->tile_proxy[tile] += lum(c);
                                acc->proxy[(size_t)Tl * T->KSp + it->ent_Sp[jj]] += lum(vscale(f, 1.0 / pa));
                            }
                        }
                    }
                }
            }
            seen_nonS = 1;
        }
        /* continue the eye sub-path by BSDF sampling */
        if (i + 1 > p->max_depth) break;
        v3 wl;
        if (!or_bsdf_sample(mz, z->n, we, or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 0),
                            or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 1),
                            or_rnd(p->seed, K_CAMERA, iteration, pu, ci, 2), &wl))
            break;
        d = wl;
        h = or_closest(s, z->p, d, z->tri);
        ++i;
    }
    if (sig_out) *sig_out = sig;
    return L;
}

void *or_create(const or_scene_desc *d) {
    or_scene_t *s = (or_scene_t *)malloc(sizeof(or_scene_t));
    or_scene_init(s, d);
    return s;
}

void or_free(void *h) {
    or_scene_free((or_scene_t *)h);
    free(h);
}

int or_entries(void *hs, const or_params *p, const int *tri, const float *bary, int cap, or_entry *out,
               int *light_index) {
    const or_scene_t *s = (const or_scene_t *)hs;
    or_iter it;
    memset(&it, 0, sizeof(it));
    build_lpaths(s, p, tri, bary, &it);
    int n = collect_entries(s, p, it.lp, cap, out, light_index, NULL);
    free(it.lp);
    return n;
}

void or_iteration(void *hs, const or_params *p, const or_tables_desc *td, int iteration, const int *tri,
                  const float *bary, int pix_lo, int pix_hi, const double *rhat_override, double *rgb,
                  uint32_t *sig, int cap, int *n_entries, double *entry_rhat, uint32_t *entry_sig,
                  double *entry_nodes, or_stats *st) {
    const or_scene_t *s = (const or_scene_t *)hs;
    or_tab T;
    tab_init(&T, td);
    or_iter it;
    /* entry outputs are written up to cap */
    int ncount;
    {
        or_iter tmp;
        memset(&tmp, 0, sizeof(tmp));
        build_lpaths(s, p, tri, bary, &tmp);
        ncount = collect_entries(s, p, tmp.lp, 0, NULL, NULL, NULL);
        free(tmp.lp);
    }
    double *nodes = (double *)calloc((size_t)ncount + 1, sizeof(double));
    uint32_t *esig = (uint32_t *)calloc((size_t)ncount + 1, sizeof(uint32_t));
    build_iter(s, p, &T, (uint32_t)iteration, tri, bary, rhat_override, &it, nodes, esig, st);
    if (n_entries) *n_entries = it.nent;
    for (int k = 0; k < it.nent && k < cap; ++k) {
        if (entry_rhat) entry_rhat[k] = it.rhat[k];
        if (entry_sig) entry_sig[k] = esig[k];
        if (entry_nodes) entry_nodes[k] = nodes[k];
    }
    for (int pix = pix_lo; pix < pix_hi; ++pix) {
        uint32_t sg;
        v3 c = eye_path(s, &T, p, &it, (uint32_t)iteration, pix, &sg, st, NULL);
        if (rgb) {
            rgb[(size_t)(pix - pix_lo) * 3] = c.x;
            rgb[(size_t)(pix - pix_lo) * 3 + 1] = c.y;
            rgb[(size_t)(pix - pix_lo) * 3 + 2] = c.z;
        }
        if (sig) sig[pix - pix_lo] = sg;
    }
    free(nodes);
    free(esig);
    free_iter(&it);
}

/* The estimates of entries [k_lo, k_hi) of one iteration, the values
 * or_iteration computes for them (lets a caller spread one iteration's
 * estimates over threads; the handle is only read). Returns the number of
 * entries of the iteration. */
int or_iteration_estimates(void *hs, const or_params *p, const or_tables_desc *td, int iteration, const int *tri,
                           const float *bary, int k_lo, int k_hi, double *out_rhat) {
    const or_scene_t *s = (const or_scene_t *)hs;
    or_tab T;
    tab_init(&T, td);
    int ncount;
    {
        or_iter tmp;
        memset(&tmp, 0, sizeof(tmp));
        build_lpaths(s, p, tri, bary, &tmp);
        ncount = collect_entries(s, p, tmp.lp, 0, NULL, NULL, NULL);
        free(tmp.lp);
    }
    double *zero = (double *)calloc((size_t)ncount + 1, sizeof(double));
    or_iter it;
    build_iter(s, p, &T, (uint32_t)iteration, tri, bary, zero, &it, NULL, NULL, NULL);
    for (int k = k_lo < 0 ? 0 : k_lo; k < k_hi && k < it.nent; ++k) {
        double nodes;
        int trunc;
        uint32_t sg;
        out_rhat[k - k_lo] = entry_estimate(s, p, &T, &it, (uint32_t)iteration, k, &nodes, &trunc, &sg);
    }
    int n = it.nent;
    free(zero);
    free_iter(&it);
    return n;
}

void or_render(void *hs, const or_params *p, const or_tables_desc *td, int iter0, int n_iter, int pix_lo,
               int pix_hi, double *film, or_stats *st) {
    const or_scene_t *s = (const or_scene_t *)hs;
    or_tab T;
    tab_init(&T, td);
    int L = p->max_depth - 1;
    int *tri = (int *)malloc(sizeof(int) * (size_t)p->M * (size_t)(L > 0 ? L : 1));
    float *bary = (float *)malloc(sizeof(float) * 2 * (size_t)p->M * (size_t)(L > 0 ? L : 1));
    for (int k = 0; k < n_iter; ++k) {
        int iteration = iter0 + k;
        or_light_pass(hs, p, iteration, tri, bary);
        or_iter it;
        build_iter(s, p, &T, (uint32_t)iteration, tri, bary, NULL, &it, NULL, NULL, st);
        for (int pix = pix_lo; pix < pix_hi; ++pix) {
            v3 c = eye_path(s, &T, p, &it, (uint32_t)iteration, pix, NULL, st, NULL);
            film[(size_t)pix * 3] += c.x;
            film[(size_t)pix * 3 + 1] += c.y;
            film[(size_t)pix * 3 + 2] += c.z;
        }
        free_iter(&it);
    }
    free(tri);
    free(bary);
}

/* ---- learning of the frozen tables ----------------------------------------
 * B(u,S',C): the largest f/q seen over n_bsamples draws per entry of the
 * learning iterations (Sec. 4.2 / App. "Optimal value for B": B = max f/q).
 * mis(u,S',C) = mean(R) / mean(R^2) over the learning entries, i.e.
 * 1/(E[R^2] Pbar) with Pbar = 1/E[R] (Sec. 5.4-5.5). Empty cells take the
 * pooled value. Gamma rows: 0.9 * normalised accumulated (unweighted)
 * contribution luminance per (T, S) + 0.1 uniform (Sec. 5.5: proportional
 * to expected contribution, learned during the first iterations, then
 * frozen). Grid: proxy share of the weighted contribution per tile; >= 5%
 * -> probability 1.0, else 0.2 (Sec. 6.1.1). */
void or_learn(void *hs, const or_params *p_in, const or_tables_desc *td, int iter0, int n_iter, int n_bsamples,
              double max_chain, float *B_out, float *mis_out, float *gconn_out, float *gproxy_out, float *pi_out) {
    const or_scene_t *s = (const or_scene_t *)hs;
    or_params p_learn = *p_in;
    p_learn.booth = 0.0;   /* statistics are learned with the paper's RRS function */
    p_learn.film = 0;
    const or_params *p = &p_learn;
    or_tab T;
    tab_init(&T, td);
    int ncell = 4 * T.KSp * (T.KC + 1);
    double *Bmax = (double *)calloc((size_t)ncell, sizeof(double));
    double *r1 = (double *)calloc((size_t)ncell, sizeof(double));
    double *r2 = (double *)calloc((size_t)ncell, sizeof(double));
    double *rn = (double *)calloc((size_t)ncell, sizeof(double));
    int L = p->max_depth - 1;
    int *tri = (int *)malloc(sizeof(int) * (size_t)p->M * (size_t)(L > 0 ? L : 1));
    float *bary = (float *)malloc(sizeof(float) * 2 * (size_t)p->M * (size_t)(L > 0 ? L : 1));
    double gmax = 0.0;
    double *fb = (double *)malloc(sizeof(double) * (size_t)(n_bsamples > 0 ? n_bsamples : 1));
    double *qb = (double *)malloc(sizeof(double) * (size_t)(n_bsamples > 0 ? n_bsamples : 1));
    /* pass 1: B from f/q samples */
    for (int k = 0; k < n_iter; ++k) {
        int iteration = iter0 + k;
        or_light_pass(hs, p, iteration, tri, bary);
        or_iter it;
        memset(&it, 0, sizeof(it));
        build_lpaths(s, p, tri, bary, &it);
        int ne = collect_entries(s, p, it.lp, 0, NULL, NULL, NULL);
        or_entry *ent = (or_entry *)malloc(sizeof(or_entry) * (size_t)(ne + 1));
        int *el = (int *)malloc(sizeof(int) * (size_t)(ne + 1));
        int *ee = (int *)malloc(sizeof(int) * (size_t)(ne + 1));
        collect_entries(s, p, it.lp, ne, ent, el, ee);
        for (int q = 0; q < ne; ++q) {
            int Sp = label_spec(&T, &it.lp[el[q]].v[ee[q]]);
            int C = ent[q].type ? label_ctrl(&T, &it.lp[el[q]].v[0]) : T.KC;
            int cell = table_cell(&T, ent[q].u, Sp, C);
            or_entry_fq(hs, &ent[q], n_bsamples, p->seed, (uint32_t)iteration, (uint32_t)q, fb, qb);
            for (int i = 0; i < n_bsamples; ++i) {
                double r = qb[i] > 0.0 ? fb[i] / qb[i] : 0.0;
                if (r > Bmax[cell]) Bmax[cell] = r;
                if (r > gmax) gmax = r;
            }
        }
        free(ent); free(el); free(ee); free(it.lp);
    }
    if (gmax <= 0.0) gmax = 1.0;
    for (int c = 0; c < ncell; ++c) B_out[c] = (float)(B_SAFETY * (Bmax[c] > 0.0 ? Bmax[c] : gmax));
    /* pass 2: reciprocal statistics with the learned B, over every entry
     * (MIS scale 1 everywhere while learning) */
    or_tables_desc t2 = *td;
    t2.mlp_w = NULL;   /* statistics are learned with the table proposal */
    t2.mlp_wp = NULL;
    t2.B_tab = B_out;
    for (int c = 0; c < ncell; ++c) mis_out[c] = 1.0f;
    t2.mis_tab = mis_out;
    or_tab T2;
    tab_init(&T2, &t2);
    double s1 = 0, s2 = 0;
    double *nsum = (double *)calloc((size_t)ncell, sizeof(double));
    double *enodes = (double *)malloc(sizeof(double) * (size_t)p->M * (size_t)(L > 0 ? L : 1));
    for (int k = 0; k < n_iter; ++k) {
        int iteration = iter0 + k;
        or_light_pass(hs, p, iteration, tri, bary);
        or_iter it;
        build_iter(s, p, &T2, (uint32_t)iteration, tri, bary, NULL, &it, enodes, NULL, NULL);
        for (int q = 0; q < it.nent; ++q) {
            int cell = table_cell(&T2, it.ent[q].u, it.ent_Sp[q], it.ent_C[q]);
            double R = it.rhat[q];
            r1[cell] += R; r2[cell] += R * R; rn[cell] += 1;
            s1 += R; s2 += R * R;
            /* a truncated estimate counts as over the bound */
            nsum[cell] += enodes[q] >= (double)p->trial_cap ? 1e30 : enodes[q];
        }
        free_iter(&it);
    }
    double pooled = (s1 > 0.0 && s2 > 0.0) ? s1 / s2 : 1.0;
    for (int c = 0; c < ncell; ++c) {
        mis_out[c] = (float)((rn[c] > 0 && r1[c] > 0.0 && r2[c] > 0.0) ? r1[c] / r2[c] : pooled);
        /* learned cost rule: cells whose estimates are too long leave the
         * proxy strategy (MIS scale 0 keeps every weight consistent) */
        if (max_chain > 0.0 && rn[c] > 0 && nsum[c] > max_chain * rn[c] * (double)p->repeats) mis_out[c] = 0.0f;
    }
    free(nsum);
    free(enodes);
    /* pass 3: selection matrices and grid from eye passes with uniform rows */
    float *gu = (float *)malloc(sizeof(float) * (size_t)T.KT * T.KS);
    float *gpu_ = (float *)malloc(sizeof(float) * (size_t)T.KT * T.KSp);
    for (int i = 0; i < T.KT * T.KS; ++i) gu[i] = 1.0f / T.KS;
    for (int i = 0; i < T.KT * T.KSp; ++i) gpu_[i] = 1.0f / T.KSp;
    float *pione = (float *)malloc(sizeof(float) * (size_t)T.gw * T.gh);
    for (int i = 0; i < T.gw * T.gh; ++i) pione[i] = 1.0f;
    or_tables_desc t3 = t2;
    t3.mis_tab = mis_out;
    t3.gamma_conn = gu;
    t3.gamma_proxy = gpu_;
    t3.pi_grid = pione;
    or_tab T3;
    tab_init(&T3, &t3);
    learn_acc acc;
    acc.conn = (double *)calloc((size_t)T.KT * T.KS, sizeof(double));
    acc.proxy = (double *)calloc((size_t)T.KT * T.KSp, sizeof(double));
    acc.tile_proxy = (double *)calloc((size_t)T.gw * T.gh, sizeof(double));
    acc.tile_all = (double *)calloc((size_t)T.gw * T.gh, sizeof(double));
    for (int k = 0; k < n_iter; ++k) {
        int iteration = iter0 + k;
        or_light_pass(hs, p, iteration, tri, bary);
        or_iter it;
        build_iter(s, p, &T3, (uint32_t)iteration, tri, bary, NULL, &it, NULL, NULL, NULL);
        for (int pix = 0; pix < s->W * s->H; ++pix)
            eye_path(s, &T3, p, &it, (uint32_t)iteration, pix, NULL, NULL, &acc);
        free_iter(&it);
    }
    for (int r = 0; r < T.KT; ++r) {
        double sc = 0, sp = 0;
        for (int c = 0; c < T.KS; ++c) sc += acc.conn[(size_t)r * T.KS + c];
        for (int c = 0; c < T.KSp; ++c) sp += acc.proxy[(size_t)r * T.KSp + c];
        for (int c = 0; c < T.KS; ++c)
            gconn_out[(size_t)r * T.KS + c] =
                (float)(sc > 0 ? 0.9 * acc.conn[(size_t)r * T.KS + c] / sc + 0.1 / T.KS : 1.0 / T.KS);
        for (int c = 0; c < T.KSp; ++c)
            gproxy_out[(size_t)r * T.KSp + c] =
                (float)(sp > 0 ? 0.9 * acc.proxy[(size_t)r * T.KSp + c] / sp + 0.1 / T.KSp : 1.0 / T.KSp);
    }
    for (int i = 0; i < T.gw * T.gh; ++i)
        pi_out[i] = (acc.tile_all[i] > 0 && acc.tile_proxy[i] / acc.tile_all[i] >= 0.05) ? 1.0f : 0.2f;
    free(acc.conn); free(acc.proxy); free(acc.tile_proxy); free(acc.tile_all);
    free(gu); free(gpu_); free(pione); free(fb); free(qb);
    free(Bmax); free(r1); free(r2); free(rn); free(tri); free(bary);
}
