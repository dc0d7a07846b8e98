/* CPU oracle (test infrastructure only): the reciprocal estimator.
 *
 * Sec. 4.2 and Appendix Alg. "Estimator I~": to estimate 1/beta with
 * beta = int f, draw x ~ q, set g = 1 - f(x)/(B q(x)), add g/B, and spawn
 * floor(r) + Bernoulli(r - floor(r)) children with the RRS function
 * r = |g| (Eq. rr), each child's estimate entering with weight g/r = sgn(g).
 * The result adds 1/B (the n = 0 Taylor term). Readings taken where the
 * printed algorithm is garbled: the loop spawns exactly r' children, the
 * factor in the loop is g0/r0, and Alg. I uses r(x0).
 *
 * Written out, the recursion is a sum over the nodes of the random tree:
 *   I~ = 1/B + sum_v (g_v / B) * prod_{a ancestor of v} sgn(g_a)
 *   I  =       sum_v (1 / B)   * prod_{a ancestor of v} sgn(g_a)   (Alg. I)
 * (with B per node under the raise rule below).
 * visit() walks the tree in pre-order and adds each node's term. Node v
 * draws its variates from the counter-based stream with word c = its
 * pre-order index. A node cap bounds the work; reaching it truncates the
 * estimate and is reported.
 *
 * Booth's Russian roulette (the baseline of the paper's RR ablation, Sec. 4.2
 * and Fig. RR-ablation) uses the same Taylor terms on one chain without
 * splitting: the k-vertex prefix continues with probability
 * rho_k = min(1, c * prod_{i<k} |g_i|), and the prefix's term is
 * prod_{i<k} g_i / prod_{1<=j<k} rho_j (Eq. RRS_estimator). The printed
 * factor is 1/r for a hyper-parameter r of order 10^2..10^3; it is read as
 * the weight cutoff 1/r, i.e. c = r (with c = 1/r every step would survive
 * with probability at most 1/r, which cannot improve as r grows to 10^3,
 * as the ablation reports). c > 0 selects this rule; c = 0 the paper's. */
#include "or_internal.h"

/* the split limit and bound rule of the stand-alone estimator entry points (pins, tests) */
static uint32_t or_split_default = 1u << 16;
static int or_fixed_default = 0;

void or_set_split_default(int split) { or_split_default = split > 0 ? (uint32_t)split : 0xFFFFFFFFu; }
void or_set_fixed_bound_default(int fixed) { or_fixed_default = fixed != 0; }

typedef struct {
    double (*ratio)(void *ctx, uint32_t node);    /* draw x ~ q, return f(x)/q(x) */
    double (*unif)(void *ctx, uint32_t node);     /* the node's RRS uniform */
    void *ctx;
    double B;
    uint32_t cap, next;
    int truncated;
    double sum_t, sum_i;
    double booth;       /* > 0: Booth's roulette with scale c (no splitting); 0: the paper's RRS */
    uint32_t split;     /* first pre-order node without splitting (see visit) */
    int fixed;          /* 1: one B for the whole estimate (the paper's walk); 0: the raise rule */
} rec_state;

/* The split limit. Alg. I~ is unbiased for any number-of-children rule
 * r(x) > 0 (with E[children] = r and the children's terms weighted by g / r):
 * each child's estimate has the same expectation whatever the rule, so the
 * recursion E[I~'] = E[g]/B + E[g] E[I~'] holds node by node, and the rule
 * may depend on the history (here: the node's pre-order index). The paper's
 * r = |g| is used up to node `split`; from there on a node with |g| > 1
 * has exactly one child of weight g (r = 1), so a chain whose bound B sits
 * far below some f/q (a tree that would split without end) finishes as a
 * chain instead of hitting the node cap. Chains shorter than `split` are
 * unchanged.
 *
 * The raise rule. The paper keeps one B for the whole estimate. Here a node
 * that splits (|g| > 1, i.e. f/q > 2B) hands its children the bound
 * B' = its own f/q. The estimate stays unbiased for any bound fixed before a
 * node's draw, because 1/beta = 1/B + (1 - beta/B) (1/beta) holds for every
 * B: a node with bound B, g = 1 - X/B and children that each estimate
 * 1/beta has expectation 1/beta. Each child enters with its own term 1/B',
 * so the node's Taylor term (the expected own term of its children) is
 * g / B'; Alg. I's term stays 1/B, the node's own. A chain whose draws stay
 * below 2B never raises its bound and is the paper's walk exactly; a tree
 * whose B sits far below the integrand's typical f/q would split without
 * end, and now grows only as far as its own ratios allow. */
static void visit(rec_state *st, double w_anc, double B) {
    for (;;) {
        if (st->next >= st->cap) {
            st->truncated = 1;
            return;
        }
        uint32_t node = st->next++;
        double X = st->ratio(st->ctx, node);
        double g = 1.0 - X / B;
        double r = fabs(g);
        double Bc = (!st->fixed && r > 1.0) ? X : B;   /* the children's bound (the raise rule above) */
        st->sum_t += w_anc * g / Bc;
        st->sum_i += w_anc / B;
        int n;
        double child_w;
        if (r > 1.0 && node >= st->split) {
            n = 1;
            child_w = w_anc * g;
        } else {
            n = (int)floor(r);
            if (st->unif(st->ctx, node) < r - (double)n) n += 1;
            child_w = w_anc * (g > 0.0 ? 1.0 : -1.0);
        }
        if (n == 0) return;
        if (!isfinite(child_w)) {   /* the weight left the double range: a truncated estimate */
            st->truncated = 1;
            return;
        }
        for (int i = 0; i < n - 1; ++i) visit(st, child_w, Bc);
        w_anc = child_w;   /* the last child continues in this loop */
        B = Bc;
    }
}

/* Booth's roulette: one chain; node k holds the k+1-vertex prefix */
static void walk_booth(rec_state *st) {
    double prod = 1.0;   /* prod_{i<=k} g_i */
    double surv = 1.0;   /* prod of the continuation probabilities taken so far */
    for (;;) {
        if (st->next >= st->cap) {
            st->truncated = 1;
            return;
        }
        uint32_t node = st->next++;
        prod *= 1.0 - st->ratio(st->ctx, node) / st->B;
        double t = prod / surv / st->B;
        if (!isfinite(t)) {   /* the weight left the double range: a truncated chain */
            st->truncated = 1;
            return;
        }
        st->sum_t += t;
        double rho = st->booth * fabs(prod);
        if (rho > 1.0) rho = 1.0;
        if (!(st->unif(st->ctx, node) < rho)) return;
        surv *= rho;
    }
}

/* one estimate: returns I~, sets *I (Alg. I; 0 under Booth's roulette),
 * *nodes, *trunc */
static double estimate(rec_state *st, double *I, double *nodes, int *trunc) {
    st->next = 0;
    st->truncated = 0;
    st->sum_t = 0.0;
    st->sum_i = 0.0;
    if (st->booth > 0.0)
        walk_booth(st);
    else
        visit(st, 1.0, st->B);
    *I = st->sum_i;
    *nodes = (double)st->next;
    *trunc = st->truncated;
    return 1.0 / st->B + st->sum_t;
}

/* ---- 1-D integrands for the estimator pins ----------------------------- */
typedef struct { int fn; uint32_t seed, run; } one_d;

static double one_d_ratio(void *c, uint32_t node) {
    one_d *o = (one_d *)c;
    double u0 = or_rnd(o->seed, K_TRAIN, o->run, 0, node, 0);
    double u1 = or_rnd(o->seed, K_TRAIN, o->run, 0, node, 1);
    double x, f, q;
    switch (o->fn) {
    case 0:
        x = u1;
        f = 1.0 + 0.5 * sin(2.0 * M_PI * x);
        q = 1.0;
        break;
    case 1:
        x = u1;
        f = 3.0 * x * x;
        q = 1.0;
        break;
    case 2:
        x = (u0 < 0.5) ? u1 : sqrt(u1);
        f = 3.0 * x * x;
        q = 0.5 * 1.0 + 0.5 * (2.0 * x);
        break;
    default:   /* f = q: the ratio is exactly 1 (integral 1) */
        (void)u0;
        return 1.0;
    }
    return f / q;
}

static double one_d_unif(void *c, uint32_t node) {
    one_d *o = (one_d *)c;
    return or_rnd(o->seed, K_TRAIN, o->run, 0, node, 2);
}

int or_recip_1d(int fn, double B, int n_runs, uint32_t seed, int trial_cap, double *out_t,
                double *out_i, double *out_n) {
    return or_recip_1d_booth(fn, B, 0.0, n_runs, seed, trial_cap, out_t, out_i, out_n);
}

int or_recip_1d_booth(int fn, double B, double c, int n_runs, uint32_t seed, int trial_cap, double *out_t,
                      double *out_i, double *out_n) {
    one_d o = {fn, seed, 0};
    rec_state st = {one_d_ratio, one_d_unif, &o, B, (uint32_t)trial_cap, 0, 0, 0, 0, c, or_split_default,
                    or_fixed_default};
    int ntr = 0;
    for (int r = 0; r < n_runs; ++r) {
        o.run = (uint32_t)r;
        int tr;
        out_t[r] = estimate(&st, &out_i[r], &out_n[r], &tr);
        ntr += tr;
    }
    return ntr;
}

/* ---- proxy-path integrand of an incomplete light sub-path ---------------
 *
 * Sec. 5.2, Eq. reciprocalFinal: P(u, h_c, y_{s-1}, w_c) is the integral
 * over the dropped vertices g = y_{s-2} .. y_{s-u-1} of
 * f(g) = p(g | h_c, w_c) p(y_{s-1} | g, h_c): the area-measure densities with
 * which the light tracer generates g and then y_{s-1}, times the indicator
 * that g has the specular/diffuse pattern the entry was built from
 * (Sec. 5.1: mismatched retraces are discarded, so only matching g occur).
 * Sec. 5.3: q is the uniform mixture of the available strategies --
 * light-source sampling (u=1, g = y_0), tracing from the control vertex
 * (u=1, h_c = y_0 on the light: cosine hemisphere), and tracing from
 * y_{s-1} (cosine hemisphere first, then the BSDF at every specular
 * vertex with the reversed incoming direction). */

typedef struct {
    const or_scene_t *s;
    or_vtx Y, H;
    int u, type;        /* type 0: L S^u, 1: L D S^u */
    int back;           /* y_{s-2} lies behind Y's normal */
    double pin;         /* share of the cosine draws at a dielectric Y toward y_{s-2}; the rest
                         * go to the other side, so q stays positive wherever f can be */
    uint32_t seed, kind, a, b;
    double last_f, last_q;
} entry_ctx;

static double R(const entry_ctx *e, uint32_t node, uint32_t d) {
    return or_rnd(e->seed, e->kind, e->a, e->b, node, d);
}

static v3 dirto(v3 a, v3 b) { return vnorm(vsub(b, a)); }

/* light-tracer area density of ys[j] given ys[j-1], ys[j-2] (Sec. 3.1,
 * Eq. tracingPdf); j=0 is light-source sampling. */
double or_fwd_density(const or_scene_t *s, const or_vtx *ys, int j) {
    if (j == 0) return or_light_pdf(s, ys[0].tri);
    v3 d = vsub(ys[j].p, ys[j - 1].p);
    double d2 = vdot(d, d);
    v3 w = vscale(d, 1.0 / sqrt(d2));
    double cos_new = fabs(vdot(ys[j].n, w));
    if (j == 1) {
        double c0 = vdot(ys[0].n, w);
        if (c0 <= 0.0) return 0.0;
        return (c0 / M_PI) * cos_new / d2;
    }
    const or_mat *m = &s->mats[ys[j - 1].mat];
    double pw = or_bsdf_pdf(m, ys[j - 1].n, dirto(ys[j - 1].p, ys[j - 2].p), w);
    return pw * cos_new / d2;
}

/* cosine density at the specular vertex Y: conductors use their front
 * hemisphere; dielectrics both, the side of y_{s-2} with probability pin. */
static double cosY_pdf(const or_scene_t *s, const or_vtx *Y, v3 w, int back, double pin) {
    const or_mat *m = &s->mats[Y->mat];
    double c = vdot(Y->n, w);
    if (m->kind == MK_DIELECTRIC) return (((c < 0.0) == (back != 0)) ? pin : 1.0 - pin) * fabs(c) / M_PI;
    return c > 0.0 ? c / M_PI : 0.0;
}

/* density that tracing from Y produces g_1..g_u (ys ordered light-first) */
static double q_from_Y(const or_scene_t *s, const or_vtx *gs, int u, const or_vtx *Y, int back, double pin) {
    /* gs[0] = Y, gs[r] = r-th retraced vertex */
    v3 d = vsub(gs[1].p, Y->p);
    double d2 = vdot(d, d);
    v3 w = vscale(d, 1.0 / sqrt(d2));
    double q = cosY_pdf(s, Y, w, back, pin) * fabs(vdot(gs[1].n, w)) / d2;
    for (int r = 1; r < u; ++r) {
        const or_mat *m = &s->mats[gs[r].mat];
        v3 dd = vsub(gs[r + 1].p, gs[r].p);
        double dd2 = vdot(dd, dd);
        v3 ww = vscale(dd, 1.0 / sqrt(dd2));
        q *= or_bsdf_pdf(m, gs[r].n, dirto(gs[r].p, gs[r - 1].p), ww) * fabs(vdot(gs[r + 1].n, ww)) / dd2;
    }
    return q;
}

/* f and q at the dropped-vertex sample gs[1..u] (gs[0] = Y); vis_* are the
 * visibilities of the segments not traced by the drawing component. */
static void eval_fq(const entry_ctx *e, const or_vtx *gs, double *f, double *q, int comp_A,
                    int vis_extra) {
    const or_scene_t *s = e->s;
    int u = e->u;
    or_vtx ys[8];
    int n = 0;
    if (e->type == 1) ys[n++] = e->H;
    for (int r = u; r >= 1; --r) ys[n++] = gs[r];
    ys[n++] = e->Y;
    ys[0].is_light = 1;
    /* pattern of the dropped vertices (Sec. 5.1) and non-absorption */
    int ok = vis_extra;
    for (int j = 1; j < n && ok; ++j) {
        const or_mat *m = &s->mats[ys[j].mat];
        int want_spec = (j == n - 1) ? 1 : (e->type == 1 && j == 1 ? 0 : 1);
        if (m->specular != want_spec) ok = 0;
        if (or_absorbing(s, &ys[j], dirto(ys[j].p, ys[j - 1].p))) ok = 0;
    }
    if (e->type == 0 && !s->mats[ys[0].mat].emitter) ok = 0;
    double fv = 0.0;
    if (ok) {
        fv = 1.0;
        for (int j = (e->type == 1 ? 1 : 0); j < n; ++j) fv *= or_fwd_density(s, ys, j);
    }
    double qB = vis_extra || !comp_A ? q_from_Y(s, gs, u, &e->Y, e->back, e->pin) : 0.0;
    double qv = qB;
    if (u == 1) {
        double qA;
        if (e->type == 0) {
            qA = or_light_pdf(s, gs[1].tri);
        } else {
            v3 d = vsub(gs[1].p, e->H.p);
            double d2 = vdot(d, d);
            v3 w = vscale(d, 1.0 / sqrt(d2));
            double c0 = vdot(e->H.n, w);
            int visHA = comp_A ? 1 : vis_extra;
            qA = (c0 > 0.0 && visHA) ? (c0 / M_PI) * fabs(vdot(gs[1].n, w)) / d2 : 0.0;
        }
        qv = 0.5 * qA + 0.5 * qB;
    }
    *f = fv;
    *q = qv;
}

static int trace_vertex(const or_scene_t *s, v3 o, v3 w, int skip, or_vtx *out) {
    or_hit h = or_closest(s, o, w, skip);
    if (h.tri < 0) return 0;
    *out = or_vertex_at(s, h.tri, h.b1, h.b2);
    return 1;
}

/* draw one sample of the dropped vertices and return f/q (node dims:
 * 0 component, 1-3 light sample, 4-5 cosine direction, 6+3(r-1).. BSDF
 * sample at the r-th specular vertex, 18 RRS uniform, 19 hemisphere side) */
static double entry_ratio(void *c, uint32_t node) {
    entry_ctx *e = (entry_ctx *)c;
    const or_scene_t *s = e->s;
    int u = e->u;
    or_vtx gs[6];
    gs[0] = e->Y;
    e->last_f = 0.0;
    e->last_q = 0.0;
    int comp_A = (u == 1) && (R(e, node, 0) < 0.5);
    if (comp_A && e->type == 0) {
        int tri;
        double b1, b2;
        if (!or_sample_light(s, R(e, node, 1), R(e, node, 2), R(e, node, 3), &tri, &b1, &b2)) return 0.0;
        gs[1] = or_vertex_at(s, tri, b1, b2);
        int vis = !or_occluded(s, gs[1].p, e->Y.p, gs[1].tri, e->Y.tri);
        double f, q;
        eval_fq(e, gs, &f, &q, 1, vis);
        e->last_f = f;
        e->last_q = q;
        return q > 0.0 ? f / q : 0.0;
    }
    if (comp_A && e->type == 1) {
        v3 w = or_cosine_dir(e->H.n, R(e, node, 4), R(e, node, 5));
        if (!trace_vertex(s, e->H.p, w, e->H.tri, &gs[1])) return 0.0;
        int vis = !or_occluded(s, gs[1].p, e->Y.p, gs[1].tri, e->Y.tri);
        double f, q;
        eval_fq(e, gs, &f, &q, 1, vis);
        e->last_f = f;
        e->last_q = q;
        return q > 0.0 ? f / q : 0.0;
    }
    /* trace from Y */
    const or_mat *mY = &s->mats[e->Y.mat];
    v3 nside = e->Y.n;
    if (mY->kind == MK_DIELECTRIC) {
        v3 nin = e->back ? vneg(e->Y.n) : e->Y.n;   /* toward y_{s-2} */
        nside = R(e, node, 19) < e->pin ? nin : vneg(nin);
    }
    v3 w = or_cosine_dir(nside, R(e, node, 4), R(e, node, 5));
    if (!trace_vertex(s, e->Y.p, w, e->Y.tri, &gs[1])) return 0.0;
    for (int r = 1; r < u; ++r) {
        const or_mat *m = &s->mats[gs[r].mat];
        v3 wg = dirto(gs[r].p, gs[r - 1].p);
        if (!m->specular || or_absorbing(s, &gs[r], wg)) return 0.0;
        v3 ws;
        uint32_t d0 = 6 + 3 * (uint32_t)(r - 1);
        if (!or_bsdf_sample(m, gs[r].n, wg, R(e, node, d0), R(e, node, d0 + 1), R(e, node, d0 + 2), &ws))
            return 0.0;
        if (!trace_vertex(s, gs[r].p, ws, gs[r].tri, &gs[r + 1])) return 0.0;
    }
    int vis = 1;
    if (e->type == 1) vis = !or_occluded(s, gs[u].p, e->H.p, gs[u].tri, e->H.tri);
    double f, q;
    eval_fq(e, gs, &f, &q, 0, vis);
    e->last_f = f;
    e->last_q = q;
    return q > 0.0 ? f / q : 0.0;
}

static double entry_unif(void *c, uint32_t node) {
    entry_ctx *e = (entry_ctx *)c;
    return R(e, node, 18);
}

static void entry_setup(entry_ctx *e, const or_scene_t *s, const or_entry *en) {
    memset(e, 0, sizeof(*e));
    e->s = s;
    e->Y = or_vertex_at(s, en->y_tri, en->y_b1, en->y_b2);
    e->u = en->u;
    e->type = en->type;
    e->back = en->back;
    e->pin = en->side_in > 0.0 ? en->side_in : 0.5;
    if (en->type == 1) {
        e->H = or_vertex_at(s, en->h_tri, en->h_b1, en->h_b2);
        e->H.is_light = 1;
    }
}

/* Reciprocal of the incomplete sub-path pdf for one entry: the mean of
 * `repeats` independent estimates I~ (Sec. 6.1.1 averages 5), with Booth's
 * roulette of scale `booth` when it is positive. Stream:
 * kind RECIP, a = iteration, b = entry*8 + repeat, c = node. */
double or_entry_rhat(const or_scene_t *s, const or_entry *en, double B, double booth, uint32_t seed,
                     uint32_t iteration, uint32_t entry, int repeats, int cap, int split, int fixed,
                     double *nodes, int *trunc, uint32_t *sig) {
    entry_ctx e;
    entry_setup(&e, s, en);
    e.seed = seed;
    e.kind = K_RECIP;
    e.a = iteration;
    rec_state st = {entry_ratio, entry_unif, &e, B, (uint32_t)cap, 0, 0, 0, 0, booth,
                    split > 0 ? (uint32_t)split : 0xFFFFFFFFu, fixed != 0};
    double acc = 0.0, nn = 0.0;
    int tr = 0;
    uint32_t h = 2166136261u;
    for (int r = 0; r < repeats; ++r) {
        e.b = entry * 8u + (uint32_t)r;
        double I, nd;
        int t;
        acc += estimate(&st, &I, &nd, &t);
        nn += nd;
        tr |= t;
        h = (h ^ (uint32_t)nd) * 16777619u;
    }
    if (nodes) *nodes = nn;
    if (trunc) *trunc = tr;
    if (sig) *sig = h;
    return acc / repeats;
}

/* B for one entry (App. "Optimal value for B": B = max f/q of the integrand
 * being estimated). f/q is drawn from the entry's own supporting
 * distribution on stream (kind PILOT, a = iteration, b = entry, c = draw),
 * which no estimate uses, in rounds of 32 draws: at least min_draws, then
 * further rounds until some draw has f > 0, at most max_draws. Returns the
 * largest f/q seen, or 0 when every draw had f = 0. Because B is fixed
 * before, and independently of, the draws of the estimate, Alg. I~ stays
 * unbiased whatever value the pilot returns. */
double or_pilot_B(const or_scene_t *s, const or_entry *en, uint32_t seed, uint32_t iteration, uint32_t entry,
                  int min_draws, int max_draws) {
    entry_ctx e;
    entry_setup(&e, s, en);
    e.seed = seed;
    e.kind = K_PILOT;
    e.a = iteration;
    e.b = entry;
    int lo = ((min_draws + 31) / 32) * 32, hi = ((max_draws + 31) / 32) * 32;
    if (lo < 32) lo = 32;
    if (hi < lo) hi = lo;
    double best = 0.0;
    for (int i = 0; i < hi; ++i) {
        if (i % 32 == 0 && i >= lo && best > 0.0) break;
        double r = entry_ratio(&e, (uint32_t)i);
        if (r > best) best = r;
    }
    return best;
}

double or_entry_pilot(void *hs, const or_entry *en, uint32_t seed, uint32_t a, uint32_t b, int min_draws,
                      int max_draws) {
    return or_pilot_B((const or_scene_t *)hs, en, seed, a, b, min_draws, max_draws);
}

void or_entry_fq(void *hs, const or_entry *en, int n, uint32_t seed, uint32_t a, uint32_t b,
                 double *f_out, double *q_out) {
    entry_ctx e;
    entry_setup(&e, (const or_scene_t *)hs, en);
    e.seed = seed;
    e.kind = K_TRAIN;
    e.a = a;
    e.b = b;
    for (int i = 0; i < n; ++i) {
        entry_ratio(&e, (uint32_t)i);
        f_out[i] = e.last_f;
        q_out[i] = e.last_q;
    }
}

int or_entry_recip(void *hs, const or_entry *en, double B, int n, uint32_t seed, int trial_cap,
                   double *out_t, double *out_i, double *out_n) {
    return or_entry_recip_booth(hs, en, B, 0.0, n, seed, trial_cap, out_t, out_i, out_n);
}

int or_entry_recip_booth(void *hs, const or_entry *en, double B, double c, int n, uint32_t seed, int trial_cap,
                         double *out_t, double *out_i, double *out_n) {
    entry_ctx e;
    entry_setup(&e, (const or_scene_t *)hs, en);
    e.seed = seed;
    e.kind = K_RECIP;
    rec_state st = {entry_ratio, entry_unif, &e, B, (uint32_t)trial_cap, 0, 0, 0, 0, c, or_split_default,
                    or_fixed_default};
    int ntr = 0;
    for (int i = 0; i < n; ++i) {
        e.a = 0xFFFFu;
        e.b = (uint32_t)i;
        int t;
        out_t[i] = estimate(&st, &out_i[i], &out_n[i], &t);
        ntr += t;
    }
    return ntr;
}
