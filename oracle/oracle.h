/* CPU oracle for proxy-tracing BDPT -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain FP64 restatement of "Proxy Tracing: Unbiased Reciprocal Estimation
 * for Optimized Sampling in BDPT" (arXiv 2503.23412): the path-integral
 * estimator of Sec. 3.1, subspace probabilistic connections (Sec. 3.2,
 * Sec. 5.5), proxy construction (Sec. 5.1), the incomplete-sub-path pdf
 * (Sec. 5.2, Eq. reciprocalFinal), the supporting distribution (Sec. 5.3),
 * the reciprocal estimator (Sec. 4.2, Eq. RRS_estimator / rr /
 * final_estimator, Appendix Alg. "Estimator I~" and "Estimator I") and the
 * MIS weight for estimated pdfs (Sec. 5.4, Eq. MIS_1).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load this library. It shares no code with the CUDA renderer. All
 * arithmetic is double precision; inputs are the float32 arrays produced by
 * paper_2503_23412_gb300/scenes.py.
 */
#ifndef ORACLE_H
#define ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nv, nt, nm;
    const float *verts;   /* nv*3 */
    const float *uvs;     /* nv*2 */
    const int *tris;      /* nt*3 */
    const int *tri_mat;   /* nt */
    const float *mats;    /* nm*12, layout in scenes.py */
    int tex_w, tex_h;
    const float *tex;     /* tex_h*tex_w*3 */
    const float *cam;     /* 12 */
} or_scene_desc;

typedef struct {
    int KT, KS, KSp, KC;
    const float *bbox_lo, *bbox_hi;   /* 3 each: feature normalisation box */
    const float *cent_T;              /* KT*9 eye subspace centroids */
    const float *cent_S;              /* KS*9 light subspace centroids */
    const float *cent_Sp;             /* KSp*6 specular subspace centroids */
    const float *cent_C;              /* KC*3 control subspace centroids */
    const float *gamma_conn;          /* KT*KS selection matrix (rows sum to 1) */
    const float *gamma_proxy;         /* KT*KSp */
    const float *B_tab;               /* 4*KSp*(KC+1): B(u,S',C), C=KC is "no control vertex" */
    const float *mis_tab;             /* 4*KSp*(KC+1): 1/(E[R^2] * Pbar) */
    int tile, grid_w, grid_h;
    const float *pi_grid;             /* grid_h*grid_w proxy probability per tile */
    const double *mlp_w;              /* learned light-subspace proposal (or_mlp.c layout), NULL: table rows */
    const double *mlp_wp;             /* learned specular-subspace proposal of the proxy strategy (or_mlp.c
                                       * layout with K = KSp), NULL: the rows Gamma'[T, .] */
} or_tables_desc;

typedef struct {
    uint32_t seed;
    int max_depth;     /* maximum number of path segments */
    int M;             /* light sub-paths per iteration */
    int M_p;           /* light sub-paths scanned for incomplete sub-paths */
    int repeats;       /* reciprocal estimates averaged per incomplete sub-path */
    int proxy;         /* proxy strategy on/off */
    int trial_cap;     /* maximum estimator nodes per repeat */
    int conn;          /* subspace connection strategy on/off */
    int pilot_min;     /* pilot draws per entry for its B, at least (rounded up to 32) */
    int pilot_max;     /* at most; 0 = no pilot (B from the table) */
    double side_in;    /* cosine draws at a dielectric y_{s-1} toward y_{s-2} (0: 0.5) */
    double booth;      /* > 0: Booth's Russian roulette of this scale in the reciprocal estimates
                        * (learning always uses the paper's RRS function) */
    int film;          /* strategies whose weighted contributions reach the pixel: 0 all, 1 the
                        * proxy strategy only, 2 all but the proxy strategy */
    int split_cap;     /* pre-order node index from which a node with |g| > 1 has one child of
                        * weight g instead of splitting (<= 0: never) */
    int fixed_bound;   /* 1: one B per estimate (the paper's walk); 0: a node with f/q > 2B hands
                        * its children the bound f/q (the raise rule) */
} or_params;

typedef struct {
    int64_t n_entries, n_truncated, n_nodes, n_conn, n_proxy, n_proxy_ok;
} or_stats;

void *or_create(const or_scene_desc *d);
/* 1: answer ray queries by brute force over all triangles (pins) */
void or_set_brute(void *h, int brute);
void or_free(void *h);

/* Philox-4x32-10 block and the uniform-variate helper (stream layout). */
void or_philox_block(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_uniform(uint32_t seed, uint32_t kind, uint32_t a, uint32_t b, uint32_t c, uint32_t d);

/* closest hit of n rays; rays: n*7 doubles (o, d, skip_tri); out: n*4 (tri, t, b1, b2) */
void or_closest_batch(void *h, int n, const double *rays, double *out);
/* occlusion of n segments; seg: n*8 (a, b, skip_a, skip_b); out: n ints */
void or_occluded_batch(void *h, int n, const double *seg, int *out);

/* BSDF of a material record (12 floats) with unit geometric normal n. */
void or_bsdf_eval_x(const float *mat, const double *n, const double *wl, const double *we, double *out3);
double or_bsdf_pdf_x(const float *mat, const double *n, const double *wg, const double *ws);
int or_bsdf_sample_x(const float *mat, const double *n, const double *wg, double u0, double u1,
                     double u2, double *ws);

/* Reciprocal estimator on a 1-D test integrand (pins; see or_recip.c).
 * fn: 0 f=1+sin(2 pi x)/2 on [0,1], q uniform; 1 f=3x^2, q uniform;
 *     2 f=3x^2, q = 0.5 uniform + 0.5 * 2x; 3 f = q (the ratio is 1).
 * out_t[i] = I~, out_i[i] = I (sign estimator), out_n[i] = nodes; returns
 * the number of truncated runs. */
int or_recip_1d(int fn, double B, int n_runs, uint32_t seed, int trial_cap, double *out_t,
                double *out_i, double *out_n);
/* The same with Booth's Russian roulette of scale c > 0 in place of the
 * paper's RRS function (one chain, no splitting; out_i is 0). */
int or_recip_1d_booth(int fn, double B, double c, int n_runs, uint32_t seed, int trial_cap, double *out_t,
                      double *out_i, double *out_n);

/* One incomplete light sub-path, as stored in the pool. */
typedef struct {
    int y_tri; double y_b1, y_b2;      /* specular end vertex y_{s-1} */
    int u;                              /* trailing specular count 1..4 */
    int type;                           /* 0: L S^u (no control vertex), 1: L D S^u (h_c = y_0) */
    int h_tri; double h_b1, h_b2;       /* control vertex h_c = y_0 (type 1) */
    int back;                           /* y_{s-2} lies behind y_{s-1}'s normal */
    double side_in;                     /* cosine draws at a dielectric y_{s-1} toward y_{s-2} (0: 0.5) */
} or_entry;

/* f and q of n proxy-path samples drawn from the supporting distribution of
 * entry e (Sec. 5.3), using stream (kind TRAIN, a, b, c=sample). */
void or_entry_fq(void *h, const or_entry *e, int n, uint32_t seed, uint32_t a, uint32_t b,
                 double *f_out, double *q_out);
/* Pilot B of entry e: the largest f/q of draws on stream (kind PILOT, a, b,
 * c = draw), at least min_draws and until one is non-zero, at most
 * max_draws (both rounded up to 32); 0 if every draw had f = 0. */
double or_entry_pilot(void *h, const or_entry *e, uint32_t seed, uint32_t a, uint32_t b, int min_draws,
                      int max_draws);
/* n independent reciprocal estimates (Alg. I~ and I) for entry e with bound B. */
int or_entry_recip(void *h, const or_entry *e, double B, int n, uint32_t seed, int trial_cap,
                   double *out_t, double *out_i, double *out_n);
/* The same with Booth's Russian roulette of scale c > 0. */
int or_entry_recip_booth(void *h, const or_entry *e, double B, double c, int n, uint32_t seed, int trial_cap,
                         double *out_t, double *out_i, double *out_n);

/* Reciprocal estimates of entries [k_lo, k_hi) of one iteration, equal to
 * those or_iteration computes (out_rhat[k - k_lo]); returns the iteration's
 * entry count. Only reads the handle, so threads may share it. */
int or_iteration_estimates(void *h, const or_params *p, const or_tables_desc *td, int iteration, const int *tri,
                           const float *bary, int k_lo, int k_hi, double *out_rhat);

/* Light pass of one iteration: light sub-path geometry. tri/bary are
 * [M][max_depth-1] (tri = -1 past the end). */
void or_light_pass(void *h, const or_params *p, int iteration, int *tri, float *bary);

/* One iteration given light geometry: pool build, reciprocal estimation,
 * eye pass over pixels [pix_lo, pix_hi). Outputs (may be NULL):
 *   rgb[(pix-pix_lo)*3] contribution of this camera sample, sig[pix-pix_lo]
 *   path signature; entry_rhat/entry_sig/entry_nodes per incomplete entry
 *   (up to cap entries; *n_entries gets the count). rhat_override, if not
 *   NULL, replaces the estimated reciprocals (one per entry). */
void or_iteration(void *h, const or_params *p, const or_tables_desc *t, int iteration,
                  const int *tri, const float *bary, int pix_lo, int pix_hi,
                  const double *rhat_override, double *rgb, uint32_t *sig,
                  int cap, int *n_entries, double *entry_rhat, uint32_t *entry_sig,
                  double *entry_nodes, or_stats *st);

/* Entries of one iteration's light geometry: out up to cap entries. */
int or_entries(void *h, const or_params *p, const int *tri, const float *bary, int cap,
               or_entry *out, int *light_index);

/* Full render: iterations [iter0, iter0+n_iter) accumulated into film
 * (W*H*3 doubles, sums) over pixels [pix_lo, pix_hi). */
void or_render(void *h, const or_params *p, const or_tables_desc *t, int iter0, int n_iter,
               int pix_lo, int pix_hi, double *film, or_stats *st);

/* Subspace labels of a vertex (nearest centroid, ties to the lowest index). */
int or_label_9(const or_tables_desc *t, const double *feat9, int K, const float *cent);

/* Learned light-subspace proposal (or_mlp.c): weights are a flat vector of
 * or_mlp_nparams(K, KT) doubles; raw features are 10 per row (normalised
 * position, facing normal, incident direction, roughness). */
size_t or_mlp_nparams(int K, int KT);
double or_bf16(double x);
void or_mlp_logits(const double *w, int K, int KT, int n, const double *raw, const int *T, int bf16, double *z);
int or_mlp_select(const double *w, int K, const double *raw, int T, const float *g, const int *start, double u,
                  double *Q);
double or_mlp_loss_grad(const double *w, int K, int KT, int n, const double *raw, const int *T, const int *S,
                        const double *wt, double *grad);
void or_mlp_adam(int np, double *w, const double *g, double *m1, double *m2, int t, double lr, double beta1,
                 double beta2, double eps);

/* split limit of or_recip_1d*, or_entry_recip* (default 2^16; <= 0: never) */
void or_set_split_default(int split);
/* bound rule of the same entry points (default 0: the raise rule; 1: one B per estimate) */
void or_set_fixed_bound_default(int fixed);

/* Statistics / selection learning (Sec. 5.4-5.5 as read in the design notes).
 * Inputs: centroids in t (gamma/B/mis/pi entries are ignored and rebuilt).
 * Outputs written to the caller's arrays. A (u, S', C) cell whose learning
 * estimates average more than max_chain estimator nodes each, or of which
 * one was truncated, gets MIS scale 0: its sub-paths are left to the other
 * strategies (max_chain <= 0: no such rule). */
void or_learn(void *h, const or_params *p, const or_tables_desc *t, int iter0, int n_iter,
              int n_bsamples, double max_chain, float *B_out, float *mis_out, float *gconn_out,
              float *gproxy_out, float *pi_out);

#ifdef __cplusplus
}
#endif
#endif
