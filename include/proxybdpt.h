/* proxybdpt -- C ABI of a GB300 (sm_103a) renderer for proxy-tracing BDPT.
 *
 * Method: "Proxy Tracing: Unbiased Reciprocal Estimation for Optimized
 * Sampling in BDPT" (arXiv 2503.23412). The renderer estimates the pixel
 * measurement I = int f(x) dmu(x) of the path-integral formulation (Sec. 3.1,
 * Eq. path intergral) with a probabilistic-connection bidirectional path
 * tracer (Sec. 3.2), adds the proxy strategy for light sub-paths that end on
 * specular vertices (Sec. 5.1-5.2) weighted by the reciprocal estimator
 * (Sec. 4.2, Appendix Alg. "Estimator I~") and the MIS weight for estimated
 * pdfs (Sec. 5.4, Eq. MIS_1), with subspace-based selection (Sec. 5.5).
 *
 * Conventions for every entry point:
 *  - Returns pb_status; PB_OK on success. No call aborts the process; on an
 *    error pb_last_error() returns a one-line description.
 *  - Pointers named host_* are host memory owned by the caller; the library
 *    copies from/to them before returning. The context owns all device memory
 *    it allocates and frees it in pb_destroy().
 *  - Calls are synchronous with respect to the host on return (work is issued
 *    on the context's stream and waited for), unless stated otherwise.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef PROXYBDPT_H
#define PROXYBDPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pb_ctx pb_ctx;

typedef enum {
    PB_OK = 0,
    PB_ERR_ARG = 1,        /* invalid argument or size */
    PB_ERR_OOM = 2,        /* device allocation failed */
    PB_ERR_CUDA = 3,       /* a CUDA call failed */
    PB_ERR_TIMEOUT = 4,    /* a bounded device loop gave up */
    PB_ERR_TRUNCATED = 5,  /* a reciprocal estimate hit its node cap (result still written) */
    PB_ERR_STATE = 6       /* call made in the wrong order (e.g. render before scene upload) */
} pb_status;

/* Scene (Sec. 3.1: surfaces, BSDFs, emitters, camera). Arrays are read
 * during the call only. Layout (float32 / int32, C order):
 *   verts[nv*3], uvs[nv*2] (may be NULL), tris[nt*3], tri_mat[nt],
 *   mats[nm*12]: kind(0 Lambert, 1 GGX conductor, 2 GGX dielectric),
 *     colour rgb, roughness (alpha = r^2; conductor/dielectric with r < 0.2
 *     is a specular vertex, Sec. 1 footnote), ior, Le rgb (front side),
 *     textured flag, 2 reserved;
 *   tex[tex_h*tex_w*3] emission texture (may be NULL when tex_w == 0);
 *   cam[12]: position, look-at, up, vertical fov (degrees), width, height;
 *     a pinhole with image x along forward x up (right-handed), image row 0
 *     at the top, and a box-filtered sample per pixel and iteration.
 * Errors: PB_ERR_ARG on empty or inconsistent sizes, out-of-range indices. */
typedef struct {
    int nv, nt, nm;
    const float *verts;
    const float *uvs;
    const int32_t *tris;
    const int32_t *tri_mat;
    const float *mats;
    int tex_w, tex_h;
    const float *tex;
    const float *cam;
} pb_scene_desc;

/* Frozen subspace tables (Sec. 5.4-5.5, Eq. subspaceApproximate):
 * centroids of the eye (T), light (S), specular (S') and control (C)
 * subspaces in bbox-normalised feature space (T, S: position, normal flipped
 * toward the incident direction, incident direction; S': position, normal;
 * C: position), the selection matrices Gamma[T,S] and Gamma'[T,S'], the
 * per-cell bound B(u,S',C) and MIS scale 1/(E[R^2] Pbar) (C = KC means "no
 * control vertex"), and the per-tile proxy probability. All float32. */
typedef struct {
    int KT, KS, KSp, KC;
    const float *bbox_lo, *bbox_hi;   /* 3 each */
    const float *cent_T;              /* KT*9 */
    const float *cent_S;              /* KS*9 */
    const float *cent_Sp;             /* KSp*6 */
    const float *cent_C;              /* KC*3 */
    const float *gamma_conn;          /* KT*KS, rows positive */
    const float *gamma_proxy;         /* KT*KSp */
    const float *B_tab;               /* 4*KSp*(KC+1), > 0 */
    const float *mis_tab;             /* 4*KSp*(KC+1), >= 0; 0 leaves the cell's sub-paths out of the proxy pool */
    int tile, grid_w, grid_h;
    const float *pi_grid;             /* grid_h*grid_w, in [0,1] */
} pb_tables_desc;

/* Render configuration. Iterations [iter0, iter0 + spp) are traced; each
 * iteration is one sample per pixel (Sec. 6: one iteration = 1 spp). */
typedef struct {
    uint32_t seed;
    int spp;
    int max_depth;     /* maximum number of path segments */
    int M;             /* light sub-paths per iteration (paper: 10,000) */
    int M_p;           /* light sub-paths scanned for incomplete sub-paths */
    int repeats;       /* reciprocal estimates averaged (paper: 5) */
    int proxy;         /* 1: proxy strategy on */
    int conn;          /* 1: subspace connections on (0 leaves PT + NEE) */
    int trial_cap;     /* node cap per reciprocal estimate (e.g. 65536) */
    int iter0;
    int batch;         /* iterations in flight per launch wave (0: automatic) */
    int count_traversal; /* 1: count BVH node fetches / triangle tests / rays (slower) */
    int chain_handoff;   /* estimator nodes a warp walks before a block takes the chain over (0: 512) */
    /* Per-entry bound B of the reciprocal estimator (App. "Optimal value for
     * B": B = max f/q of the integrand being estimated): the largest f/q of
     * draws from the entry's supporting distribution on its own stream, in
     * rounds of 32 -- at least pilot_min draws (0: 64), then until one has
     * f > 0, at most pilot_max (0: 1024; negative: no pilot). An entry whose
     * draws all had f = 0, or every entry with the pilot off, uses the learned
     * table value. */
    int pilot_min;
    int pilot_max;
    /* Light-subspace proposal of the subspace connection (Sec. 3.2): 0 = the
     * table row Gamma[T, .]; 1 = the learned network mixed with the table,
     * Q(S | x) = 0.9 softmax(MLP(x))_S + 0.1 Gamma[T, S] / Z_T over occupied
     * subspaces (needs a network: pb_mlp_upload or pb_train_proposal);
     * 2 = also the proxy strategy's specular subspace S' from its own network,
     * Q'(S' | x) = 0.9 softmax(MLP'(x))_S' + 0.1 Gamma'[T, S'] / Z'_T over the
     * subspaces that hold incomplete sub-paths, in place of the row
     * Gamma'[T, .] of Sec. 5.5 (needs pb_mlp_proxy_upload or training with
     * pb_train_desc.proxy = 1). The proxy estimate divides by the drawn
     * subspace's Q', so it stays unbiased. */
    int proposal;
    /* 1: capture the render's waves as a CUDA graph the first time this
     * configuration is seen on the context, then replay it (iter0 becomes a
     * device scalar set before each replay). Results are identical to the
     * eager path. The cache is dropped when the scene, the tables or the
     * buffers it points to change. */
    int graph;
    /* Supporting distribution (Sec. 5.3): share of the cosine draws at a
     * dielectric y_{s-1} that go to the side of the dropped vertex y_{s-2}
     * (0: 0.5, an even split; must be < 1 so that q covers both sides). */
    float side_in;
    /* Reciprocal-estimator schedule; the estimates are the same either way:
     * 0 = wavefront (all chains' node windows evaluated in stages, ray queries
     * answered by traversal-only kernels, then a warp walk per chain);
     * 1 = a warp phase then a block phase per chain. */
    int estimator;
    /* Russian roulette of the reciprocal estimator (Sec. 4.2): 0 = the
     * paper's RRS function r = |g| with splitting (Eq. rr); c > 0 = Booth's
     * roulette, the baseline of the paper's RR ablation: one chain without
     * splitting, whose k-node prefix continues with probability
     * min(1, c * prod_{i<k} |g_i|) (the printed factor 1/r read as a weight
     * cutoff, c = r). Both are unbiased. Booth's runs on the wavefront
     * schedule only (estimator 0; PB_ERR_ARG otherwise); table learning
     * always uses the paper's function. */
    float booth;
    /* How the wavefront estimator's trace stages and the eye pass's
     * occlusion answers map queries to threads: 0 = one query per thread;
     * 1 = persistent warps whose lanes take the next query as soon as theirs
     * is answered (ray replacement). The answers are the same either way. */
    int trace;
    /* Strategies whose weighted contributions reach the film: 0 = all; 1 =
     * only the proxy strategy (the paper's subspace-selection comparison
     * renders these paths alone); 2 = all but the proxy strategy. Sampling
     * and MIS weights are the same in every mode, so the modes' films add up
     * to the full one. */
    int film;
    /* Split limit of the reciprocal estimator (Alg. I~ with r = |g|): from
     * this pre-order node of an estimate on, a node with |g| > 1 has one child
     * entering with weight g instead of floor(|g|) + Bernoulli children of
     * weight sign(g). The estimate stays unbiased for any such rule; a tree
     * that would split without end (a bound B far below some f/q) continues
     * as a chain instead of reaching trial_cap. 0: 65536; negative: never
     * (the paper's rule throughout). */
    int split_cap;
    /* Bound of the reciprocal estimator's nodes. 0: the raise rule -- a node
     * that splits (|g| > 1, i.e. f/q > 2B) hands its children the bound
     * B' = its own f/q, and its Taylor term becomes g / B'. The estimate stays
     * unbiased for any bound fixed before a node's draw (1/beta = 1/B +
     * (1 - beta/B) / beta for every B), chains whose draws stay below 2B are
     * the paper's walk exactly, and a tree whose B sits far below the
     * integrand's f/q (outside the convergence condition 0 < beta/B < 2)
     * grows only as far as its own ratios instead of without end. 1: one B
     * for the whole estimate (the paper's walk throughout). */
    int fixed_bound;
} pb_config;

typedef struct {
    double ms;                 /* device time of the call */
    double mpaths_per_s;       /* W*H*spp / seconds */
    int64_t n_entries;         /* incomplete light sub-paths estimated */
    int64_t n_truncated;       /* estimates that hit trial_cap */
    int64_t n_nodes;           /* estimator nodes evaluated (trials) */
    int64_t n_conn, n_proxy, n_proxy_ok;
    double ms_light, ms_pool, ms_recip, ms_eye;   /* device time per stage (pb_render) */
    int64_t n_launches;                           /* kernels launched by the call */
    int64_t n_waves;                              /* launch waves (iterations in flight per wave) */
    /* traversal work when count_traversal = 1: the eye shading pass (proxy
     * retrace) and the estimator */
    int64_t eye_nodes, eye_tris, eye_rays, rec_nodes, rec_tris, rec_rays;
    double ms_mlp;             /* device time of the proposal's feature pass and network (proposal = 1) */
    double batch_ms;           /* pb_render_batch: device time of the whole batch (first entry only) */
    /* the eye side's stages (pb_render): camera sub-paths traced by the
     * feature pass (its time is in ms_mlp with the learned proposal, in
     * ms_eye otherwise) and the traversal-only occlusion answers (in ms_eye);
     * with count_traversal = 1 their traversal work (the eye_* counts above
     * keep the shading pass's own: the proxy retrace) */
    double ms_eye_feat, ms_eye_occ;
    int64_t cam_nodes, cam_tris, cam_rays, shd_nodes, shd_tris, shd_rays;
} pb_stats;

/* Creates a context on CUDA device `device`. cuda_stream: a cudaStream_t
 * the caller owns and keeps alive (all work of the context is issued on it),
 * or NULL for a stream the context creates and owns. *out receives the
 * context. PB_ERR_ARG for a NULL out, PB_ERR_CUDA if the device cannot be
 * used (no context is returned then). */
pb_status pb_create(pb_ctx **out, int device, void *cuda_stream /* NULL: own stream */);
/* Waits for the context's work, frees all its device memory, captured
 * graphs and its own stream (never a caller's stream). NULL is a no-op. */
void pb_destroy(pb_ctx *ctx);
/* One-line description of the last error on ctx ("null context" for NULL);
 * the string stays valid until the next call on ctx. */
const char *pb_last_error(const pb_ctx *ctx);

/* Builds the BVH on the host (binned SAH), checks its structure, and uploads
 * scene and BVH. Replaces any earlier scene and drops captured graphs. */
pb_status pb_scene_upload(pb_ctx *ctx, const pb_scene_desc *scene);
/* Copies the tables to the device, replacing earlier ones and dropping
 * captured graphs. PB_ERR_ARG on sizes out of range (every K >= 1, KS and
 * KSp <= 1023, KC <= 1000, tile >= 1, grid_w x grid_h = the image in tiles),
 * a NULL array or a B entry that is not positive; PB_ERR_STATE before a
 * scene upload. */
pb_status pb_tables_upload(pb_ctx *ctx, const pb_tables_desc *tables);

/* Renders n scenes (one context each, same device, each context at most
 * once) with their own configurations as ONE graph launch: each scene's
 * render graph (captured as with cfg.graph = 1) becomes a child of a parent
 * graph, so the scenes run concurrently and fill the GPU however uneven
 * their sizes. Each film receives exactly what pb_render would add;
 * stats[i] (may be NULL) is scene i's, stats[0].batch_ms the whole batch's.
 * Errors are reported on ctxs[0]. Returns PB_ERR_TRUNCATED if any scene's
 * estimator hit its cap. */
pb_status pb_render_batch(pb_ctx *const *ctxs, const pb_config *cfgs, int n, pb_stats *stats);

/* Autotuner: times trial renders of trial_iters iterations (0: 32; never
 * added to the film) over iterations in flight {4, 8, 16, 32} x estimator
 * schedule {wavefront, warp/block phases} and writes cfg with the fastest
 * pair into *best. Results are cached per size bucket (log2 of the triangle and
 * pixel counts, depth, M, M_p, repeats, proposal, proxy) for the process;
 * *from_cache (may be NULL) tells whether the cache answered. Neither
 * parameter changes an image beyond the estimator's summation order. With
 * booth > 0 only the wavefront schedule is tried, under its own cache key. */
pb_status pb_autotune(pb_ctx *ctx, const pb_config *cfg, int trial_iters, pb_config *best, int *from_cache);
/* the cache as text lines "bucket batch estimator ms_per_iteration" */
pb_status pb_autotune_cache_save(const char *path);
pb_status pb_autotune_cache_load(const char *path);
void pb_autotune_cache_clear(void);

/* Table learning (Sec. 5.4-5.5): n_iter learning iterations, numbered from
 * iter0 and never added to the film, build on the device
 *  - k-means centroids of the eye, light, specular and control subspaces
 *    (lloyd_iters Lloyd steps from evenly spaced samples), unless
 *    keep_centroids = 1 keeps those of the uploaded tables;
 *  - B(u,S',C) = b_safety (0: 1.0) x the largest f/q of n_bsamples draws per
 *    incomplete sub-path (App. "Optimal value for B": B = max f/q);
 *  - the MIS scale mean(R)/mean(R^2) per cell (Sec. 5.4, Eq. MIS_1);
 *  - Gamma rows proportional to the accumulated unweighted contribution
 *    (0.9 x normalised + 0.1 uniform) and the 10x10-tile proxy probability
 *    (1.0 where the proxy share is >= 5 %, else 0.2; Sec. 6.1.1);
 *  - a cost bound on the proxy strategy's sub-path types, extending the
 *    paper's own limits (Sec. 6.1.1: only L S^u and L D S^u with u <= 4 are
 *    estimated, the rest is left to the subspace connections): a cell whose
 *    learning estimates average more than max_chain estimator nodes each
 *    (0: 4096; negative: no bound), or in which one entry's estimates took
 *    trial_cap nodes or more in total, gets MIS scale 0. Its sub-paths then
 *    never enter the proxy pool, and every strategy's weight already gives
 *    the proxy no share of such paths, so the image stays unbiased.
 * The learned tables replace the current ones. Table sizes KT, KS, KSp, KC
 * and tile apply when the centroids are learned (KS, KSp <= 1023). */
typedef struct {
    int KT, KS, KSp, KC, tile;
    int n_iter;
    uint32_t iter0;
    int n_bsamples;
    int lloyd_iters;
    int keep_centroids;
    float b_safety;
    float max_chain;
} pb_learn_desc;
pb_status pb_prepare(pb_ctx *ctx, const pb_config *cfg, const pb_learn_desc *learn, pb_stats *stats_or_null);

/* Copies the current tables to caller buffers sized as in pb_tables_desc.
 * Sizes (K*, tile, grid) are always written; if any pointer is NULL only the
 * sizes are returned. */
typedef struct {
    int KT, KS, KSp, KC, tile, grid_w, grid_h;
    float *bbox_lo, *bbox_hi, *cent_T, *cent_S, *cent_Sp, *cent_C;
    float *gamma_conn, *gamma_proxy, *B_tab, *mis_tab, *pi_grid;
} pb_tables_host;
pb_status pb_tables_readback(pb_ctx *ctx, pb_tables_host *out);

/* Traces cfg->spp iterations and adds them to the film. PB_ERR_TRUNCATED
 * if any estimate hit the cap (the film is still updated). */
pb_status pb_render(pb_ctx *ctx, const pb_config *cfg, pb_stats *stats_or_null);
pb_status pb_film_clear(pb_ctx *ctx);
/* Mean radiance per pixel, W*H*3 floats (host_rgb must hold n_floats). */
pb_status pb_film_readback(pb_ctx *ctx, float *host_rgb, size_t n_floats);
/* Device pointer of the film sum (W*H*3 float32) and its iteration count. */
pb_status pb_film_device(pb_ctx *ctx, float **dev_sum, int64_t *iterations);

/* ---- queries used by the parity tests ------------------------------------ */
/* Closest hits: host_rays n*7 (origin, direction, skip tri); host_hits n*4
 * (tri or -1, t, b1, b2). Stackless BVH traversal. */
pb_status pb_trace(pb_ctx *ctx, const float *host_rays, int n, float *host_hits);
/* Occlusion of segments a->b: host_seg n*8 (a, b, skip_a, skip_b). */
pb_status pb_occluded(pb_ctx *ctx, const float *host_seg, int n, int32_t *host_out);
/* Light pass of one iteration: geometry [M][max_depth-1] (tri, b1 b2). */
pb_status pb_light_pass(pb_ctx *ctx, const pb_config *cfg, int iteration, int32_t *host_tri,
                        float *host_bary);
/* One iteration on given light geometry: pool build, reciprocal estimation
 * (or host_rhat_override if not NULL: M*(max_depth-1) doubles of which the
 * first n_entries, in (light path, vertex) order, are used), eye pass.
 * Triangle indices must lie in [-1, nt) (PB_ERR_ARG otherwise). Outputs per
 * pixel: this sample's radiance (W*H*3) and path signature (W*H); per entry
 * up to cap: estimate, signature, nodes. */
pb_status pb_iteration(pb_ctx *ctx, const pb_config *cfg, int iteration, const int32_t *host_tri,
                       const float *host_bary, const double *host_rhat_override,
                       float *host_pix_rgb, uint32_t *host_pix_sig, int cap, int *n_entries,
                       float *host_entry_rhat, uint32_t *host_entry_sig, float *host_entry_nodes,
                       pb_stats *stats_or_null);

/* ---- allocation-free reciprocal estimates ---------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory while they run -- an engine that
 * reserves all of its device memory up front, a process whose allocations
 * are capped or pooled by another runtime, or a latency-critical path where
 * cudaMalloc/cudaFree's implicit synchronisation is not acceptable.
 *
 * It computes the averaged reciprocal estimate of n incomplete light
 * sub-paths on the context's scene -- the same values pb_iteration computes
 * for its pool when given the same entries in (light path, vertex) order,
 * the same iteration, seed, repeats, trial_cap, side_in and B -- and
 * allocates nothing: its scratch is a file-scope device array of
 * PB_NOALLOC_MAX_ESTIMATES (entry, repeat) slots (about 200 KB) that a device
 * keeps from the library's first use on it until the process exits.
 * pb_create looks up the array's device address for its context (that
 * set-up may load the library's device code and place the array on the
 * device); this call then only launches kernels and copies 12 bytes back.
 * Calls with n * cfg->repeats above that maximum return PB_ERR_ARG. All
 * calls share the array and it keeps the last call's contents (each call
 * clears its counters first): calls whose work overlaps on the GPU (two
 * contexts or streams at once) race on it. The call is synchronous.
 *
 * Device inputs (caller-owned): d_tri[2n] (y_{s-1} triangle, h_c triangle),
 * d_bary[4n] (their barycentrics), d_info[n] (u | type << 3 | back << 30, type 1 =
 * L D S^u, back 1 when y_{s-2} lies behind y_{s-1}'s normal),
 * d_B[n] (bound B > 0 per entry). Device outputs: d_rhat[n], d_nodes[n] (total
 * estimator nodes over the repeats, may be NULL). *n_truncated (may be NULL)
 * counts entries with a repeat that hit trial_cap or its split stack. From
 * cfg only seed, repeats (1..8), trial_cap (> 0), side_in ([0, 1), 0 for an
 * even split), split_cap and fixed_bound are read; the roulette is always the paper's RRS
 * function.
 * An entry whose B is not positive (or NaN) gets a NaN estimate and the call
 * returns PB_ERR_ARG after writing the other entries' estimates. */
#define PB_NOALLOC_MAX_ESTIMATES 16384
pb_status pb_recip_estimates_noalloc(pb_ctx *ctx, const pb_config *cfg, int iteration, int n,
                                     const int32_t *d_tri, const float *d_bary, const int32_t *d_info,
                                     const float *d_B, float *d_rhat, float *d_nodes, int *n_truncated);

/* ---- learned light-subspace proposal --------------------------------------
 * Not in the paper, which selects the light subspace of a connection from the
 * learned table Gamma[T, .] (Sec. 3.2, Sec. 5.5). The network maps features
 * of the eye vertex x = (position normalised to the table box, normal facing
 * the incident direction, incident direction, roughness, a 4-d embedding of
 * T, 1, 0) through 16 -> 64 ReLU -> 64 ReLU -> KS logits. Weights are a flat
 * fp32 vector, row-major with the output index first:
 *   W1[64][16] | W2[64][64] | b2[64] | W3[KS][64] | b3[KS] | E[KT][4]
 * with KS, KT those of the uploaded tables (KS <= 384). Inference runs with
 * bf16 operands and fp32 accumulation on the tensor cores; training in fp32.
 * The loss of a batch is -(1/n) sum_b w_b log softmax(z_b)[S_b]. All calls
 * are synchronous. */
size_t pb_mlp_nparams(int KS, int KT);
/* copies the n = pb_mlp_nparams weights (host) and resets Adam's moments */
pb_status pb_mlp_upload(pb_ctx *ctx, const float *w, size_t n);
pb_status pb_mlp_readback(pb_ctx *ctx, float *w, size_t n);
/* the proxy strategy's network: the same layout with KSp outputs, n =
 * pb_mlp_nparams(KSp, KT) with the tables' KSp (<= 384) */
pb_status pb_mlp_proxy_upload(pb_ctx *ctx, const float *w, size_t n);
pb_status pb_mlp_proxy_readback(pb_ctx *ctx, float *w, size_t n);
/* logits of n rows: raw features n x 10 (host), eye subspaces T (host); z is
 * n x KS (host). Runs the tensor-core kernel of the render path. */
pb_status pb_mlp_logits(pb_ctx *ctx, int n, const float *raw, const int32_t *T, float *z);
/* gradient of the batch loss (host arrays: raw n x 10, T, S, w; grad has
 * pb_mlp_nparams entries); loss may be NULL */
pb_status pb_mlp_grad(pb_ctx *ctx, int n, const float *raw, const int32_t *T, const int32_t *S, const float *w,
                      float *grad, float *loss);
/* one Adam step (beta 0.9 / 0.999, eps 1e-8) on the gradient of the batch */
pb_status pb_mlp_train_batch(pb_ctx *ctx, int n, const float *raw, const int32_t *T, const int32_t *S,
                             const float *w, float lr, float *loss);

typedef struct {
    int samples;               /* training samples collected per round (buffer size) */
    int rounds;                /* collect-then-train rounds */
    int steps;                 /* Adam steps per round */
    int batch;                 /* samples per step, drawn with replacement from the round's samples */
    float lr;                  /* Adam step size (0: 1e-3) */
    uint32_t seed;             /* initialisation and mini-batch draws */
    int iter0;                 /* first iteration number of the collection renders */
    int max_iters_per_round;   /* collection iterations per round at most (0: 256) */
    int iters_per_wave;        /* iterations in flight while collecting (0: 8) */
    int reinit;                /* 1: start from a fresh initialisation even if a network is loaded */
    int learned_first;         /* 1: the first round already collects with the network */
    int proxy;                 /* 1: also train the proxy strategy's network (proposal 2) */
} pb_train_desc;

typedef struct {
    int64_t iterations, samples, steps;
    double loss_first, loss_last;
    int64_t samples_proxy;     /* the proxy network's training samples (proxy = 1) */
    double loss_proxy_first, loss_proxy_last;
} pb_train_stats;

/* Online training: each round renders collection iterations (never added to
 * the film) with the current proposal -- the table in the first round unless
 * learned_first -- and records one sample per connection with a non-zero
 * contribution (features, T, the chosen S, the unweighted contribution
 * luminance, which already carries the 1/Q(S) of the proposal that drew it),
 * then takes `steps` Adam steps on mini-batches of those samples. With
 * proxy = 1 each successful proxy connection also records a sample (its S',
 * the unweighted contribution luminance clamped at 0, since the reciprocal
 * estimate in it is signed) and the proxy network takes its own steps. */
pb_status pb_train_proposal(pb_ctx *ctx, const pb_config *cfg, const pb_train_desc *td, pb_train_stats *out);

/* Moments of the subspace-connection estimate under cfg->proposal: renders
 * iterations [iter0, iter0 + spp) without touching the film and returns
 * out[0] = connections made, out[1] = sum of their unweighted contribution
 * luminance, out[2] = sum of its squares. Both proposals are unbiased, so
 * out[1] / out[0] agrees between them up to noise, and the proposal with the
 * smaller out[2] / out[0] is the better one. */
pb_status pb_connection_moments(pb_ctx *ctx, const pb_config *cfg, double *out);

/* ---- memory read bandwidth (measurement) -----------------------------------
 * The paper has no counterpart; this gives the roofline denominators of the
 * traversal kernels on the machine at hand. Allocates `bytes` on `device`,
 * reads it once to warm up, then `reps` times with loads cached in L2 only,
 * and writes the read rate in GB/s (10^9 bytes/s) to *gbs. Below the L2
 * size this is the L2 read rate, far above it the HBM read rate. Synchronous;
 * frees everything it allocates. PB_ERR_ARG for bytes < 4096, reps < 1 or a
 * NULL gbs; PB_ERR_OOM when the buffer cannot be allocated. */
pb_status pb_read_bandwidth(int device, size_t bytes, int reps, double *gbs);

#ifdef __cplusplus
}
#endif
#endif
