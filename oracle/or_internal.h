/* CPU oracle for proxy-tracing BDPT -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 restatement of the method of "Proxy Tracing: Unbiased
 * Reciprocal Estimation for Optimized Sampling in BDPT" (arXiv 2503.23412).
 * It shares no code with the CUDA renderer and is used only by tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline leg.
 *
 * Internal header: vector helpers and data types used by the oracle's .c files.
 */
#ifndef OR_INTERNAL_H
#define OR_INTERNAL_H

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct { double x, y, z; } v3;

static inline v3 v3m(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static inline v3 vadd(v3 a, v3 b) { return v3m(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline v3 vsub(v3 a, v3 b) { return v3m(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline v3 vscale(v3 a, double s) { return v3m(a.x * s, a.y * s, a.z * s); }
static inline v3 vneg(v3 a) { return v3m(-a.x, -a.y, -a.z); }
static inline double vdot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline v3 vcross(v3 a, v3 b) {
    return v3m(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static inline double vlen(v3 a) { return sqrt(vdot(a, a)); }
static inline v3 vnorm(v3 a) { return vscale(a, 1.0 / vlen(a)); }
static inline v3 vmul(v3 a, v3 b) { return v3m(a.x * b.x, a.y * b.y, a.z * b.z); }
static inline double vmaxc(v3 a) { return fmax(a.x, fmax(a.y, a.z)); }
static inline double vsumc(v3 a) { return a.x + a.y + a.z; }

/* ---- Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ---------------- */
void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* uniform in [0,1): the top 24 bits of one Philox output word times 2^-24
 * (exactly representable in float and double). Stream layout: key =
 * (seed, kind), counter = (a, b, c, d >> 2), word d & 3. */
double or_rnd(uint32_t seed, uint32_t kind, uint32_t a, uint32_t b, uint32_t c, uint32_t d);

enum { K_CAMERA = 1, K_LIGHT = 2, K_RECIP = 3, K_TRAIN = 4, K_PILOT = 6 };

/* ---- scene --------------------------------------------------------------- */
enum { MK_LAMBERT = 0, MK_CONDUCTOR = 1, MK_DIELECTRIC = 2 };

typedef struct {
    int kind;
    v3 color;
    double rough, alpha, ior;
    v3 Le;
    int textured;
    int specular;   /* S vertex: conductor/dielectric with roughness < 0.2 */
    int emitter;    /* Le > 0 */
} or_mat;

typedef struct {
    int nv, nt, nm;
    v3 *P;
    double *UV;
    int *T, *tm;
    v3 *N;          /* unit geometric normal (v1-v0)x(v2-v0) */
    double *area;
    or_mat *mats;
    int tw, th;
    const float *tex;
    int ne;          /* emitter triangles */
    int *etri;
    double *ecdf;    /* cumulative power share, last entry 1 */
    double *epmf;    /* per emitter triangle: probability of choosing it */
    int *tri2e;      /* triangle -> emitter slot, -1 if not an emitter */
    v3 lo, hi;
    double extent, eps_t;
    v3 cpos, cfwd, cright, cup;
    double tanh_, aspect;
    int W, H;
    /* bounding-volume hierarchy used to accelerate or_closest/or_occluded;
     * it changes no result (every triangle whose box the ray meets is
     * tested with the same predicate and tie rule as the brute force). */
    int nnodes;
    double *blo, *bhi;   /* 3 per node */
    int *bl, *br;        /* children (internal) or -1 */
    int *bfirst, *bcount;
    int *order;          /* triangle indices in leaf order */
    int brute;           /* 1: ignore the hierarchy */
} or_scene_t;

typedef struct { int tri; double t, b1, b2; } or_hit;

/* a path vertex in world space */
typedef struct {
    v3 p, n;         /* position, unit geometric normal */
    int tri, mat;
    int is_light;    /* x_0 of a full path (emitter sample or emitter hit) */
    double b1, b2;   /* barycentrics on tri */
} or_vtx;

/* scene.c */
int or_scene_init(or_scene_t *s, const or_scene_desc *d);
void or_scene_free(or_scene_t *s);
or_hit or_closest(const or_scene_t *s, v3 o, v3 d, int skip);
or_hit or_closest_brute(const or_scene_t *s, v3 o, v3 d, int skip);
int or_occluded(const or_scene_t *s, v3 a, v3 b, int skip_a, int skip_b);
or_vtx or_vertex_at(const or_scene_t *s, int tri, double b1, double b2);
v3 or_emitted(const or_scene_t *s, const or_vtx *v, v3 w);   /* Le toward w (front only) */
double or_light_pdf(const or_scene_t *s, int tri);             /* area density p_L */
int or_sample_light(const or_scene_t *s, double u0, double u1, double u2, int *tri, double *b1, double *b2);
void or_onb(v3 n, v3 *t, v3 *b);
v3 or_cosine_dir(v3 n, double u1, double u2);
int or_is_specular(const or_scene_t *s, int tri);
int or_absorbing(const or_scene_t *s, const or_vtx *v, v3 w_in);

/* bsdf.c: directions are unit and point away from the surface.
 * eval: radiance BSDF for light arriving from w_light scattered to w_eye.
 * pdf:  solid-angle density of sampling w_s given w_g.
 * sample: draws w_s given w_g; returns 0 on failure. */
v3 or_bsdf_eval(const or_mat *m, v3 n, v3 w_light, v3 w_eye);
double or_bsdf_pdf(const or_mat *m, v3 n, v3 w_g, v3 w_s);
int or_bsdf_sample(const or_mat *m, v3 n, v3 w_g, double u0, double u1, double u2, v3 *w_s);

#endif
