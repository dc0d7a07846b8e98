/* CPU oracle (test infrastructure only): the learned light-subspace proposal.
 *
 * The method selects the light subspace S of a connection from the row
 * Gamma[T, .] of its eye subspace T (Sec. 3.2 and Sec. 5.5, "proportional to
 * expected contribution"). This file is the learned alternative: a small
 * network maps features x of the eye vertex to logits over the KS light
 * subspaces; the proposal mixes its softmax (renormalised over the
 * subspaces that hold light vertices) with the table row,
 *     Q(S | x) = (1 - eps) p(S | x) + eps gamma(S),   eps = 0.1,
 * so Q(S) > 0 wherever the table is positive and the connection estimate
 * f / (M Q(S) / |S|) stays unbiased (Sec. 3.2). The network is trained to
 * minimise the cross-entropy between the contribution-weighted selections
 * and p, i.e. loss = -(1/n) sum_b w_b log p(S_b | x_b), with w_b the
 * connection's unweighted contribution luminance (which already carries the
 * 1 / Q(S_b) of the proposal that drew it): the per-sample form of the KL
 * gradient used for neural importance sampling (Mueller et al. 2019).
 *
 * Network: x (16) -> 64 ReLU -> 64 ReLU -> KS logits.
 *   x = [position normalised to the table box (3), normal facing the
 *        incident direction (3), incident direction (3), roughness (1),
 *        embedding of T (4), 1 (bias of the first layer), 0]
 * Flat weight vector (row-major, output index first):
 *   W1[64][16] | W2[64][64] | b2[64] | W3[KS][64] | b3[KS] | E[KT][4]
 * The device runs the forward pass with bf16 operands and fp32 sums; with
 * `bf16` set the oracle rounds x, the weights and the hidden activations to
 * bf16 at the same points (round to nearest even), so both sides take the
 * same sampling decisions. Gradients and Adam are plain FP64. */
#include "or_internal.h"

#define H 64
#define NX 16
#define EPS_MIX 0.1

static size_t off_W2(void) { return (size_t)H * NX; }
static size_t off_b2(void) { return off_W2() + (size_t)H * H; }
static size_t off_W3(void) { return off_b2() + H; }
static size_t off_b3(int K) { return off_W3() + (size_t)K * H; }
static size_t off_E(int K) { return off_b3(K) + (size_t)K; }

size_t or_mlp_nparams(int K, int KT) { return off_E(K) + 4 * (size_t)KT; }

/* round to bf16 (8-bit significand), nearest even, via the float value */
double or_bf16(double x) {
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (double)f;   /* inf / nan unchanged */
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double rnd(double x, int bf16) { return bf16 ? or_bf16(x) : x; }
static double as_f32(double x) { return (double)(float)x; }

/* x from the raw features (10) and the embedding row of T */
static void make_x(const double *w, int K, const double *raw, int T, double *x) {
    for (int i = 0; i < 10; ++i) x[i] = raw[i];
    for (int i = 0; i < 4; ++i) x[10 + i] = w[off_E(K) + 4 * (size_t)T + i];
    x[14] = 1.0;
    x[15] = 0.0;
}

static void forward(const double *w, int K, const double *x_in, int bf16, double *x, double *h1, double *h2,
                    double *z) {
    for (int c = 0; c < NX; ++c) x[c] = rnd(x_in[c], bf16);
    for (int i = 0; i < H; ++i) {
        double s = 0.0;
        for (int c = 0; c < NX; ++c) s += rnd(w[(size_t)i * NX + c], bf16) * x[c];
        h1[i] = rnd(s > 0.0 ? s : 0.0, bf16);
    }
    for (int i = 0; i < H; ++i) {
        double s = 0.0;
        for (int j = 0; j < H; ++j) s += rnd(w[off_W2() + (size_t)i * H + j], bf16) * h1[j];
        s += bf16 ? as_f32(w[off_b2() + i]) : w[off_b2() + i];
        h2[i] = rnd(s > 0.0 ? s : 0.0, bf16);
    }
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int j = 0; j < H; ++j) s += rnd(w[off_W3() + (size_t)k * H + j], bf16) * h2[j];
        z[k] = s + (bf16 ? as_f32(w[off_b3(K) + k]) : w[off_b3(K) + k]);
    }
}

/* logits of n rows of raw features (n x 10) with eye subspaces T */
void or_mlp_logits(const double *w, int K, int KT, int n, const double *raw, const int *T, int bf16, double *z) {
    (void)KT;
    double xin[NX], x[NX], h1[H], h2[H];
    for (int b = 0; b < n; ++b) {
        make_x(w, K, raw + 10 * (size_t)b, T[b], xin);
        forward(w, K, xin, bf16, x, h1, h2, z + (size_t)b * K);
    }
}

/* Proposal of one eye vertex: S and Q(S). `g` is the table row Gamma[T, .],
 * `start` the bucket starts of the light subspaces (S holds light vertices
 * iff start[S+1] > start[S]). One uniform u chooses the mixture component:
 * u < eps draws S from the table row restricted to occupied subspaces with
 * u / eps; otherwise S is drawn from the renormalised softmax with
 * (u - eps) / (1 - eps). Returns -1 when no subspace is occupied. */
int or_mlp_select(const double *w, int K, const double *raw, int T, const float *g, const int *start, double u,
                  double *Q) {
    double xin[NX], x[NX], h1[H], h2[H];
    double *z = (double *)malloc(sizeof(double) * (size_t)K);
    make_x(w, K, raw, T, xin);
    forward(w, K, xin, 1, x, h1, h2, z);
    double m = -INFINITY, Zg = 0.0;
    int last = -1;
    for (int k = 0; k < K; ++k) {
        if (start[k + 1] == start[k]) continue;
        if (z[k] > m) m = z[k];
        Zg += g[k];
        last = k;
    }
    if (last < 0) {
        free(z);
        return -1;
    }
    double Z = 0.0;
    for (int k = 0; k < K; ++k)
        if (start[k + 1] > start[k]) Z += exp(z[k] - m);
    int pick = last;
    if (u < EPS_MIX) {
        double ut = u / EPS_MIX, cum = 0.0;
        for (int k = 0; k < K; ++k) {
            if (start[k + 1] == start[k]) continue;
            cum += g[k] / Zg;
            if (ut < cum) {
                pick = k;
                break;
            }
        }
    } else {
        double target = (u - EPS_MIX) / (1.0 - EPS_MIX) * Z, cum = 0.0;
        for (int k = 0; k < K; ++k) {
            if (start[k + 1] == start[k]) continue;
            cum += exp(z[k] - m);
            if (target < cum) {
                pick = k;
                break;
            }
        }
    }
    *Q = (1.0 - EPS_MIX) * exp(z[pick] - m) / Z + EPS_MIX * g[pick] / Zg;
    free(z);
    return pick;
}

/* loss = -(1/n) sum_b w_b log softmax(z_b)[S_b] over all K logits, and its
 * gradient with respect to the flat weight vector (added into `grad`). */
double or_mlp_loss_grad(const double *w, int K, int KT, int n, const double *raw, const int *T, const int *S,
                        const double *wt, double *grad) {
    (void)KT;
    double xin[NX], x[NX], h1[H], h2[H], dh1[H], dh2[H];
    double *z = (double *)malloc(sizeof(double) * (size_t)K);
    double *dz = (double *)malloc(sizeof(double) * (size_t)K);
    double loss = 0.0;
    for (int b = 0; b < n; ++b) {
        make_x(w, K, raw + 10 * (size_t)b, T[b], xin);
        forward(w, K, xin, 0, x, h1, h2, z);
        double m = -INFINITY;
        for (int k = 0; k < K; ++k)
            if (z[k] > m) m = z[k];
        double Z = 0.0;
        for (int k = 0; k < K; ++k) Z += exp(z[k] - m);
        double lse = m + log(Z);
        double a = wt[b] / n;
        loss += -a * (z[S[b]] - lse);
        /* d/dz_k = a (p_k - [k = S]) */
        for (int k = 0; k < K; ++k) dz[k] = a * (exp(z[k] - lse) - (k == S[b] ? 1.0 : 0.0));
        for (int j = 0; j < H; ++j) dh2[j] = 0.0;
        for (int k = 0; k < K; ++k) {
            grad[off_b3(K) + k] += dz[k];
            for (int j = 0; j < H; ++j) {
                grad[off_W3() + (size_t)k * H + j] += dz[k] * h2[j];
                dh2[j] += dz[k] * w[off_W3() + (size_t)k * H + j];
            }
        }
        for (int i = 0; i < H; ++i) {
            if (!(h2[i] > 0.0)) dh2[i] = 0.0;
            grad[off_b2() + i] += dh2[i];
        }
        for (int j = 0; j < H; ++j) dh1[j] = 0.0;
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < H; ++j) {
                grad[off_W2() + (size_t)i * H + j] += dh2[i] * h1[j];
                dh1[j] += dh2[i] * w[off_W2() + (size_t)i * H + j];
            }
        for (int i = 0; i < H; ++i)
            if (!(h1[i] > 0.0)) dh1[i] = 0.0;
        for (int i = 0; i < H; ++i)
            for (int c = 0; c < NX; ++c) grad[(size_t)i * NX + c] += dh1[i] * x[c];
        /* the embedding enters through x[10..13] */
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int i = 0; i < H; ++i) s += dh1[i] * w[(size_t)i * NX + 10 + c];
            grad[off_E(K) + 4 * (size_t)T[b] + c] += s;
        }
    }
    free(z);
    free(dz);
    return loss;
}

/* Adam (Kingma and Ba 2015), step t >= 1, bias-corrected moments */
void or_mlp_adam(int np, double *w, const double *g, double *m1, double *m2, int t, double lr, double beta1,
                 double beta2, double eps) {
    double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
    for (int i = 0; i < np; ++i) {
        m1[i] = beta1 * m1[i] + (1.0 - beta1) * g[i];
        m2[i] = beta2 * m2[i] + (1.0 - beta2) * g[i] * g[i];
        w[i] -= lr * (m1[i] / c1) / (sqrt(m2[i] / c2) + eps);
    }
}
