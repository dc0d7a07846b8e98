// Reciprocal estimates for caller-supplied incomplete light sub-paths with no
// device allocation in the call (pb_recip_estimates_noalloc).
//
// Some callers cannot allocate device memory while they run: a host engine
// that owns all device memory up front and forbids later allocation, a
// process whose allocations are capped or pooled by another runtime, or code
// on a path where cudaMalloc's implicit synchronisation is not acceptable.
// This entry point serves them. Its inputs and outputs are the caller's
// device buffers; its scratch -- one estimate, node count and status flag
// per (entry, repeat), plus a work counter -- lives in the file-scope array
// below, sized for PB_NOALLOC_MAX_ESTIMATES estimates. A device holds that
// array from the library's first use on it until the process exits;
// pb_create looks up its address once per context (pb_noalloc_setup), so the
// entry point itself never allocates or loads anything.
//
// The kernel is a one-phase form of the estimator (Sec. 4.2, App. Alg. I~):
// one warp per (entry, repeat) draws 32 pre-order nodes at a time and
// replays the sequential walk with a stack of 48 frames (children whose
// weight and bound match the top frame join it). It uses the same
// streams as the pooled estimator in pb_light.cu, so both produce the same
// estimates.
#include "pb_ctx.h"
#include "pb_estimator.cuh"

namespace {

constexpr int NA_MAXF = 48;

// the walk state a warp keeps (every lane holds the same copy)
struct NAStack {
    float cur_sign, cur_ib;
    int sp;
    float fr_sign[NA_MAXF], fr_ib[NA_MAXF];
    int fr_rem[NA_MAXF];
};

struct NAScratch {
    int work;        // next (entry, repeat) to claim; cleared at the start of each call
    int ntrunc;      // entries with a truncated repeat; cleared at the start of each call
    int nbad;        // entries whose bound B is not positive; cleared at the start of each call
    int pad[61];
    float est[PB_NOALLOC_MAX_ESTIMATES];
    float nodes[PB_NOALLOC_MAX_ESTIMATES];
    int flag[PB_NOALLOC_MAX_ESTIMATES];   // 1 truncated, 2 bound not positive
};

// In host code `g_na_scratch` names a host-side stand-in, not device memory:
// kernels get the address obtained from cudaGetSymbolAddress in
// pb_noalloc_setup.
static __device__ __align__(256) NAScratch g_na_scratch;

__global__ void __launch_bounds__(128) k_na_recip(DScene S, KParams P, uint32_t iteration, int n,
                                                  const int32_t *tri, const float *bary, const int32_t *info,
                                                  const float *Bv, NAScratch *sc) {
    int lane = threadIdx.x & 31;
    int total = n * P.repeats;
    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&sc->work, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        int k = item / P.repeats, rep = item % P.repeats;
        Entry E;
        E.Y = vertex_at(S, tri[2 * k], bary[4 * k], bary[4 * k + 1]);
        E.H = vertex_at(S, tri[2 * k + 1], bary[4 * k + 2], bary[4 * k + 3]);
        E.u = info[k] & 7;
        E.type = (info[k] >> 3) & 1;
        E.back = (info[k] >> 30) & 1;
        E.pin = P.side_in;
        const float Bk = Bv[k];
        if (!(Bk > 0.0f)) {   // not a valid bound (zero, negative or NaN): no estimate
            if (lane == 0) {
                sc->est[item] = __int_as_float(0x7fc00000);
                sc->nodes[item] = 0.0f;
                sc->flag[item] = 2;
            }
            continue;
        }
        float invB = 1.0f / Bk;
        double sum_t = 0.0;
        int nodes = 0;
        bool done = false, trunc = false;
        NAStack ws;
        ws.cur_sign = 1.0f;
        ws.cur_ib = invB;
        ws.sp = 0;
        for (int base = 0; !done; base += 32) {
            int v = base + lane;
            float g = 1.0f, x = 0.0f, u = 1.0f;
            int nch = 0;
            if (v < P.trial_cap) {
                Rng R;
                R.init(P.seed, K_RECIP, iteration, (uint32_t)(k * 8 + rep), (uint32_t)v);
                x = entry_ratio<false>(S, E, R, nullptr);
                u = R.u(18);
                g = est_g(x, invB);
                nch = est_children(g, u, (uint32_t)v, P.split);
            }
            for (int j = 0; j < 32; ++j) {
                const float gj = __shfl_sync(0xffffffffu, g, j), xj = __shfl_sync(0xffffffffu, x, j);
                const float uj = __shfl_sync(0xffffffffu, u, j);
                const int nj = __shfl_sync(0xffffffffu, nch, j);
                if (done) continue;
                if (base + j >= P.trial_cap) {
                    done = true;
                    trunc = true;
                    continue;
                }
                const EstStep e = est_step(ws, xj, uj, gj, nj, invB, (uint32_t)(base + j), P);
                nodes++;
                const int r = est_take<NA_MAXF>(ws, e, sum_t);
                if (r) {
                    done = true;
                    trunc = r == 2;
                }
            }
        }
        if (lane == 0) {
            sc->est[item] = (float)((double)invB + sum_t);
            sc->nodes[item] = (float)nodes;
            sc->flag[item] = trunc ? 1 : 0;
        }
    }
}

__global__ void k_na_finish(KParams P, int n, NAScratch *sc, float *rhat, float *nodes_out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double acc = 0.0;
    float nn = 0.0f;
    int fl = 0;
    for (int r = 0; r < P.repeats; ++r) {
        acc += (double)sc->est[k * P.repeats + r];
        nn += sc->nodes[k * P.repeats + r];
        fl |= sc->flag[k * P.repeats + r];
    }
    rhat[k] = (float)(acc / (double)P.repeats);
    if (nodes_out) nodes_out[k] = nn;
    if (fl & 2) atomicAdd(&sc->nbad, 1);
    else if (fl & 1) atomicAdd(&sc->ntrunc, 1);
}

}  // namespace

void pb_noalloc_setup(pb_ctx *ctx) {
    // called by pb_create with ctx's device current: the lookup may load the
    // library's device code and place the array on this device, so it
    // belongs to set-up, not to the allocation-free call
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e == cudaSuccess && p) {
        ctx->na_scratch = p;
    } else {
        ctx->na_scratch = nullptr;
        ctx->na_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        cudaGetLastError();
    }
}

extern "C" pb_status pb_recip_estimates_noalloc(pb_ctx *ctx, const pb_config *cfg, int iteration, int n,
                                                const int32_t *d_tri, const float *d_bary, const int32_t *d_info,
                                                const float *d_B, float *d_rhat, float *d_nodes, int *n_truncated) {
    if (!ctx) return PB_ERR_ARG;
    if (!ctx->has_scene) return pb_fail(ctx, PB_ERR_STATE, "no scene uploaded");
    if (!cfg || cfg->repeats < 1 || cfg->repeats > 8 || cfg->trial_cap < 1)
        return pb_fail(ctx, PB_ERR_ARG, "noalloc: repeats must be in [1, 8] and trial_cap positive");
    if (!(cfg->side_in >= 0.0f && cfg->side_in < 1.0f))
        return pb_fail(ctx, PB_ERR_ARG, "noalloc: side_in must lie in [0, 1)");
    if (n < 0 || (n > 0 && (!d_tri || !d_bary || !d_info || !d_B || !d_rhat)))
        return pb_fail(ctx, PB_ERR_ARG, "noalloc: null input or output");
    if ((long long)n * cfg->repeats > PB_NOALLOC_MAX_ESTIMATES)
        return pb_fail(ctx, PB_ERR_ARG,
                       "noalloc: entries x repeats exceeds PB_NOALLOC_MAX_ESTIMATES (" +
                           std::to_string(PB_NOALLOC_MAX_ESTIMATES) + ")");
    if (!ctx->na_scratch) return pb_fail(ctx, PB_ERR_CUDA, "noalloc: scratch array unavailable: " + ctx->na_err);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return pb_fail(ctx, PB_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    NAScratch *sc = (NAScratch *)ctx->na_scratch;
    if (n_truncated) *n_truncated = 0;
    if (n == 0) return PB_OK;
    KParams P = pb_kparams(ctx, cfg);
    // the work counter and the status counts start at zero each call
    e = cudaMemsetAsync(sc, 0, 3 * sizeof(int), ctx->stream);
    if (e != cudaSuccess) return pb_fail(ctx, PB_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    k_na_recip<<<ctx->num_sms * 8, 128, 0, ctx->stream>>>(ctx->S, P, (uint32_t)iteration, n, d_tri, d_bary, d_info,
                                                          d_B, sc);
    k_na_finish<<<(n + 127) / 128, 128, 0, ctx->stream>>>(P, n, sc, d_rhat, d_nodes);
    int cnt[3] = {0, 0, 0};
    e = cudaMemcpyAsync(cnt, sc, sizeof(cnt), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return pb_fail(ctx, PB_ERR_CUDA, std::string("noalloc estimator: ") + cudaGetErrorString(e));
    if (n_truncated) *n_truncated = cnt[1];
    if (cnt[2] > 0)
        return pb_fail(ctx, PB_ERR_ARG, "noalloc: " + std::to_string(cnt[2]) +
                                            " entries have a bound B that is not positive (their estimates are NaN)");
    return PB_OK;
}
