// Reciprocal estimates for caller-supplied incomplete light sub-paths with no
// device allocation in the call (pb_recip_estimates_noalloc).
//
// Some callers cannot allocate device memory while they run: a host engine
// that owns all device memory up front and forbids later allocation, a
// process whose allocations are capped or pooled by another runtime, or code
// on a path where cudaMalloc's implicit synchronisation is not acceptable.
// This entry point serves them. Its inputs and outputs are the caller's
// device buffers; its scratch -- one estimate, node count and truncation flag
// per (entry, repeat), plus a work counter -- lives in the file-scope array
// below, sized for PB_NOALLOC_MAX_ESTIMATES estimates. Every GPU that loads
// the library holds that array until the process exits.
//
// The kernel is a one-phase form of the estimator (Sec. 4.2, App. Alg. I~):
// one warp per (entry, repeat) draws 32 pre-order nodes at a time and
// replays the sequential walk with a 48-frame stack. It uses the same
// streams as the pooled estimator in pb_light.cu, so both produce the same
// estimates.
#include <mutex>

#include "pb_ctx.h"
#include "pb_estimator.cuh"

namespace {

constexpr int NA_MAXF = 48;

struct NAScratch {
    int work;        // next (entry, repeat) to claim; cleared at the start of each call
    int pad[63];
    float est[PB_NOALLOC_MAX_ESTIMATES];
    float nodes[PB_NOALLOC_MAX_ESTIMATES];
    int trunc[PB_NOALLOC_MAX_ESTIMATES];
};

// In host code `g_na_scratch` names a host-side stand-in, not device memory:
// kernels get the address obtained from cudaGetSymbolAddress below.
static __device__ __align__(256) NAScratch g_na_scratch;

std::mutex g_na_mutex;
void *g_na_ptr[256] = {nullptr};   // per device ordinal

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
        float invB = 1.0f / Bv[k];
        double sum_t = 0.0;
        int nodes = 0;
        bool done = false, trunc = false;
        float fr_sign[NA_MAXF];
        int fr_rem[NA_MAXF];
        int sp = 0;
        float cur_sign = 1.0f;
        for (int base = 0; !done; base += 32) {
            int v = base + lane;
            float g = 1.0f;
            int nch = 0;
            if (v < P.trial_cap) {
                Rng R;
                R.init(P.seed, K_RECIP, iteration, (uint32_t)(k * 8 + rep), (uint32_t)v);
                float ratio = entry_ratio<false>(S, E, R, nullptr);
                g = 1.0f - ratio * invB;
                float r = fabsf(g);
                nch = (int)floorf(r);
                if (R.u(18) < r - (float)nch) nch += 1;
            }
            for (int j = 0; j < 32; ++j) {
                float gj = __shfl_sync(0xffffffffu, g, j);
                int nj = __shfl_sync(0xffffffffu, nch, j);
                if (done) continue;
                if (base + j >= P.trial_cap) {
                    done = true;
                    trunc = true;
                    continue;
                }
                sum_t += (double)(cur_sign * gj * invB);
                nodes++;
                if (nj >= 1) {
                    if (sp >= NA_MAXF) {
                        done = true;
                        trunc = true;
                        continue;
                    }
                    fr_sign[sp] = cur_sign * (gj > 0.0f ? 1.0f : -1.0f);
                    fr_rem[sp] = nj;
                    ++sp;
                }
                if (sp == 0) {
                    done = true;
                    continue;
                }
                cur_sign = fr_sign[sp - 1];
                if (--fr_rem[sp - 1] == 0) --sp;
            }
        }
        if (lane == 0) {
            sc->est[item] = (float)((double)invB + sum_t);
            sc->nodes[item] = (float)nodes;
            sc->trunc[item] = trunc ? 1 : 0;
        }
    }
}

__global__ void k_na_finish(KParams P, int n, const NAScratch *sc, float *rhat, float *nodes_out, int *ntrunc) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double acc = 0.0;
    float nn = 0.0f;
    int tr = 0;
    for (int r = 0; r < P.repeats; ++r) {
        acc += (double)sc->est[k * P.repeats + r];
        nn += sc->nodes[k * P.repeats + r];
        tr |= sc->trunc[k * P.repeats + r];
    }
    rhat[k] = (float)(acc / (double)P.repeats);
    if (nodes_out) nodes_out[k] = nn;
    if (tr) atomicAdd(ntrunc, 1);
}

}  // namespace

extern "C" pb_status pb_recip_estimates_noalloc(pb_ctx *ctx, const pb_config *cfg, int iteration, int n,
                                                const int32_t *d_tri, const float *d_bary, const int32_t *d_info,
                                                const float *d_B, float *d_rhat, float *d_nodes, int *n_truncated) {
    if (!ctx) return PB_ERR_ARG;
    if (!ctx->has_scene) return pb_fail(ctx, PB_ERR_STATE, "no scene uploaded");
    if (!cfg || cfg->repeats < 1 || cfg->repeats > 8 || cfg->trial_cap < 1)
        return pb_fail(ctx, PB_ERR_ARG, "noalloc: repeats must be in [1, 8] and trial_cap positive");
    if (n < 0 || (n > 0 && (!d_tri || !d_bary || !d_info || !d_B || !d_rhat)))
        return pb_fail(ctx, PB_ERR_ARG, "noalloc: null input or output");
    if ((long long)n * cfg->repeats > PB_NOALLOC_MAX_ESTIMATES)
        return pb_fail(ctx, PB_ERR_ARG,
                       "noalloc: entries x repeats exceeds PB_NOALLOC_MAX_ESTIMATES (" +
                           std::to_string(PB_NOALLOC_MAX_ESTIMATES) + ")");
    if (ctx->device < 0 || ctx->device >= 256) return pb_fail(ctx, PB_ERR_ARG, "noalloc: device ordinal out of range");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return pb_fail(ctx, PB_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    NAScratch *sc;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[ctx->device]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_na_scratch);
            if (e != cudaSuccess || !p)
                return pb_fail(ctx, PB_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_na_ptr[ctx->device] = p;
        }
        sc = (NAScratch *)g_na_ptr[ctx->device];
    }
    if (n_truncated) *n_truncated = 0;
    if (n == 0) return PB_OK;
    KParams P = pb_kparams(ctx, cfg);
    // the work counter and the caller's truncation count start at zero each call
    e = cudaMemsetAsync(&sc->work, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return pb_fail(ctx, PB_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    int *d_ntr = reinterpret_cast<int *>(&sc->pad[0]);
    e = cudaMemsetAsync(d_ntr, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return pb_fail(ctx, PB_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    k_na_recip<<<ctx->num_sms * 8, 128, 0, ctx->stream>>>(ctx->S, P, (uint32_t)iteration, n, d_tri, d_bary, d_info,
                                                          d_B, sc);
    k_na_finish<<<(n + 127) / 128, 128, 0, ctx->stream>>>(P, n, sc, d_rhat, d_nodes, d_ntr);
    int ntr = 0;
    e = cudaMemcpyAsync(&ntr, d_ntr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return pb_fail(ctx, PB_ERR_CUDA, std::string("noalloc estimator: ") + cudaGetErrorString(e));
    if (n_truncated) *n_truncated = ntr;
    return PB_OK;
}
