// Internal definition of the opaque context (include/proxybdpt.h) shared by
// the host translation units.
#pragma once
#include <string>
#include <vector>

#include "../../include/proxybdpt.h"
#include "pb_kernels.h"

// learned proposal: network, Adam state, eye-pass rows, training buffers
struct MlpState {
    int K = 0, KT = 0, Kpad = 0;
    size_t np = 0;
    float *w = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;   // fp32 master weights, gradient, moments
    int step = 0;
    bool ready = false;                 // bf16 images are current
    uint8_t *img = nullptr;             // bf16 operand images of W1, W2, W3
    float *bias = nullptr;              // b2 | b3 (padded)
    uint16_t *emb = nullptr;            // bf16 E[KT][4]
    int *err = nullptr;                 // set by the tensor-core kernel when a wait times out
    uint16_t *rows = nullptr;
    int32_t *rowT = nullptr, *rowPos = nullptr, *sel = nullptr;
    float *selq = nullptr;
    int4 *hits = nullptr;
    unsigned int *rcount = nullptr;
    size_t cap_rows16 = 0, cap_rowT = 0, cap_rowPos = 0, cap_sel = 0, cap_selq = 0, cap_hits = 0;
    float *s_raw = nullptr, *s_w = nullptr;
    int32_t *s_T = nullptr, *s_S = nullptr;
    unsigned int *s_count = nullptr;
    size_t s_cap = 0;
    int b_cap = 0;
    float *b_X = nullptr, *b_a = nullptr, *b_H1 = nullptr, *b_H2 = nullptr, *b_DH1 = nullptr, *b_DH2 = nullptr,
          *b_DZ = nullptr, *b_DE = nullptr, *b_loss = nullptr;
    int32_t *b_T = nullptr, *b_S = nullptr;
};

// a render captured as a CUDA graph (one per configuration; iter0 is a device scalar)
struct RenderGraph {
    pb_config cfg;
    int slots = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> ev;     // per wave stage events
    std::vector<cudaEvent_t> ends;   // start and end of the render
};

struct pb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 1;
    std::string err;
    std::vector<void *> scene_mem, table_mem, pool_mem;
    bool has_scene = false, has_tables = false;
    int scene_nm = 0;    // materials of the uploaded scene
    DScene S{};
    DTables T{};
    float3 scene_lo{}, scene_hi{};
    // iteration-slot buffers and their capacity
    Pool B{};
    int cap_slots = 0, cap_ML = 0, cap_rep = 0, cap_KT = 0, cap_KS = 0, cap_KSp = 0;
    float4 *Lbuf = nullptr;
    uint32_t *sigbuf = nullptr;
    int cap_Lslots = 0;
    float *film = nullptr;
    int64_t film_iters = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    MlpState mlp;        // the connection's network (K = KS)
    MlpState mlp_p;      // the proxy strategy's network (K = KSp), proposal = 2
    std::vector<RenderGraph *> graphs;
    uint32_t *d_iter0 = nullptr;     // iteration base of graph replays
    // wavefront estimator buffers (allocated on first use)
    WfBufs wf{};
    std::vector<void *> wf_mem;
    int wf_chain_cap = 0;
    // camera-side wavefront of the eye pass: stored hits (table proposal; the
    // learned proposal's feature pass has its own), occlusion queries, answers
    int4 *eye_hits = nullptr;
    float4 *eye_qa = nullptr, *eye_qb = nullptr;
    int32_t *eye_dst = nullptr;
    unsigned int *eye_count = nullptr;
    uint8_t *eye_vis = nullptr;
    size_t eye_cap_q = 0, eye_cap_px = 0;   // queries, slot-vertex-pixels
    std::vector<void *> eye_mem;
    // device address of the allocation-free estimator's scratch array on this
    // context's device (looked up once in pb_create), or null with the reason
    void *na_scratch = nullptr;
    std::string na_err;
};

// shared by the host translation units
pb_status pb_ensure_pool(pb_ctx *ctx, int slots, int ML, int repeats);
pb_status pb_fail(pb_ctx *c, pb_status s, const std::string &m);
pb_status pb_run_wave(pb_ctx *ctx, const KParams &P, int slots, uint32_t iter_base, bool with_light,
                      bool with_recip, uint32_t *sig);
KParams pb_kparams(const pb_ctx *ctx, const pb_config *c);
pb_status pb_check_cfg(pb_ctx *ctx, const pb_config *c);
// the eye pass of one wave as the camera-side wavefront (pb_api.cu): the
// feature pass (unless P.mlp.hits is already filled), the query pass, the
// traversal-only answers and the shading pass into ctx->Lbuf
// events recorded between the eye stages (null: none); flags as for cudaEventRecordWithFlags
struct EyeEvents {
    cudaEvent_t feat_end = nullptr, emit_end = nullptr, occ_end = nullptr;
    unsigned int flags = 0;
};
pb_status pb_eye_stages(pb_ctx *ctx, const KParams &P, int slots, uint32_t iter_base, uint32_t *sig, cudaStream_t st,
                        const EyeEvents *ev = nullptr);
pb_status pb_eye_ensure(pb_ctx *ctx, int slots, int depth);
// allocation-free estimator (pb_noalloc.cu): looks up the device address of
// its scratch array with ctx's device current; called once by pb_create
void pb_noalloc_setup(pb_ctx *ctx);
// learned proposal (pb_mlp.cu)
void mlp_free(pb_ctx *ctx);
pb_status mlp_prepare(pb_ctx *ctx, int slots, int depth, int proposal);
void free_graphs(pb_ctx *ctx);
pb_status wf_ensure(pb_ctx *ctx);
pb_status wf_check(pb_ctx *ctx);
pb_status mlp_wave(pb_ctx *ctx, KParams &P, int slots, uint32_t iter_base, const EyeEvents *ev = nullptr);
pb_status mlp_check_err(pb_ctx *ctx);
// one wave of iterations that records proposal training samples and leaves the film alone (pb_api.cu)
pb_status pb_collect_wave(pb_ctx *ctx, const pb_config *cfg, int slots, uint32_t iter_base, const SampleSink &sink,
                          const SampleSink &sink_proxy = SampleSink{});
