// Internal definition of the opaque context (include/proxybdpt.h) shared by
// the host translation units.
#pragma once
#include <string>
#include <vector>

#include "../../include/proxybdpt.h"
#include "pb_kernels.h"

struct pb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 1;
    std::string err;
    std::vector<void *> scene_mem, table_mem, pool_mem;
    bool has_scene = false, has_tables = false;
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
};

// shared by the host translation units
pb_status pb_ensure_pool(pb_ctx *ctx, int slots, int ML, int repeats);
pb_status pb_fail(pb_ctx *c, pb_status s, const std::string &m);
pb_status pb_run_wave(pb_ctx *ctx, const KParams &P, int slots, uint32_t iter_base, bool with_light,
                      bool with_recip, uint32_t *sig);
KParams pb_kparams(const pb_ctx *ctx, const pb_config *c);
pb_status pb_check_cfg(pb_ctx *ctx, const pb_config *c);
