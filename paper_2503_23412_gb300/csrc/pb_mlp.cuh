// Learned light-subspace proposal: sizes, the flat weight layout and the
// network's input row, shared by the eye feature pass and the network
// kernels.
//
// The proposal replaces the table row Gamma[T, .] of the subspace
// connection (Sec. 3.2, Sec. 5.5) by
//     Q(S | x) = (1 - eps) softmax(MLP(x))_S + eps Gamma[T, S] / Z_T
// over the light subspaces that hold stored vertices (eps = 0.1). The
// connection estimate divides by M Q(S) / |S|, so it stays unbiased.
//
// Network: x (16) -> 64 ReLU -> 64 ReLU -> KS logits, with
//   x = [position normalised to the table box (3), normal facing the
//        incident direction (3), incident direction (3), roughness (1),
//        embedding E[T] (4), 1, 0].
// Flat fp32 weights, row-major with the output index first:
//   W1[64][16] | W2[64][64] | b2[64] | W3[KS][64] | b3[KS] | E[KT][4]
// (the first layer's bias is W1[:, 14], fed by the constant input).
#pragma once
#include <cuda_bf16.h>

#include "pb_device.cuh"

constexpr int MLP_H = 64;
constexpr int MLP_NX = 16;
constexpr int MLP_NRAW = 10;
constexpr int MLP_KMAX = 384;     // TMEM: 64 + 64 + KS (padded to 16) columns of 512
constexpr float MLP_EPS = 0.1f;

__host__ __device__ inline size_t mlp_off_W2() { return (size_t)MLP_H * MLP_NX; }
__host__ __device__ inline size_t mlp_off_b2() { return mlp_off_W2() + (size_t)MLP_H * MLP_H; }
__host__ __device__ inline size_t mlp_off_W3() { return mlp_off_b2() + MLP_H; }
__host__ __device__ inline size_t mlp_off_b3(int K) { return mlp_off_W3() + (size_t)K * MLP_H; }
__host__ __device__ inline size_t mlp_off_E(int K) { return mlp_off_b3(K) + (size_t)K; }
__host__ __device__ inline size_t mlp_nparams(int K, int KT) { return mlp_off_E(K) + 4 * (size_t)KT; }
__host__ __device__ inline int mlp_kpad(int K) { return (K + 15) / 16 * 16; }

// raw features of an eye vertex: normalised position, normal facing we, we, roughness
__device__ __forceinline__ void mlp_raw(const DScene &S, const Vtx &z, float3 we, float *f) {
    feat_pos(S, z.p, f);
    float3 n = dot(z.n, we) >= 0.0f ? z.n : -z.n;
    f[3] = n.x; f[4] = n.y; f[5] = n.z;
    f[6] = we.x; f[7] = we.y; f[8] = we.z;
    f[9] = S.mats[z.mat].rough;
}

__device__ __forceinline__ uint32_t bf16_pair(float lo, float hi) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

// the 16-wide bf16 input row (32 bytes, 16-byte aligned destination)
__device__ __forceinline__ void mlp_pack_row(const float *raw, int T, const uint16_t *emb, uint16_t *dst) {
    uint4 a, b;
    a.x = bf16_pair(raw[0], raw[1]);
    a.y = bf16_pair(raw[2], raw[3]);
    a.z = bf16_pair(raw[4], raw[5]);
    a.w = bf16_pair(raw[6], raw[7]);
    b.x = bf16_pair(raw[8], raw[9]);
    const uint16_t *e = emb + 4 * (size_t)T;
    b.y = (uint32_t)e[0] | ((uint32_t)e[1] << 16);
    b.z = (uint32_t)e[2] | ((uint32_t)e[3] << 16);
    b.w = bf16_pair(1.0f, 0.0f);
    reinterpret_cast<uint4 *>(dst)[0] = a;
    reinterpret_cast<uint4 *>(dst)[1] = b;
}
