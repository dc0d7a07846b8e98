// Learned light-subspace proposal on the device.
//
// Inference (k_mlp_select) runs the three layers on the 5th-generation
// tensor cores: one CTA per SM walks 128-row tiles; operands sit in shared
// memory in the no-swizzle K-major layout (8-row x 16-byte core matrices),
// tcgen05.mma (kind::f16, bf16 x bf16 -> fp32) accumulates into tensor
// memory, and the epilogues read the accumulators back with tcgen05.ld:
// bias and ReLU, rounding to bf16 as the next layer's operand, and finally
// the masked softmax, the mixture with the table row, and the draw of S
// with the camera stream's connection uniform (dimension 6).
//
// Training (forward, backward, Adam) runs in fp32 on the CUDA cores over
// mini-batches gathered from samples the renderer records.
#include <cmath>
#include <cstring>

#include "pb_ctx.h"
#include "pb_mlp.cuh"

namespace {

constexpr int TILE_M = 128;
constexpr uint32_t K_MLPTRAIN = 7;   // stream kind of the mini-batch draws

// ---- tcgen05 / mbarrier helpers (inline PTX) ------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, start / leading (K-adjacent
// core matrices) / stride (8-row groups) byte offsets, descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor: kind::f16 with fp32 accumulator, bf16 A and B,
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_smem_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// waits for the mbarrier phase; gives up after `ns` nanoseconds
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, uint64_t ns) {
    uint64_t t0 = globaltimer();
    for (uint32_t i = 0;; ++i) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
        if ((i & 63) == 63 && globaltimer() - t0 > ns) return false;
    }
}

// 32 lanes x 32 consecutive fp32 columns of this warp's quarter of TMEM
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of element (r, k) in the canonical no-swizzle K-major layout
// of an operand with `kdim` columns: core matrix (r/8, k/8) of 8 rows x 16 B
__host__ __device__ inline uint32_t canon_off(int r, int k, int kdim) {
    return (uint32_t)((r >> 3) * (kdim / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// ---- weight images ----------------------------------------------------------
struct ImgLayout {
    uint32_t w1, w2, w3, bytes;   // byte offsets of the bf16 operand images
};
__host__ __device__ inline ImgLayout img_layout(int Kpad) {
    ImgLayout L;
    L.w1 = 0;
    L.w2 = L.w1 + MLP_H * MLP_NX * 2;
    L.w3 = L.w2 + MLP_H * MLP_H * 2;
    L.bytes = L.w3 + (uint32_t)Kpad * MLP_H * 2;
    return L;
}

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

// fp32 master weights -> bf16 operand images, fp32 biases, bf16 embedding
__global__ void k_mlp_pack(const float *w, int K, int KT, uint8_t *img, float *bias, uint16_t *emb) {
    int Kpad = mlp_kpad(K);
    ImgLayout L = img_layout(Kpad);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int n1 = MLP_H * MLP_NX, n2 = MLP_H * MLP_H, n3 = Kpad * MLP_H;
    if (i < n1) {
        int r = i / MLP_NX, k = i % MLP_NX;
        *reinterpret_cast<uint16_t *>(img + L.w1 + canon_off(r, k, MLP_NX)) = bf16_bits(w[i]);
    } else if ((i -= n1) < n2) {
        int r = i / MLP_H, k = i % MLP_H;
        *reinterpret_cast<uint16_t *>(img + L.w2 + canon_off(r, k, MLP_H)) = bf16_bits(w[mlp_off_W2() + i]);
    } else if ((i -= n2) < n3) {
        int r = i / MLP_H, k = i % MLP_H;
        float v = r < K ? w[mlp_off_W3() + (size_t)r * MLP_H + k] : 0.0f;
        *reinterpret_cast<uint16_t *>(img + L.w3 + canon_off(r, k, MLP_H)) = bf16_bits(v);
    } else if ((i -= n3) < MLP_H + Kpad) {
        bias[i] = i < MLP_H ? w[mlp_off_b2() + i] : (i - MLP_H < K ? w[mlp_off_b3(K) + (i - MLP_H)] : 0.0f);
    } else if ((i -= MLP_H + Kpad) < 4 * KT) {
        emb[i] = bf16_bits(w[mlp_off_E(K) + i]);
    }
}

__global__ void k_mlp_rows_from_raw(int n, const float *raw, const int32_t *T, const uint16_t *emb, uint16_t *rows) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    mlp_pack_row(raw + (size_t)MLP_NRAW * b, T[b], emb, rows + (size_t)MLP_NX * b);
}

// ---- inference --------------------------------------------------------------
struct SelArgs {
    const uint8_t *img;
    const float *bias;
    int K, Kpad;
    const uint16_t *rows;
    const int32_t *rowT;
    const int32_t *rowPos;       // dense index of each row (selection mode)
    const unsigned int *count;   // selection mode: rows to process (read on the device)
    long long nrows;             // logits mode: rows to process; selection mode: capacity
    // selection mode
    int A, npix, slots, KT;
    uint32_t seed, iter_base;
    const uint32_t *iter_dev;    // graph replay: iteration numbers are *iter_dev + iter_base
    const int32_t *bstart;   // slots x (K + 1)
    const float *gC;         // KT x K
    const float *ZC;         // slots x KT
    const float *cdfC;       // slots x KT x K
    int32_t *sel;
    float *selq;
    int udim;                // camera dimension of the selection uniform (6 connection, 9 proxy)
    int tcols;               // TMEM columns the CTA allocates (128, 256 or 512)
    // logits mode
    float *logits;           // nrows x K
    int *err;
};

__device__ __forceinline__ int select_cdf_row(const float *cdf, int K, float u) {
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (u < cdf[mid]) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// 8 warps: warp w reads TMEM lanes 32 (w % 4) .. (the rows of its quarter)
// and handles half h = w / 4 of each accumulator's columns. TMEM: layer 1 in
// columns 0..63, layer 2 in 64..127, layer 3 from column 0 again (both hidden
// accumulators are read before its MMAs start), so a CTA needs
// max(128, Kpad) columns, rounded up to a power of two, and small networks
// fit several CTAs on an SM.
constexpr int SEL_THREADS = 256;
__host__ __device__ inline int sel_tcols(int Kpad) { return Kpad <= 128 ? 128 : (Kpad <= 256 ? 256 : 512); }
constexpr int MASK_WORDS = MLP_KMAX / 32;
constexpr int MAX_SLOTS = 64;

struct SelSmem {
    uint32_t a1, a23, bias, mask, part, bar, tslot, abort_, bytes;
};
__host__ __device__ inline SelSmem sel_smem(int Kpad) {
    SelSmem s;
    uint32_t o = (img_layout(Kpad).bytes + 127) / 128 * 128;
    s.a1 = o;
    o += TILE_M * MLP_NX * 2;
    s.a23 = o;
    o += TILE_M * MLP_H * 2;
    s.bias = o;
    o += (MLP_H + MLP_KMAX) * 4;
    s.mask = o;
    o += MAX_SLOTS * MASK_WORDS * 4;
    s.part = o;                     // per half and row: max, sum, last occupied S, its logit, pick, its weight
    o += 2 * TILE_M * 6 * 4;
    s.bar = o;
    o += 8;
    s.tslot = o;
    o += 4;
    s.abort_ = o;
    o += 4;
    s.bytes = (o + 127) / 128 * 128;
    return s;
}

// hidden-layer epilogue: 32 columns (col0 + 32 h) of this thread's row plus
// bias, ReLU, bf16 into the next layer's A operand
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem_row, int col0, int h, const float *bias, uint8_t *a23,
                                                int r) {
    float v[32];
    tmem_ld32(tmem_row + (uint32_t)(col0 + 32 * h), v);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        uint4 q;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float t = v[8 * g + e] + (bias ? bias[32 * h + 8 * g + e] : 0.0f);
            x[e] = t > 0.0f ? t : 0.0f;
        }
        q.x = bf16_pair(x[0], x[1]);
        q.y = bf16_pair(x[2], x[3]);
        q.z = bf16_pair(x[4], x[5]);
        q.w = bf16_pair(x[6], x[7]);
        *reinterpret_cast<uint4 *>(a23 + canon_off(r, 32 * h + 8 * g, MLP_H)) = q;
    }
}

template <bool LOGITS>
__global__ void __launch_bounds__(SEL_THREADS, 2) k_mlp_select(SelArgs a) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int r = 32 * quarter + lane;   // this thread's row within the tile
    const SelSmem SL = sel_smem(a.Kpad);
    const ImgLayout IL = img_layout(a.Kpad);
    uint8_t *a1 = sm + SL.a1, *a23 = sm + SL.a23;
    float *sbias = reinterpret_cast<float *>(sm + SL.bias);
    uint32_t *smask = reinterpret_cast<uint32_t *>(sm + SL.mask);
    float *part = reinterpret_cast<float *>(sm + SL.part);   // [half][field][row]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + SL.tslot);
    volatile int *abort_ = reinterpret_cast<int *>(sm + SL.abort_);
    const uint32_t bar = smem_u32(sm + SL.bar);

    // weights and biases into shared memory
    for (uint32_t o = 16 * tid; o < IL.bytes; o += 16 * SEL_THREADS)
        *reinterpret_cast<uint4 *>(sm + o) = *reinterpret_cast<const uint4 *>(a.img + o);
    for (int i = tid; i < MLP_H + a.Kpad; i += SEL_THREADS) sbias[i] = a.bias[i];
    const int nchunk = (a.Kpad + 31) / 32;
    if (!LOGITS) {
        // occupied light subspaces of every slot
        for (int i = tid; i < a.slots * nchunk; i += SEL_THREADS) {
            int s = i / nchunk, wd = i % nchunk;
            uint32_t m = 0;
            const int32_t *st = a.bstart + (size_t)s * (a.K + 1);
            for (int b = 0; b < 32; ++b) {
                int S = 32 * wd + b;
                if (S < a.K && st[S + 1] > st[S]) m |= 1u << b;
            }
            smask[s * MASK_WORDS + wd] = m;
        }
    }
    if (tid == 0) {
        *abort_ = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(a.tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    async_smem_fence();
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot;
    const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);   // this warp's TMEM lanes
    const uint32_t d1 = tmem, d2 = tmem + 64, d3 = tmem;
    const uint32_t sa1 = smem_u32(a1), sa23 = smem_u32(a23);
    const uint32_t sw1 = smem_u32(sm + IL.w1), sw2 = smem_u32(sm + IL.w2), sw3 = smem_u32(sm + IL.w3);
    const uint64_t TIMEOUT = 1000000000ull;   // 1 s per wait
    uint32_t phase = 0;
    long long nrows = a.nrows;
    if (!LOGITS) nrows = min((long long)*a.count, a.nrows);
    const long long ntiles = (nrows + TILE_M - 1) / TILE_M;
    bool pending = false;   // an MMA group was committed and not yet waited for
    // column chunks of this half: [c0, c1)
    const int cmid = (nchunk + 1) / 2;
    const int c0 = half ? cmid : 0, c1 = half ? nchunk : cmid;

    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // A tile of layer 1: each of the 128 rows is 32 bytes, one 16-byte half per thread
        {
            const int rr = tid >> 1, hh = tid & 1;
            const long long row = tile * TILE_M + rr;
            uint4 q = make_uint4(0, 0, 0, 0);
            if (row < nrows) q = reinterpret_cast<const uint4 *>(a.rows + (size_t)MLP_NX * row)[hh];
            *reinterpret_cast<uint4 *>(a1 + canon_off(rr, 8 * hh, MLP_NX)) = q;
        }
        async_smem_fence();
        __syncthreads();
        // layer 1: D1 = A1 (128 x 16) W1^T
        if (tid == 0) {
            tc_after();
            umma(d1, sdesc(sa1, 128, 2 * 128), sdesc(sw1, 128, 2 * 128), idesc_bf16(TILE_M, MLP_H), 0);
            umma_commit(bar);
        }
        pending = true;
        // while the MMAs run: this row's cell, position and uniform, and the
        // table draw (none of them depends on the logits)
        const long long row = tile * TILE_M + r;
        const bool inrow = row < nrows;
        int T = -1, pos = 0, slot = 0, av = 0, pix = 0, gpick = -1;
        float u = 0.0f;
        if (!LOGITS && inrow) {
            T = a.rowT[row];
            pos = a.rowPos[row];
            const long long per_slot = (long long)a.A * a.npix;
            slot = (int)(pos / per_slot);
            const long long rem = pos - (long long)slot * per_slot;
            av = (int)(rem / a.npix) + 1;
            pix = (int)(rem % a.npix);
            if (T >= 0) {
                Rng R;
                const uint32_t ib = a.iter_dev ? a.iter_base + *a.iter_dev : a.iter_base;
                R.init(a.seed, K_CAMERA, ib + (uint32_t)slot, (uint32_t)pix, (uint32_t)av);
                u = R.u(a.udim);
                if (u < MLP_EPS) gpick = select_cdf_row(a.cdfC + ((size_t)slot * a.KT + T) * a.K, a.K, u / MLP_EPS);
            }
        }
        if (mbar_wait(bar, phase, TIMEOUT)) {
            pending = false;
            phase ^= 1;
        } else {
            *abort_ = 1;
        }
        __syncthreads();
        if (*abort_) break;
        tc_after();
        hidden_epilogue(trow, 0, half, nullptr, a23, r);
        async_smem_fence();
        tc_before();
        __syncthreads();
        // layer 2: D2 = H1 (128 x 64) W2^T, four K = 16 steps
        if (tid == 0) {
            tc_after();
            for (int s = 0; s < 4; ++s)
                umma(d2, sdesc(sa23 + 256 * s, 128, 8 * 128), sdesc(sw2 + 256 * s, 128, 8 * 128),
                     idesc_bf16(TILE_M, MLP_H), s > 0);
            umma_commit(bar);
        }
        pending = true;
        if (mbar_wait(bar, phase, TIMEOUT)) {
            pending = false;
            phase ^= 1;
        } else {
            *abort_ = 1;
        }
        __syncthreads();
        if (*abort_) break;
        tc_after();
        hidden_epilogue(trow, 64, half, sbias, a23, r);
        async_smem_fence();
        tc_before();
        __syncthreads();
        // layer 3: D3 = H2 (128 x 64) W3^T in column chunks of at most 256
        if (tid == 0) {
            tc_after();
            for (int n0 = 0; n0 < a.Kpad; n0 += 256) {
                int nc = min(256, a.Kpad - n0);
                for (int s = 0; s < 4; ++s)
                    umma(d3 + n0, sdesc(sa23 + 256 * s, 128, 8 * 128),
                         sdesc(sw3 + (uint32_t)(n0 / 8) * 1024 + 256 * s, 128, 8 * 128), idesc_bf16(TILE_M, nc),
                         s > 0);
            }
            umma_commit(bar);
        }
        pending = true;
        if (mbar_wait(bar, phase, TIMEOUT)) {
            pending = false;
            phase ^= 1;
        } else {
            *abort_ = 1;
        }
        __syncthreads();
        if (*abort_) break;
        tc_after();
        const float *b3 = sbias + MLP_H;
        float v[32];
        if (LOGITS) {
            for (int c = c0; c < c1; ++c) {
                tmem_ld32(trow + 32 * c, v);
                if (row < nrows)
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        int S = 32 * c + k;
                        if (S < a.K) a.logits[(size_t)row * a.K + S] = v[k] + b3[S];
                    }
            }
        } else {
            const uint32_t *mk = smask + slot * MASK_WORDS;
            // pass A over this half: online max and normaliser, last occupied subspace
            float m = -INFINITY, Z = 0.0f, vlast = 0.0f;
            int last = -1;
            for (int c = c0; c < c1; ++c) {
                tmem_ld32(trow + 32 * c, v);
                const uint32_t bits = mk[c];
                float cm = -INFINITY;
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    v[k] += b3[32 * c + k];
                    if ((bits >> k) & 1u) cm = fmaxf(cm, v[k]);
                }
                if (cm == -INFINITY) continue;
                float nm = fmaxf(m, cm);
                float s = 0.0f;
#pragma unroll
                for (int k = 0; k < 32; ++k) s += ((bits >> k) & 1u) ? __expf(v[k] - nm) : 0.0f;
                Z = Z * __expf(m - nm) + s;
                m = nm;
                const int hb = 31 - __clz(bits);
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (k == hb) vlast = v[k];
                last = 32 * c + hb;
            }
            float *P0 = part + (size_t)(half * 6) * TILE_M;
            P0[0 * TILE_M + r] = m;
            P0[1 * TILE_M + r] = Z;
            P0[2 * TILE_M + r] = __int_as_float(last);
            P0[3 * TILE_M + r] = vlast;
            __syncthreads();
            const float *Q0 = part, *Q1 = part + 6 * TILE_M;
            const float m0 = Q0[r], m1 = Q1[r];
            const float mg = fmaxf(m0, m1);
            const float Zh0 = m0 == -INFINITY ? 0.0f : Q0[TILE_M + r] * __expf(m0 - mg);
            const float Zh1 = m1 == -INFINITY ? 0.0f : Q1[TILE_M + r] * __expf(m1 - mg);
            const float Zg = Zh0 + Zh1;
            const bool valid = T >= 0 && mg > -INFINITY;
            // one uniform picks the mixture component (the table row: gpick, drawn
            // above) and the subspace
            float target = 0.0f;
            if (valid && gpick < 0) target = (u - MLP_EPS) / (1.0f - MLP_EPS) * Zg;
            // pass B over this half: the cumulative search (softmax branch, the
            // half that holds the target) or the drawn subspace's weight
            int pick = -1;
            float e_pick = 0.0f;
            const bool mine = valid && (gpick >= 0 ? (gpick >= 32 * c0 && gpick < 32 * c1)
                                                   : (half == 0 ? target < Zh0 : target >= Zh0));
            float cum = half ? Zh0 : 0.0f;
            for (int c = c0; c < c1; ++c) {
                if (__all_sync(0xffffffffu, !mine || pick >= 0)) break;
                tmem_ld32(trow + 32 * c, v);
                if (!mine || pick >= 0) continue;
                const uint32_t bits = mk[c];
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const int S = 32 * c + k;
                    const bool occ = (bits >> k) & 1u;
                    const float e = occ ? __expf(v[k] + b3[S] - mg) : 0.0f;
                    if (gpick >= 0) {
                        if (pick < 0 && S == gpick) {
                            pick = S;
                            e_pick = e;
                        }
                    } else if (pick < 0 && occ) {
                        cum += e;
                        if (target < cum) {
                            pick = S;
                            e_pick = e;
                        }
                    }
                }
            }
            P0[4 * TILE_M + r] = __int_as_float(pick);
            P0[5 * TILE_M + r] = e_pick;
            __syncthreads();
            if (half == 0 && inrow) {
                int pk = __float_as_int(Q0[4 * TILE_M + r]);
                float ep = Q0[5 * TILE_M + r];
                if (pk < 0) {
                    pk = __float_as_int(Q1[4 * TILE_M + r]);
                    ep = Q1[5 * TILE_M + r];
                }
                if (valid && pk < 0) {
                    // rounding left the target past the last occupied subspace
                    int l1 = __float_as_int(Q1[2 * TILE_M + r]);
                    pk = l1 >= 0 ? l1 : __float_as_int(Q0[2 * TILE_M + r]);
                    ep = __expf((l1 >= 0 ? Q1[3 * TILE_M + r] : Q0[3 * TILE_M + r]) - mg);
                }
                if (valid) {
                    const float gam = a.gC[(size_t)T * a.K + pk] / a.ZC[(size_t)slot * a.KT + T];
                    a.sel[pos] = pk;
                    a.selq[pos] = (1.0f - MLP_EPS) * ep / Zg + MLP_EPS * gam;
                } else {
                    a.sel[pos] = -1;
                    a.selq[pos] = 0.0f;
                }
            }
        }
        tc_before();
        __syncthreads();
    }
    if (*abort_ && tid == 0) atomicExch(a.err, 1);
    // an abandoned wait: give the committed group one more bounded wait
    if (pending) mbar_wait(bar, phase, TIMEOUT);
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tcols) : "memory");
}

// ---- training (fp32, CUDA cores) -------------------------------------------
struct Batch {
    int n;
    float *X;      // n x 16 inputs (raw, E[T], 1, 0)
    int32_t *T, *S;
    float *a;      // per-sample factor w_b / n
    float *H1, *H2, *DH1, *DH2;   // n x 64
    float *DZ;     // n x Kpad
    float *DE;     // n x 4
    float *loss;   // per-block partial losses
};

__global__ void k_tr_gather(int n, int nsrc, const float *raw, const int32_t *T, const int32_t *S, const float *w,
                            uint32_t seed, uint32_t step, const float *wt, int K, Batch b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = i;
    if (nsrc > 0) {
        Rng R;
        R.init(seed, K_MLPTRAIN, step, (uint32_t)i, 0);
        j = min((int)(R.u(0) * (float)nsrc), nsrc - 1);
    }
    const float *r = raw + (size_t)MLP_NRAW * j;
    float *x = b.X + (size_t)MLP_NX * i;
    for (int c = 0; c < MLP_NRAW; ++c) x[c] = r[c];
    for (int c = 0; c < 4; ++c) x[10 + c] = wt[mlp_off_E(K) + 4 * (size_t)T[j] + c];
    x[14] = 1.0f;
    x[15] = 0.0f;
    b.T[i] = T[j];
    b.S[i] = S[j];
    b.a[i] = w[j] / (float)n;
}

__global__ void __launch_bounds__(128) k_tr_fwd(const float *wt, int K, int Kpad, Batch b) {
    __shared__ float red[128];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float lossv = 0.0f;
    if (i < b.n) {
        const float *x = b.X + (size_t)MLP_NX * i;
        float xs[MLP_NX], h1[MLP_H], h2[MLP_H];
        for (int c = 0; c < MLP_NX; ++c) xs[c] = x[c];
        for (int o = 0; o < MLP_H; ++o) {
            float s = 0.0f;
            for (int c = 0; c < MLP_NX; ++c) s = fmaf(wt[o * MLP_NX + c], xs[c], s);
            h1[o] = s > 0.0f ? s : 0.0f;
        }
        for (int o = 0; o < MLP_H; ++o) {
            float s = wt[mlp_off_b2() + o];
            for (int j = 0; j < MLP_H; ++j) s = fmaf(wt[mlp_off_W2() + o * MLP_H + j], h1[j], s);
            h2[o] = s > 0.0f ? s : 0.0f;
        }
        for (int o = 0; o < MLP_H; ++o) {
            b.H1[(size_t)i * MLP_H + o] = h1[o];
            b.H2[(size_t)i * MLP_H + o] = h2[o];
        }
        const float *W3 = wt + mlp_off_W3(), *b3 = wt + mlp_off_b3(K);
        float m = -INFINITY, Z = 0.0f;
        for (int k = 0; k < K; ++k) {
            float s = b3[k];
            for (int j = 0; j < MLP_H; ++j) s = fmaf(W3[(size_t)k * MLP_H + j], h2[j], s);
            if (s > m) {
                Z = Z * expf(m - s) + 1.0f;
                m = s;
            } else {
                Z += expf(s - m);
            }
        }
        float lse = m + logf(Z);
        float av = b.a[i];
        int St = b.S[i];
        for (int k = 0; k < Kpad; ++k) {
            float dz = 0.0f;
            if (k < K) {
                float s = b3[k];
                for (int j = 0; j < MLP_H; ++j) s = fmaf(W3[(size_t)k * MLP_H + j], h2[j], s);
                if (k == St) lossv = -av * (s - lse);
                dz = av * (expf(s - lse) - (k == St ? 1.0f : 0.0f));
            }
            b.DZ[(size_t)i * Kpad + k] = dz;
        }
    }
    red[threadIdx.x] = lossv;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) b.loss[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(128) k_tr_bwd(const float *wt, int K, int Kpad, Batch b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.n) return;
    const float *W3 = wt + mlp_off_W3();
    float dh2[MLP_H], dh1[MLP_H];
    for (int j = 0; j < MLP_H; ++j) dh2[j] = 0.0f;
    for (int k = 0; k < K; ++k) {
        float dz = b.DZ[(size_t)i * Kpad + k];
        if (dz == 0.0f) continue;
        for (int j = 0; j < MLP_H; ++j) dh2[j] = fmaf(dz, W3[(size_t)k * MLP_H + j], dh2[j]);
    }
    for (int j = 0; j < MLP_H; ++j) {
        if (!(b.H2[(size_t)i * MLP_H + j] > 0.0f)) dh2[j] = 0.0f;
        b.DH2[(size_t)i * MLP_H + j] = dh2[j];
        dh1[j] = 0.0f;
    }
    for (int o = 0; o < MLP_H; ++o) {
        if (dh2[o] == 0.0f) continue;
        for (int j = 0; j < MLP_H; ++j) dh1[j] = fmaf(dh2[o], wt[mlp_off_W2() + o * MLP_H + j], dh1[j]);
    }
    for (int j = 0; j < MLP_H; ++j) {
        if (!(b.H1[(size_t)i * MLP_H + j] > 0.0f)) dh1[j] = 0.0f;
        b.DH1[(size_t)i * MLP_H + j] = dh1[j];
    }
    for (int c = 0; c < 4; ++c) {
        float s = 0.0f;
        for (int o = 0; o < MLP_H; ++o) s = fmaf(dh1[o], wt[o * MLP_NX + 10 + c], s);
        b.DE[(size_t)i * 4 + c] = s;
    }
}

// G[m][n] = sum_b A[b][m] B[b][n] (m < M, n < N), fixed summation order
__global__ void k_tr_outer(int nb, const float *A, int lda, int M, const float *Bm, int ldb, int N, float *G) {
    __shared__ float sa[32][33], sb[32][33];
    int tm = threadIdx.y, tn = threadIdx.x;
    int m = blockIdx.y * 32 + tm, nn = blockIdx.x * 32 + tn;
    float acc = 0.0f;
    for (int b0 = 0; b0 < nb; b0 += 32) {
        int bb = b0 + tm;   // rows staged by threadIdx.y
        int ma = blockIdx.y * 32 + tn;
        sa[tm][tn] = (bb < nb && ma < M) ? A[(size_t)bb * lda + ma] : 0.0f;
        int nb_ = blockIdx.x * 32 + tn;
        sb[tm][tn] = (bb < nb && nb_ < N) ? Bm[(size_t)bb * ldb + nb_] : 0.0f;
        __syncthreads();
        for (int k = 0; k < 32; ++k) acc = fmaf(sa[k][tm], sb[k][tn], acc);
        __syncthreads();
    }
    if (m < M && nn < N) G[(size_t)m * N + nn] = acc;
}

__global__ void k_tr_colsum(int nb, const float *A, int lda, int M, float *g) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    float s = 0.0f;
    for (int b = 0; b < nb; ++b) s += A[(size_t)b * lda + m];
    g[m] = s;
}

__global__ void k_tr_embgrad(int nb, const int32_t *T, const float *DE, int KT, float *g) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * KT) return;
    int t = i / 4, c = i % 4;
    float s = 0.0f;
    for (int b = 0; b < nb; ++b)
        if (T[b] == t) s += DE[(size_t)b * 4 + c];
    g[i] = s;
}

__global__ void k_adam(int np, float *w, const float *g, float *m1, float *m2, float lr, float beta1, float beta2,
                       float c1, float c2, float eps) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    float gi = g[i];
    float a = beta1 * m1[i] + (1.0f - beta1) * gi;
    float v = beta2 * m2[i] + (1.0f - beta2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    w[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
#define CK(x)                                                                          \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) return pb_fail(ctx, PB_ERR_CUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
static cudaError_t grow(T **p, size_t &cap, size_t n) {
    if (*p && cap >= n) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (n ? n : 1));
    if (e == cudaSuccess) cap = n;
    return e;
}

static pb_status mlp_check(pb_ctx *ctx) {
    if (!ctx->has_tables) return pb_fail(ctx, PB_ERR_STATE, "mlp: no tables uploaded");
    if (ctx->T.KS > MLP_KMAX) return pb_fail(ctx, PB_ERR_ARG, "mlp: more than 384 light subspaces");
    if (ctx->T.KSp > MLP_KMAX) return pb_fail(ctx, PB_ERR_ARG, "mlp: more than 384 specular subspaces");
    return PB_OK;
}

static void free_state(MlpState &M) {
    void *ps[] = {M.w, M.g, M.m1, M.m2, M.img, M.bias, M.emb, M.err, M.rows, M.rowT, M.rowPos, M.hits, M.rcount,
                  M.sel, M.selq, M.s_raw,
                  M.s_T, M.s_S, M.s_w, M.s_count, M.b_X, M.b_T, M.b_S, M.b_a, M.b_H1, M.b_H2, M.b_DH1, M.b_DH2,
                  M.b_DZ, M.b_DE, M.b_loss};
    for (void *p : ps)
        if (p) cudaFree(p);
    M = MlpState{};
}

// the network of the connection (K = KS) or of the proxy strategy (K = KSp)
static MlpState &net(pb_ctx *ctx, bool proxy) { return proxy ? ctx->mlp_p : ctx->mlp; }

// (re)shape a network for the current tables
static pb_status mlp_shape(pb_ctx *ctx, bool proxy = false) {
    MlpState &M = net(ctx, proxy);
    int K = proxy ? ctx->T.KSp : ctx->T.KS, KT = ctx->T.KT;
    if (M.K == K && M.KT == KT && M.w) return PB_OK;
    free_graphs(ctx);
    free_state(M);
    M.K = K;
    M.KT = KT;
    M.Kpad = mlp_kpad(K);
    M.np = mlp_nparams(K, KT);
    CK(cudaMalloc(&M.w, 4 * M.np));
    CK(cudaMalloc(&M.g, 4 * M.np));
    CK(cudaMalloc(&M.m1, 4 * M.np));
    CK(cudaMalloc(&M.m2, 4 * M.np));
    CK(cudaMemsetAsync(M.m1, 0, 4 * M.np, ctx->stream));
    CK(cudaMemsetAsync(M.m2, 0, 4 * M.np, ctx->stream));
    CK(cudaMalloc(&M.img, img_layout(M.Kpad).bytes));
    CK(cudaMalloc(&M.bias, 4 * (MLP_H + M.Kpad)));
    CK(cudaMalloc(&M.emb, 2 * 4 * (size_t)KT));
    CK(cudaMalloc(&M.err, sizeof(int)));
    CK(cudaMemsetAsync(M.err, 0, sizeof(int), ctx->stream));
    M.step = 0;
    M.ready = false;
    return PB_OK;
}

void mlp_free(pb_ctx *ctx) {
    free_state(ctx->mlp);
    free_state(ctx->mlp_p);
}

static pb_status mlp_pack(pb_ctx *ctx, bool proxy = false) {
    MlpState &M = net(ctx, proxy);
    int n = MLP_H * MLP_NX + MLP_H * MLP_H + M.Kpad * MLP_H + MLP_H + M.Kpad + 4 * M.KT;
    k_mlp_pack<<<(n + 255) / 256, 256, 0, ctx->stream>>>(M.w, M.K, M.KT, M.img, M.bias, M.emb);
    CK(cudaGetLastError());
    M.ready = true;
    return PB_OK;
}

static pb_status set_select_attr(pb_ctx *ctx) {
    static bool done = false;
    if (done) return PB_OK;
    int smem = 120 * 1024;
    CK(cudaFuncSetAttribute(k_mlp_select<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    CK(cudaFuncSetAttribute(k_mlp_select<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    done = true;
    return PB_OK;
}

static pb_status run_select(pb_ctx *ctx, SelArgs &a, bool device_count) {
    // as many CTAs per SM as registers, shared memory and TMEM columns allow
    const int smem_req = (int)sel_smem(a.Kpad).bytes;
    if (smem_req > 120 * 1024) return pb_fail(ctx, PB_ERR_ARG, "mlp: shared memory layout too large");
    pb_status s0 = set_select_attr(ctx);
    if (s0 != PB_OK) return s0;
    a.tcols = sel_tcols(a.Kpad);
    int occ = 1;
    if (a.logits) CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mlp_select<true>, SEL_THREADS, smem_req));
    else CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mlp_select<false>, SEL_THREADS, smem_req));
    const int per_sm = std::max(1, std::min(occ, 512 / a.tcols));
    long long ntiles = (a.nrows + TILE_M - 1) / TILE_M;
    // with the row count on the device every CTA slot gets a CTA; idle ones exit at once
    const long long slots_ = (long long)ctx->num_sms * per_sm;
    int grid = device_count ? (int)slots_ : (int)std::min<long long>(ntiles, slots_);
    if (grid < 1) return PB_OK;
    if (a.logits) k_mlp_select<true><<<grid, SEL_THREADS, smem_req, ctx->stream>>>(a);
    else k_mlp_select<false><<<grid, SEL_THREADS, smem_req, ctx->stream>>>(a);
    CK(cudaGetLastError());
    return PB_OK;
}

static SelArgs sel_base(pb_ctx *ctx, bool proxy = false) {
    MlpState &M = net(ctx, proxy);
    SelArgs a{};
    a.img = M.img;
    a.bias = M.bias;
    a.K = M.K;
    a.Kpad = M.Kpad;
    a.KT = M.KT;
    a.err = M.err;
    a.udim = 6;
    return a;
}

// rows, hits and selections of `slots` iterations of the eye pass (the
// proxy network's rows and selections use the same dense layout; it stores
// no hits)
pb_status mlp_ensure_rows(pb_ctx *ctx, int slots, int A, int depth, bool proxy) {
    MlpState &M = net(ctx, proxy);
    size_t npix = (size_t)ctx->S.W * ctx->S.H;
    size_t n = (size_t)slots * A * npix;
    size_t nh = proxy ? 0 : (size_t)slots * depth * npix;
    if (M.cap_rowT < n || M.cap_hits < nh) free_graphs(ctx);
    CK(grow(&M.rows, M.cap_rows16, MLP_NX * n));
    CK(grow(&M.rowT, M.cap_rowT, n));
    CK(grow(&M.rowPos, M.cap_rowPos, n));
    CK(grow(&M.sel, M.cap_sel, n));
    CK(grow(&M.selq, M.cap_selq, n));
    if (!proxy) CK(grow(&M.hits, M.cap_hits, nh));
    if (!M.rcount) CK(cudaMalloc(&M.rcount, sizeof(unsigned int)));
    return PB_OK;
}

// everything a wave of the learned proposal allocates or configures, done
// before a render is enqueued (and possibly captured); proposal 2 also the
// proxy strategy's network
pb_status mlp_prepare(pb_ctx *ctx, int slots, int depth, int proposal) {
    if (!ctx->mlp.ready) return pb_fail(ctx, PB_ERR_STATE, "learned proposal requested but no network is loaded");
    if (proposal == 2 && !ctx->mlp_p.ready)
        return pb_fail(ctx, PB_ERR_STATE, "learned proxy proposal requested but no proxy network is loaded");
    if (depth - 2 < 1) return PB_OK;
    pb_status s = mlp_ensure_rows(ctx, slots, depth - 2, depth, false);
    if (s != PB_OK) return s;
    if (proposal == 2 && (s = mlp_ensure_rows(ctx, slots, depth - 2, depth, true)) != PB_OK) return s;
    return set_select_attr(ctx);
}

// feature pass, network and selection for one wave of iterations; sets P.mlp
pb_status mlp_wave(pb_ctx *ctx, KParams &P, int slots, uint32_t iter_base, const EyeEvents *ev) {
    MlpState &M = ctx->mlp;
    if (!M.ready) return pb_fail(ctx, PB_ERR_STATE, "learned proposal requested but no network is loaded");
    if (slots > MAX_SLOTS) return pb_fail(ctx, PB_ERR_ARG, "mlp: too many iterations in flight");
    const bool prox = P.proposal == 2;
    MlpState &MP = ctx->mlp_p;
    if (prox && !MP.ready) return pb_fail(ctx, PB_ERR_STATE, "learned proxy proposal requested but no proxy network");
    int A = P.max_depth - 2;
    if (A < 1) return PB_OK;
    pb_status s = mlp_ensure_rows(ctx, slots, A, P.max_depth, false);
    if (s != PB_OK) return s;
    if (prox && (s = mlp_ensure_rows(ctx, slots, A, P.max_depth, true)) != PB_OK) return s;
    size_t n = (size_t)slots * A * P.npix;
    CK(cudaMemsetAsync(M.rcount, 0, sizeof(unsigned int), ctx->stream));
    P.mlp = MlpRows{M.rows, M.rowT, M.rowPos, M.rcount, (int)n, M.hits, nullptr, nullptr, M.emb, A};
    if (prox) {
        CK(cudaMemsetAsync(MP.rcount, 0, sizeof(unsigned int), ctx->stream));
        P.mlpp = MlpRows{MP.rows, MP.rowT, MP.rowPos, MP.rcount, (int)n, nullptr, nullptr, nullptr, MP.emb, A};
    }
    launch_eye_feat(ctx->S, ctx->T, P, ctx->B, slots, iter_base, ctx->stream);
    CK(cudaGetLastError());
    if (ev && ev->feat_end) CK(cudaEventRecordWithFlags(ev->feat_end, ctx->stream, ev->flags));
    SelArgs a = sel_base(ctx);
    a.rows = M.rows;
    a.rowT = M.rowT;
    a.rowPos = M.rowPos;
    a.count = M.rcount;
    a.nrows = (long long)n;
    a.A = A;
    a.npix = P.npix;
    a.slots = slots;
    a.seed = P.seed;
    a.iter_base = iter_base;
    a.iter_dev = P.iter_dev;
    a.bstart = ctx->B.bstart;
    a.gC = ctx->T.gC;
    a.ZC = ctx->B.ZC;
    a.cdfC = ctx->B.cdfC;
    a.sel = M.sel;
    a.selq = M.selq;
    s = run_select(ctx, a, true);
    if (s != PB_OK) return s;
    P.mlp.rows = nullptr;
    P.mlp.sel = M.sel;
    P.mlp.selq = M.selq;
    if (prox) {
        // the proxy strategy's specular subspace S' of each proxy row: the same
        // kernel with the proxy network, Gamma' as the defensive part, the
        // occupancy of the incomplete sub-paths and camera dimension 9
        SelArgs b = sel_base(ctx, true);
        b.rows = MP.rows;
        b.rowT = MP.rowT;
        b.rowPos = MP.rowPos;
        b.count = MP.rcount;
        b.nrows = (long long)n;
        b.A = A;
        b.npix = P.npix;
        b.slots = slots;
        b.seed = P.seed;
        b.iter_base = iter_base;
        b.iter_dev = P.iter_dev;
        b.bstart = ctx->B.estart;
        b.gC = ctx->T.gP;
        b.ZC = ctx->B.ZP;
        b.cdfC = ctx->B.cdfP;
        b.sel = MP.sel;
        b.selq = MP.selq;
        b.udim = 9;
        s = run_select(ctx, b, true);
        if (s != PB_OK) return s;
        P.mlpp.rows = nullptr;
        P.mlpp.sel = MP.sel;
        P.mlpp.selq = MP.selq;
    }
    return PB_OK;
}

pb_status mlp_check_err(pb_ctx *ctx) {
    for (MlpState *Mp : {&ctx->mlp, &ctx->mlp_p}) {
        MlpState &M = *Mp;
        if (!M.err) continue;
        int e = 0;
        CK(cudaMemcpyAsync(&e, M.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (e) {
            CK(cudaMemsetAsync(M.err, 0, sizeof(int), ctx->stream));
            return pb_fail(ctx, PB_ERR_TIMEOUT, "mlp: tensor-core wait timed out");
        }
    }
    return PB_OK;
}

static pb_status ensure_batch(pb_ctx *ctx, int n, bool proxy = false) {
    MlpState &M = net(ctx, proxy);
    if (M.b_cap >= n) return PB_OK;
    void *ps[] = {M.b_X, M.b_T, M.b_S, M.b_a, M.b_H1, M.b_H2, M.b_DH1, M.b_DH2, M.b_DZ, M.b_DE, M.b_loss};
    for (void *p : ps)
        if (p) cudaFree(p);
    CK(cudaMalloc(&M.b_X, 4 * (size_t)n * MLP_NX));
    CK(cudaMalloc(&M.b_T, 4 * (size_t)n));
    CK(cudaMalloc(&M.b_S, 4 * (size_t)n));
    CK(cudaMalloc(&M.b_a, 4 * (size_t)n));
    CK(cudaMalloc(&M.b_H1, 4 * (size_t)n * MLP_H));
    CK(cudaMalloc(&M.b_H2, 4 * (size_t)n * MLP_H));
    CK(cudaMalloc(&M.b_DH1, 4 * (size_t)n * MLP_H));
    CK(cudaMalloc(&M.b_DH2, 4 * (size_t)n * MLP_H));
    CK(cudaMalloc(&M.b_DZ, 4 * (size_t)n * M.Kpad));
    CK(cudaMalloc(&M.b_DE, 4 * (size_t)n * 4));
    CK(cudaMalloc(&M.b_loss, 4 * (size_t)((n + 127) / 128)));
    M.b_cap = n;
    return PB_OK;
}

static Batch batch_view(MlpState &M, int n) {
    return Batch{n, M.b_X, M.b_T, M.b_S, M.b_a, M.b_H1, M.b_H2, M.b_DH1, M.b_DH2, M.b_DZ, M.b_DE, M.b_loss};
}

// gradient of the batch loss into M.g (flat layout)
static pb_status batch_grad(pb_ctx *ctx, int n, bool proxy = false) {
    MlpState &M = net(ctx, proxy);
    Batch b = batch_view(M, n);
    cudaStream_t st = ctx->stream;
    int nb = (n + 127) / 128;
    k_tr_fwd<<<nb, 128, 0, st>>>(M.w, M.K, M.Kpad, b);
    k_tr_bwd<<<nb, 128, 0, st>>>(M.w, M.K, M.Kpad, b);
    dim3 t(32, 32);
    k_tr_outer<<<dim3(1, 2), t, 0, st>>>(n, M.b_DH1, MLP_H, MLP_H, M.b_X, MLP_NX, MLP_NX, M.g);
    k_tr_outer<<<dim3(2, 2), t, 0, st>>>(n, M.b_DH2, MLP_H, MLP_H, M.b_H1, MLP_H, MLP_H, M.g + mlp_off_W2());
    k_tr_colsum<<<1, 64, 0, st>>>(n, M.b_DH2, MLP_H, MLP_H, M.g + mlp_off_b2());
    k_tr_outer<<<dim3(2, (M.K + 31) / 32), t, 0, st>>>(n, M.b_DZ, M.Kpad, M.K, M.b_H2, MLP_H, MLP_H,
                                                       M.g + mlp_off_W3());
    k_tr_colsum<<<(M.K + 127) / 128, 128, 0, st>>>(n, M.b_DZ, M.Kpad, M.K, M.g + mlp_off_b3(M.K));
    k_tr_embgrad<<<(4 * M.KT + 127) / 128, 128, 0, st>>>(n, M.b_T, M.b_DE, M.KT, M.g + mlp_off_E(M.K));
    CK(cudaGetLastError());
    return PB_OK;
}

static pb_status adam_step(pb_ctx *ctx, float lr, bool proxy = false) {
    MlpState &M = net(ctx, proxy);
    M.step++;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = (float)(1.0 - std::pow((double)b1, M.step)), c2 = (float)(1.0 - std::pow((double)b2, M.step));
    k_adam<<<(int)((M.np + 255) / 256), 256, 0, ctx->stream>>>((int)M.np, M.w, M.g, M.m1, M.m2, lr, b1, b2, c1, c2,
                                                               1e-8f);
    CK(cudaGetLastError());
    return PB_OK;
}

static pb_status upload_batch(pb_ctx *ctx, int n, const float *raw, const int32_t *T, const int32_t *S,
                              const float *w) {
    MlpState &M = ctx->mlp;
    pb_status s = ensure_batch(ctx, n);
    if (s != PB_OK) return s;
    for (int i = 0; i < n; ++i)
        if (T[i] < 0 || T[i] >= M.KT || S[i] < 0 || S[i] >= M.K) return pb_fail(ctx, PB_ERR_ARG, "mlp: T or S out of range");
    // host rows go through the device gather with the identity order
    float *draw;
    int32_t *dT, *dS;
    float *dw;
    CK(cudaMallocAsync(&draw, 4 * (size_t)n * MLP_NRAW, ctx->stream));
    CK(cudaMallocAsync(&dT, 4 * (size_t)n, ctx->stream));
    CK(cudaMallocAsync(&dS, 4 * (size_t)n, ctx->stream));
    CK(cudaMallocAsync(&dw, 4 * (size_t)n, ctx->stream));
    CK(cudaMemcpyAsync(draw, raw, 4 * (size_t)n * MLP_NRAW, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dT, T, 4 * (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dS, S, 4 * (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dw, w, 4 * (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
    k_tr_gather<<<(n + 127) / 128, 128, 0, ctx->stream>>>(n, 0, draw, dT, dS, dw, 0, 0, M.w, M.K,
                                                          batch_view(M, n));
    CK(cudaGetLastError());
    CK(cudaFreeAsync(draw, ctx->stream));
    CK(cudaFreeAsync(dT, ctx->stream));
    CK(cudaFreeAsync(dS, ctx->stream));
    CK(cudaFreeAsync(dw, ctx->stream));
    return PB_OK;
}

static float batch_loss(pb_ctx *ctx, int n, bool proxy = false) {
    MlpState &M = net(ctx, proxy);
    int nb = (n + 127) / 128;
    std::vector<float> h(nb);
    if (cudaMemcpyAsync(h.data(), M.b_loss, 4 * (size_t)nb, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
        return NAN;
    cudaStreamSynchronize(ctx->stream);
    double s = 0.0;
    for (float v : h) s += v;
    return (float)s;
}

// deterministic initialisation: uniform He fan-in for the hidden layers,
// small output layer, N(0, 0.5)-like embedding (sum of uniforms)
static void init_weights(std::vector<float> &w, int K, int KT, uint32_t seed) {
    uint64_t st = 0x9E3779B97F4A7C15ull ^ seed;
    auto nxt = [&]() {
        st ^= st << 13;
        st ^= st >> 7;
        st ^= st << 17;
        return (double)(st >> 11) * (1.0 / 9007199254740992.0);
    };
    std::fill(w.begin(), w.end(), 0.0f);
    for (size_t i = 0; i < (size_t)MLP_H * MLP_NX; ++i) w[i] = (float)((2 * nxt() - 1) * std::sqrt(6.0 / 16));
    for (size_t i = 0; i < (size_t)MLP_H * MLP_H; ++i) w[mlp_off_W2() + i] = (float)((2 * nxt() - 1) * std::sqrt(6.0 / 64));
    for (size_t i = 0; i < (size_t)K * MLP_H; ++i) w[mlp_off_W3() + i] = (float)((2 * nxt() - 1) * 0.05);
    for (size_t i = 0; i < 4 * (size_t)KT; ++i) w[mlp_off_E(K) + i] = (float)((nxt() + nxt() + nxt() - 1.5) * 0.8);
}

extern "C" {

size_t pb_mlp_nparams(int K, int KT) { return mlp_nparams(K, KT); }

pb_status pb_mlp_upload(pb_ctx *ctx, const float *w, size_t n) {
    if (!ctx) return PB_ERR_ARG;
    pb_status s = mlp_check(ctx);
    if (s != PB_OK) return s;
    if ((s = mlp_shape(ctx)) != PB_OK) return s;
    if (!w || n != ctx->mlp.np) return pb_fail(ctx, PB_ERR_ARG, "mlp: weight count differs from pb_mlp_nparams");
    CK(cudaMemcpyAsync(ctx->mlp.w, w, 4 * n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->mlp.m1, 0, 4 * n, ctx->stream));
    CK(cudaMemsetAsync(ctx->mlp.m2, 0, 4 * n, ctx->stream));
    ctx->mlp.step = 0;
    if ((s = mlp_pack(ctx)) != PB_OK) return s;
    CK(cudaStreamSynchronize(ctx->stream));
    return PB_OK;
}

pb_status pb_mlp_proxy_upload(pb_ctx *ctx, const float *w, size_t n) {
    if (!ctx) return PB_ERR_ARG;
    pb_status s = mlp_check(ctx);
    if (s != PB_OK) return s;
    if ((s = mlp_shape(ctx, true)) != PB_OK) return s;
    MlpState &M = ctx->mlp_p;
    if (!w || n != M.np) return pb_fail(ctx, PB_ERR_ARG, "mlp: proxy weight count differs from pb_mlp_nparams(KSp, KT)");
    CK(cudaMemcpyAsync(M.w, w, 4 * n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(M.m1, 0, 4 * n, ctx->stream));
    CK(cudaMemsetAsync(M.m2, 0, 4 * n, ctx->stream));
    M.step = 0;
    if ((s = mlp_pack(ctx, true)) != PB_OK) return s;
    CK(cudaStreamSynchronize(ctx->stream));
    return PB_OK;
}

pb_status pb_mlp_proxy_readback(pb_ctx *ctx, float *w, size_t n) {
    if (!ctx) return PB_ERR_ARG;
    MlpState &M = ctx->mlp_p;
    if (!M.w) return pb_fail(ctx, PB_ERR_STATE, "mlp: no proxy network");
    if (!w || n != M.np) return pb_fail(ctx, PB_ERR_ARG, "mlp: proxy weight count differs from pb_mlp_nparams(KSp, KT)");
    CK(cudaMemcpyAsync(w, M.w, 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PB_OK;
}

pb_status pb_mlp_readback(pb_ctx *ctx, float *w, size_t n) {
    if (!ctx) return PB_ERR_ARG;
    if (!ctx->mlp.w) return pb_fail(ctx, PB_ERR_STATE, "mlp: no network");
    if (!w || n != ctx->mlp.np) return pb_fail(ctx, PB_ERR_ARG, "mlp: weight count differs from pb_mlp_nparams");
    CK(cudaMemcpyAsync(w, ctx->mlp.w, 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PB_OK;
}

pb_status pb_mlp_logits(pb_ctx *ctx, int n, const float *raw, const int32_t *T, float *z) {
    if (!ctx) return PB_ERR_ARG;
    MlpState &M = ctx->mlp;
    if (!M.ready) return pb_fail(ctx, PB_ERR_STATE, "mlp: no network");
    if (n < 0 || (n > 0 && (!raw || !T || !z))) return pb_fail(ctx, PB_ERR_ARG, "mlp: null argument");
    if (n == 0) return PB_OK;
    for (int i = 0; i < n; ++i)
        if (T[i] < 0 || T[i] >= M.KT) return pb_fail(ctx, PB_ERR_ARG, "mlp: T out of range");
    float *draw, *dz;
    int32_t *dT;
    uint16_t *drows;
    CK(cudaMallocAsync(&draw, 4 * (size_t)n * MLP_NRAW, ctx->stream));
    CK(cudaMallocAsync(&dT, 4 * (size_t)n, ctx->stream));
    CK(cudaMallocAsync(&drows, 2 * (size_t)n * MLP_NX, ctx->stream));
    CK(cudaMallocAsync(&dz, 4 * (size_t)n * M.K, ctx->stream));
    CK(cudaMemcpyAsync(draw, raw, 4 * (size_t)n * MLP_NRAW, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dT, T, 4 * (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
    k_mlp_rows_from_raw<<<(n + 127) / 128, 128, 0, ctx->stream>>>(n, draw, dT, M.emb, drows);
    CK(cudaGetLastError());
    SelArgs a = sel_base(ctx);
    a.rows = drows;
    a.nrows = n;
    a.logits = dz;
    pb_status s = run_select(ctx, a, false);
    if (s != PB_OK) return s;
    CK(cudaMemcpyAsync(z, dz, 4 * (size_t)n * M.K, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaFreeAsync(draw, ctx->stream));
    CK(cudaFreeAsync(dT, ctx->stream));
    CK(cudaFreeAsync(drows, ctx->stream));
    CK(cudaFreeAsync(dz, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return mlp_check_err(ctx);
}

pb_status pb_mlp_grad(pb_ctx *ctx, int n, const float *raw, const int32_t *T, const int32_t *S, const float *w,
                      float *grad, float *loss) {
    if (!ctx) return PB_ERR_ARG;
    MlpState &M = ctx->mlp;
    if (!M.w) return pb_fail(ctx, PB_ERR_STATE, "mlp: no network");
    if (n < 1 || !raw || !T || !S || !w || !grad) return pb_fail(ctx, PB_ERR_ARG, "mlp: null argument or empty batch");
    pb_status s = upload_batch(ctx, n, raw, T, S, w);
    if (s != PB_OK) return s;
    if ((s = batch_grad(ctx, n)) != PB_OK) return s;
    CK(cudaMemcpyAsync(grad, M.g, 4 * M.np, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (loss) *loss = batch_loss(ctx, n);
    return PB_OK;
}

pb_status pb_mlp_train_batch(pb_ctx *ctx, int n, const float *raw, const int32_t *T, const int32_t *S,
                             const float *w, float lr, float *loss) {
    if (!ctx) return PB_ERR_ARG;
    MlpState &M = ctx->mlp;
    if (!M.w) return pb_fail(ctx, PB_ERR_STATE, "mlp: no network");
    if (n < 1 || !raw || !T || !S || !w) return pb_fail(ctx, PB_ERR_ARG, "mlp: null argument or empty batch");
    pb_status s = upload_batch(ctx, n, raw, T, S, w);
    if (s != PB_OK) return s;
    if ((s = batch_grad(ctx, n)) != PB_OK) return s;
    if (loss) *loss = batch_loss(ctx, n);
    if ((s = adam_step(ctx, lr)) != PB_OK) return s;
    if ((s = mlp_pack(ctx)) != PB_OK) return s;
    CK(cudaStreamSynchronize(ctx->stream));
    return PB_OK;
}

pb_status pb_train_proposal(pb_ctx *ctx, const pb_config *cfg, const pb_train_desc *td, pb_train_stats *out) {
    if (!ctx) return PB_ERR_ARG;
    pb_status s = pb_check_cfg(ctx, cfg);
    if (s != PB_OK) return s;
    if ((s = mlp_check(ctx)) != PB_OK) return s;
    if (!td || td->samples < 1 || td->rounds < 1 || td->steps < 0 || td->batch < 1)
        return pb_fail(ctx, PB_ERR_ARG, "train: samples, rounds and batch must be positive");
    const bool prox = td->proxy != 0;
    for (int h = 0; h < (prox ? 2 : 1); ++h) {
        if ((s = mlp_shape(ctx, h == 1)) != PB_OK) return s;
        MlpState &Mh = net(ctx, h == 1);
        if (!Mh.ready || td->reinit) {
            std::vector<float> w(Mh.np);
            init_weights(w, Mh.K, Mh.KT, td->seed + 977u * (uint32_t)h);
            CK(cudaMemcpyAsync(Mh.w, w.data(), 4 * Mh.np, cudaMemcpyHostToDevice, ctx->stream));
            CK(cudaMemsetAsync(Mh.m1, 0, 4 * Mh.np, ctx->stream));
            CK(cudaMemsetAsync(Mh.m2, 0, 4 * Mh.np, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            Mh.step = 0;
            if ((s = mlp_pack(ctx, h == 1)) != PB_OK) return s;
        }
        // sample buffer
        size_t cap = (size_t)td->samples;
        if (Mh.s_cap < cap) {
            void *ps[] = {Mh.s_raw, Mh.s_T, Mh.s_S, Mh.s_w};
            for (void *p : ps)
                if (p) cudaFree(p);
            CK(cudaMalloc(&Mh.s_raw, 4 * cap * MLP_NRAW));
            CK(cudaMalloc(&Mh.s_T, 4 * cap));
            CK(cudaMalloc(&Mh.s_S, 4 * cap));
            CK(cudaMalloc(&Mh.s_w, 4 * cap));
            Mh.s_cap = cap;
        }
        if (!Mh.s_count) CK(cudaMalloc(&Mh.s_count, sizeof(unsigned int)));
        if ((s = ensure_batch(ctx, td->batch, h == 1)) != PB_OK) return s;
    }
    MlpState &M = ctx->mlp;
    const size_t cap = (size_t)td->samples;
    pb_config c = *cfg;
    c.proposal = 0;
    int64_t iters = 0, nsamp_total = 0, nsamp_proxy = 0;
    double loss_first = NAN, loss_last = NAN, lp_first = NAN, lp_last = NAN;
    uint32_t it = (uint32_t)td->iter0;
    for (int r = 0; r < td->rounds; ++r) {
        // collect: render iterations (not accumulated) with the current proposal
        c.proposal = (r == 0 && !td->learned_first) ? 0 : (prox ? 2 : 1);
        CK(cudaMemsetAsync(M.s_count, 0, sizeof(unsigned int), ctx->stream));
        if (prox) CK(cudaMemsetAsync(ctx->mlp_p.s_count, 0, sizeof(unsigned int), ctx->stream));
        unsigned int cnt = 0, cntp = 0;
        int max_it = td->max_iters_per_round > 0 ? td->max_iters_per_round : 256;
        int done = 0;
        while (done < max_it) {
            int wave = std::min(td->iters_per_wave > 0 ? td->iters_per_wave : 8, max_it - done);
            SampleSink sink{M.s_raw, M.s_T, M.s_S, M.s_w, M.s_count, (int)cap};
            MlpState &MP = ctx->mlp_p;
            SampleSink sinkp{};
            if (prox) sinkp = SampleSink{MP.s_raw, MP.s_T, MP.s_S, MP.s_w, MP.s_count, (int)cap};
            if ((s = pb_collect_wave(ctx, &c, wave, it, sink, sinkp)) != PB_OK) return s;
            it += (uint32_t)wave;
            done += wave;
            iters += wave;
            CK(cudaMemcpyAsync(&cnt, M.s_count, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
            if (prox) CK(cudaMemcpyAsync(&cntp, MP.s_count, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            if (cnt >= cap) break;
        }
        // train each network on its own samples
        for (int h = 0; h < (prox ? 2 : 1); ++h) {
            MlpState &Mh = net(ctx, h == 1);
            int nsrc = (int)std::min<size_t>(h ? cntp : cnt, cap);
            (h ? nsamp_proxy : nsamp_total) += nsrc;
            if (nsrc == 0) continue;
            for (int k = 0; k < td->steps; ++k) {
                Batch b = batch_view(Mh, td->batch);
                k_tr_gather<<<(td->batch + 127) / 128, 128, 0, ctx->stream>>>(
                    td->batch, nsrc, Mh.s_raw, Mh.s_T, Mh.s_S, Mh.s_w, td->seed + 977u * (uint32_t)h,
                    (uint32_t)Mh.step, Mh.w, Mh.K, b);
                CK(cudaGetLastError());
                if ((s = batch_grad(ctx, td->batch, h == 1)) != PB_OK) return s;
                if (k == 0 || k == td->steps - 1) {
                    float l = batch_loss(ctx, td->batch, h == 1);
                    double &lf = h ? lp_first : loss_first;
                    if (std::isnan(lf)) lf = l;
                    (h ? lp_last : loss_last) = l;
                }
                if ((s = adam_step(ctx, td->lr > 0.0f ? td->lr : 1e-3f, h == 1)) != PB_OK) return s;
            }
            if ((s = mlp_pack(ctx, h == 1)) != PB_OK) return s;
        }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    if (out) {
        out->iterations = iters;
        out->samples = nsamp_total;
        out->steps = M.step;
        out->loss_first = loss_first;
        out->loss_last = loss_last;
        out->samples_proxy = nsamp_proxy;
        out->loss_proxy_first = lp_first;
        out->loss_proxy_last = lp_last;
    }
    return PB_OK;
}

pb_status pb_connection_moments(pb_ctx *ctx, const pb_config *cfg, double *out) {
    if (!ctx) return PB_ERR_ARG;
    pb_status s = pb_check_cfg(ctx, cfg);
    if (s != PB_OK) return s;
    if (!out) return pb_fail(ctx, PB_ERR_ARG, "moments: null output");
    if (cfg->proposal && !ctx->mlp.ready) return pb_fail(ctx, PB_ERR_STATE, "moments: no network loaded");
    MlpState &M = ctx->mlp;
    const int wave = 8;
    int A = std::max(1, cfg->max_depth - 2);
    size_t cap = (size_t)wave * A * ctx->S.W * ctx->S.H;
    float *draw, *dw;
    int32_t *dT, *dS;
    unsigned int *dcnt;
    CK(cudaMallocAsync(&draw, 4 * cap * MLP_NRAW, ctx->stream));
    CK(cudaMallocAsync(&dw, 4 * cap, ctx->stream));
    CK(cudaMallocAsync(&dT, 4 * cap, ctx->stream));
    CK(cudaMallocAsync(&dS, 4 * cap, ctx->stream));
    CK(cudaMallocAsync(&dcnt, sizeof(unsigned int), ctx->stream));
    double n_conn = 0.0, s1 = 0.0, s2 = 0.0;
    std::vector<float> hw(cap);
    for (int done = 0; done < cfg->spp; done += wave) {
        int ns = std::min(wave, cfg->spp - done);
        CK(cudaMemsetAsync(dcnt, 0, sizeof(unsigned int), ctx->stream));
        s = pb_ensure_pool(ctx, ns, cfg->M * (cfg->max_depth - 1), cfg->repeats);
        if (s != PB_OK) return s;
        CK(cudaMemsetAsync(ctx->B.counters, 0, sizeof(unsigned long long) * CNT_N, ctx->stream));
        SampleSink sink{draw, dT, dS, dw, dcnt, (int)cap};
        if ((s = pb_collect_wave(ctx, cfg, ns, (uint32_t)(cfg->iter0 + done), sink)) != PB_OK) return s;
        unsigned int cnt = 0;
        unsigned long long nc = 0;
        CK(cudaMemcpyAsync(&cnt, dcnt, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(&nc, ctx->B.counters + CNT_CONN, sizeof(nc), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        size_t k = std::min<size_t>(cnt, cap);
        CK(cudaMemcpyAsync(hw.data(), dw, 4 * k, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        n_conn += (double)nc;
        for (size_t i = 0; i < k; ++i) {
            s1 += hw[i];
            s2 += (double)hw[i] * hw[i];
        }
    }
    CK(cudaFreeAsync(draw, ctx->stream));
    CK(cudaFreeAsync(dw, ctx->stream));
    CK(cudaFreeAsync(dT, ctx->stream));
    CK(cudaFreeAsync(dS, ctx->stream));
    CK(cudaFreeAsync(dcnt, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    (void)M;
    out[0] = n_conn;
    out[1] = s1;
    out[2] = s2;
    return PB_OK;
}

}  // extern "C"
