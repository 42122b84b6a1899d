// The regression network of the learned ranking path: 16-64-64-1 with ReLU
// on standardised node features, trained with a mean-squared-error loss on
// exact EF by Adam (Kingma and Ba, Algorithm 1).
//
// Every matrix product runs on the tensor cores as BF16 mma.sync m16n8k16
// with FP32 accumulation:
// - inference and the training forward pass take 16 rows per warp;
// - the backward pass computes the data gradients per tile in the same
//   registers;
// - the weight gradients are separate reductions over the batch
//   (k_mlp_wgrad).
// The work is tiny next to the exact EF pass (5.3k parameters): inference
// reads 64 bytes of features per node and is bound by HBM, so the
// warp-level BF16 instructions suffice here (tcgen05 would not pay).
//
// Fragment layouts of m16n8k16 (g = lane / 4, t = lane % 4):
// - A 16x16 row-major: {A[g][2t..2t+1]}, {A[g+8][2t..]}, {A[g][2t+8..]},
//   {A[g+8][2t+8..]};
// - B 16x8: {B[2t..2t+1][g]}, {B[2t+8..2t+9][g]};
// - C 16x8: c0,c1 = C[g][2t..2t+1], c2,c3 = C[g+8][2t..2t+1].
// Two adjacent C tiles of a layer form the A fragment of the next layer's
// 16-wide k-chunk.
#include "ef_internal.cuh"

#include <cuda_bf16.h>

namespace ef {

__device__ __forceinline__ float bf16_to_float(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }

__device__ __forceinline__ uint32_t pair_u16(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The model as one CTA holds it in shared memory.  Weight rows are padded
// (16 -> 24 and 64 -> 72 elements) so that the eight row groups of a
// fragment load fall in different banks (unpadded, 64-element rows put them
// all in one bank: an 8-way conflict that made inference bound by shared
// memory).
constexpr int W1S = 24, W2S = 72;

struct MlpSmem {
    __align__(16) uint16_t w1t[MLP_H * W1S];
    __align__(16) uint16_t w2t[MLP_H * W2S];
    __align__(16) uint16_t w2r[MLP_H * W2S];
    float b1[MLP_H], b2[MLP_H], w3[MLP_H], mean[MLP_F], istd[MLP_F];
    float b3;
};

__device__ void load_model(const ModelDev *M, MlpSmem &s, bool with_w2r) {
    // 16-byte chunks: 2 per W1 row, 8 per W2 row
    const uint4 *src1 = reinterpret_cast<const uint4 *>(M->w1t);
    const uint4 *src2 = reinterpret_cast<const uint4 *>(M->w2t);
    const uint4 *src3 = reinterpret_cast<const uint4 *>(M->w2r);
    for (int i = threadIdx.x; i < MLP_H * 2; i += blockDim.x)
        reinterpret_cast<uint4 *>(s.w1t + (i >> 1) * W1S)[i & 1] = src1[i];
    for (int i = threadIdx.x; i < MLP_H * 8; i += blockDim.x) {
        reinterpret_cast<uint4 *>(s.w2t + (i >> 3) * W2S)[i & 7] = src2[i];
        if (with_w2r) reinterpret_cast<uint4 *>(s.w2r + (i >> 3) * W2S)[i & 7] = src3[i];
    }
    for (int i = threadIdx.x; i < MLP_H; i += blockDim.x) {
        s.b1[i] = M->p[P_B1 + i];
        s.b2[i] = M->p[P_B2 + i];
        s.w3[i] = M->p[P_W3 + i];
    }
    for (int i = threadIdx.x; i < MLP_F; i += blockDim.x) {
        s.mean[i] = M->mean[i];
        s.istd[i] = 1.0f / M->stdv[i];
    }
    if (threadIdx.x == 0) s.b3 = M->p[P_B3];
}

// Forward pass of one 16-row tile.  Rows g and g+8 of this thread are the
// feature rows xg, xg8 (nullptr: a padding row, all zero).
struct Tile {
    uint32_t a1[4];       // standardised features as the layer-1 A fragment
    float h1[8][4];       // layer-1 activations (C tiles)
    float h2[8][4];       // layer-2 activations
    float p0, p1;         // predictions of rows g and g+8 (all four lanes of a group)
};

// The four features a thread needs of one row (2t, 2t+1, 2t+8, 2t+9).
struct RowPart {
    float2 lo, hi;
};

__device__ __forceinline__ RowPart load_row(const float *x) {
    const int t = threadIdx.x & 3;
    if (!x) return RowPart{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    return RowPart{__ldg(reinterpret_cast<const float2 *>(x + 2 * t)),
                   __ldg(reinterpret_cast<const float2 *>(x + 2 * t + 8))};
}

__device__ __forceinline__ void tile_forward(const MlpSmem &s, RowPart rg, RowPart rg8, bool vg, bool vg8, Tile &T);
__device__ __forceinline__ void tile_layers(const MlpSmem &s, Tile &T);

__device__ __forceinline__ void tile_forward(const MlpSmem &s, const float *xg, const float *xg8, Tile &T) {
    tile_forward(s, load_row(xg), load_row(xg8), xg != nullptr, xg8 != nullptr, T);
}

__device__ __forceinline__ void tile_forward(const MlpSmem &s, RowPart rg, RowPart rg8, bool vg, bool vg8, Tile &T) {
    const int t = threadIdx.x & 3;
    const int f0 = 2 * t, f1 = 2 * t + 8;
    float z[2][4];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const RowPart &p = rr ? rg8 : rg;
        const bool v = rr ? vg8 : vg;
        z[rr][0] = v ? (p.lo.x - s.mean[f0]) * s.istd[f0] : 0.f;
        z[rr][1] = v ? (p.lo.y - s.mean[f0 + 1]) * s.istd[f0 + 1] : 0.f;
        z[rr][2] = v ? (p.hi.x - s.mean[f1]) * s.istd[f1] : 0.f;
        z[rr][3] = v ? (p.hi.y - s.mean[f1 + 1]) * s.istd[f1 + 1] : 0.f;
    }
    T.a1[0] = pack_bf16(z[0][0], z[0][1]);
    T.a1[1] = pack_bf16(z[1][0], z[1][1]);
    T.a1[2] = pack_bf16(z[0][2], z[0][3]);
    T.a1[3] = pack_bf16(z[1][2], z[1][3]);
    tile_layers(s, T);
}

// Layers 1-3 of a tile whose first-layer operand T.a1 is set.
__device__ __forceinline__ void tile_layers(const MlpSmem &s, Tile &T) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int n = 8 * j + g;
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(c, T.a1, *reinterpret_cast<const uint32_t *>(&s.w1t[n * W1S + 2 * t]),
                 *reinterpret_cast<const uint32_t *>(&s.w1t[n * W1S + 2 * t + 8]));
        const float bb0 = s.b1[8 * j + 2 * t], bb1 = s.b1[8 * j + 2 * t + 1];
        T.h1[j][0] = fmaxf(c[0] + bb0, 0.f);
        T.h1[j][1] = fmaxf(c[1] + bb1, 0.f);
        T.h1[j][2] = fmaxf(c[2] + bb0, 0.f);
        T.h1[j][3] = fmaxf(c[3] + bb1, 0.f);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) T.h2[j][0] = T.h2[j][1] = T.h2[j][2] = T.h2[j][3] = 0.f;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
        const uint32_t a[4] = {pack_bf16(T.h1[2 * kc][0], T.h1[2 * kc][1]), pack_bf16(T.h1[2 * kc][2], T.h1[2 * kc][3]),
                               pack_bf16(T.h1[2 * kc + 1][0], T.h1[2 * kc + 1][1]),
                               pack_bf16(T.h1[2 * kc + 1][2], T.h1[2 * kc + 1][3])};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = 8 * j + g;
            mma16816(T.h2[j], a, *reinterpret_cast<const uint32_t *>(&s.w2t[n * W2S + 16 * kc + 2 * t]),
                     *reinterpret_cast<const uint32_t *>(&s.w2t[n * W2S + 16 * kc + 2 * t + 8]));
        }
    }
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c0 = 8 * j + 2 * t;
        const float bb0 = s.b2[c0], bb1 = s.b2[c0 + 1];
        T.h2[j][0] = fmaxf(T.h2[j][0] + bb0, 0.f);
        T.h2[j][1] = fmaxf(T.h2[j][1] + bb1, 0.f);
        T.h2[j][2] = fmaxf(T.h2[j][2] + bb0, 0.f);
        T.h2[j][3] = fmaxf(T.h2[j][3] + bb1, 0.f);
        p0 += T.h2[j][0] * s.w3[c0] + T.h2[j][1] * s.w3[c0 + 1];
        p1 += T.h2[j][2] * s.w3[c0] + T.h2[j][3] * s.w3[c0 + 1];
    }
    p0 += __shfl_xor_sync(FULL, p0, 1);
    p0 += __shfl_xor_sync(FULL, p0, 2);
    p1 += __shfl_xor_sync(FULL, p1, 1);
    p1 += __shfl_xor_sync(FULL, p1, 2);
    T.p0 = p0 + s.b3;
    T.p1 = p1 + s.b3;
}

constexpr int MLP_WARPS = 8;

__global__ void __launch_bounds__(MLP_WARPS * 32, 4) k_mlp_infer(const ModelDev *__restrict__ M,
                                                              const float *__restrict__ X, int32_t n,
                                                              float *__restrict__ out) {
    __shared__ MlpSmem s;
    load_model(M, s, false);
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
    const int64_t tiles = ((int64_t)n + 15) / 16;
    const int64_t step = (int64_t)gridDim.x * MLP_WARPS;
    auto row = [&](int64_t r) { return r < n ? X + r * MLP_F : nullptr; };
    int64_t tile = (int64_t)blockIdx.x * MLP_WARPS + w;
    // the next tile's rows are loaded before the current tile is computed
    RowPart a = load_row(row(tile * 16 + g)), b = load_row(row(tile * 16 + g + 8));
    for (; tile < tiles; tile += step) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        const RowPart ca = a, cb = b;
        const int64_t nx = tile + step;
        if (nx < tiles) {
            a = load_row(row(nx * 16 + g));
            b = load_row(row(nx * 16 + g + 8));
        }
        Tile T;
        tile_forward(s, ca, cb, r0 < n, r1 < n, T);
        if (t == 0) {
            if (r0 < n) out[r0] = T.p0;
            if (r1 < n) out[r1] = T.p1;
        }
    }
}

// Inference on standardised BF16 rows (8 words per row, word q holding
// features 2q and 2q + 1): lane (g, t) reads words t and t + 4 of rows g and
// g + 8, which are the first-layer A fragment as it is, so the predictions
// equal k_mlp_infer's on the FP32 rows bit for bit.
__global__ void __launch_bounds__(MLP_WARPS * 32, 4) k_mlp_infer_bf16(const ModelDev *__restrict__ M,
                                                                   const uint32_t *__restrict__ Xb, int32_t n,
                                                                   float *__restrict__ out) {
    __shared__ MlpSmem s;
    load_model(M, s, false);
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
    const int64_t tiles = ((int64_t)n + 15) / 16;
    const int64_t step = (int64_t)gridDim.x * MLP_WARPS;
    auto word = [&](int64_t r, int q) { return r < n ? __ldg(Xb + r * (MLP_F / 2) + q) : 0u; };
    int64_t tile = (int64_t)blockIdx.x * MLP_WARPS + w;
    // the next tile's words are loaded before the current tile is computed
    uint32_t a0 = word(tile * 16 + g, t), a1 = word(tile * 16 + g + 8, t);
    uint32_t a2 = word(tile * 16 + g, t + 4), a3 = word(tile * 16 + g + 8, t + 4);
    for (; tile < tiles; tile += step) {
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        Tile T;
        T.a1[0] = a0;
        T.a1[1] = a1;
        T.a1[2] = a2;
        T.a1[3] = a3;
        const int64_t nx = tile + step;
        if (nx < tiles) {
            a0 = word(nx * 16 + g, t);
            a1 = word(nx * 16 + g + 8, t);
            a2 = word(nx * 16 + g, t + 4);
            a3 = word(nx * 16 + g + 8, t + 4);
        }
        tile_layers(s, T);
        if (t == 0) {
            if (r0 < n) out[r0] = T.p0;
            if (r1 < n) out[r1] = T.p1;
        }
    }
}

// Counter-based row sampling: row r of training step `step` (splitmix64).
__device__ __forceinline__ int sample_row(uint64_t seed, int32_t step, int r, int32_t n) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * ((uint64_t)(uint32_t)step * 0x100000000ull + (uint32_t)r + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (int)(z % (uint64_t)n);
}

// Activations kept for the weight gradients, BF16, per padded batch row:
// Z [16], H1 [64], dA2 [64], dA1 [64].
size_t mlp_act_bytes(int32_t batch) {
    const size_t rows = ((size_t)batch + 15) / 16 * 16;
    return rows * (MLP_F + 3 * MLP_H) * sizeof(uint16_t);
}

struct Acts {
    uint16_t *z, *h1, *e2, *e1;
};

__host__ __device__ inline Acts acts_of(uint16_t *base, int32_t batch) {
    const size_t rows = ((size_t)batch + 15) / 16 * 16;
    return Acts{base, base + rows * MLP_F, base + rows * (MLP_F + MLP_H), base + rows * (MLP_F + 2 * MLP_H)};
}

// Zero the gradient and loss; optionally advance the step counter (which
// seeds the row sampling and Adam's bias corrections).
__global__ void k_mlp_zero(ModelDev *M, bool count_step) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P_N; i += gridDim.x * blockDim.x) M->grad[i] = 0.f;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        M->loss_sum = 0.f;
        if (count_step) M->step += 1;
    }
}

// Forward and data-gradient pass of a batch: per 16-row tile the loss, the
// bias and w3 gradients (reduced here) and the activations the weight
// gradients need (written as BF16).  dL/dp = 2 (p - y) / batch.
__global__ void __launch_bounds__(MLP_WARPS * 32) k_mlp_fwd_bwd(ModelDev *M, const float *__restrict__ X,
                                                                const float *__restrict__ Y, int32_t n,
                                                                int32_t batch, uint64_t seed, bool sample,
                                                                uint16_t *acts_base) {
    __shared__ MlpSmem s;
    load_model(M, s, true);
    __syncthreads();
    const Acts A = acts_of(acts_base, batch);
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
    const int32_t step = M->step;
    const float inv_b = 1.0f / (float)batch;
    float gw3[8][2] = {}, gb2[8][2] = {}, gb1[8][2] = {};
    float gb3 = 0.f, loss = 0.f;
    const int tiles = (batch + 15) / 16;
    for (int tile = blockIdx.x * MLP_WARPS + w; tile < tiles; tile += gridDim.x * MLP_WARPS) {
        const int r0 = tile * 16 + g, r1 = r0 + 8;
        const int v0 = r0 < batch ? (sample ? sample_row(seed, step, r0, n) : r0) : -1;
        const int v1 = r1 < batch ? (sample ? sample_row(seed, step, r1, n) : r1) : -1;
        Tile T;
        tile_forward(s, v0 >= 0 ? X + (int64_t)v0 * MLP_F : nullptr, v1 >= 0 ? X + (int64_t)v1 * MLP_F : nullptr, T);
        const float e0 = v0 >= 0 ? T.p0 - Y[v0] : 0.f, e1 = v1 >= 0 ? T.p1 - Y[v1] : 0.f;
        if (t == 0) loss += e0 * e0 + e1 * e1;
        const float d0 = 2.f * e0 * inv_b, d1 = 2.f * e1 * inv_b;
        if (t == 0) gb3 += d0 + d1;
        // layer 3 and 2: dw3, dA2 = d * w3 * [h2 > 0], db2
        float e2[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c0 = 8 * j + 2 * t;
            gw3[j][0] += d0 * T.h2[j][0] + d1 * T.h2[j][2];
            gw3[j][1] += d0 * T.h2[j][1] + d1 * T.h2[j][3];
            e2[j][0] = T.h2[j][0] > 0.f ? d0 * s.w3[c0] : 0.f;
            e2[j][1] = T.h2[j][1] > 0.f ? d0 * s.w3[c0 + 1] : 0.f;
            e2[j][2] = T.h2[j][2] > 0.f ? d1 * s.w3[c0] : 0.f;
            e2[j][3] = T.h2[j][3] > 0.f ? d1 * s.w3[c0 + 1] : 0.f;
            gb2[j][0] += e2[j][0] + e2[j][2];
            gb2[j][1] += e2[j][1] + e2[j][3];
        }
        // layer 1: dA1 = (dA2 W2^T) * [h1 > 0]; B[k = j][n = i] = W2[i][j] = w2r[i][j]
        float e1v[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) e1v[j][0] = e1v[j][1] = e1v[j][2] = e1v[j][3] = 0.f;
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            const uint32_t a[4] = {pack_bf16(e2[2 * kc][0], e2[2 * kc][1]), pack_bf16(e2[2 * kc][2], e2[2 * kc][3]),
                                   pack_bf16(e2[2 * kc + 1][0], e2[2 * kc + 1][1]),
                                   pack_bf16(e2[2 * kc + 1][2], e2[2 * kc + 1][3])};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int nn = 8 * j + g;
                mma16816(e1v[j], a, *reinterpret_cast<const uint32_t *>(&s.w2r[nn * W2S + 16 * kc + 2 * t]),
                         *reinterpret_cast<const uint32_t *>(&s.w2r[nn * W2S + 16 * kc + 2 * t + 8]));
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            e1v[j][0] = T.h1[j][0] > 0.f ? e1v[j][0] : 0.f;
            e1v[j][1] = T.h1[j][1] > 0.f ? e1v[j][1] : 0.f;
            e1v[j][2] = T.h1[j][2] > 0.f ? e1v[j][2] : 0.f;
            e1v[j][3] = T.h1[j][3] > 0.f ? e1v[j][3] : 0.f;
            gb1[j][0] += e1v[j][0] + e1v[j][2];
            gb1[j][1] += e1v[j][1] + e1v[j][3];
        }
        // activations for the weight gradients (rows r0, r1 of the padded batch)
        uint32_t *z0 = reinterpret_cast<uint32_t *>(A.z + (size_t)r0 * MLP_F);
        uint32_t *z1 = reinterpret_cast<uint32_t *>(A.z + (size_t)r1 * MLP_F);
        z0[t] = T.a1[0];
        z1[t] = T.a1[1];
        z0[t + 4] = T.a1[2];
        z1[t + 4] = T.a1[3];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c0 = 8 * j + 2 * t;
            *reinterpret_cast<uint32_t *>(A.h1 + (size_t)r0 * MLP_H + c0) = pack_bf16(T.h1[j][0], T.h1[j][1]);
            *reinterpret_cast<uint32_t *>(A.h1 + (size_t)r1 * MLP_H + c0) = pack_bf16(T.h1[j][2], T.h1[j][3]);
            *reinterpret_cast<uint32_t *>(A.e2 + (size_t)r0 * MLP_H + c0) = pack_bf16(e2[j][0], e2[j][1]);
            *reinterpret_cast<uint32_t *>(A.e2 + (size_t)r1 * MLP_H + c0) = pack_bf16(e2[j][2], e2[j][3]);
            *reinterpret_cast<uint32_t *>(A.e1 + (size_t)r0 * MLP_H + c0) = pack_bf16(e1v[j][0], e1v[j][1]);
            *reinterpret_cast<uint32_t *>(A.e1 + (size_t)r1 * MLP_H + c0) = pack_bf16(e1v[j][2], e1v[j][3]);
        }
    }
    // reduce over the 8 groups (lanes with equal t hold the same columns)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                gw3[j][q] += __shfl_xor_sync(FULL, gw3[j][q], o);
                gb2[j][q] += __shfl_xor_sync(FULL, gb2[j][q], o);
                gb1[j][q] += __shfl_xor_sync(FULL, gb1[j][q], o);
            }
    if (g == 0) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int c = 8 * j + 2 * t + q;
                atomicAdd(&M->grad[P_W3 + c], gw3[j][q]);
                atomicAdd(&M->grad[P_B2 + c], gb2[j][q]);
                atomicAdd(&M->grad[P_B1 + c], gb1[j][q]);
            }
    }
    gb3 = warp_sum(gb3);
    loss = warp_sum(loss);
    if (lane == 0) {
        atomicAdd(&M->grad[P_B3], gb3);
        atomicAdd(&M->loss_sum, loss);
    }
}

// Weight gradients over the batch: dW2 = H1^T dA2 (64 x 64) and
// dW1 = Z^T dA1 (16 x 64), K = batch rows.  A CTA takes WG_ROWS rows; warp w
// owns dW2 row tile (w & 3) x column tiles 4 (w >> 2) .. +3 and dW1 column
// tile w.  Operands are read from the BF16 activations with the transposed
// fragment layout.
constexpr int WG_ROWS = 256;

__global__ void __launch_bounds__(MLP_WARPS * 32) k_mlp_wgrad(ModelDev *M, int32_t batch,
                                                              const uint16_t *__restrict__ acts_base) {
    const Acts A = acts_of(const_cast<uint16_t *>(acts_base), batch);
    const int rows = (batch + 15) / 16 * 16;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
    const int mi = w & 3, nj0 = (w >> 2) * 4;
    float acc2[4][4] = {}, acc1[4] = {};
    for (int r0 = blockIdx.x * WG_ROWS; r0 < rows; r0 += gridDim.x * WG_ROWS) {
        const int rend = min(r0 + WG_ROWS, rows);
        for (int rb = r0; rb < rend; rb += 16) {
            // A = H1^T rows 16 mi .. + 15 (hidden units), k = batch rows rb .. rb + 15
            const uint16_t *h = A.h1 + (size_t)rb * MLP_H;
            const int i0 = 16 * mi + g;
            const uint32_t a2[4] = {pair_u16(h[(2 * t) * MLP_H + i0], h[(2 * t + 1) * MLP_H + i0]),
                                    pair_u16(h[(2 * t) * MLP_H + i0 + 8], h[(2 * t + 1) * MLP_H + i0 + 8]),
                                    pair_u16(h[(2 * t + 8) * MLP_H + i0], h[(2 * t + 9) * MLP_H + i0]),
                                    pair_u16(h[(2 * t + 8) * MLP_H + i0 + 8], h[(2 * t + 9) * MLP_H + i0 + 8])};
            const uint16_t *e = A.e2 + (size_t)rb * MLP_H;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 8 * (nj0 + q) + g;
                mma16816(acc2[q], a2, pair_u16(e[(2 * t) * MLP_H + c], e[(2 * t + 1) * MLP_H + c]),
                         pair_u16(e[(2 * t + 8) * MLP_H + c], e[(2 * t + 9) * MLP_H + c]));
            }
            // A = Z^T (16 features), B = dA1 column tile w
            const uint16_t *z = A.z + (size_t)rb * MLP_F;
            const uint32_t a1[4] = {pair_u16(z[(2 * t) * MLP_F + g], z[(2 * t + 1) * MLP_F + g]),
                                    pair_u16(z[(2 * t) * MLP_F + g + 8], z[(2 * t + 1) * MLP_F + g + 8]),
                                    pair_u16(z[(2 * t + 8) * MLP_F + g], z[(2 * t + 9) * MLP_F + g]),
                                    pair_u16(z[(2 * t + 8) * MLP_F + g + 8], z[(2 * t + 9) * MLP_F + g + 8])};
            const uint16_t *e1 = A.e1 + (size_t)rb * MLP_H;
            const int c1 = 8 * w + g;
            mma16816(acc1, a1, pair_u16(e1[(2 * t) * MLP_H + c1], e1[(2 * t + 1) * MLP_H + c1]),
                     pair_u16(e1[(2 * t + 8) * MLP_H + c1], e1[(2 * t + 9) * MLP_H + c1]));
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = 16 * mi + g, c = 8 * (nj0 + q) + 2 * t;
        atomicAdd(&M->grad[P_W2 + i * MLP_H + c], acc2[q][0]);
        atomicAdd(&M->grad[P_W2 + i * MLP_H + c + 1], acc2[q][1]);
        atomicAdd(&M->grad[P_W2 + (i + 8) * MLP_H + c], acc2[q][2]);
        atomicAdd(&M->grad[P_W2 + (i + 8) * MLP_H + c + 1], acc2[q][3]);
    }
    {
        const int f = g, c = 8 * w + 2 * t;
        atomicAdd(&M->grad[P_W1 + f * MLP_H + c], acc1[0]);
        atomicAdd(&M->grad[P_W1 + f * MLP_H + c + 1], acc1[1]);
        atomicAdd(&M->grad[P_W1 + (f + 8) * MLP_H + c], acc1[2]);
        atomicAdd(&M->grad[P_W1 + (f + 8) * MLP_H + c + 1], acc1[3]);
    }
}

// BF16 copies of the weights in the fragment layouts.
__device__ __forceinline__ void pack_param(ModelDev *M, int i) {
    const uint16_t b = __bfloat16_as_ushort(__float2bfloat16_rn(M->p[i]));
    if (i < P_B1) {
        const int f = (i - P_W1) / MLP_H, j = (i - P_W1) % MLP_H;
        M->w1t[j * MLP_F + f] = b;
    } else if (i >= P_W2 && i < P_B2) {
        const int a = (i - P_W2) / MLP_H, j = (i - P_W2) % MLP_H;
        M->w2t[j * MLP_H + a] = b;
        M->w2r[a * MLP_H + j] = b;
    }
}

__global__ void k_model_pack(ModelDev *M) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P_N; i += gridDim.x * blockDim.x) pack_param(M, i);
}

// One Adam step (bias-corrected moments) with step t = M->step >= 1.
__global__ void k_adam(ModelDev *M, float lr) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const int tstep = M->step;
    const float c1 = 1.f - powf(b1, (float)tstep), c2 = 1.f - powf(b2, (float)tstep);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P_N; i += gridDim.x * blockDim.x) {
        const float gr = M->grad[i];
        const float m = b1 * M->m[i] + (1.f - b1) * gr;
        const float v = b2 * M->v[i] + (1.f - b2) * gr * gr;
        M->m[i] = m;
        M->v[i] = v;
        M->p[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
        pack_param(M, i);
    }
}

// Mean and standard deviation of each feature over the rows (FP64 sums).
__global__ void k_feature_sums(const float *__restrict__ X, int32_t n, double *tmp) {
    __shared__ double s[2 * MLP_F];
    if (threadIdx.x < 2 * MLP_F) s[threadIdx.x] = 0.0;
    __syncthreads();
    const int f = threadIdx.x & (MLP_F - 1);
    double a = 0.0, b = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)n * MLP_F;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = X[i];   // blockDim and the stride are multiples of 16: column f throughout
        a += x;
        b += x * x;
    }
    atomicAdd(&s[f], a);
    atomicAdd(&s[MLP_F + f], b);
    __syncthreads();
    if (threadIdx.x < 2 * MLP_F) atomicAdd(&tmp[threadIdx.x], s[threadIdx.x]);
}

__global__ void k_feature_stats(const double *tmp, int32_t n, ModelDev *M) {
    const int f = threadIdx.x;
    if (f < MLP_F) {
        const double mu = tmp[f] / n, var = tmp[MLP_F + f] / n - mu * mu;
        const double sd = var > 1e-12 ? sqrt(var) : 1.0;
        M->mean[f] = (float)mu;
        M->stdv[f] = (float)sd;
    }
}

int launch_feature_stats(const float *x, int32_t n, ModelDev *M, double *tmp, cudaStream_t st) {
    if (n <= 0) return -1;
    if (cudaMemsetAsync(tmp, 0, 2 * MLP_F * sizeof(double), st) != cudaSuccess) return -1;
    k_feature_sums<<<256, 256, 0, st>>>(x, n, tmp);
    k_feature_stats<<<1, 32, 0, st>>>(tmp, n, M);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_model_pack(ModelDev *M, cudaStream_t st) {
    k_model_pack<<<(P_N + 255) / 256, 256, 0, st>>>(M);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_mlp_infer(const ModelDev *M, const float *x, int32_t n, float *out, int num_sms, cudaStream_t st) {
    const int64_t tiles = ((int64_t)n + 15) / 16;
    int64_t g = (tiles + MLP_WARPS - 1) / MLP_WARPS;
    if (g > (int64_t)num_sms * 8) g = (int64_t)num_sms * 8;
    if (g < 1) g = 1;
    k_mlp_infer<<<(unsigned)g, MLP_WARPS * 32, 0, st>>>(M, x, n, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_mlp_infer_bf16(const ModelDev *M, const uint32_t *xb, int32_t n, float *out, int num_sms,
                          cudaStream_t st) {
    const int64_t tiles = ((int64_t)n + 15) / 16;
    int64_t g = (tiles + MLP_WARPS - 1) / MLP_WARPS;
    if (g > (int64_t)num_sms * 8) g = (int64_t)num_sms * 8;
    if (g < 1) g = 1;
    k_mlp_infer_bf16<<<(unsigned)g, MLP_WARPS * 32, 0, st>>>(M, xb, n, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// One training (or gradient-only) step over `batch` rows: zero, forward +
// data gradients, weight gradients, and (adam) the update.
int launch_mlp_step(ModelDev *M, const float *x, const float *y, int32_t n, int32_t batch, uint64_t seed, bool sample,
                    bool count_step, bool adam, float lr, uint16_t *acts, int num_sms, cudaStream_t st) {
    k_mlp_zero<<<(P_N + 255) / 256, 256, 0, st>>>(M, count_step);
    const int tiles = (batch + 15) / 16;
    int gf = (tiles + MLP_WARPS - 1) / MLP_WARPS;
    if (gf > num_sms * 4) gf = num_sms * 4;
    k_mlp_fwd_bwd<<<gf < 1 ? 1 : gf, MLP_WARPS * 32, 0, st>>>(M, x, y, n, batch, seed, sample, acts);
    int gw = (batch + WG_ROWS - 1) / WG_ROWS;
    if (gw > num_sms * 2) gw = num_sms * 2;
    k_mlp_wgrad<<<gw < 1 ? 1 : gw, MLP_WARPS * 32, 0, st>>>(M, batch, acts);
    if (adam) k_adam<<<(P_N + 255) / 256, 256, 0, st>>>(M, lr);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ef
