// mlp.cu -- the learned surrogate of a cacheable node: a per-material MLP on Fourier
// features of (u, v), trained and evaluated with BF16 tensor-core MMAs (mma.sync
// m16n8k16, FP32 accumulation).
//
// Network: g(u, v) = [sin pi k u, cos pi k u, sin pi k v, cos pi k v]_{k=1..16}
// (64; half-range frequencies, so the network need not repeat from u = 0 to 1)
// -> relu(g W1 + b1) (64) -> relu(h1 W2 + b2) (64) -> h2 W3 + b3 (3); 8,515
// parameters W1 [64][64], b1, W2 [64][64], b2, W3 [64][3], b3.  Operands (features,
// weights, activations) are rounded to BF16, products accumulate in FP32, FP32 master
// weights take Adam steps.
//
// Fragment layouts of mma.m16n8k16 with g = lane / 4, t = lane % 4 (PTX ISA):
//   A 16x16 row-major: {A[g][2t..2t+1]}, {A[g+8][2t..]}, {A[g][2t+8..]}, {A[g+8][2t+8..]}
//   B 16x8 (k, n):     {B[2t..2t+1][g]}, {B[2t+8..2t+9][g]}
//   C 16x8:            C[g][2t], C[g][2t+1], C[g+8][2t], C[g+8][2t+1]
// The C fragments of n-tiles 2q and 2q+1 are exactly the A fragment of k-chunk q, so a
// layer's activations feed the next layer from registers.
#include <cuda_bf16.h>

#include <cstdint>

#include "nodes.cuh"
#include "pmc_internal.h"

namespace pmc {

namespace {

constexpr int P_W1 = 0, P_B1 = 4096, P_W2 = 4160, P_B2 = 8256, P_W3 = 8320, P_B3 = 8512;
constexpr int MB = 128;       // training rows per step: 8 warps x 16
constexpr int WS = 72;        // shared row stride (bf16) of 64-wide weight rows: conflict-free
constexpr int AS = MB + 8;    // shared row stride of transposed activations
constexpr unsigned FULL = 0xFFFFFFFFu;

struct Smem {                 // byte offsets into dynamic shared memory
    static constexpr int w1t = 0;                       // [64 out][WS]  forward B of layer 1
    static constexpr int w2t = w1t + 64 * WS * 2;       // [64 out][WS]  forward B of layer 2
    static constexpr int w3t = w2t + 64 * WS * 2;       // [8 out][WS]   forward B of layer 3
    static constexpr int bias = w3t + 8 * WS * 2;       // b1[64], b2[64], b3[8] fp32
    static constexpr int infer_end = bias + 136 * 4;
    static constexpr int w2r = infer_end;               // [64 in][WS]   backward B, dH1 = dH2 W2^T
    static constexpr int w3r = w2r + 64 * WS * 2;       // [64 in][8]    backward B, dH2 = dY W3^T
    static constexpr int gT = w3r + 64 * 8 * 2;         // [64 feature][AS] transposed activations
    static constexpr int h1T = gT + 64 * AS * 2;
    static constexpr int h2T = h1T + 64 * AS * 2;
    static constexpr int d1T = h2T + 64 * AS * 2;
    static constexpr int d2T = d1T + 64 * AS * 2;
    static constexpr int dyT = d2T + 64 * AS * 2;       // [8 out][AS]
    static constexpr int train_end = dyT + 8 * AS * 2;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf_lo(uint32_t x) { return __uint_as_float(x << 16); }
__device__ __forceinline__ float bf_hi(uint32_t x) { return __uint_as_float(x & 0xFFFF0000u); }
__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <typename T>
__device__ __forceinline__ T* at(unsigned char* base, int off) { return reinterpret_cast<T*>(base + off); }

// Copies FP32 parameters into the BF16 shared layouts (all threads of the block).
__device__ void load_weights(unsigned char* sm, const float* __restrict__ th, bool train) {
    __nv_bfloat16* w1t = at<__nv_bfloat16>(sm, Smem::w1t);
    __nv_bfloat16* w2t = at<__nv_bfloat16>(sm, Smem::w2t);
    __nv_bfloat16* w3t = at<__nv_bfloat16>(sm, Smem::w3t);
    float* bias = at<float>(sm, Smem::bias);
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
        const int in = i >> 6, out = i & 63;
        w1t[out * WS + in] = __float2bfloat16_rn(th[P_W1 + i]);
        const __nv_bfloat16 w2 = __float2bfloat16_rn(th[P_W2 + i]);
        w2t[out * WS + in] = w2;
        if (train) at<__nv_bfloat16>(sm, Smem::w2r)[in * WS + out] = w2;
    }
    for (int i = threadIdx.x; i < 64 * 8; i += blockDim.x) {
        const int in = i >> 3, out = i & 7;
        const __nv_bfloat16 w3 = __float2bfloat16_rn(out < 3 ? th[P_W3 + in * 3 + out] : 0.0f);
        w3t[out * WS + in] = w3;
        if (train) at<__nv_bfloat16>(sm, Smem::w3r)[in * 8 + out] = w3;
    }
    for (int i = threadIdx.x; i < 136; i += blockDim.x)
        bias[i] = i < 64 ? th[P_B1 + i] : (i < 128 ? th[P_B2 + i - 64] : (i < 131 ? th[P_B3 + i - 128] : 0.0f));
}

// Features of rows g and g+8 as the A fragments of the four 16-column chunks
// (sin u, cos u, sin v, cos v); optionally their transposed BF16 copy.
__device__ __forceinline__ void features(float u0, float v0, float u1, float v1, uint32_t (&af)[4][4],
                                         __nv_bfloat16* gT, int b0) {
    const int t = threadIdx.x & 3;
    const int cols[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
    float su[2][4], cu[2][4], sv[2][4], cv[2][4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float k = (float)(cols[c] + 1);   // the angle is pi k u (k u exact in FP32)
        sincospif(k * u0, &su[0][c], &cu[0][c]);
        sincospif(k * u1, &su[1][c], &cu[1][c]);
        sincospif(k * v0, &sv[0][c], &cv[0][c]);
        sincospif(k * v1, &sv[1][c], &cv[1][c]);
    }
    float (*F[4])[4] = {su, cu, sv, cv};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        af[q][0] = pack_bf16(F[q][0][0], F[q][0][1]);
        af[q][1] = pack_bf16(F[q][1][0], F[q][1][1]);
        af[q][2] = pack_bf16(F[q][0][2], F[q][0][3]);
        af[q][3] = pack_bf16(F[q][1][2], F[q][1][3]);
        if (gT) {
            const int g = (threadIdx.x & 31) >> 2;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                gT[(16 * q + cols[c]) * AS + b0 + g] = __float2bfloat16_rn(F[q][0][c]);
                gT[(16 * q + cols[c]) * AS + b0 + g + 8] = __float2bfloat16_rn(F[q][1][c]);
            }
        }
    }
}

// One hidden layer: acc = A (16x64) x W (64x64) from wT [out][in]; relu(acc + b) as the A
// fragments of the next layer; optionally stored transposed (BF16) at hT.
__device__ __forceinline__ void hidden(const uint32_t (&ain)[4][4], const __nv_bfloat16* wT, const float* b,
                                       uint32_t (&aout)[4][4], __nv_bfloat16* hT, int b0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const __nv_bfloat16* wr = wT + (8 * j + g) * WS + 16 * q + 2 * t;
            mma16816(acc[j], ain[q], ld_pair(wr), ld_pair(wr + 8));
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = 8 * j + 2 * t;
        acc[j][0] = fmaxf(acc[j][0] + b[c], 0.0f);
        acc[j][1] = fmaxf(acc[j][1] + b[c + 1], 0.0f);
        acc[j][2] = fmaxf(acc[j][2] + b[c], 0.0f);
        acc[j][3] = fmaxf(acc[j][3] + b[c + 1], 0.0f);
        if (hT) {
            hT[c * AS + b0 + g] = __float2bfloat16_rn(acc[j][0]);
            hT[(c + 1) * AS + b0 + g] = __float2bfloat16_rn(acc[j][1]);
            hT[c * AS + b0 + g + 8] = __float2bfloat16_rn(acc[j][2]);
            hT[(c + 1) * AS + b0 + g + 8] = __float2bfloat16_rn(acc[j][3]);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        aout[q][0] = pack_bf16(acc[2 * q][0], acc[2 * q][1]);
        aout[q][1] = pack_bf16(acc[2 * q][2], acc[2 * q][3]);
        aout[q][2] = pack_bf16(acc[2 * q + 1][0], acc[2 * q + 1][1]);
        aout[q][3] = pack_bf16(acc[2 * q + 1][2], acc[2 * q + 1][3]);
    }
}

// Output layer: y (16 x 8, columns >= 3 zero) = h2 x W3 + b3.
__device__ __forceinline__ void output(const uint32_t (&a2)[4][4], const __nv_bfloat16* w3t, const float* b3,
                                       float (&y)[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    y[0] = y[1] = y[2] = y[3] = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat16* wr = w3t + g * WS + 16 * q + 2 * t;
        mma16816(y, a2[q], ld_pair(wr), ld_pair(wr + 8));
    }
    const int o = 2 * t;
    const float bl = o < 3 ? b3[o] : 0.0f, bh = o + 1 < 3 ? b3[o + 1] : 0.0f;
    y[0] += bl;
    y[1] += bh;
    y[2] += bl;
    y[3] += bh;
}

// relu'(h) > 0 of the activation at C position (row g or g+8, column 8j + 2t + k) from
// the A fragments that hold it.
__device__ __forceinline__ bool active(const uint32_t (&a)[4][4], int j, int idx) {
    const uint32_t w = a[j >> 1][(j & 1) * 2 + (idx >> 1)];
    return ((idx & 1) ? bf_hi(w) : bf_lo(w)) > 0.0f;
}

// dW tile group of one warp: C (16 x 8 tiles) = A^T-rows (m = feature) x B (k = batch row).
__device__ __forceinline__ void weight_grad(const __nv_bfloat16* aT, const __nv_bfloat16* bT, int mt, int j0, int nj,
                                            float (&gw)[4][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) gw[jj][0] = gw[jj][1] = gw[jj][2] = gw[jj][3] = 0.0f;
#pragma unroll 2
    for (int ks = 0; ks < MB / 16; ++ks) {
        const __nv_bfloat16* ar = aT + (16 * mt + g) * AS + 16 * ks + 2 * t;
        const uint32_t a[4] = {ld_pair(ar), ld_pair(ar + 8 * AS), ld_pair(ar + 8), ld_pair(ar + 8 * AS + 8)};
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            if (jj >= nj) break;
            const __nv_bfloat16* br = bT + (8 * (j0 + jj) + g) * AS + 16 * ks + 2 * t;
            mma16816(gw[jj], a, ld_pair(br), ld_pair(br + 8));
        }
    }
}

struct TrainArgs {
    float* theta;            // n_mats x 8515 FP32 masters
    float* adam_m;
    float* adam_v;
    float* grad;             // gradient mode: accumulated gradient (n_mats x 8515)
    const float* data;       // per material: n_data rows of (u, v, r, g, b)
    float* loss;             // per material: summed loss of the steps run
    uint32_t n_data;         // rows per material (a power of two in training mode)
    uint32_t steps;          // steps in this launch
    uint64_t sample0;        // rows consumed before this launch (per material)
    uint32_t step0;          // Adam steps taken before this launch
    uint32_t total_steps;    // for the learning-rate schedule
    float lr;
    float grad_scale;        // dL/dy = grad_scale * (y - t)
    int mode;                // 0: train (Adam), 1: accumulate the gradient only
};

__device__ __forceinline__ void apply(const TrainArgs& A, size_t base, int idx, float gr, float lr_t, float bc1,
                                      float bc2) {
    const size_t k = base + idx;
    if (A.mode == 1) {
        atomicAdd(&A.grad[k], gr);
        return;
    }
    const float m = 0.9f * A.adam_m[k] + 0.1f * gr;
    const float v = 0.999f * A.adam_v[k] + 0.001f * gr * gr;
    A.adam_m[k] = m;
    A.adam_v[k] = v;
    A.theta[k] -= lr_t * (m / bc1) / (sqrtf(v / bc2) + 1e-8f);
}

// One block per material (blockIdx.y) runs `steps` minibatch steps: forward, backward and
// the Adam update of all 8,515 parameters.  In gradient mode blockIdx.x splits the rows.
__global__ void __launch_bounds__(256) k_mlp_train(TrainArgs A) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint32_t mat = blockIdx.y;
    const size_t pbase = (size_t)mat * MLP_PARAMS;
    const float* th = A.theta + pbase;
    const float* data = A.data + (size_t)mat * A.n_data * 5;
    __nv_bfloat16* gT = at<__nv_bfloat16>(sm, Smem::gT);
    __nv_bfloat16* h1T = at<__nv_bfloat16>(sm, Smem::h1T);
    __nv_bfloat16* h2T = at<__nv_bfloat16>(sm, Smem::h2T);
    __nv_bfloat16* d1T = at<__nv_bfloat16>(sm, Smem::d1T);
    __nv_bfloat16* d2T = at<__nv_bfloat16>(sm, Smem::d2T);
    __nv_bfloat16* dyT = at<__nv_bfloat16>(sm, Smem::dyT);
    const float* bias = at<float>(sm, Smem::bias);
    float loss = 0.0f;
    const uint32_t log2n = 31 - __clz(A.n_data);
    for (uint32_t s = 0; s < A.steps; ++s) {
        const uint32_t step = s * gridDim.x + blockIdx.x;
        load_weights(sm, th, true);
        __syncthreads();
        // ---- rows of this warp: g and g + 8 of tile `warp`
        const int b0 = warp * 16;
        uint32_t rows[2];
        float uu[2], vv[2], tg[2][3];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const uint64_t k = A.sample0 + (uint64_t)step * MB + b0 + g + 8 * r;
            if (A.mode == 1) {
                rows[r] = (uint32_t)k;
            } else {
                const uint32_t epoch = (uint32_t)(k >> log2n);
                rows[r] = (uint32_t)(k * 2654435761ull + (uint64_t)epoch * 0x9E3779B9ull) & (A.n_data - 1);
            }
            const float* d = data + (size_t)rows[r] * 5;
            uu[r] = d[0];
            vv[r] = d[1];
            tg[r][0] = d[2];
            tg[r][1] = d[3];
            tg[r][2] = d[4];
        }
        uint32_t a0[4][4], a1[4][4], a2[4][4];
        features(uu[0], vv[0], uu[1], vv[1], a0, gT, b0);
        hidden(a0, at<__nv_bfloat16>(sm, Smem::w1t), bias, a1, h1T, b0);
        hidden(a1, at<__nv_bfloat16>(sm, Smem::w2t), bias + 64, a2, h2T, b0);
        float y[4];
        output(a2, at<__nv_bfloat16>(sm, Smem::w3t), bias + 128, y);
        // ---- dL/dy and the loss
        float dy[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int o = 2 * t + (k & 1), r = k >> 1;
            const float e = o < 3 ? y[k] - tg[r][o] : 0.0f;
            dy[k] = A.grad_scale * e;
            loss += e * e;
            dyT[o * AS + b0 + g + 8 * r] = __float2bfloat16_rn(dy[k]);
        }
        // ---- dH2 = dY W3^T masked by relu'(h2)
        uint32_t ad[4] = {pack_bf16(dy[0], dy[1]), pack_bf16(dy[2], dy[3]), 0u, 0u};
        const __nv_bfloat16* w3r = at<__nv_bfloat16>(sm, Smem::w3r);
        float acc[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
            mma16816(acc[j], ad, ld_pair(w3r + (8 * j + g) * 8 + 2 * t), 0u);
        }
        uint32_t ad2[4][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = 8 * j + 2 * t;
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[j][k] = active(a2, j, k) ? acc[j][k] : 0.0f;
            d2T[c * AS + b0 + g] = __float2bfloat16_rn(acc[j][0]);
            d2T[(c + 1) * AS + b0 + g] = __float2bfloat16_rn(acc[j][1]);
            d2T[c * AS + b0 + g + 8] = __float2bfloat16_rn(acc[j][2]);
            d2T[(c + 1) * AS + b0 + g + 8] = __float2bfloat16_rn(acc[j][3]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            ad2[q][0] = pack_bf16(acc[2 * q][0], acc[2 * q][1]);
            ad2[q][1] = pack_bf16(acc[2 * q][2], acc[2 * q][3]);
            ad2[q][2] = pack_bf16(acc[2 * q + 1][0], acc[2 * q + 1][1]);
            ad2[q][3] = pack_bf16(acc[2 * q + 1][2], acc[2 * q + 1][3]);
        }
        // ---- dH1 = dH2 W2^T masked by relu'(h1)
        const __nv_bfloat16* w2r = at<__nv_bfloat16>(sm, Smem::w2r);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const __nv_bfloat16* wr = w2r + (8 * j + g) * WS + 16 * q + 2 * t;
                mma16816(acc[j], ad2[q], ld_pair(wr), ld_pair(wr + 8));
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = 8 * j + 2 * t;
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[j][k] = active(a1, j, k) ? acc[j][k] : 0.0f;
            d1T[c * AS + b0 + g] = __float2bfloat16_rn(acc[j][0]);
            d1T[(c + 1) * AS + b0 + g] = __float2bfloat16_rn(acc[j][1]);
            d1T[c * AS + b0 + g + 8] = __float2bfloat16_rn(acc[j][2]);
            d1T[(c + 1) * AS + b0 + g + 8] = __float2bfloat16_rn(acc[j][3]);
        }
        __syncthreads();
        // ---- weight gradients over the 128 rows, tiles split across the 8 warps
        const uint32_t adam_t = A.step0 + step + 1;
        const float frac = A.total_steps > 1 ? (float)(A.step0 + step) / (float)(A.total_steps - 1) : 0.0f;
        const float lr_t = A.lr * (0.05f + 0.95f * 0.5f * (1.0f + cospif(fminf(frac, 1.0f))));
        const float bc1 = 1.0f - powf(0.9f, (float)adam_t), bc2 = 1.0f - powf(0.999f, (float)adam_t);
        float gw[4][4];
        const int mt = warp >> 1, j0 = 4 * (warp & 1);
        weight_grad(gT, d1T, mt, j0, 4, gw);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int in = 16 * mt + g, out = 8 * (j0 + jj) + 2 * t;
            apply(A, pbase, P_W1 + in * 64 + out, gw[jj][0], lr_t, bc1, bc2);
            apply(A, pbase, P_W1 + in * 64 + out + 1, gw[jj][1], lr_t, bc1, bc2);
            apply(A, pbase, P_W1 + (in + 8) * 64 + out, gw[jj][2], lr_t, bc1, bc2);
            apply(A, pbase, P_W1 + (in + 8) * 64 + out + 1, gw[jj][3], lr_t, bc1, bc2);
        }
        weight_grad(h1T, d2T, mt, j0, 4, gw);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int in = 16 * mt + g, out = 8 * (j0 + jj) + 2 * t;
            apply(A, pbase, P_W2 + in * 64 + out, gw[jj][0], lr_t, bc1, bc2);
            apply(A, pbase, P_W2 + in * 64 + out + 1, gw[jj][1], lr_t, bc1, bc2);
            apply(A, pbase, P_W2 + (in + 8) * 64 + out, gw[jj][2], lr_t, bc1, bc2);
            apply(A, pbase, P_W2 + (in + 8) * 64 + out + 1, gw[jj][3], lr_t, bc1, bc2);
        }
        if (warp < 4) {
            weight_grad(h2T, dyT, warp, 0, 1, gw);
            const int in = 16 * warp + g, out = 2 * t;
            if (out < 3) {
                apply(A, pbase, P_W3 + in * 3 + out, gw[0][0], lr_t, bc1, bc2);
                apply(A, pbase, P_W3 + (in + 8) * 3 + out, gw[0][2], lr_t, bc1, bc2);
            }
            if (out + 1 < 3) {
                apply(A, pbase, P_W3 + in * 3 + out + 1, gw[0][1], lr_t, bc1, bc2);
                apply(A, pbase, P_W3 + (in + 8) * 3 + out + 1, gw[0][3], lr_t, bc1, bc2);
            }
        }
        // ---- bias gradients: row sums of the transposed activation gradients
        if (threadIdx.x < 131) {
            const int i = threadIdx.x;
            const __nv_bfloat16* row = i < 64 ? d1T + i * AS : (i < 128 ? d2T + (i - 64) * AS : dyT + (i - 128) * AS);
            float sum = 0.0f;
            for (int b = 0; b < MB; ++b) sum += __bfloat162float(row[b]);
            apply(A, pbase, i < 64 ? P_B1 + i : (i < 128 ? P_B2 + i - 64 : P_B3 + i - 128), sum, lr_t, bc1, bc2);
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(FULL, loss, o);
    if (lane == 0) atomicAdd(&A.loss[mat], loss);
}

// Training pairs of the exact evaluator: uniform (u, v) from a counter-based generator
// (SplitMix64 of seed ^ (material, row)), value = the cacheable node's standalone program.
__global__ void __launch_bounds__(128) k_root_samples(const uint4* __restrict__ prog, const float* __restrict__ params,
                                                      const RootInfo* __restrict__ rinfo, const uint32_t* __restrict__ groots,
                                                      uint32_t n_train_mats, uint32_t n_rows, uint64_t seed, float* data,
                                                      uint32_t max_slots) {
    extern __shared__ float s_val[];
    __shared__ float2 s_grad[8];
    init_gradients(s_grad);
    __syncthreads();
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* V = s_val + (size_t)warp * max_slots * 96u + lane;
    const uint32_t chunks = (n_rows + 31) / 32;
    for (uint32_t item = blockIdx.x * 4 + warp; item < n_train_mats * chunks; item += gridDim.x * 4) {
        const uint32_t mi = item / chunks, row = (item % chunks) * 32 + lane;
        const RootInfo ri = rinfo[groots[mi]];
        PointIn pt{0, 0, 0, 0, 0, 0, 0, 0};
        const uint64_t z = seed ^ (((uint64_t)mi << 32) | row);
        const uint64_t h = z + 0x9E3779B97F4A7C15ull;
        uint64_t x = (h ^ (h >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        x ^= x >> 31;
        pt.u = (float)(uint32_t)(x >> 40) * (1.0f / 16777216.0f);
        pt.v = (float)(uint32_t)((x >> 8) & 0xFFFFFFu) * (1.0f / 16777216.0f);
        for (uint32_t pc = 0; pc < ri.prog_len; ++pc) {
            const uint4 ins = __ldg(&prog[ri.prog_start + pc]);
            const uint32_t op = ins.x & 0xFFu;
            if (op == OP_LOAD_ROOT) {
                // a cacheable node below this one: the sample uses its exact value too,
                // evaluated by running that node's own program is not available here;
                // such nodes are rejected when surrogates are chosen
                continue;
            }
            if (row < n_rows) exec_node(op, ins, V, pt, params, s_grad);
        }
        if (row < n_rows) {
            float* d = data + ((size_t)mi * n_rows + row) * 5;
            d[0] = pt.u;
            d[1] = pt.v;
            d[2] = V[(ri.out_slot * 3) * 32];
            d[3] = V[(ri.out_slot * 3 + 1) * 32];
            d[4] = V[(ri.out_slot * 3 + 2) * 32];
        }
    }
}

}  // namespace

size_t mlp_train_smem() { return Smem::train_end; }
size_t mlp_infer_smem() { return Smem::infer_end; }

cudaError_t launch_mlp_train(float* theta, float* adam_m, float* adam_v, float* grad, const float* data, float* loss,
                             uint32_t n_mats, uint32_t n_data, uint32_t steps, uint64_t sample0, uint32_t step0,
                             uint32_t total_steps, float lr, float grad_scale, int mode, uint32_t splits,
                             cudaStream_t s) {
    TrainArgs A{theta, adam_m, adam_v, grad, data, loss, n_data, steps, sample0, step0, total_steps, lr, grad_scale, mode};
    cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Smem::train_end);
    if (e != cudaSuccess) return e;
    k_mlp_train<<<dim3(splits, n_mats), 256, Smem::train_end, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_root_samples(const uint4* prog, const float* params, const RootInfo* rinfo, const uint32_t* groots,
                                uint32_t n_train_mats, uint32_t n_rows, uint64_t seed, float* data, uint32_t max_slots,
                                int num_sms, cudaStream_t s) {
    const size_t smem = (size_t)4 * max_slots * 96u * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_root_samples, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_root_samples<<<num_sms * 16, 128, smem, s>>>(prog, params, rinfo, groots, n_train_mats, n_rows, seed, data,
                                                   max_slots);
    return cudaGetLastError();
}

}  // namespace pmc
