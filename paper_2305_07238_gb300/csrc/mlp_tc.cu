// mlp_tc.cu -- the learned surrogate on the 5th-generation tensor cores: inference and
// training with tcgen05.mma (kind::f16, BF16 operands from shared memory, FP32 accumulators
// in tensor memory), completion tracked by an mbarrier, accumulators read back with
// tcgen05.ld.
//
// A CTA of 128 threads evaluates tiles of 128 points: thread t owns row t of every
// activation matrix and lane t of tensor memory (warp w reads lanes 32w..32w+31).
//   layer 1: D1[128x64] = G[128x64] W1      (G: features, K = 64 in four K = 16 steps)
//   layer 2: D2[128x64] = relu(D1 + b1) W2
//   layer 3: D3[128x16] = relu(D2 + b2) W3  (outputs 0..2 used, W3 padded to 16 columns)
// Operands live in shared memory in the no-swizzle K-major layout: 8x8 BF16 "core
// matrices" of 128 contiguous bytes, core matrices adjacent along K 128 B apart (leading
// byte offset) and 8-row groups 1024 B apart (stride byte offset).  The network and
// its BF16 rounding points are those of mlp.cu (features, weights and hidden
// activations rounded to BF16, FP32 accumulation).
#include <cuda_bf16.h>

#include <cstdint>

#include "nodes.cuh"
#include "pmc_internal.h"

namespace pmc {

namespace {

constexpr int P_W1 = 0, P_B1 = 4096, P_W2 = 4160, P_B2 = 8256, P_W3 = 8320, P_B3 = 8512;
constexpr uint32_t TC_ROWS = 128;
constexpr uint32_t TC_COLS = 64;                // tensor-memory columns: D1, D2 and D3 all at column 0
constexpr uint32_t TC_CTAS_PER_SM = 6;          // resident inference CTAs (shared memory and TMEM allow 6)
constexpr uint32_t WAIT_POLLS = 1u << 22;       // bound of every mbarrier wait

// One activation operand serves the three layers: a layer's epilogue overwrites it only after
// the product that read it has completed (the mbarrier wait), and likewise one 64-column
// accumulator, read out completely before the next product is issued.  35 KB of shared
// memory and 64 TMEM columns per CTA let six CTAs share an SM.
struct Sm {                                     // byte offsets into dynamic shared memory
    static constexpr uint32_t a0 = 0;           // 128 x 64 BF16: features, then layer-1, then layer-2 output
    static constexpr uint32_t w1 = 16384;       // 64 x 64 BF16: W1 transposed (n rows, k columns)
    static constexpr uint32_t w2 = 24576;       // 64 x 64 BF16: W2 transposed
    static constexpr uint32_t w3 = 32768;       // 16 x 64 BF16: W3 transposed, rows 3..15 zero
    static constexpr uint32_t bias = 34816;     // b1[64], b2[64], b3[4] FP32
    static constexpr uint32_t mbar = 35344;     // 8-byte mbarrier of the products
    static constexpr uint32_t mbar_w = 35352;   // 8-byte mbarrier of the operand-image copy
    static constexpr uint32_t tmem = 35360;     // tensor-memory base written by tcgen05.alloc
    static constexpr uint32_t end = 35368;
};
// the operand image of a network is shared memory [w1, bias end), in that layout
static_assert(Sm::bias + 132 * 4 - Sm::w1 == SURR_IMG_BYTES, "operand image = weights and biases of Sm");
static_assert(Sm::w1 % 16 == 0, "bulk copies land on 16-byte boundaries");
static_assert(TC_CTAS_PER_SM * (Sm::end + 1024) <= 228 * 1024, "inference CTAs per SM by shared memory");
static_assert(TC_CTAS_PER_SM * TC_COLS <= 512, "inference CTAs per SM by tensor memory");

// Byte offset of element (r, c) of a 64-column operand in the core-matrix layout.
__device__ __forceinline__ uint32_t cm_off(uint32_t r, uint32_t c) {
    return (r >> 3) * 1024u + (c >> 3) * 128u + (r & 7u) * 16u + (c & 7u) * 2u;
}

// The same for an operand of K columns: 8-row groups K * 16 bytes apart.
__device__ __forceinline__ uint32_t cm_off_k(uint32_t r, uint32_t c, uint32_t k) {
    return (r >> 3) * (k * 16u) + (c >> 3) * 128u + (r & 7u) * 16u + (c & 7u) * 2u;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading byte offset 128, stride byte
// offset 1024, the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// The same for an operand of K columns (stride byte offset K * 16).
__device__ __forceinline__ uint64_t sdesc_k(uint32_t saddr, uint32_t k) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)((k * 16u) >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc(uint32_t m, uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits for the mbarrier phase with the given parity; false if the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < WAIT_POLLS && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
    }
    return done != 0;
}

// 16 consecutive FP32 accumulator columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// FP32 parameters -> BF16 transposed operands and FP32 biases in shared memory (all 128
// threads); the async-proxy fence is issued by the caller before the next MMA.
// The network's operands from its FP32 parameters, written at dst in the layout of Sm from
// w1 on (shared memory, or a network's operand image in global memory).  The loads of W1
// and W2 are issued eight per matrix at a time, so that a thread has 16 in flight instead
// of one (the parameters are FP32 and 4-byte aligned only).
__device__ void tc_write_weights(unsigned char* dst, const float* __restrict__ th) {
    unsigned char* sm = dst - Sm::w1;   // offsets below are Sm's
    static_assert(64u * 64u % (TC_ROWS * 8u) == 0, "W1/W2 batches");
    for (uint32_t i0 = threadIdx.x; i0 < 64u * 64u; i0 += 8u * TC_ROWS) {
        float w1[8], w2[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            w1[k] = __ldg(th + P_W1 + i0 + k * TC_ROWS);
            w2[k] = __ldg(th + P_W2 + i0 + k * TC_ROWS);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t i = i0 + k * TC_ROWS, in = i >> 6, out = i & 63u;
            *reinterpret_cast<__nv_bfloat16*>(sm + Sm::w1 + cm_off(out, in)) = __float2bfloat16_rn(w1[k]);
            *reinterpret_cast<__nv_bfloat16*>(sm + Sm::w2 + cm_off(out, in)) = __float2bfloat16_rn(w2[k]);
        }
    }
    for (uint32_t i = threadIdx.x; i < 16u * 64u; i += blockDim.x) {
        const uint32_t out = i >> 6, in = i & 63u;
        const float w = out < 3 ? th[P_W3 + in * 3 + out] : 0.0f;
        *reinterpret_cast<__nv_bfloat16*>(sm + Sm::w3 + cm_off(out, in)) = __float2bfloat16_rn(w);
    }
    float* bias = reinterpret_cast<float*>(sm + Sm::bias);
    for (uint32_t i = threadIdx.x; i < 132u; i += blockDim.x)
        bias[i] = i < 64 ? th[P_B1 + i] : (i < 128 ? th[P_B2 + i - 64] : (i < 131 ? th[P_B3 + i - 128] : 0.0f));
}

__device__ __forceinline__ void tc_load_weights(unsigned char* sm, const float* __restrict__ th) {
    tc_write_weights(sm + Sm::w1, th);
}

// The operand image of one network: block b writes slot b's.
__global__ void __launch_bounds__(TC_ROWS) k_surr_images(const float* __restrict__ theta, unsigned char* img) {
    tc_write_weights(img + (size_t)blockIdx.x * SURR_IMG_BYTES, theta + (size_t)blockIdx.x * MLP_PARAMS);
}

// One bulk copy (the tensor memory accelerator's linear form) of a network's operand image
// into shared memory [w1, bias end), completing on mbar_w with its byte count: issued by
// thread 0 after every thread is done with the previous network's operands (the caller's
// barrier); every thread then waits (bounded).  False if the wait ran out.
__device__ __forceinline__ bool tc_copy_image(unsigned char* sm, const unsigned char* src, uint32_t* phase_w) {
    const uint32_t base = smem_u32(sm), mbar = base + Sm::mbar_w;
    if (threadIdx.x == 0) {
        fence_async_smem();
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(SURR_IMG_BYTES)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(base +
                                                                                                           Sm::w1),
            "l"(src), "r"(SURR_IMG_BYTES), "r"(mbar)
            : "memory");
    }
    const bool done = mbar_wait(mbar, *phase_w);
    *phase_w ^= 1u;
    return !__syncthreads_or(!done);
}

// BF16 pair {relu(lo), relu(hi)} (lo in the low half) in one conversion: each value is
// clamped below at 0, then rounded to nearest even, as pack2(fmaxf(lo, 0), fmaxf(hi, 0)).
__device__ __forceinline__ uint32_t pack2_relu(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Row t of the feature matrix: [sin pi k u, cos pi k u, sin pi k v, cos pi k v], k = 1..16.
// sincospif gives the anchors k = 1 and k = 9 of both coordinates; from each anchor, seven
// steps of the angle-addition formulas
//   sin(a + b) = sin a cos b + cos a sin b,  cos(a + b) = cos a cos b - sin a sin b
// with b = pi x give the next seven frequencies.  Every quantity is a (u, v) pair, so one
// packed instruction steps both coordinates.  A step adds about an ulp of error, so every
// feature is within a few ulps of sincospif's, far below the BF16 rounding the features
// then take.  The features are packed to BF16 as soon as two neighbours exist.
__device__ __forceinline__ void tc_features(unsigned char* sm, uint32_t t, float u, float v) {
    float s1u, c1u, s1v, c1v;
    sincospif(u, &s1u, &c1u);
    sincospif(v, &s1v, &c1v);
    const float2 S1 = f2(s1u, s1v), C1 = f2(c1u, c1v), nS1 = f2(-s1u, -s1v);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float2 sk, ck;
        if (half == 0) {
            sk = S1;
            ck = C1;
        } else {
            float su, cu, sv, cv;
            sincospif(9.0f * u, &su, &cu);
            sincospif(9.0f * v, &sv, &cv);
            sk = f2(su, sv);
            ck = f2(cu, cv);
        }
        uint32_t wsu[4], wcu[4], wsv[4], wcv[4];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            const float2 sn = fma2(sk, C1, mul2(ck, S1));
            const float2 cn = fma2(ck, C1, mul2(sk, nS1));
            wsu[j / 2] = pack2(sk.x, sn.x);
            wcu[j / 2] = pack2(ck.x, cn.x);
            wsv[j / 2] = pack2(sk.y, sn.y);
            wcv[j / 2] = pack2(ck.y, cn.y);
            if (j < 6) {
                sk = fma2(sn, C1, mul2(cn, S1));
                ck = fma2(cn, C1, mul2(sn, nS1));
            }
        }
        const uint32_t k0 = 8u * half;   // first frequency of this anchor, minus one
        *reinterpret_cast<uint4*>(sm + Sm::a0 + cm_off(t, k0)) = make_uint4(wsu[0], wsu[1], wsu[2], wsu[3]);
        *reinterpret_cast<uint4*>(sm + Sm::a0 + cm_off(t, 16 + k0)) = make_uint4(wcu[0], wcu[1], wcu[2], wcu[3]);
        *reinterpret_cast<uint4*>(sm + Sm::a0 + cm_off(t, 32 + k0)) = make_uint4(wsv[0], wsv[1], wsv[2], wsv[3]);
        *reinterpret_cast<uint4*>(sm + Sm::a0 + cm_off(t, 48 + k0)) = make_uint4(wcv[0], wcv[1], wcv[2], wcv[3]);
    }
}

// relu(acc + bias) of 64 accumulator columns -> row t of a BF16 operand.
__device__ __forceinline__ void tc_hidden(unsigned char* sm, uint32_t dst, uint32_t taddr, const float* bias,
                                          uint32_t t) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float v[16];
        tmem_ld16(taddr + 16u * q, v);
        uint32_t p[8];
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            const float4 b = *reinterpret_cast<const float4*>(bias + 16 * q + 2 * k);
            const float2 x0 = add2(f2(v[2 * k], v[2 * k + 1]), f2(b.x, b.y));
            const float2 x1 = add2(f2(v[2 * k + 2], v[2 * k + 3]), f2(b.z, b.w));
            p[k] = pack2_relu(x0.x, x0.y);
            p[k + 1] = pack2_relu(x1.x, x1.y);
        }
        *reinterpret_cast<uint4*>(sm + dst + cm_off(t, 16 * q)) = make_uint4(p[0], p[1], p[2], p[3]);
        *reinterpret_cast<uint4*>(sm + dst + cm_off(t, 16 * q + 8)) = make_uint4(p[4], p[5], p[6], p[7]);
    }
}

// Issues the four K = 16 steps of one layer (one thread).
__device__ __forceinline__ void tc_layer(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr, uint32_t id) {
#pragma unroll
    for (uint32_t s = 0; s < 4; ++s) mma_bf16(d_tmem, sdesc(a_saddr + 256u * s), sdesc(b_saddr + 256u * s), id, s > 0);
}

// The network for this CTA's 128 rows (row t = this thread's point); y = raw outputs.
// Every thread returns the same value: false if a wait for the tensor cores ran out.
__device__ bool tc_forward(unsigned char* sm, uint32_t tmem, uint32_t t, float u, float v, float (&y)[3],
                           uint32_t* phase) {
    const uint32_t base = smem_u32(sm), mbar = base + Sm::mbar;
    const uint32_t lane_addr = tmem + (((t >> 5) * 32u) << 16);
    const float* bias = reinterpret_cast<const float*>(sm + Sm::bias);
    tc_features(sm, t, u, v);
    const uint32_t a0 = base + Sm::a0;
    const uint32_t srcB[3] = {base + Sm::w1, base + Sm::w2, base + Sm::w3};
    const uint32_t ids[3] = {idesc(128, 64), idesc(128, 64), idesc(128, 16)};
#pragma unroll
    for (int layer = 0; layer < 3; ++layer) {
        // the operand rows written by every thread become visible to the tensor cores
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (t == 0) {
            fence_after();
            tc_layer(tmem, a0, srcB[layer], ids[layer]);
            mma_commit(mbar);
        }
        const bool done = mbar_wait(mbar, *phase);
        *phase ^= 1u;
        if (__syncthreads_or(!done)) return false;
        fence_after();
        if (layer == 0) tc_hidden(sm, Sm::a0, lane_addr, bias, t);
        else if (layer == 1) tc_hidden(sm, Sm::a0, lane_addr, bias + 64, t);
        else {
            float o[4];
            tmem_ld4(lane_addr + 0u, o);
            y[0] = o[0] + bias[128];
            y[1] = o[1] + bias[129];
            y[2] = o[2] + bias[130];
        }
        fence_before();
    }
    return true;
}

__device__ __forceinline__ uint32_t tc_setup(unsigned char* sm) {
    const uint32_t base = smem_u32(sm);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(base + Sm::mbar));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(base + Sm::mbar_w));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + Sm::tmem),
                     "r"(TC_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    return *reinterpret_cast<volatile uint32_t*>(sm + Sm::tmem);
}

__device__ __forceinline__ void tc_teardown(uint32_t tmem) {
    fence_before();
    __syncthreads();
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS));
}

// Stand-alone network over n points (planar 3 x n output).
__global__ void __launch_bounds__(TC_ROWS) k_mlp_forward_tc(const float* __restrict__ theta, const float* __restrict__ u,
                                                            const float* __restrict__ v, uint32_t n, float* out,
                                                            int clamp, uint32_t* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t t = threadIdx.x;
    const uint32_t tmem = tc_setup(sm);
    tc_load_weights(sm, theta);
    uint32_t phase = 0;
    bool ok = true;
    const uint32_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    // each tile's (u, v) is loaded while the previous tile runs through the network
    uint32_t r = blockIdx.x * TC_ROWS + t;
    float uu = r < n ? u[r] : 0.0f, vv = r < n ? v[r] : 0.0f;
    for (uint32_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const uint32_t rn = r + gridDim.x * TC_ROWS;
        const float un = rn < n ? u[rn] : 0.0f, vn = rn < n ? v[rn] : 0.0f;
        float y[3];
        ok = tc_forward(sm, tmem, t, uu, vv, y, &phase);
        if (ok && r < n) {
#pragma unroll
            for (int k = 0; k < 3; ++k) out[(size_t)k * n + r] = clamp ? __saturatef(y[k]) : y[k];
        }
        r = rn;
        uu = un;
        vv = vn;
    }
    if (!ok) {
        // a wait for the tensor cores ran out: this CTA's remaining rows read NaN
        for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
            const uint32_t r = tile * TC_ROWS + t;
            if (r < n)
                for (int k = 0; k < 3; ++k) out[(size_t)k * n + r] = __int_as_float(0x7FC00000);
        }
        if (err && t == 0) atomicOr(err, ERR_TIMEOUT);
    }
    tc_teardown(tmem);
}

// In-pass inference: contiguous ranges of 128-point items (grouped points of a material
// whose cacheable node has a surrogate); the node's value goes into the points' probe
// records as a value computed this pass.
__global__ void __launch_bounds__(TC_ROWS) k_surrogate_tc(BatchArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t t = threadIdx.x;
    const uint32_t tmem = tc_setup(sm);
    const uint32_t n_items = a.ctl->n_surr_items;
    const uint32_t per = (n_items + gridDim.x - 1) / gridDim.x;
    const uint32_t i_end = min(n_items, (blockIdx.x + 1) * per);
    uint32_t loaded = 0xFFFFFFFFu, phase = 0, phase_w = 0;
    unsigned long long n_eval = 0;
    bool ok = true;
    // an item's material is the largest m with surr_item_base[m] <= item; the CTA's items are
    // consecutive, so the bisection runs only when an item passes the current material's end
    uint32_t m = 0, next_base = 0, ibase = 0, cnt = 0, s0 = 0, pre_item = 0xFFFFFFFFu;
    float uu = 0.0f, vv = 0.0f;
    size_t rbase = 0;   // the first probe record of the node's column in material m
    for (uint32_t item = blockIdx.x * per; item < i_end && ok; ++item) {
        if (item >= next_base) {
            uint32_t lo = 0, hi = a.n_mats;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (a.surr_item_base[mid] <= item) lo = mid;
                else hi = mid;
            }
            m = lo;
            ibase = a.surr_item_base[m];
            next_base = a.surr_item_base[m + 1];
            cnt = a.counts[m];
            s0 = a.seg_start[m];
            rbase = (size_t)a.probe_base[m] + (size_t)(uint32_t)a.surr_ord[m] * cnt;
        }
        if (m != loaded) {
            __syncthreads();   // the previous network's tile is finished everywhere
            if (a.surr_img) {
                if (!tc_copy_image(sm, a.surr_img + (size_t)a.surr_slot[m] * SURR_IMG_BYTES, &phase_w)) {
                    ok = false;
                    break;
                }
            } else {
                tc_load_weights(sm, a.surr_theta + (size_t)a.surr_slot[m] * MLP_PARAMS);
            }
            loaded = m;
        }
        const uint32_t j = (item - ibase) * TC_ROWS + t;
        // this item's (u, v) were loaded during the previous item if it had the same material
        if (item != pre_item) {
            uu = j < cnt ? a.su[s0 + j] : 0.0f;
            vv = j < cnt ? a.sv[s0 + j] : 0.0f;
        }
        const uint32_t jn = j + TC_ROWS;
        const bool pre = item + 1 < i_end && item + 1 < next_base;
        const float un = (pre && jn < cnt) ? a.su[s0 + jn] : 0.0f, vn = (pre && jn < cnt) ? a.sv[s0 + jn] : 0.0f;
        pre_item = pre ? item + 1 : 0xFFFFFFFFu;
        float y[3];
        ok = tc_forward(sm, tmem, t, uu, vv, y, &phase);
        if (ok && j < cnt) {
            const size_t rec = rbase + j;
            a.probes[rec] = make_float4(__saturatef(y[0]), __saturatef(y[1]), __saturatef(y[2]), __uint_as_float(3u));
            n_eval++;
        }
        uu = un;
        vv = vn;
    }
    if (!ok && t == 0) atomicOr(&a.ctl->err, ERR_TIMEOUT);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_eval += __shfl_xor_sync(0xFFFFFFFFu, n_eval, o);
    if ((t & 31u) == 0 && n_eval) atomicAdd(&a.stats[ST_SURR], n_eval);
    tc_teardown(tmem);
}


// =======================================================================================
// Training on the tensor cores.  A CTA of 128 threads takes minibatches of 128 rows of one
// network; thread t owns row t of every activation and lane t of tensor memory.
//   forward:   Z1 = G W1, H1 = relu(Z1 + b1); Z2 = H1 W2, H2 = relu(Z2 + b2); Y = H2 W3 + b3
//   backward:  dY = s (Y - T); dZ2 = (dY W3^T) . [H2 > 0]; dZ1 = (dZ2 W2^T) . [H1 > 0]
//   gradients: dW1 = G^T dZ1 and dW2 = H1^T dZ2 as one M = 128, N = 128 product
//              [G^T; H1^T] [dZ1^T; dZ2^T]^T (its two diagonal blocks), dW3 = H2^T dY from
//              [H1^T; H2^T] dY (its lower half); biases: column sums of dZ1, dZ2, dY
// Every product takes BF16 operands from shared memory and accumulates in FP32 in tensor
// memory; the batch-dimension products read transposed copies the epilogues write.  Then
// FP32 Adam on the master weights.
// =======================================================================================
constexpr uint32_t TR_COLS = 256;               // tensor-memory columns of the training kernel

struct St {                                     // byte offsets into dynamic shared memory
    static constexpr uint32_t a0 = 0;           // [128][64] features, then H2 (A of layers 1, 3)
    static constexpr uint32_t a1 = 16384;       // [128][64] H1 (A of layer 2)
    static constexpr uint32_t dz2 = 32768;      // [128][64] dZ2 (A of dH1 = dZ2 W2^T)
    static constexpr uint32_t dy = 49152;       // [128][16] dY, columns >= 3 zero (A of dH2)
    static constexpr uint32_t gT = 53248;       // [64][128] G^T   \ gT, h1T: one 128-row operand
    static constexpr uint32_t h1T = 69632;      // [64][128] H1^T  / h1T, h2T: another
    static constexpr uint32_t h2T = 86016;      // [64][128] H2^T
    static constexpr uint32_t dz1T = 102400;    // [64][128] dZ1^T \ one 128-row operand
    static constexpr uint32_t dz2T = 118784;    // [64][128] dZ2^T /
    static constexpr uint32_t dyT = 135168;     // [16][128] dY^T, rows >= 3 zero
    static constexpr uint32_t w1t = 139264;     // [64][64] W1^T (B of layer 1)
    static constexpr uint32_t w2t = 147456;     // [64][64] W2^T (B of layer 2)
    static constexpr uint32_t w3t = 155648;     // [16][64] W3^T, rows >= 3 zero (B of layer 3)
    static constexpr uint32_t w2n = 157696;     // [64][64] W2 (B of dH1)
    static constexpr uint32_t w3n = 165888;     // [64][16] W3, columns >= 3 zero (B of dH2)
    static constexpr uint32_t bias = 167936;    // b1[64], b2[64], b3[4] FP32
    static constexpr uint32_t mbar = 168464;    // 8-byte mbarrier
    static constexpr uint32_t tmem = 168472;    // tensor-memory base written by tcgen05.alloc
    // one step's gradient, FP32: rows of W1 and of W2 at a stride of GROW floats (a padded
    // stride spreads the rows written by the 32 lanes of a warp over the banks), then W3, b1,
    // b2, b3 in parameter order
    static constexpr uint32_t GROW = 68;
    static constexpr uint32_t gw1 = 168960;
    static constexpr uint32_t gw2 = gw1 + 64 * GROW * 4;
    static constexpr uint32_t grest = gw2 + 64 * GROW * 4;   // W3 (192), b1 (64), b2 (64), b3 (3)
    static constexpr uint32_t end = grest + 324 * 4;
};
static_assert(St::end <= 227 * 1024, "shared memory of the training kernel");

struct TcTrainArgs {
    float* theta;            // n_mats x MLP_PARAMS FP32 masters
    float* adam_m;
    float* adam_v;
    float* grad;             // gradient mode: accumulated gradient
    const float* data;       // per material: n_data rows of (u, v, r, g, b)
    float* loss;             // per material: summed squared error of the steps run
    uint32_t* err;           // ERR_TIMEOUT if a wait for the tensor cores ran out (may be null)
    uint32_t n_data;
    uint32_t steps;
    uint64_t sample0;
    uint32_t step0;
    uint32_t total_steps;
    float lr;
    float grad_scale;        // dL/dy = grad_scale (y - t)
    int mode;                // 0: Adam steps, 1: accumulate the gradient only
};

__device__ __forceinline__ void put_bf16(unsigned char* sm, uint32_t off, float x) {
    *reinterpret_cast<__nv_bfloat16*>(sm + off) = __float2bfloat16_rn(x);
}

// The network's parameters as BF16 operands (both orientations where the backward pass
// needs them) and FP32 biases.
__device__ void tr_load_weights(unsigned char* sm, const float* __restrict__ th) {
    for (uint32_t i = threadIdx.x; i < 64u * 64u; i += blockDim.x) {
        const uint32_t in = i >> 6, out = i & 63u;
        put_bf16(sm, St::w1t + cm_off(out, in), th[P_W1 + i]);
        const float w2 = th[P_W2 + i];
        put_bf16(sm, St::w2t + cm_off(out, in), w2);
        put_bf16(sm, St::w2n + cm_off(in, out), w2);
    }
    for (uint32_t i = threadIdx.x; i < 16u * 64u; i += blockDim.x) {
        const uint32_t out = i >> 6, in = i & 63u;
        const float w = out < 3 ? th[P_W3 + in * 3 + out] : 0.0f;
        put_bf16(sm, St::w3t + cm_off_k(out, in, 64), w);
        put_bf16(sm, St::w3n + cm_off_k(in, out, 16), w);
    }
    float* bias = reinterpret_cast<float*>(sm + St::bias);
    for (uint32_t i = threadIdx.x; i < 132u; i += blockDim.x)
        bias[i] = i < 64 ? th[P_B1 + i] : (i < 128 ? th[P_B2 + i - 64] : (i < 131 ? th[P_B3 + i - 128] : 0.0f));
}

// Makes the operand rows written by every thread visible to the tensor cores, issues
// `k16` K = 16 steps of one product from thread 0 and waits for it.  False if the wait
// ran out (every thread gets the same answer).
__device__ __forceinline__ bool tr_mma(uint32_t mbar, uint32_t* phase, uint32_t d, uint32_t a, uint32_t ka,
                                       uint32_t b, uint32_t kb, uint32_t id, uint32_t k16) {
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_after();
        for (uint32_t s = 0; s < k16; ++s) mma_bf16(d, sdesc_k(a + 256u * s, ka), sdesc_k(b + 256u * s, kb), id, s > 0);
        mma_commit(mbar);
    }
    const bool done = mbar_wait(mbar, *phase);
    *phase ^= 1u;
    const bool ok = !__syncthreads_or(!done);
    fence_after();
    return ok;
}

// relu(acc + bias) of 64 accumulator columns: row t of a [128][64] operand, column t of a
// [64][128] transposed one, and the relu'(h) > 0 mask of the BF16 values.
__device__ __forceinline__ uint64_t tr_hidden(unsigned char* sm, uint32_t dst, uint32_t dstT, uint32_t taddr,
                                              const float* bias, uint32_t t) {
    uint64_t mask = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float v[16];
        tmem_ld16(taddr + 16u * q, v);
        uint32_t p[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            p[k] = pack2(fmaxf(v[2 * k] + bias[16 * q + 2 * k], 0.0f), fmaxf(v[2 * k + 1] + bias[16 * q + 2 * k + 1], 0.0f));
            const uint32_t c = 16 * q + 2 * k;
            *reinterpret_cast<uint16_t*>(sm + dstT + cm_off_k(c, t, 128)) = (uint16_t)(p[k] & 0xFFFFu);
            *reinterpret_cast<uint16_t*>(sm + dstT + cm_off_k(c + 1, t, 128)) = (uint16_t)(p[k] >> 16);
            mask |= (uint64_t)((p[k] & 0x7FFFu) != 0 && !(p[k] & 0x8000u)) << c;
            mask |= (uint64_t)(((p[k] >> 16) & 0x7FFFu) != 0 && !(p[k] & 0x80000000u)) << (c + 1);
        }
        *reinterpret_cast<uint4*>(sm + dst + cm_off(t, 16 * q)) = make_uint4(p[0], p[1], p[2], p[3]);
        *reinterpret_cast<uint4*>(sm + dst + cm_off(t, 16 * q + 8)) = make_uint4(p[4], p[5], p[6], p[7]);
    }
    return mask;
}

// acc . mask of 64 accumulator columns as BF16: row t of a [128][64] operand (dst != ~0u)
// and column t of a [64][128] transposed one.
__device__ __forceinline__ void tr_masked(unsigned char* sm, uint32_t dst, uint32_t dstT, uint32_t taddr, uint64_t mask,
                                          uint32_t t) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float v[16];
        tmem_ld16(taddr + 16u * q, v);
        uint32_t p[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t c = 16 * q + 2 * k;
            p[k] = pack2(((mask >> c) & 1u) ? v[2 * k] : 0.0f, ((mask >> (c + 1)) & 1u) ? v[2 * k + 1] : 0.0f);
            *reinterpret_cast<uint16_t*>(sm + dstT + cm_off_k(c, t, 128)) = (uint16_t)(p[k] & 0xFFFFu);
            *reinterpret_cast<uint16_t*>(sm + dstT + cm_off_k(c + 1, t, 128)) = (uint16_t)(p[k] >> 16);
        }
        if (dst != ~0u) {
            *reinterpret_cast<uint4*>(sm + dst + cm_off(t, 16 * q)) = make_uint4(p[0], p[1], p[2], p[3]);
            *reinterpret_cast<uint4*>(sm + dst + cm_off(t, 16 * q + 8)) = make_uint4(p[4], p[5], p[6], p[7]);
        }
    }
}

// Sum of row r of a [rows][128] BF16 operand (a bias gradient: a column sum over the batch).
__device__ __forceinline__ float tr_row_sum(const unsigned char* sm, uint32_t base, uint32_t r) {
    float s = 0.0f;
#pragma unroll 4
    for (uint32_t c = 0; c < 128; c += 8) {
        const uint4 w = *reinterpret_cast<const uint4*>(sm + base + cm_off_k(r, c, 128));
        const uint32_t x[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) s += __uint_as_float(x[k] << 16) + __uint_as_float(x[k] & 0xFFFF0000u);
    }
    return s;
}

// One CTA per (split, material) runs `steps` minibatch steps of 128 rows.
__global__ void __launch_bounds__(TC_ROWS) k_mlp_train_tc(TcTrainArgs A) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t t = threadIdx.x;
    const uint32_t base = smem_u32(sm), mbar = base + St::mbar;
    const uint32_t mat = blockIdx.y;
    const size_t pbase = (size_t)mat * MLP_PARAMS;
    const float* data = A.data + (size_t)mat * A.n_data * 5;
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (t < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + St::tmem),
                     "r"(TR_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // the zero columns of dY and zero rows of dY^T stay zero: only outputs 0..2 are written
    for (uint32_t i = t; i < 128u * 16u; i += TC_ROWS) {
        *reinterpret_cast<uint16_t*>(sm + St::dy + cm_off_k(i >> 4, i & 15u, 16)) = 0;
        *reinterpret_cast<uint16_t*>(sm + St::dyT + cm_off_k(i & 15u, i >> 4, 128)) = 0;
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + St::tmem);
    const uint32_t lane_addr = tmem + (((t >> 5) * 32u) << 16);
    const float* bias = reinterpret_cast<const float*>(sm + St::bias);
    const uint32_t log2n = 31 - __clz(A.n_data);
    uint32_t phase = 0;
    float loss = 0.0f;
    bool ok = true;
    tr_load_weights(sm, A.theta + pbase);   // later steps update the operands in place
    __syncthreads();
    for (uint32_t s = 0; s < A.steps && ok; ++s) {
        const uint32_t step = s * gridDim.x + blockIdx.x;
        // ---- row t of the minibatch: in order (gradient mode) or a fixed per-epoch shuffle
        const uint64_t k = A.sample0 + (uint64_t)step * TC_ROWS + t;
        uint32_t row;
        if (A.mode == 1) {
            row = (uint32_t)k;
        } else {
            const uint32_t epoch = (uint32_t)(k >> log2n);
            row = (uint32_t)(k * 2654435761ull + (uint64_t)epoch * 0x9E3779B9ull) & (A.n_data - 1);
        }
        const float* d = data + (size_t)row * 5;
        const float u = d[0], v = d[1], tg0 = d[2], tg1 = d[3], tg2 = d[4];
        // ---- features: row t of G, column t of G^T
        tc_features(sm, t, u, v);
        for (uint32_t c = 0; c < 64; c += 8) {
            const uint4 w = *reinterpret_cast<const uint4*>(sm + St::a0 + cm_off(t, c));
            const uint32_t x[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                *reinterpret_cast<uint16_t*>(sm + St::gT + cm_off_k(c + 2 * q, t, 128)) = (uint16_t)(x[q] & 0xFFFFu);
                *reinterpret_cast<uint16_t*>(sm + St::gT + cm_off_k(c + 2 * q + 1, t, 128)) = (uint16_t)(x[q] >> 16);
            }
        }
        // ---- forward
        ok = tr_mma(mbar, &phase, tmem + 0u, base + St::a0, 64, base + St::w1t, 64, idesc(128, 64), 4);
        if (!ok) break;
        const uint64_t mask1 = tr_hidden(sm, St::a1, St::h1T, lane_addr + 0u, bias, t);
        fence_before();
        ok = tr_mma(mbar, &phase, tmem + 64u, base + St::a1, 64, base + St::w2t, 64, idesc(128, 64), 4);
        if (!ok) break;
        const uint64_t mask2 = tr_hidden(sm, St::a0, St::h2T, lane_addr + 64u, bias + 64, t);
        fence_before();
        ok = tr_mma(mbar, &phase, tmem + 128u, base + St::a0, 64, base + St::w3t, 64, idesc(128, 16), 4);
        if (!ok) break;
        // ---- dL/dy and the loss
        {
            float o[4];
            tmem_ld4(lane_addr + 128u, o);
            const float e[3] = {o[0] + bias[128] - tg0, o[1] + bias[129] - tg1, o[2] + bias[130] - tg2};
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                loss += e[q] * e[q];
                const float g = A.grad_scale * e[q];
                put_bf16(sm, St::dy + cm_off_k(t, q, 16), g);
                put_bf16(sm, St::dyT + cm_off_k(q, t, 128), g);
            }
        }
        fence_before();
        // ---- dH2 = dY W3^T, masked
        ok = tr_mma(mbar, &phase, tmem + 0u, base + St::dy, 16, base + St::w3n, 16, idesc(128, 64), 1);
        if (!ok) break;
        tr_masked(sm, St::dz2, St::dz2T, lane_addr + 0u, mask2, t);
        fence_before();
        // ---- dH1 = dZ2 W2^T, masked
        ok = tr_mma(mbar, &phase, tmem + 64u, base + St::dz2, 64, base + St::w2n, 64, idesc(128, 64), 4);
        if (!ok) break;
        tr_masked(sm, ~0u, St::dz1T, lane_addr + 64u, mask1, t);
        fence_before();
        // ---- weight gradients: [G^T; H1^T] x [dZ1^T; dZ2^T]^T and [H1^T; H2^T] x dY
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (t == 0) {
            fence_after();
            for (uint32_t q = 0; q < 8; ++q)
                mma_bf16(tmem + 0u, sdesc_k(base + St::gT + 256u * q, 128), sdesc_k(base + St::dz1T + 256u * q, 128),
                         idesc(128, 128), q > 0);
            for (uint32_t q = 0; q < 8; ++q)
                mma_bf16(tmem + 128u, sdesc_k(base + St::h1T + 256u * q, 128), sdesc_k(base + St::dyT + 256u * q, 128),
                         idesc(128, 16), q > 0);
            mma_commit(mbar);
        }
        // bias gradients while the tensor cores run: column sums of dZ1, dZ2 and dY
        const float gb = t < 64 ? tr_row_sum(sm, St::dz1T, t) : tr_row_sum(sm, St::dz2T, t - 64);
        const float gb3 = t < 3 ? tr_row_sum(sm, St::dyT, t) : 0.0f;
        const bool done = mbar_wait(mbar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!done)) {
            ok = false;
            break;
        }
        fence_after();
        // ---- the step's gradient into shared memory: thread t < 64 holds row t of dW1 (tensor-
        // memory lane t, columns 0..63), thread t >= 64 row t - 64 of dW2 (columns 64..127)
        // and of dW3 (columns 128..130)
        float* gw1 = reinterpret_cast<float*>(sm + St::gw1);
        float* gw2 = reinterpret_cast<float*>(sm + St::gw2);
        float* grest = reinterpret_cast<float*>(sm + St::grest);
        {
            float* row = t < 64 ? gw1 + t * St::GROW : gw2 + (t - 64) * St::GROW;
            const uint32_t col0 = t < 64 ? 0u : 64u;
#pragma unroll
            for (uint32_t q = 0; q < 4; ++q) {
                float g[16];
                tmem_ld16(lane_addr + col0 + 16u * q, g);
#pragma unroll
                for (int k = 0; k < 16; k += 4)
                    *reinterpret_cast<float4*>(row + 16 * q + k) = make_float4(g[k], g[k + 1], g[k + 2], g[k + 3]);
            }
            if (t >= 64) {
                float g3[4];
                tmem_ld4(lane_addr + 128u, g3);
                for (uint32_t o = 0; o < 3; ++o) grest[(t - 64) * 3 + o] = g3[o];
            }
            grest[192 + t] = gb;                  // b1 (t < 64), then b2
            if (t < 3) grest[320 + t] = gb3;
        }
        fence_before();
        __syncthreads();
        // ---- Adam (or gradient accumulation) over the parameters in order, coalesced; the
        // updated weights go straight into the BF16 operands of the next step
        const uint32_t adam_t = A.step0 + step + 1;
        const float frac = A.total_steps > 1 ? (float)(A.step0 + step) / (float)(A.total_steps - 1) : 0.0f;
        const float lr_t = A.lr * (0.05f + 0.95f * 0.5f * (1.0f + cospif(fminf(frac, 1.0f))));
        const float bc1 = 1.0f - powf(0.9f, (float)adam_t), bc2 = 1.0f - powf(0.999f, (float)adam_t);
        float* bias_w = reinterpret_cast<float*>(sm + St::bias);
#pragma unroll 4
        for (uint32_t i = t; i < MLP_PARAMS; i += TC_ROWS) {
            float g;
            if (i < (uint32_t)P_B1) g = gw1[(i >> 6) * St::GROW + (i & 63u)];
            else if (i < (uint32_t)P_W2) g = grest[192 + (i - P_B1)];
            else if (i < (uint32_t)P_B2) g = gw2[((i - P_W2) >> 6) * St::GROW + ((i - P_W2) & 63u)];
            else if (i < (uint32_t)P_W3) g = grest[256 + (i - P_B2)];
            else if (i < (uint32_t)P_B3) g = grest[i - P_W3];
            else g = grest[320 + (i - P_B3)];
            const size_t k = pbase + i;
            if (A.mode == 1) {
                atomicAdd(&A.grad[k], g);
                continue;
            }
            const float m1 = 0.9f * A.adam_m[k] + 0.1f * g;
            const float m2 = 0.999f * A.adam_v[k] + 0.001f * g * g;
            A.adam_m[k] = m1;
            A.adam_v[k] = m2;
            const float w = A.theta[k] - lr_t * (m1 / bc1) / (sqrtf(m2 / bc2) + 1e-8f);
            A.theta[k] = w;
            if (i < (uint32_t)P_B1) {
                put_bf16(sm, St::w1t + cm_off(i & 63u, i >> 6), w);
            } else if (i < (uint32_t)P_W2) {
                bias_w[i - P_B1] = w;
            } else if (i < (uint32_t)P_B2) {
                const uint32_t j = i - P_W2, in = j >> 6, out = j & 63u;
                put_bf16(sm, St::w2t + cm_off(out, in), w);
                put_bf16(sm, St::w2n + cm_off(in, out), w);
            } else if (i < (uint32_t)P_W3) {
                bias_w[64 + (i - P_B2)] = w;
            } else if (i < (uint32_t)P_B3) {
                const uint32_t j = i - P_W3, in = j / 3u, out = j % 3u;
                put_bf16(sm, St::w3t + cm_off_k(out, in, 64), w);
                put_bf16(sm, St::w3n + cm_off_k(in, out, 16), w);
            } else {
                bias_w[128 + (i - P_B3)] = w;
            }
        }
        fence_before();
        __syncthreads();   // the next step reads the updated operands
    }
    if (!ok) {
        if (t == 0) {
            if (A.err) atomicOr(A.err, ERR_TIMEOUT);
            atomicExch(&A.loss[mat], __int_as_float(0x7FC00000));
        }
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xFFFFFFFFu, loss, o);
        if ((t & 31u) == 0) atomicAdd(&A.loss[mat], loss);
    }
    fence_before();
    __syncthreads();
    if (t < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TR_COLS));
}

}  // namespace

cudaError_t launch_mlp_train(float* theta, float* adam_m, float* adam_v, float* grad, const float* data, float* loss,
                             uint32_t* err, uint32_t n_mats, uint32_t n_data, uint32_t steps, uint64_t sample0,
                             uint32_t step0, uint32_t total_steps, float lr, float grad_scale, int mode, uint32_t splits,
                             cudaStream_t s) {
    TcTrainArgs A{theta, adam_m, adam_v, grad, data, loss, err, n_data, steps, sample0, step0, total_steps, lr,
                  grad_scale, mode};
    cudaError_t e = cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)St::end);
    if (e != cudaSuccess) return e;
    k_mlp_train_tc<<<dim3(splits, n_mats), TC_ROWS, St::end, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_surrogate(const BatchArgs& a, int num_sms, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_surrogate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::end);
    if (e != cudaSuccess) return e;
    // six CTAs per SM: their tensor-memory allocations (6 x 64 columns) fit the SM's 512
    k_surrogate_tc<<<num_sms * TC_CTAS_PER_SM, TC_ROWS, Sm::end, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_surrogate_images(const float* theta, uint32_t n_slots, unsigned char* img, cudaStream_t s) {
    if (n_slots == 0) return cudaSuccess;
    k_surr_images<<<n_slots, TC_ROWS, 0, s>>>(theta, img);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward_tc(const float* theta, const float* u, const float* v, uint32_t n, float* out, int clamp,
                                  uint32_t* err, int num_sms, cudaStream_t s) {
    const uint32_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    const uint32_t full = (uint32_t)num_sms * TC_CTAS_PER_SM;
    uint32_t blocks = tiles < full ? tiles : full;
    if (blocks == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::end);
    if (e != cudaSuccess) return e;
    k_mlp_forward_tc<<<blocks, TC_ROWS, Sm::end, s>>>(theta, u, v, n, out, clamp, err);
    return cudaGetLastError();
}

}  // namespace pmc
