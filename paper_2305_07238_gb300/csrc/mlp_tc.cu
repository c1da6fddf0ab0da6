// mlp_tc.cu -- inference of the learned surrogate on the 5th-generation tensor cores:
// tcgen05.mma (kind::f16, BF16 operands from shared memory, FP32 accumulators in tensor
// memory), completion tracked by an mbarrier, accumulators read back with tcgen05.ld.
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
constexpr uint32_t TC_COLS = 128;               // tensor-memory columns: D1 at 0, D2 at 64, D3 at 0
constexpr uint32_t WAIT_POLLS = 1u << 22;       // bound of every mbarrier wait

struct Sm {                                     // byte offsets into dynamic shared memory
    static constexpr uint32_t a0 = 0;           // 128 x 64 BF16: features, then layer-2 output
    static constexpr uint32_t a1 = 16384;       // 128 x 64 BF16: layer-1 output
    static constexpr uint32_t w1 = 32768;       // 64 x 64 BF16: W1 transposed (n rows, k columns)
    static constexpr uint32_t w2 = 40960;       // 64 x 64 BF16: W2 transposed
    static constexpr uint32_t w3 = 49152;       // 16 x 64 BF16: W3 transposed, rows 3..15 zero
    static constexpr uint32_t bias = 51200;     // b1[64], b2[64], b3[4] FP32
    static constexpr uint32_t mbar = 51744;     // 8-byte mbarrier
    static constexpr uint32_t tmem = 51752;     // tensor-memory base written by tcgen05.alloc
    static constexpr uint32_t end = 51760;
};

// Byte offset of element (r, c) of a 64-column operand in the core-matrix layout.
__device__ __forceinline__ uint32_t cm_off(uint32_t r, uint32_t c) {
    return (r >> 3) * 1024u + (c >> 3) * 128u + (r & 7u) * 16u + (c & 7u) * 2u;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading byte offset 128, stride byte
// offset 1024, the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
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
__device__ void tc_load_weights(unsigned char* sm, const float* __restrict__ th) {
    for (uint32_t i = threadIdx.x; i < 64u * 64u; i += blockDim.x) {
        const uint32_t in = i >> 6, out = i & 63u;
        *reinterpret_cast<__nv_bfloat16*>(sm + Sm::w1 + cm_off(out, in)) = __float2bfloat16_rn(th[P_W1 + i]);
        *reinterpret_cast<__nv_bfloat16*>(sm + Sm::w2 + cm_off(out, in)) = __float2bfloat16_rn(th[P_W2 + i]);
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

// Row t of the feature matrix: [sin pi k u, cos pi k u, sin pi k v, cos pi k v], k = 1..16.
__device__ __forceinline__ void tc_features(unsigned char* sm, uint32_t t, float u, float v) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const float x = half ? v : u;
        float s[16], c[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) sincospif((float)(k + 1) * x, &s[k], &c[k]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const uint4 ws = make_uint4(pack2(s[8 * q], s[8 * q + 1]), pack2(s[8 * q + 2], s[8 * q + 3]),
                                        pack2(s[8 * q + 4], s[8 * q + 5]), pack2(s[8 * q + 6], s[8 * q + 7]));
            const uint4 wc = make_uint4(pack2(c[8 * q], c[8 * q + 1]), pack2(c[8 * q + 2], c[8 * q + 3]),
                                        pack2(c[8 * q + 4], c[8 * q + 5]), pack2(c[8 * q + 6], c[8 * q + 7]));
            *reinterpret_cast<uint4*>(sm + Sm::a0 + cm_off(t, 32 * half + 8 * q)) = ws;
            *reinterpret_cast<uint4*>(sm + Sm::a0 + cm_off(t, 32 * half + 16 + 8 * q)) = wc;
        }
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
        for (int k = 0; k < 8; ++k)
            p[k] = pack2(fmaxf(v[2 * k] + bias[16 * q + 2 * k], 0.0f), fmaxf(v[2 * k + 1] + bias[16 * q + 2 * k + 1], 0.0f));
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
    const uint32_t a0 = base + Sm::a0, a1 = base + Sm::a1;
    const uint32_t srcA[3] = {a0, a1, a0};
    const uint32_t srcB[3] = {base + Sm::w1, base + Sm::w2, base + Sm::w3};
    const uint32_t dcol[3] = {0u, 64u, 0u};
    const uint32_t ids[3] = {idesc(128, 64), idesc(128, 64), idesc(128, 16)};
#pragma unroll
    for (int layer = 0; layer < 3; ++layer) {
        // the operand rows written by every thread become visible to the tensor cores
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (t == 0) {
            fence_after();
            tc_layer(tmem + dcol[layer], srcA[layer], srcB[layer], ids[layer]);
            mma_commit(mbar);
        }
        const bool done = mbar_wait(mbar, *phase);
        *phase ^= 1u;
        if (__syncthreads_or(!done)) return false;
        fence_after();
        if (layer == 0) tc_hidden(sm, Sm::a1, lane_addr + 0u, bias, t);
        else if (layer == 1) tc_hidden(sm, Sm::a0, lane_addr + 64u, bias + 64, t);
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
    for (uint32_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const uint32_t r = tile * TC_ROWS + t;
        const float uu = r < n ? u[r] : 0.0f, vv = r < n ? v[r] : 0.0f;
        float y[3];
        ok = tc_forward(sm, tmem, t, uu, vv, y, &phase);
        if (ok && r < n) {
#pragma unroll
            for (int k = 0; k < 3; ++k) out[(size_t)k * n + r] = clamp ? __saturatef(y[k]) : y[k];
        }
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
    uint32_t loaded = 0xFFFFFFFFu, phase = 0;
    unsigned long long n_eval = 0;
    bool ok = true;
    for (uint32_t item = blockIdx.x * per; item < i_end && ok; ++item) {
        uint32_t lo = 0, hi = a.n_mats;   // largest m with surr_item_base[m] <= item
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.surr_item_base[mid] <= item) lo = mid;
            else hi = mid;
        }
        const uint32_t m = lo;
        if (m != loaded) {
            __syncthreads();   // the previous network's tile is finished everywhere
            tc_load_weights(sm, a.surr_theta + (size_t)a.surr_slot[m] * MLP_PARAMS);
            loaded = m;
        }
        const uint32_t cnt = a.counts[m], r = (uint32_t)a.surr_ord[m];
        const uint32_t j = (item - a.surr_item_base[m]) * TC_ROWS + t;
        const uint32_t s0 = a.seg_start[m];
        const float uu = j < cnt ? a.su[s0 + j] : 0.0f, vv = j < cnt ? a.sv[s0 + j] : 0.0f;
        float y[3];
        ok = tc_forward(sm, tmem, t, uu, vv, y, &phase);
        if (ok && j < cnt) {
            const size_t rec = (size_t)a.probe_base[m] + (size_t)r * cnt + j;
            a.probes[rec] = make_float4(__saturatef(y[0]), __saturatef(y[1]), __saturatef(y[2]), __uint_as_float(3u));
            n_eval++;
        }
    }
    if (!ok && t == 0) atomicOr(&a.ctl->err, ERR_TIMEOUT);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_eval += __shfl_xor_sync(0xFFFFFFFFu, n_eval, o);
    if ((t & 31u) == 0 && n_eval) atomicAdd(&a.stats[ST_SURR], n_eval);
    tc_teardown(tmem);
}

}  // namespace

cudaError_t launch_surrogate(const BatchArgs& a, int num_sms, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_surrogate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::end);
    if (e != cudaSuccess) return e;
    // four CTAs per SM: their tensor-memory allocations (4 x 128 columns) fit the SM's 512
    k_surrogate_tc<<<num_sms * 4, TC_ROWS, Sm::end, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward_tc(const float* theta, const float* u, const float* v, uint32_t n, float* out, int clamp,
                                  uint32_t* err, int num_sms, cudaStream_t s) {
    const uint32_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    uint32_t blocks = tiles < (uint32_t)num_sms * 4u ? tiles : (uint32_t)num_sms * 4u;
    if (blocks == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sm::end);
    if (e != cudaSuccess) return e;
    k_mlp_forward_tc<<<blocks, TC_ROWS, Sm::end, s>>>(theta, u, v, n, out, clamp, err);
    return cudaGetLastError();
}

}  // namespace pmc
