// mlp.cu -- training data of the learned surrogate of a cacheable node: the node's
// standalone program run by the exact FP32 evaluator at (u, v) drawn from SplitMix64.  The
// network itself (inference and training on the tcgen05 tensor cores) is in mlp_tc.cu.
#include <cstdint>

#include "nodes.cuh"
#include "pmc_internal.h"

namespace pmc {

namespace {

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
    char* Vb = reinterpret_cast<char*>(s_val + (size_t)warp * max_slots * 96u + lane);
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
            if (row < n_rows) exec_node(op, ins, Vb, pt, params, s_grad);
        }
        if (row < n_rows) {
            float* d = data + ((size_t)mi * n_rows + row) * 5;
            d[0] = pt.u;
            d[1] = pt.v;
            d[2] = slot_ch(Vb, ri.out_slot * SLOT_BYTES, 0);
            d[3] = slot_ch(Vb, ri.out_slot * SLOT_BYTES, 1);
            d[4] = slot_ch(Vb, ri.out_slot * SLOT_BYTES, 2);
        }
    }
}

}  // namespace

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
