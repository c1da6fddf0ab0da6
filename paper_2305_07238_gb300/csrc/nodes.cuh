// nodes.cuh -- device code shared by the pass kernels and the surrogate kernels:
// descriptors and hashes (Sec. 3.1, Eq. 1, Alg. 1), the FP32 node primitives and one
// interpreter step of a compiled material program (Sec. 2).
#pragma once

#include <cstdint>

#include "pmc_internal.h"

namespace pmc {

// =======================================================================================
// Descriptor and hashes (Sec. 3.1, Eq. 1, Alg. 1)
// =======================================================================================
__device__ __forceinline__ uint32_t d_fmix32(uint32_t h) {
    // MurmurHash3 32-bit finaliser (Appleby)
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ uint64_t d_fmix64(uint64_t k) {
    // MurmurHash3 64-bit finaliser (Appleby)
    k ^= k >> 33;
    k *= 0xFF51AFD7ED558CCDull;
    k ^= k >> 33;
    k *= 0xC4CEB9FE1A85EC53ull;
    k ^= k >> 33;
    return k;
}

__device__ __forceinline__ uint64_t d_splitmix(uint64_t z) {
    // SplitMix64 output function (Steele, Lea & Flood 2014)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Texel index on a virtual texture of 2^level texels per axis.  u * 2^level is exact in
// FP32, so the index is the same as in any wider precision.  fmaxf maps NaN to 0.
__device__ __forceinline__ uint32_t d_texel(float u, uint32_t level) {
    float x = fminf(fmaxf(u, 0.0f), 1.0f);
    uint32_t res = 1u << level;
    uint32_t t = (uint32_t)floorf(x * (float)res);
    return min(t, res - 1u);
}

// Mip level of the virtual texture from the ray-cone footprint (Sec. 3.1, Eq. 1):
// floor(-log2(min(|g1|, |g2|))) + offset, clamped to [0, 13].  The squared norms are formed
// in FP32 with every product and the sum rounded to nearest (no fused multiply-add), and
// the floor is read off the exponent E and fraction f of the smaller one, s = (1 + f) 2^E:
// -log2(sqrt(s)) = -(E + log2(1 + f)) / 2, whose floor is -ceil(E / 2) when f = 0 and
// -floor(E / 2) - 1 otherwise.  A zero or subnormal s (level 63 or more) gives 13 for any
// offset of at least -13; an infinite or NaN one gives 0.
__device__ __forceinline__ uint32_t d_level(float g1u, float g1v, float g2u, float g2v, int32_t offset) {
    const float s1 = __fadd_rn(__fmul_rn(g1u, g1u), __fmul_rn(g1v, g1v));
    const float s2 = __fadd_rn(__fmul_rn(g2u, g2u), __fmul_rn(g2v, g2v));
    if (s1 != s1 || s2 != s2) return 0u;
    const uint32_t b = __float_as_uint(fminf(s1, s2));
    const int be = (int)(b >> 23);   // s >= 0: the sign bit is clear
    if (be == 0) return 13u;
    if (be == 255) return 0u;
    const int E = be - 127;
    const int L = (b & 0x7FFFFFu) ? -((E + 2) >> 1) : -((E + 1) >> 1);
    return (uint32_t)min(13, max(0, L + offset));
}

__device__ __forceinline__ uint64_t d_key(uint32_t mat, uint32_t node, uint32_t level,
                                          uint32_t iu, uint32_t iv) {
    return ((uint64_t)mat << 48) | ((uint64_t)node << 32) | ((uint64_t)level << 26) |
           ((uint64_t)iu << 13) | (uint64_t)iv;
}

// Voxel of one position coordinate on a grid of 2^-level world units: floor(p 2^level)
// clamped to [-512, 511] and offset to [0, 1023]; p 2^level is exact in FP32 (a power-of-two
// scale), so the index is the same in any wider precision; NaN takes the lowest voxel.
__device__ __forceinline__ uint32_t d_voxel(float p, uint32_t level) {
    float x = p * __int_as_float((int)(127u + level) << 23);
    if (!(x >= -512.0f)) x = -512.0f;
    if (x > 511.0f) x = 511.0f;
    return (uint32_t)((int)floorf(x) + 512);
}

// World-position descriptor: (material, node, voxel of the position); bit 31 set.
__device__ __forceinline__ uint64_t d_key_pos(uint32_t mat, uint32_t node, uint32_t level, float px, float py,
                                              float pz) {
    return ((uint64_t)mat << 48) | ((uint64_t)node << 32) | (1ull << 31) | ((uint64_t)d_voxel(px, level) << 20) |
           ((uint64_t)d_voxel(py, level) << 10) | (uint64_t)d_voxel(pz, level);
}

__device__ __forceinline__ void d_address(uint64_t key, uint64_t n_cells, uint32_t pow2_mask,
                                          uint32_t* cell, uint32_t* h2) {
    uint64_t h1 = d_splitmix(key);
    *cell = pow2_mask ? (uint32_t)(h1 & (uint64_t)pow2_mask) : (uint32_t)(h1 % n_cells);
    uint32_t c = (uint32_t)(d_fmix64(key ^ 0x9E3779B97F4A7C15ull) >> 32);
    *h2 = c ? c : 1u;
}

// =======================================================================================
// Node primitives in FP32
// =======================================================================================
__device__ __forceinline__ uint32_t d_lattice(int i, int j, uint32_t seed) {
    // Teschner et al. 2003 primes, xor-combined, then fmix32
    return d_fmix32(((uint32_t)i * 73856093u) ^ ((uint32_t)j * 19349663u) ^ (seed * 83492791u));
}

// The 8 unit gradients at multiples of 45 degrees, indexed by hash & 7; each kernel that
// evaluates noise keeps a copy in shared memory (one 8-byte load per lattice corner).
__device__ __forceinline__ void init_gradients(float2* g) {
    if (threadIdx.x < 8) {
        const float R = 0.70710678118654752f;
        const float gx[8] = {1.0f, R, 0.0f, -R, -1.0f, -R, 0.0f, R};
        const float gy[8] = {0.0f, R, 1.0f, R, 0.0f, -R, -1.0f, -R};
        g[threadIdx.x] = make_float2(gx[threadIdx.x], gy[threadIdx.x]);
    }
}

__device__ __forceinline__ float d_fade(float t) {
    return t * t * t * fmaf(t, fmaf(t, 6.0f, -15.0f), 10.0f);
}

__device__ __forceinline__ float d_perlin(float x, float y, uint32_t seed, const float2* grad) {
    float fx0 = floorf(x), fy0 = floorf(y);
    int ix = (int)fx0, iy = (int)fy0;
    float fx = x - fx0, fy = y - fy0;
    float fx1 = fx - 1.0f, fy1 = fy - 1.0f;
    const float2 g00 = grad[d_lattice(ix, iy, seed) & 7u];
    const float2 g10 = grad[d_lattice(ix + 1, iy, seed) & 7u];
    const float2 g01 = grad[d_lattice(ix, iy + 1, seed) & 7u];
    const float2 g11 = grad[d_lattice(ix + 1, iy + 1, seed) & 7u];
    float d00 = fmaf(g00.x, fx, g00.y * fy);
    float d10 = fmaf(g10.x, fx1, g10.y * fy);
    float d01 = fmaf(g01.x, fx, g01.y * fy1);
    float d11 = fmaf(g11.x, fx1, g11.y * fy1);
    float su = d_fade(fx), sv = d_fade(fy);
    float a = fmaf(su, d10 - d00, d00);
    float b = fmaf(su, d11 - d01, d01);
    return fmaf(sv, b - a, a);
}

// clamp to [0, 1] (NaN to 0) as a saturating modifier of the producing instruction
__device__ __forceinline__ float d_clamp01(float x) { return __saturatef(x); }

__device__ __forceinline__ float d_fbm(float x, float y, const float* p, const float2* grad) {
    float scale = p[0], lac = p[1], gain = p[2], inv_norm = p[3];
    int oct = __float_as_int(p[4]);
    uint32_t seed = (uint32_t)__float_as_int(p[5]);
    float sum = 0.0f, amp = 1.0f, freq = scale;
    for (int k = 0; k < oct; ++k) {
        sum = fmaf(amp, d_perlin(x * freq, y * freq, seed + (uint32_t)k, grad), sum);
        amp *= gain;
        freq *= lac;
    }
    return d_clamp01(fmaf(sum, inv_norm, 0.5f));
}

__device__ __forceinline__ float d_voronoi(float x, float y, const float* p) {
    float sx = x * p[0], sy = y * p[0];
    uint32_t seed = (uint32_t)__float_as_int(p[1]);
    float fx0 = floorf(sx), fy0 = floorf(sy);
    int ix = (int)fx0, iy = (int)fy0;
    float fx = sx - fx0, fy = sy - fy0;
    float best = 3.0e38f;
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
#pragma unroll
        for (int a = -1; a <= 1; ++a) {
            uint32_t h = d_lattice(ix + a, iy + b, seed);
            float ox = fmaf((float)(h & 0xFFFFu), 0.5f / 65536.0f, (float)a + 0.25f);
            float oy = fmaf((float)(h >> 16), 0.5f / 65536.0f, (float)b + 0.25f);
            float dx = ox - fx, dy = oy - fy;
            best = fminf(best, fmaf(dx, dx, dy * dy));
        }
    }
    return d_clamp01(sqrtf(best));
}

struct PointIn {
    float u, v, px, py, pz, nx, ny, nz;
};

// One node instruction for one lane.  V points at the lane's slot file, laid out
// [slot][channel][lane] so that the 32 lanes of a warp touch 32 consecutive words.
__device__ __forceinline__ void exec_node(uint32_t op, const uint4& ins, float* V, const PointIn& pt,
                                          const float* __restrict__ params, const float2* grad) {
    const uint32_t out = ins.y & 0xFFFFu;
    const uint32_t i0 = ins.y >> 16, i1 = ins.z & 0xFFFFu, i2 = ins.z >> 16;
    // a node's parameters start on a 16-byte boundary: vector loads fetch them
    const float* p = params + ins.w;
    const float4* p4 = reinterpret_cast<const float4*>(p);
    float r0 = 0.f, r1 = 0.f, r2 = 0.f;
    switch (op) {
    case PMC_OP_UV: r0 = pt.u; r1 = pt.v; break;
    case PMC_OP_POSITION: r0 = pt.px; r1 = pt.py; r2 = pt.pz; break;
    case PMC_OP_NORMAL: r0 = pt.nx; r1 = pt.ny; r2 = pt.nz; break;
    case PMC_OP_CONST: {
        const float4 q = __ldg(p4);
        r0 = q.x; r1 = q.y; r2 = q.z;
        break;
    }
    case PMC_OP_UV_AFFINE: {
        const float4 q = __ldg(p4);
        const float4 t = __ldg(p4 + 1);
        float x = V[(i0 * 3) * 32], y = V[(i0 * 3 + 1) * 32];
        r0 = fmaf(q.x, x, fmaf(q.y, y, t.x));
        r1 = fmaf(q.z, x, fmaf(q.w, y, t.y));
        break;
    }
    case PMC_OP_FBM: {
        const float4 q = __ldg(p4);
        const float4 t = __ldg(p4 + 1);
        const float pp[6] = {q.x, q.y, q.z, q.w, t.x, t.y};
        r0 = r1 = r2 = d_fbm(V[(i0 * 3) * 32], V[(i0 * 3 + 1) * 32], pp, grad);
        break;
    }
    case PMC_OP_VORONOI: {
        const float4 q = __ldg(p4);
        const float pp[2] = {q.x, q.y};
        r0 = r1 = r2 = d_voronoi(V[(i0 * 3) * 32], V[(i0 * 3 + 1) * 32], pp);
        break;
    }
    case PMC_OP_CHECKER: {
        const float4 q = __ldg(p4);
        const float4 t = __ldg(p4 + 1);
        const float sc = q.x;
        long long k = (long long)floorf(V[(i0 * 3) * 32] * sc) + (long long)floorf(V[(i0 * 3 + 1) * 32] * sc);
        const bool odd = (k & 1) != 0;
        r0 = d_clamp01(odd ? t.x : q.y); r1 = d_clamp01(odd ? t.y : q.z); r2 = d_clamp01(odd ? t.z : q.w);
        break;
    }
    case PMC_OP_RAMP: {
        int ns = __float_as_int(__ldg(&p[0]));
        const float* pos = p + 1;
        const float* col = p + 5;
        float t = d_clamp01(V[(i0 * 3) * 32]);
        if (t <= __ldg(&pos[0])) {
            r0 = __ldg(&col[0]); r1 = __ldg(&col[1]); r2 = __ldg(&col[2]);
        } else if (t >= __ldg(&pos[ns - 1])) {
            r0 = __ldg(&col[3 * (ns - 1)]); r1 = __ldg(&col[3 * (ns - 1) + 1]); r2 = __ldg(&col[3 * (ns - 1) + 2]);
        } else {
            int k = 0;
            while (k + 2 < ns && t >= __ldg(&pos[k + 1])) ++k;
            float p0 = __ldg(&pos[k]), p1 = __ldg(&pos[k + 1]);
            float w = (t - p0) / (p1 - p0);
            float a0 = __ldg(&col[3 * k]), a1 = __ldg(&col[3 * k + 1]), a2 = __ldg(&col[3 * k + 2]);
            r0 = fmaf(w, __ldg(&col[3 * k + 3]) - a0, a0);
            r1 = fmaf(w, __ldg(&col[3 * k + 4]) - a1, a1);
            r2 = fmaf(w, __ldg(&col[3 * k + 5]) - a2, a2);
        }
        r0 = d_clamp01(r0); r1 = d_clamp01(r1); r2 = d_clamp01(r2);
        break;
    }
    case PMC_OP_MIX: {
        float f = d_clamp01(i2 != 0xFFFFu ? V[(i2 * 3) * 32] : __ldg(&p[0]));
        float a0 = V[(i0 * 3) * 32], a1 = V[(i0 * 3 + 1) * 32], a2 = V[(i0 * 3 + 2) * 32];
        r0 = d_clamp01(fmaf(f, V[(i1 * 3) * 32] - a0, a0));
        r1 = d_clamp01(fmaf(f, V[(i1 * 3 + 1) * 32] - a1, a1));
        r2 = d_clamp01(fmaf(f, V[(i1 * 3 + 2) * 32] - a2, a2));
        break;
    }
    case PMC_OP_ADD:
        r0 = d_clamp01(V[(i0 * 3) * 32] + V[(i1 * 3) * 32]);
        r1 = d_clamp01(V[(i0 * 3 + 1) * 32] + V[(i1 * 3 + 1) * 32]);
        r2 = d_clamp01(V[(i0 * 3 + 2) * 32] + V[(i1 * 3 + 2) * 32]);
        break;
    case PMC_OP_MUL:
        r0 = d_clamp01(V[(i0 * 3) * 32] * V[(i1 * 3) * 32]);
        r1 = d_clamp01(V[(i0 * 3 + 1) * 32] * V[(i1 * 3 + 1) * 32]);
        r2 = d_clamp01(V[(i0 * 3 + 2) * 32] * V[(i1 * 3 + 2) * 32]);
        break;
    case PMC_OP_POW: {
        float e = __ldg(&p[0]);
        r0 = d_clamp01(powf(fmaxf(V[(i0 * 3) * 32], 0.0f), e));
        r1 = d_clamp01(powf(fmaxf(V[(i0 * 3 + 1) * 32], 0.0f), e));
        r2 = d_clamp01(powf(fmaxf(V[(i0 * 3 + 2) * 32], 0.0f), e));
        break;
    }
    case PMC_OP_FACING: {
        const float4 q = __ldg(p4);
        float d = fmaf(V[(i0 * 3) * 32], q.x, fmaf(V[(i0 * 3 + 1) * 32], q.y, V[(i0 * 3 + 2) * 32] * q.z));
        r0 = r1 = r2 = d_clamp01(fabsf(d));
        break;
    }
    default:
        break;
    }
    V[(out * 3) * 32] = r0;
    V[(out * 3 + 1) * 32] = r1;
    V[(out * 3 + 2) * 32] = r2;
}


}  // namespace pmc
