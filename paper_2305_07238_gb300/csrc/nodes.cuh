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

// Pairs of independent FP32 operations issue as one instruction (Blackwell's packed FP32);
// each lane of a pair rounds exactly as the scalar operation would.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// quintic fade 6t^5 - 15t^4 + 10t^3 of both coordinates at once
__device__ __forceinline__ float2 d_fade2(float2 t) {
    const float2 t3 = mul2(mul2(t, t), t);
    return mul2(t3, fma2(t, fma2(t, f2(6.0f, 6.0f), f2(-15.0f, -15.0f)), f2(10.0f, 10.0f)));
}

__device__ __forceinline__ float d_fade(float t) {
    return t * t * t * fmaf(t, fmaf(t, 6.0f, -15.0f), 10.0f);
}

__device__ __forceinline__ float d_perlin(float x, float y, uint32_t seed, const float2* grad) {
    const float2 p = f2(x, y);
    const float2 f0 = f2(floorf(x), floorf(y));
    const int ix = (int)f0.x, iy = (int)f0.y;
    const float2 fr = fma2(f0, f2(-1.0f, -1.0f), p);          // (fx, fy) = p - floor(p)
    const float2 fr1 = add2(fr, f2(-1.0f, -1.0f));            // (fx - 1, fy - 1)
    // lattice hashes of the four corners: the prime products of x + 1 and y + 1 are those
    // of x and y plus the prime
    const uint32_t ax = (uint32_t)ix * 73856093u, by = (uint32_t)iy * 19349663u, sz = seed * 83492791u;
    const uint32_t ax1 = ax + 73856093u, by1 = by + 19349663u;
    const float2 g00 = grad[d_fmix32(ax ^ by ^ sz) & 7u];
    const float2 g10 = grad[d_fmix32(ax1 ^ by ^ sz) & 7u];
    const float2 g01 = grad[d_fmix32(ax ^ by1 ^ sz) & 7u];
    const float2 g11 = grad[d_fmix32(ax1 ^ by1 ^ sz) & 7u];
    // corner dot products g . (p - corner), each as fmaf(gx, dx, gy dy); scalar, since the
    // corners' gradients arrive in separate registers
    const float2 dA = f2(fmaf(g00.x, fr.x, g00.y * fr.y), fmaf(g01.x, fr.x, g01.y * fr1.y));    // (d00, d01)
    const float2 dB = f2(fmaf(g10.x, fr1.x, g10.y * fr.y), fmaf(g11.x, fr1.x, g11.y * fr1.y));  // (d10, d11)
    const float2 s = d_fade2(fr);
    // (a, b) = dA + s.x (dB - dA); result = a + s.y (b - a)
    const float2 ab = fma2(f2(s.x, s.x), fma2(dA, f2(-1.0f, -1.0f), dB), dA);
    return fmaf(s.y, ab.y - ab.x, ab.x);
}

// The same noise at two points A and B, every FP32 quantity held as an (A, B) pair so that
// each packed instruction serves both points; the result is (noise(A), noise(B)) with the
// roundings of d_perlin.
__device__ __forceinline__ float2 d_perlin2(float2 X, float2 Y, uint32_t seed, const float2* grad) {
    const float2 fX = f2(floorf(X.x), floorf(X.y)), fY = f2(floorf(Y.x), floorf(Y.y));
    const float2 rX = fma2(fX, f2(-1.0f, -1.0f), X), rY = fma2(fY, f2(-1.0f, -1.0f), Y);   // fx, fy
    const float2 rX1 = add2(rX, f2(-1.0f, -1.0f)), rY1 = add2(rY, f2(-1.0f, -1.0f));       // fx - 1, fy - 1
    const uint32_t sz = seed * 83492791u;
    const uint32_t axA = (uint32_t)(int)fX.x * 73856093u, byA = (uint32_t)(int)fY.x * 19349663u;
    const uint32_t axB = (uint32_t)(int)fX.y * 73856093u, byB = (uint32_t)(int)fY.y * 19349663u;
    const uint32_t axA1 = axA + 73856093u, byA1 = byA + 19349663u;
    const uint32_t axB1 = axB + 73856093u, byB1 = byB + 19349663u;
    const float2 a00 = grad[d_fmix32(axA ^ byA ^ sz) & 7u], b00 = grad[d_fmix32(axB ^ byB ^ sz) & 7u];
    const float2 a10 = grad[d_fmix32(axA1 ^ byA ^ sz) & 7u], b10 = grad[d_fmix32(axB1 ^ byB ^ sz) & 7u];
    const float2 a01 = grad[d_fmix32(axA ^ byA1 ^ sz) & 7u], b01 = grad[d_fmix32(axB ^ byB1 ^ sz) & 7u];
    const float2 a11 = grad[d_fmix32(axA1 ^ byA1 ^ sz) & 7u], b11 = grad[d_fmix32(axB1 ^ byB1 ^ sz) & 7u];
    const float2 d00 = f2(fmaf(a00.x, rX.x, a00.y * rY.x), fmaf(b00.x, rX.y, b00.y * rY.y));
    const float2 d10 = f2(fmaf(a10.x, rX1.x, a10.y * rY.x), fmaf(b10.x, rX1.y, b10.y * rY.y));
    const float2 d01 = f2(fmaf(a01.x, rX.x, a01.y * rY1.x), fmaf(b01.x, rX.y, b01.y * rY1.y));
    const float2 d11 = f2(fmaf(a11.x, rX1.x, a11.y * rY1.x), fmaf(b11.x, rX1.y, b11.y * rY1.y));
    const float2 sX = d_fade2(rX), sY = d_fade2(rY);
    const float2 a = fma2(sX, fma2(d00, f2(-1.0f, -1.0f), d10), d00);
    const float2 b = fma2(sX, fma2(d01, f2(-1.0f, -1.0f), d11), d01);
    return fma2(sY, fma2(a, f2(-1.0f, -1.0f), b), a);
}

// clamp to [0, 1] (NaN to 0) as a saturating modifier of the producing instruction
__device__ __forceinline__ float d_clamp01(float x) { return __saturatef(x); }

// q = {scale, lacunarity, gain, 1 / sum of gains}, t = {octaves, seed} (integers in floats)
__device__ __forceinline__ float d_fbm(float x, float y, const float4 q, const float4 t, const float2* grad) {
    const float scale = q.x, lac = q.y, gain = q.z, inv_norm = q.w;
    const int oct = __float_as_int(t.x);
    const uint32_t seed = (uint32_t)__float_as_int(t.y);
    float sum = 0.0f, amp = 1.0f, freq = scale;
    for (int k = 0; k < oct; ++k) {
        const float2 q = mul2(f2(x, y), f2(freq, freq));
        sum = fmaf(amp, d_perlin(q.x, q.y, seed + (uint32_t)k, grad), sum);
        const float2 af = mul2(f2(amp, freq), f2(gain, lac));
        amp = af.x;
        freq = af.y;
    }
    return d_clamp01(fmaf(sum, inv_norm, 0.5f));
}

// d_fbm at two points in one octave loop (the amplitude and frequency updates are shared)
__device__ __forceinline__ float2 d_fbm2(float2 X, float2 Y, const float4 q, const float4 t, const float2* grad) {
    const float scale = q.x, lac = q.y, gain = q.z, inv_norm = q.w;
    const int oct = __float_as_int(t.x);
    const uint32_t seed = (uint32_t)__float_as_int(t.y);
    float2 sum = f2(0.0f, 0.0f);
    float amp = 1.0f, freq = scale;
    for (int k = 0; k < oct; ++k) {
        const float2 n = d_perlin2(mul2(X, f2(freq, freq)), mul2(Y, f2(freq, freq)), seed + (uint32_t)k, grad);
        sum = fma2(f2(amp, amp), n, sum);
        const float2 af = mul2(f2(amp, freq), f2(gain, lac));
        amp = af.x;
        freq = af.y;
    }
    const float2 r = fma2(sum, f2(inv_norm, inv_norm), f2(0.5f, 0.5f));
    return f2(d_clamp01(r.x), d_clamp01(r.y));
}

// The two 16-bit halves of a hash h as m = 1 + h16 2^-16, exactly: an FP32 number whose
// fraction holds h16 in its top 16 bits.  One shift and one masked or per half, no
// integer-to-float conversion.
__device__ __forceinline__ float2 d_halves(uint32_t h) {
    return f2(__uint_as_float(((h << 7) & 0x7FFF80u) | 0x3F800000u),
              __uint_as_float(((h >> 9) & 0x7FFF80u) | 0x3F800000u));
}

__device__ __forceinline__ float d_voronoi(float x, float y, float scale, uint32_t seed) {
    const float2 sc = mul2(f2(x, y), f2(scale, scale));
    const float2 f0 = f2(floorf(sc.x), floorf(sc.y));
    const int ix = (int)f0.x, iy = (int)f0.y;
    const float2 fr = fma2(f0, f2(-1.0f, -1.0f), sc);
    const uint32_t sz = seed * 83492791u;
    const uint32_t ax = (uint32_t)ix * 73856093u;
    const uint32_t axs[3] = {ax - 73856093u, ax, ax + 73856093u};
    float best = 3.0e38f;
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
        const uint32_t by = ((uint32_t)iy * 19349663u + (uint32_t)b * 19349663u) ^ sz;
#pragma unroll
        for (int a = -1; a <= 1; ++a) {
            // feature point at cell + 0.25 + 0.5 h16 2^-16 per axis: with m = 1 + h16 2^-16,
            // fmaf(m, 0.5, a - 0.25) is that same real number under one rounding, the value
            // fmaf(h16, 0.5 / 65536, a + 0.25) gives
            const float2 m = d_halves(d_fmix32(axs[a + 1] ^ by));
            const float2 o = fma2(m, f2(0.5f, 0.5f), f2((float)a - 0.25f, (float)b - 0.25f));
            const float2 d = fma2(fr, f2(-1.0f, -1.0f), o);
            best = fminf(best, fmaf(d.x, d.x, d.y * d.y));
        }
    }
    // sqrt(best) as best / sqrt(best) through the reciprocal square root (within a few ulp);
    // best = 0 gives 0 x inf = NaN, which the clamp maps to 0 = sqrt(0)
    return d_clamp01(best * rsqrtf(best));
}

// Parity of an integer-valued FP32 number f as 0 or 1: f - 2 floor(f / 2), exact for every
// finite f (integers beyond 2^24 are even, and the formula gives 0 there).
__device__ __forceinline__ float d_parity(float f) { return fmaf(-2.0f, floorf(f * 0.5f), f); }

struct PointIn {
    float u, v, px, py, pz, nx, ny, nz;
};

// A node's value slots, laid out [slot][channel][lane] per warp: the 32 lanes of a warp
// touch 32 consecutive words.  Programs name slots by byte offsets from the lane's base
// (slot x SLOT_BYTES), so an operand is one add away from its address.
constexpr uint32_t CH_BYTES = 32u * 4u;

__device__ __forceinline__ float slot_ch(const char* Vb, uint32_t off, int ch) {
    return *reinterpret_cast<const float*>(Vb + off + ch * CH_BYTES);
}
__device__ __forceinline__ void slot_store(char* Vb, uint32_t off, float r0, float r1, float r2) {
    float* o = reinterpret_cast<float*>(Vb + off);
    o[0] = r0;
    o[32] = r1;
    o[64] = r2;
}

// One node instruction for one lane.  Vb is the lane's base in the slot file; the
// instruction's y = out | in0 << 16, z = in1 | in2 << 16 are byte offsets from it.
__device__ __forceinline__ void exec_node(uint32_t op, const uint4& ins, char* Vb, const PointIn& pt,
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
        const float x = slot_ch(Vb, i0, 0), y = slot_ch(Vb, i0, 1);
        r0 = fmaf(q.x, x, fmaf(q.y, y, t.x));
        r1 = fmaf(q.z, x, fmaf(q.w, y, t.y));
        break;
    }
    case PMC_OP_FBM: {
        const float4 q = __ldg(p4);
        const float4 t = __ldg(p4 + 1);
        r0 = r1 = r2 = d_fbm(slot_ch(Vb, i0, 0), slot_ch(Vb, i0, 1), q, t, grad);
        break;
    }
    case PMC_OP_VORONOI: {
        const float4 q = __ldg(p4);
        r0 = r1 = r2 = d_voronoi(slot_ch(Vb, i0, 0), slot_ch(Vb, i0, 1), q.x, (uint32_t)__float_as_int(q.y));
        break;
    }
    case PMC_OP_CHECKER: {
        // colour B iff floor(x s) + floor(y s) is odd, i.e. the two parities differ
        const float4 q = __ldg(p4);
        const float4 t = __ldg(p4 + 1);
        const float2 f = mul2(f2(slot_ch(Vb, i0, 0), slot_ch(Vb, i0, 1)), f2(q.x, q.x));
        const bool odd = d_parity(floorf(f.x)) != d_parity(floorf(f.y));
        r0 = d_clamp01(odd ? t.x : q.y); r1 = d_clamp01(odd ? t.y : q.z); r2 = d_clamp01(odd ? t.z : q.w);
        break;
    }
    case PMC_OP_RAMP: {
        // parameters: {first stop, last stop, second, third (2 if absent)}, (stop, 1 / segment
        // length) of segments 0..2, padding, colours of stops 0..3 and of the last stop, four
        // floats each
        const float4 q = __ldg(p4);
        const float t = d_clamp01(slot_ch(Vb, i0, 0));
        const int k = (t >= q.z ? 1 : 0) + (t >= q.w ? 1 : 0);   // interior stops at or below t
        const float2 seg = __ldg(reinterpret_cast<const float2*>(p + 4) + k);
        const float4 ca = __ldg(p4 + 3 + k);
        const float4 cb = __ldg(p4 + 4 + k);
        const float w = (t - seg.x) * seg.y;
        r0 = fmaf(w, cb.x - ca.x, ca.x);
        r1 = fmaf(w, cb.y - ca.y, ca.y);
        r2 = fmaf(w, cb.z - ca.z, ca.z);
        if (t <= q.x) {
            const float4 c0 = __ldg(p4 + 3);
            r0 = c0.x; r1 = c0.y; r2 = c0.z;
        } else if (t >= q.y) {
            const float4 cl = __ldg(p4 + 7);
            r0 = cl.x; r1 = cl.y; r2 = cl.z;
        }
        r0 = d_clamp01(r0); r1 = d_clamp01(r1); r2 = d_clamp01(r2);
        break;
    }
    case PMC_OP_MIX: {
        const float f = d_clamp01(((ins.x >> 8) & FLAG_IN2) ? slot_ch(Vb, i2, 0) : __ldg(&p[0]));
        const float a0 = slot_ch(Vb, i0, 0), a1 = slot_ch(Vb, i0, 1), a2 = slot_ch(Vb, i0, 2);
        r0 = d_clamp01(fmaf(f, slot_ch(Vb, i1, 0) - a0, a0));
        r1 = d_clamp01(fmaf(f, slot_ch(Vb, i1, 1) - a1, a1));
        r2 = d_clamp01(fmaf(f, slot_ch(Vb, i1, 2) - a2, a2));
        break;
    }
    case PMC_OP_ADD:
        r0 = d_clamp01(slot_ch(Vb, i0, 0) + slot_ch(Vb, i1, 0));
        r1 = d_clamp01(slot_ch(Vb, i0, 1) + slot_ch(Vb, i1, 1));
        r2 = d_clamp01(slot_ch(Vb, i0, 2) + slot_ch(Vb, i1, 2));
        break;
    case PMC_OP_MUL:
        r0 = d_clamp01(slot_ch(Vb, i0, 0) * slot_ch(Vb, i1, 0));
        r1 = d_clamp01(slot_ch(Vb, i0, 1) * slot_ch(Vb, i1, 1));
        r2 = d_clamp01(slot_ch(Vb, i0, 2) * slot_ch(Vb, i1, 2));
        break;
    case PMC_OP_POW: {
        // x^e for x >= 0 through the hardware base-2 logarithm and exponential (__powf);
        // x = 0 gives 0 for every e > 0
        const float e = __ldg(&p[0]);
        r0 = d_clamp01(__powf(fmaxf(slot_ch(Vb, i0, 0), 0.0f), e));
        r1 = d_clamp01(__powf(fmaxf(slot_ch(Vb, i0, 1), 0.0f), e));
        r2 = d_clamp01(__powf(fmaxf(slot_ch(Vb, i0, 2), 0.0f), e));
        break;
    }
    case PMC_OP_FACING: {
        const float4 q = __ldg(p4);
        float d = fmaf(slot_ch(Vb, i0, 0), q.x, fmaf(slot_ch(Vb, i0, 1), q.y, slot_ch(Vb, i0, 2) * q.z));
        r0 = r1 = r2 = d_clamp01(fabsf(d));
        break;
    }
    default:
        break;
    }
    slot_store(Vb, out, r0, r1, r2);
}


// Two points per lane: the slot file is [slot][channel][lane][2], so a slot is 2 x SLOT_BYTES
// and a channel row 2 x CH_BYTES; an operand's byte offset in a program doubles.  One
// decode, dispatch and parameter load serve both points, and their two independent
// computations overlap.
__device__ __forceinline__ float2 slot2(const char* Vb, uint32_t off, int ch) {
    return *reinterpret_cast<const float2*>(Vb + 2u * off + ch * (2u * CH_BYTES));
}
__device__ __forceinline__ void slot2_store(char* Vb, uint32_t off, float2 r0, float2 r1, float2 r2) {
    float2* o = reinterpret_cast<float2*>(Vb + 2u * off);
    o[0] = r0;
    o[32] = r1;
    o[64] = r2;
}
__device__ __forceinline__ float2 sat2(float2 x) { return f2(d_clamp01(x.x), d_clamp01(x.y)); }

// exec_node for points A (.x of every pair) and B (.y).
__device__ __forceinline__ void exec_node2(uint32_t op, const uint4& ins, char* Vb, const PointIn& A, const PointIn& B,
                                           const float* __restrict__ params, const float2* grad) {
    const uint32_t out = ins.y & 0xFFFFu;
    const uint32_t i0 = ins.y >> 16, i1 = ins.z & 0xFFFFu, i2 = ins.z >> 16;
    const float* p = params + ins.w;
    const float4* p4 = reinterpret_cast<const float4*>(p);
    // every case stores its own result: no values merge after the switch
    switch (op) {
    case PMC_OP_UV: slot2_store(Vb, out, f2(A.u, B.u), f2(A.v, B.v), f2(0.f, 0.f)); break;
    case PMC_OP_POSITION: slot2_store(Vb, out, f2(A.px, B.px), f2(A.py, B.py), f2(A.pz, B.pz)); break;
    case PMC_OP_NORMAL: slot2_store(Vb, out, f2(A.nx, B.nx), f2(A.ny, B.ny), f2(A.nz, B.nz)); break;
    case PMC_OP_CONST: {
        const float4 q = __ldg(p4);
        slot2_store(Vb, out, f2(q.x, q.x), f2(q.y, q.y), f2(q.z, q.z));
        break;
    }
    case PMC_OP_UV_AFFINE: {
        const float4 q = __ldg(p4);
        const float4 t = __ldg(p4 + 1);
        const float2 x = slot2(Vb, i0, 0), y = slot2(Vb, i0, 1);
        slot2_store(Vb, out, fma2(f2(q.x, q.x), x, fma2(f2(q.y, q.y), y, f2(t.x, t.x))),
                    fma2(f2(q.z, q.z), x, fma2(f2(q.w, q.w), y, f2(t.y, t.y))), f2(0.f, 0.f));
        break;
    }
    case PMC_OP_FBM: {
        const float4 q = __ldg(p4);
        const float4 t = __ldg(p4 + 1);
        const float2 r = d_fbm2(slot2(Vb, i0, 0), slot2(Vb, i0, 1), q, t, grad);
        slot2_store(Vb, out, r, r, r);
        break;
    }
    case PMC_OP_VORONOI: {
        const float4 q = __ldg(p4);
        const float2 x = slot2(Vb, i0, 0), y = slot2(Vb, i0, 1);
        const uint32_t seed = (uint32_t)__float_as_int(q.y);
        const float2 r = f2(d_voronoi(x.x, y.x, q.x, seed), d_voronoi(x.y, y.y, q.x, seed));
        slot2_store(Vb, out, r, r, r);
        break;
    }
    case PMC_OP_CHECKER: {
        const float4 q = __ldg(p4);
        const float4 t = __ldg(p4 + 1);
        const float2 fx = mul2(slot2(Vb, i0, 0), f2(q.x, q.x)), fy = mul2(slot2(Vb, i0, 1), f2(q.x, q.x));
        const bool oa = d_parity(floorf(fx.x)) != d_parity(floorf(fy.x));
        const bool ob = d_parity(floorf(fx.y)) != d_parity(floorf(fy.y));
        slot2_store(Vb, out, sat2(f2(oa ? t.x : q.y, ob ? t.x : q.y)), sat2(f2(oa ? t.y : q.z, ob ? t.y : q.z)),
                    sat2(f2(oa ? t.z : q.w, ob ? t.z : q.w)));
        break;
    }
    case PMC_OP_RAMP: {
        const float4 q = __ldg(p4);
        const float2 tt = sat2(slot2(Vb, i0, 0));
        const float ts[2] = {tt.x, tt.y};
        float o[2][3];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float t = ts[s];
            const int k = (t >= q.z ? 1 : 0) + (t >= q.w ? 1 : 0);
            const float2 seg = __ldg(reinterpret_cast<const float2*>(p + 4) + k);
            const float4 ca = __ldg(p4 + 3 + k);
            const float4 cb = __ldg(p4 + 4 + k);
            const float w = (t - seg.x) * seg.y;
            o[s][0] = fmaf(w, cb.x - ca.x, ca.x);
            o[s][1] = fmaf(w, cb.y - ca.y, ca.y);
            o[s][2] = fmaf(w, cb.z - ca.z, ca.z);
            if (t <= q.x) {
                const float4 c0 = __ldg(p4 + 3);
                o[s][0] = c0.x; o[s][1] = c0.y; o[s][2] = c0.z;
            } else if (t >= q.y) {
                const float4 cl = __ldg(p4 + 7);
                o[s][0] = cl.x; o[s][1] = cl.y; o[s][2] = cl.z;
            }
        }
        slot2_store(Vb, out, sat2(f2(o[0][0], o[1][0])), sat2(f2(o[0][1], o[1][1])), sat2(f2(o[0][2], o[1][2])));
        break;
    }
    case PMC_OP_MIX: {
        const float2 f = sat2(((ins.x >> 8) & FLAG_IN2) ? slot2(Vb, i2, 0) : f2(__ldg(&p[0]), __ldg(&p[0])));
        const float2 a0 = slot2(Vb, i0, 0), a1 = slot2(Vb, i0, 1), a2 = slot2(Vb, i0, 2);
        // a + f (b - a), each product and sum rounded as fmaf(f, b - a, a) rounds them
        slot2_store(Vb, out, sat2(fma2(f, fma2(a0, f2(-1.0f, -1.0f), slot2(Vb, i1, 0)), a0)),
                    sat2(fma2(f, fma2(a1, f2(-1.0f, -1.0f), slot2(Vb, i1, 1)), a1)),
                    sat2(fma2(f, fma2(a2, f2(-1.0f, -1.0f), slot2(Vb, i1, 2)), a2)));
        break;
    }
    case PMC_OP_ADD:
        slot2_store(Vb, out, sat2(add2(slot2(Vb, i0, 0), slot2(Vb, i1, 0))), sat2(add2(slot2(Vb, i0, 1), slot2(Vb, i1, 1))),
                    sat2(add2(slot2(Vb, i0, 2), slot2(Vb, i1, 2))));
        break;
    case PMC_OP_MUL:
        slot2_store(Vb, out, sat2(mul2(slot2(Vb, i0, 0), slot2(Vb, i1, 0))), sat2(mul2(slot2(Vb, i0, 1), slot2(Vb, i1, 1))),
                    sat2(mul2(slot2(Vb, i0, 2), slot2(Vb, i1, 2))));
        break;
    case PMC_OP_POW: {
        const float e = __ldg(&p[0]);
        const float2 x0 = slot2(Vb, i0, 0), x1 = slot2(Vb, i0, 1), x2 = slot2(Vb, i0, 2);
        slot2_store(Vb, out, sat2(f2(__powf(fmaxf(x0.x, 0.0f), e), __powf(fmaxf(x0.y, 0.0f), e))),
                    sat2(f2(__powf(fmaxf(x1.x, 0.0f), e), __powf(fmaxf(x1.y, 0.0f), e))),
                    sat2(f2(__powf(fmaxf(x2.x, 0.0f), e), __powf(fmaxf(x2.y, 0.0f), e))));
        break;
    }
    case PMC_OP_FACING: {
        const float4 q = __ldg(p4);
        const float2 d = fma2(slot2(Vb, i0, 0), f2(q.x, q.x),
                              fma2(slot2(Vb, i0, 1), f2(q.y, q.y), mul2(slot2(Vb, i0, 2), f2(q.z, q.z))));
        const float2 r = sat2(f2(fabsf(d.x), fabsf(d.y)));
        slot2_store(Vb, out, r, r, r);
        break;
    }
    default:
        slot2_store(Vb, out, f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f));
        break;
    }
}

}  // namespace pmc
