// kernels.cu -- sm_103a kernels of one progressive pass (Sec. 3, Alg. 1).
//
//   k_hist     material histogram of the batch (+ range check of material indices)
//   k_scan     per-material segment offsets, probe offsets and warp work items
//   k_scatter  groups the points by material into structure-of-arrays copies
//   k_lookup   warp-cooperative probes of every (point, cacheable node) against the
//              table as it was when the pass started (Sec. 3.2, Fig. 3)
//   k_eval     warp-uniform interpreter of the material programs (Sec. 2); hit blocks
//              are skipped, missed cacheable nodes become insert candidates (Sec. 3)
//   k_claim /  rounds of the insert: every live candidate targets the first slot of
//   k_resolve  its cell holding its hash2 (duplicate) or 0 (free, Alg. 1); the smallest
//              (point index, node ID) per cell wins by atomicMin and writes its slot
//   k_finish   advances the claim epoch and the batch counters
#include <cstdio>

#include "pmc_internal.h"

namespace pmc {

#define FULL_MASK 0xFFFFFFFFu

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

__device__ __forceinline__ uint64_t d_key(uint32_t mat, uint32_t node, uint32_t level,
                                          uint32_t iu, uint32_t iv) {
    return ((uint64_t)mat << 48) | ((uint64_t)node << 32) | ((uint64_t)level << 26) |
           ((uint64_t)iu << 13) | (uint64_t)iv;
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

// Gradient k of the 8 unit vectors at multiples of 45 degrees: x component.
// |gx| = 1 for k in {0,4}, 0 for {2,6}, sqrt(1/2) for odd k; negative for k in {3,4,5}.
__device__ __forceinline__ float d_gx(uint32_t k) {
    float m = (k & 1u) ? 0.70710678118654752f : ((k & 2u) ? 0.0f : 1.0f);
    return ((k + 1u) & 4u) ? -m : m;
}
// y component: the x component of the gradient 90 degrees earlier.
__device__ __forceinline__ float d_gy(uint32_t k) { return d_gx((k + 6u) & 7u); }

__device__ __forceinline__ float d_fade(float t) {
    return t * t * t * fmaf(t, fmaf(t, 6.0f, -15.0f), 10.0f);
}

__device__ __forceinline__ float d_perlin(float x, float y, uint32_t seed) {
    float fx0 = floorf(x), fy0 = floorf(y);
    int ix = (int)fx0, iy = (int)fy0;
    float fx = x - fx0, fy = y - fy0;
    float fx1 = fx - 1.0f, fy1 = fy - 1.0f;
    uint32_t h00 = d_lattice(ix, iy, seed) & 7u;
    uint32_t h10 = d_lattice(ix + 1, iy, seed) & 7u;
    uint32_t h01 = d_lattice(ix, iy + 1, seed) & 7u;
    uint32_t h11 = d_lattice(ix + 1, iy + 1, seed) & 7u;
    float d00 = fmaf(d_gx(h00), fx, d_gy(h00) * fy);
    float d10 = fmaf(d_gx(h10), fx1, d_gy(h10) * fy);
    float d01 = fmaf(d_gx(h01), fx, d_gy(h01) * fy1);
    float d11 = fmaf(d_gx(h11), fx1, d_gy(h11) * fy1);
    float su = d_fade(fx), sv = d_fade(fy);
    float a = fmaf(su, d10 - d00, d00);
    float b = fmaf(su, d11 - d01, d01);
    return fmaf(sv, b - a, a);
}

__device__ __forceinline__ float d_clamp01(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }

__device__ __forceinline__ float d_fbm(float x, float y, const float* p) {
    float scale = p[0], lac = p[1], gain = p[2], inv_norm = p[3];
    int oct = __float_as_int(p[4]);
    uint32_t seed = (uint32_t)__float_as_int(p[5]);
    float sum = 0.0f, amp = 1.0f, freq = scale;
    for (int k = 0; k < oct; ++k) {
        sum = fmaf(amp, d_perlin(x * freq, y * freq, seed + (uint32_t)k), sum);
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

// =======================================================================================
// Small helpers
// =======================================================================================
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ void warp_add_u64(unsigned long long* dst, unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    if (lane_id() == 0 && v) atomicAdd(dst, v);
}

// Appends the lanes with `pred` to a list; returns each lane's index (undefined for others).
__device__ __forceinline__ uint32_t warp_append(uint32_t* counter, bool pred) {
    unsigned m = __ballot_sync(FULL_MASK, pred);
    uint32_t base = 0;
    if (m) {
        int leader = __ffs(m) - 1;
        if ((int)lane_id() == leader) base = atomicAdd(counter, (uint32_t)__popc(m));
        base = __shfl_sync(FULL_MASK, base, leader);
    }
    return base + __popc(m & ((1u << lane_id()) - 1u));
}

__device__ __forceinline__ uint32_t find_material(const uint32_t* item_base, uint32_t n_mats,
                                                  uint32_t item) {
    // largest m with item_base[m] <= item (item_base is non-decreasing, item_base[0] = 0)
    uint32_t lo = 0, hi = n_mats;  // invariant: item_base[lo] <= item < item_base[hi]
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(&item_base[mid]) <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

// =======================================================================================
// Grouping by material
// =======================================================================================
__global__ void k_hist(BatchArgs a) {
    uint32_t stride = gridDim.x * blockDim.x;
    uint32_t n_round = (a.n + 31u) & ~31u;
    unsigned long long bad = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        bool act = i < a.n;
        uint32_t m = act ? a.mat[i] : 0u;
        bool ok = act && m < a.n_mats;
        if (act && !ok) bad++;
        unsigned vmask = __ballot_sync(FULL_MASK, ok);
        if (ok) {
            unsigned peers = __match_any_sync(vmask, m);
            int leader = __ffs(peers) - 1;
            if ((int)lane_id() == leader) atomicAdd(&a.counts[m], (uint32_t)__popc(peers));
        }
    }
    unsigned long long tot = bad;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(FULL_MASK, tot, o);
    if (lane_id() == 0 && tot) {
        atomicAdd(&a.stats[ST_BAD], tot);
        atomicOr(&a.ctl->err, ERR_BAD_MAT);
    }
}

// One block: exclusive scans of counts, counts * roots and ceil(counts / 32).
__global__ void k_scan(BatchArgs a) {
    __shared__ uint32_t s_tot[3][1024];
    const uint32_t T = blockDim.x, t = threadIdx.x;
    const uint32_t per = (a.n_mats + T - 1) / T;
    const uint32_t lo = min(t * per, a.n_mats), hi = min(lo + per, a.n_mats);
    uint32_t c0 = 0, c1 = 0, c2 = 0;
    for (uint32_t m = lo; m < hi; ++m) {
        uint32_t c = a.counts[m];
        uint32_t k = a.use_cache ? a.mats[m].n_roots : 0u;
        c0 += c;
        c1 += c * k;
        c2 += (c + 31u) >> 5;
    }
    s_tot[0][t] = c0; s_tot[1][t] = c1; s_tot[2][t] = c2;
    __syncthreads();
    // Hillis-Steele inclusive scan over the per-thread totals
    for (uint32_t off = 1; off < T; off <<= 1) {
        uint32_t v0 = 0, v1 = 0, v2 = 0;
        if (t >= off) { v0 = s_tot[0][t - off]; v1 = s_tot[1][t - off]; v2 = s_tot[2][t - off]; }
        __syncthreads();
        s_tot[0][t] += v0; s_tot[1][t] += v1; s_tot[2][t] += v2;
        __syncthreads();
    }
    uint32_t b0 = t ? s_tot[0][t - 1] : 0, b1 = t ? s_tot[1][t - 1] : 0, b2 = t ? s_tot[2][t - 1] : 0;
    for (uint32_t m = lo; m < hi; ++m) {
        uint32_t c = a.counts[m];
        uint32_t k = a.use_cache ? a.mats[m].n_roots : 0u;
        a.seg_start[m] = b0;
        a.cursor[m] = b0;
        a.probe_base[m] = b1;
        a.item_base[m] = b2;
        b0 += c;
        b1 += c * k;
        b2 += (c + 31u) >> 5;
    }
    if (t == T - 1) {
        a.seg_start[a.n_mats] = s_tot[0][t];
        a.probe_base[a.n_mats] = s_tot[1][t];
        a.item_base[a.n_mats] = s_tot[2][t];
        a.ctl->n_items = s_tot[2][t];
        a.ctl->total_probes = s_tot[1][t];
        if (s_tot[1][t] > a.probe_cap) atomicOr(&a.ctl->err, ERR_BOUNDS);
        atomicAdd(&a.stats[ST_POINTS], (unsigned long long)a.n);
    }
}

__global__ void k_scatter(BatchArgs a) {
    uint32_t stride = gridDim.x * blockDim.x;
    uint32_t n_round = (a.n + 31u) & ~31u;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        bool act = i < a.n;
        uint32_t m = act ? a.mat[i] : 0u;
        bool ok = act && m < a.n_mats;
        unsigned vmask = __ballot_sync(FULL_MASK, ok);
        if (ok) {
            unsigned peers = __match_any_sync(vmask, m);
            int leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if ((int)lane_id() == leader) base = atomicAdd(&a.cursor[m], (uint32_t)__popc(peers));
            base = __shfl_sync(peers, base, leader);
            uint32_t pos = base + __popc(peers & ((1u << lane_id()) - 1u));
            a.su[pos] = a.u[i];
            a.sv[pos] = a.v[i];
            a.spx[pos] = a.px[i];
            a.spy[pos] = a.py[i];
            a.spz[pos] = a.pz[i];
            a.snx[pos] = a.nx[i];
            a.sny[pos] = a.ny[i];
            a.snz[pos] = a.nz[i];
            a.sidx[pos] = i;
        } else if (act) {
            // out-of-range material: zero output, no probes
            a.out_rgb[i] = 0.0f;
            a.out_rgb[(size_t)a.n + i] = 0.0f;
            a.out_rgb[2 * (size_t)a.n + i] = 0.0f;
            if (a.out_hits) a.out_hits[i] = 0;
        }
    }
}

// =======================================================================================
// Lookup (Sec. 3.2): G lanes read one cell (one 16-byte slot each) per step
// =======================================================================================
constexpr uint32_t PROBE_HIT = 1u;

template <int G>
__global__ void __launch_bounds__(256) k_lookup(BatchArgs a) {
    constexpr int P = 32 / G;  // probes per step
    __shared__ uint32_t s_cell[8][32];
    __shared__ uint32_t s_h2[8][32];
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t warps_total = gridDim.x * (blockDim.x >> 5);
    const uint32_t n_items = a.ctl->n_items;
    const uint32_t ne = a.n_entries;
    unsigned long long n_look = 0, n_hit = 0, n_slots = 0;
    for (uint32_t item = blockIdx.x * (blockDim.x >> 5) + warp; item < n_items; item += warps_total) {
        uint32_t m = find_material(a.item_base, a.n_mats, item);
        uint32_t cnt = __ldg(&a.counts[m]);
        uint32_t j = (item - __ldg(&a.item_base[m])) * 32u + lane;
        bool valid = j < cnt;
        uint32_t s = __ldg(&a.seg_start[m]) + j;
        uint32_t iu = 0, iv = 0;
        if (valid) {
            iu = d_texel(a.su[s], a.level);
            iv = d_texel(a.sv[s], a.level);
        }
        const MatInfo mi = a.mats[m];
        const uint32_t pbase = __ldg(&a.probe_base[m]);
        for (uint32_t r = 0; r < mi.n_roots; ++r) {
            uint32_t node = __ldg(&a.roots[mi.root_base + r]);
            uint32_t cell = 0, h2 = 0;
            if (valid) d_address(d_key(m, node, a.level, iu, iv), a.n_cells, a.cells_pow2_mask, &cell, &h2);
            s_cell[warp][lane] = cell;
            s_h2[warp][lane] = valid ? h2 : 0u;
            __syncwarp();
            const uint32_t e = lane % G;
            const uint32_t grp = lane / G;
#pragma unroll
            for (int step = 0; step < G; ++step) {
                const uint32_t q = step * P + grp;      // probe of this lane in this step
                const uint32_t qh2 = s_h2[warp][q];     // 0 = invalid probe
                const uint32_t qcell = s_cell[warp][q];
                uint4 slot = make_uint4(0xFFFFFFFFu, 0, 0, 0);
                bool ld = qh2 != 0u && e < ne;
                if (ld) slot = __ldg(&a.table[(size_t)qcell * ne + e]);
                bool match = ld && slot.x == qh2;
                bool stop = ld && (slot.x == qh2 || slot.x == 0u);
                unsigned sb = __ballot_sync(FULL_MASK, stop);
                unsigned mb = __ballot_sync(FULL_MASK, match);
                const unsigned gmask = (G == 32) ? FULL_MASK : (((1u << G) - 1u) << (grp * G));
                unsigned gs = sb & gmask;
                int first = gs ? (__ffs(gs) - 1) : -1;   // lane index of the first stop
                if (qh2 != 0u) {
                    size_t rec = (size_t)pbase + (size_t)r * cnt + (item - __ldg(&a.item_base[m])) * 32u + q;
                    bool hit = first >= 0 && ((mb >> first) & 1u);
                    if (hit && (int)lane == first) {
                        a.probes[rec] = make_float4(__uint_as_float(slot.y), __uint_as_float(slot.z),
                                                    __uint_as_float(slot.w), __uint_as_float(PROBE_HIT));
                    }
                    if (e == 0) {
                        n_look++;
                        n_slots += first >= 0 ? (uint32_t)(first - (int)(grp * G)) + 1u : ne;
                        if (hit) n_hit++;
                        if (!hit)
                            a.probes[rec] = make_float4(__uint_as_float(qcell), __uint_as_float(qh2), 0.0f,
                                                        __uint_as_float(0u));
                    }
                }
            }
            __syncwarp();
        }
    }
    warp_add_u64(&a.stats[ST_LOOKUPS], n_look);
    warp_add_u64(&a.stats[ST_HITS], n_hit);
    warp_add_u64(&a.stats[ST_MISSES], n_look - n_hit);
    warp_add_u64(&a.stats[ST_SLOTS], n_slots);
}

// =======================================================================================
// Evaluation (Sec. 2, Sec. 3): one warp runs one material's program for 32 points
// =======================================================================================
constexpr uint32_t EVAL_WARPS = 4;

size_t eval_smem_bytes(uint32_t max_slots) {
    return (size_t)EVAL_WARPS * max_slots * 3u * 32u * sizeof(float);
}

__global__ void __launch_bounds__(EVAL_WARPS * 32) k_eval(BatchArgs a, uint32_t* item_ctr) {
    extern __shared__ float s_val[];
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    float* V = s_val + (size_t)warp * a.max_slots * 96u + lane;   // V[(slot*3 + c) * 32]
    const uint32_t n_items = a.ctl->n_items;
    unsigned long long n_nodes = 0, n_flops = 0;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(item_ctr, 1u);
        item = __shfl_sync(FULL_MASK, item, 0);
        if (item >= n_items) break;
        const uint32_t m = find_material(a.item_base, a.n_mats, item);
        const uint32_t cnt = __ldg(&a.counts[m]);
        const uint32_t j = (item - __ldg(&a.item_base[m])) * 32u + lane;
        const bool valid = j < cnt;
        const uint32_t s = __ldg(&a.seg_start[m]) + (valid ? j : 0u);
        float u = 0, v = 0, px = 0, py = 0, pz = 0, nx = 0, ny = 0, nz = 0;
        uint32_t orig = 0;
        if (valid) {
            u = a.su[s]; v = a.sv[s];
            px = a.spx[s]; py = a.spy[s]; pz = a.spz[s];
            nx = a.snx[s]; ny = a.sny[s]; nz = a.snz[s];
            orig = a.sidx[s];
        }
        const MatInfo mi = a.mats[m];
        const uint4* prog = a.prog + mi.prog_start;
        const uint32_t pbase = __ldg(&a.probe_base[m]);
        int skip_end = -1;          // lane inactive while pc <= skip_end
        uint32_t hits = 0, cand_cell = 0, cand_h2 = 0, cand_node = 0;
        for (int pc = 0; pc < (int)mi.prog_len; ++pc) {
            const uint4 ins = __ldg(&prog[pc]);
            const uint32_t op = ins.x & 0xFFu;
            if (op == OP_ROOT_BEGIN) {
                const uint32_t slot = ins.y & 0xFFFFu, r = ins.y >> 16;
                bool need = valid;
                if (a.use_cache && valid) {
                    float4 rec = a.probes[(size_t)pbase + (size_t)r * cnt + j];
                    if (__float_as_uint(rec.w) == PROBE_HIT) {
                        V[(slot * 3 + 0) * 32] = rec.x;
                        V[(slot * 3 + 1) * 32] = rec.y;
                        V[(slot * 3 + 2) * 32] = rec.z;
                        hits++;
                        need = false;
                    } else {
                        cand_cell = __float_as_uint(rec.x);
                        cand_h2 = __float_as_uint(rec.y);
                        cand_node = ins.z;
                    }
                }
                if (!need) skip_end = pc + (int)ins.w;
                if (__all_sync(FULL_MASK, !need)) pc += (int)ins.w;
                continue;
            }
            const bool act = valid && pc > skip_end;
            const uint32_t out = ins.y & 0xFFFFu;
            const uint32_t i0 = ins.y >> 16, i1 = ins.z & 0xFFFFu, i2 = ins.z >> 16;
            const float* p = a.params + ins.w;
            if (act) {
                float r0 = 0.f, r1 = 0.f, r2 = 0.f;
                switch (op) {
                case PMC_OP_UV: r0 = u; r1 = v; break;
                case PMC_OP_POSITION: r0 = px; r1 = py; r2 = pz; break;
                case PMC_OP_NORMAL: r0 = nx; r1 = ny; r2 = nz; break;
                case PMC_OP_CONST: r0 = __ldg(&p[0]); r1 = __ldg(&p[1]); r2 = __ldg(&p[2]); break;
                case PMC_OP_UV_AFFINE: {
                    float x = V[(i0 * 3) * 32], y = V[(i0 * 3 + 1) * 32];
                    r0 = fmaf(__ldg(&p[0]), x, fmaf(__ldg(&p[1]), y, __ldg(&p[4])));
                    r1 = fmaf(__ldg(&p[2]), x, fmaf(__ldg(&p[3]), y, __ldg(&p[5])));
                    break;
                }
                case PMC_OP_FBM: {
                    float pp[6];
#pragma unroll
                    for (int k = 0; k < 6; ++k) pp[k] = __ldg(&p[k]);
                    r0 = r1 = r2 = d_fbm(V[(i0 * 3) * 32], V[(i0 * 3 + 1) * 32], pp);
                    break;
                }
                case PMC_OP_VORONOI: {
                    float pp[2] = {__ldg(&p[0]), __ldg(&p[1])};
                    r0 = r1 = r2 = d_voronoi(V[(i0 * 3) * 32], V[(i0 * 3 + 1) * 32], pp);
                    break;
                }
                case PMC_OP_CHECKER: {
                    float sc = __ldg(&p[0]);
                    long long k = (long long)floorf(V[(i0 * 3) * 32] * sc) + (long long)floorf(V[(i0 * 3 + 1) * 32] * sc);
                    const float* c = (k & 1) ? p + 4 : p + 1;
                    r0 = d_clamp01(__ldg(&c[0])); r1 = d_clamp01(__ldg(&c[1])); r2 = d_clamp01(__ldg(&c[2]));
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
                    float d = fmaf(V[(i0 * 3) * 32], __ldg(&p[0]),
                                   fmaf(V[(i0 * 3 + 1) * 32], __ldg(&p[1]), V[(i0 * 3 + 2) * 32] * __ldg(&p[2])));
                    r0 = r1 = r2 = d_clamp01(fabsf(d));
                    break;
                }
                default:
                    break;
                }
                V[(out * 3) * 32] = r0;
                V[(out * 3 + 1) * 32] = r1;
                V[(out * 3 + 2) * 32] = r2;
                n_nodes++;
                n_flops += ins.x >> 16;
            }
            if (a.use_cache && ((ins.x >> 8) & FLAG_ROOT)) {
                // a missed cacheable node was evaluated: offer it to the table (Sec. 3)
                const bool emit = act;
                uint32_t idx = warp_append(&a.ctl->n_cand, emit);
                if (emit) {
                    Candidate c;
                    c.prio = ((unsigned long long)orig << 16) | cand_node;
                    c.cell = cand_cell;
                    c.h2 = cand_h2;
                    c.r = V[(out * 3) * 32];
                    c.g = V[(out * 3 + 1) * 32];
                    c.b = V[(out * 3 + 2) * 32];
                    c.target = 0;
                    if (idx < a.probe_cap) a.cands[idx] = c;
                    else atomicOr(&a.ctl->err, ERR_BOUNDS);
                }
            }
        }
        if (valid) {
            a.out_rgb[orig] = V[(mi.out_slot * 3) * 32];
            a.out_rgb[(size_t)a.n + orig] = V[(mi.out_slot * 3 + 1) * 32];
            a.out_rgb[2 * (size_t)a.n + orig] = V[(mi.out_slot * 3 + 2) * 32];
            if (a.out_hits) a.out_hits[orig] = (uint16_t)min(hits, 65535u);
        }
    }
    warp_add_u64(&a.stats[ST_NODES], n_nodes);
    warp_add_u64(&a.stats[ST_FLOPS], n_flops);
}

// =======================================================================================
// Insert (Alg. 1 semantics, deterministic): rounds of claim / resolve
// =======================================================================================
__device__ __forceinline__ unsigned long long claim_word(uint32_t epoch, unsigned long long prio) {
    return ((unsigned long long)(EPOCH_MAX - epoch) << 44) | prio;
}

__global__ void k_claim(BatchArgs a, uint32_t round, int final_round) {
    const uint32_t n_in = round == 0 ? min(a.ctl->n_cand, a.probe_cap) : a.ctl->out_count[round - 1];
    const uint32_t* list_in = round == 0 ? nullptr : a.lists[(round - 1) & 1u];
    const uint32_t epoch = a.ctl->epoch + round;
    const uint32_t ne = a.n_entries;
    uint32_t stride = gridDim.x * blockDim.x;
    uint32_t n_round = (n_in + 31u) & ~31u;
    unsigned long long n_dup = 0, n_full = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        bool act = i < n_in;
        bool live = false;
        uint32_t idx = 0;
        if (act) {
            idx = list_in ? list_in[i] : i;
            Candidate c = a.cands[idx];
            const uint4* cell = a.table + (size_t)c.cell * ne;
            int target = -1;
            bool dup = false;
            for (uint32_t e = 0; e < ne; ++e) {
                uint32_t h = cell[e].x;   // plain load: earlier rounds wrote the table
                if (h == c.h2) { dup = true; break; }
                if (h == 0u) { target = (int)e; break; }
            }
            if (dup) n_dup++;
            else if (target < 0) n_full++;
            else if (final_round) atomicOr(&a.ctl->err, ERR_INSERT);
            else {
                a.cands[idx].target = (uint32_t)target;
                atomicMin(&a.claims[c.cell], claim_word(epoch, c.prio));
                live = true;
            }
        }
        uint32_t pos = warp_append(&a.ctl->mid_count[round], live);
        if (live) a.lists[2][pos] = idx;
    }
    warp_add_u64(&a.stats[ST_DUP], n_dup);
    warp_add_u64(&a.stats[ST_FULL], n_full);
}

__global__ void k_resolve(BatchArgs a, uint32_t round) {
    const uint32_t n_mid = a.ctl->mid_count[round];
    const uint32_t epoch = a.ctl->epoch + round;
    uint32_t* list_out = a.lists[round & 1u];
    uint32_t stride = gridDim.x * blockDim.x;
    uint32_t n_round = (n_mid + 31u) & ~31u;
    unsigned long long n_ins = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        bool act = i < n_mid;
        bool lose = false;
        uint32_t idx = 0;
        if (act) {
            idx = a.lists[2][i];
            const Candidate c = a.cands[idx];
            if (a.claims[c.cell] == claim_word(epoch, c.prio)) {
                a.table[(size_t)c.cell * a.n_entries + c.target] =
                    make_uint4(c.h2, __float_as_uint(c.r), __float_as_uint(c.g), __float_as_uint(c.b));
                n_ins++;
            } else {
                lose = true;
            }
        }
        uint32_t pos = warp_append(&a.ctl->out_count[round], lose);
        if (lose) list_out[pos] = idx;
    }
    warp_add_u64(&a.stats[ST_INSERTED], n_ins);
}

__global__ void k_finish(BatchArgs a) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        uint32_t nc = min(a.ctl->n_cand, a.probe_cap);
        if (a.use_cache) a.ctl->epoch += a.n_entries + 1u;
        a.stats[ST_CANDIDATES] += nc;
        a.stats[ST_BATCHES] += 1ull;
    }
}

// =======================================================================================
// Stand-alone key computation (parity checks of descriptors and addressing)
// =======================================================================================
__global__ void k_keys(const uint32_t* mat, const uint32_t* node, const float* u, const float* v,
                       uint64_t n, uint32_t level, uint64_t n_cells, uint32_t pow2_mask,
                       uint64_t* key, uint64_t* cell, uint32_t* h2) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = d_key(mat[i], node[i], level, d_texel(u[i], level), d_texel(v[i], level));
        uint32_t c, h;
        d_address(k, n_cells, pow2_mask, &c, &h);
        key[i] = k;
        cell[i] = c;
        h2[i] = h;
    }
}

// =======================================================================================
// Host-side launch sequences
// =======================================================================================
cudaError_t launch_keys(const uint32_t* mat, const uint32_t* node, const float* u, const float* v,
                        uint64_t n, uint32_t level, uint64_t n_cells, uint64_t* key, uint64_t* cell,
                        uint32_t* h2, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    uint32_t mask = (n_cells && (n_cells & (n_cells - 1)) == 0 && n_cells <= (1ull << 32)) ? (uint32_t)(n_cells - 1) : 0u;
    if (n_cells == 1) mask = 0;  // h1 % 1 == 0 either way
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_keys<<<(unsigned)blocks, 256, 0, s>>>(mat, node, u, v, n, level, n_cells, mask, key, cell, h2);
    return cudaGetLastError();
}

cudaError_t launch_reset(uint4* table, size_t slots, unsigned long long* claims, size_t cells,
                         Control* ctl, unsigned long long* stats, cudaStream_t s) {
    cudaError_t e;
    if (slots && (e = cudaMemsetAsync(table, 0, slots * sizeof(uint4), s)) != cudaSuccess) return e;
    if (cells && (e = cudaMemsetAsync(claims, 0xFF, cells * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ctl, 0, sizeof(Control), s)) != cudaSuccess) return e;
    return cudaMemsetAsync(stats, 0, ST_COUNT * sizeof(unsigned long long), s);
}

cudaError_t launch_batch(const BatchArgs& a, cudaStream_t s, int num_sms, cudaEvent_t* ev,
                         uint64_t* launches) {
    cudaError_t e;
    uint64_t nl = 0;
    auto mark = [&](int k) { return ev ? cudaEventRecord(ev[k], s) : cudaSuccess; };
    if ((e = mark(0)) != cudaSuccess) return e;
    // per-batch counters: items, probes, candidates, round counts (epoch and err persist)
    if ((e = cudaMemsetAsync(a.ctl, 0, 3 * sizeof(uint32_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.ctl->mid_count, 0, 2 * (MAX_ENTRIES + 2) * sizeof(uint32_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.counts, 0, (a.n_mats + 1) * sizeof(uint32_t), s)) != cudaSuccess) return e;
    // counts has n_mats + 1 entries; the last one is the eval work-item counter
    uint32_t* item_ctr = a.counts + a.n_mats;
    const int gs_blocks = num_sms * 4;
    if (a.n > 0) {
        k_hist<<<gs_blocks, 256, 0, s>>>(a);
        nl++;
    }
    k_scan<<<1, 1024, 0, s>>>(a);
    nl++;
    if (a.n > 0) {
        k_scatter<<<gs_blocks, 256, 0, s>>>(a);
        nl++;
    }
    if ((e = mark(1)) != cudaSuccess) return e;
    if (a.n > 0 && a.use_cache) {
        uint32_t ne = a.n_entries;
        int lb = num_sms * 8;
        if (ne <= 4) k_lookup<4><<<lb, 256, 0, s>>>(a);
        else if (ne <= 8) k_lookup<8><<<lb, 256, 0, s>>>(a);
        else if (ne <= 16) k_lookup<16><<<lb, 256, 0, s>>>(a);
        else k_lookup<32><<<lb, 256, 0, s>>>(a);
        nl++;
    }
    if ((e = mark(2)) != cudaSuccess) return e;
    if (a.n > 0) {
        size_t smem = eval_smem_bytes(a.max_slots);
        if (smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(k_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        k_eval<<<num_sms * 16, EVAL_WARPS * 32, smem, s>>>(a, item_ctr);
        nl++;
    }
    if ((e = mark(3)) != cudaSuccess) return e;
    if (a.n > 0 && a.use_cache) {
        for (uint32_t r = 0; r < a.n_entries; ++r) {
            k_claim<<<gs_blocks, 256, 0, s>>>(a, r, 0);
            k_resolve<<<gs_blocks, 256, 0, s>>>(a, r);
            nl += 2;
        }
        k_claim<<<gs_blocks, 256, 0, s>>>(a, a.n_entries, 1);
        nl++;
    }
    if ((e = mark(4)) != cudaSuccess) return e;
    k_finish<<<1, 32, 0, s>>>(a);
    nl++;
    if ((e = mark(5)) != cudaSuccess) return e;
    if (launches) *launches += nl;
    return cudaGetLastError();
}

}  // namespace pmc
