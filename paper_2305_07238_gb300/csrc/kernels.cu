// kernels.cu -- sm_103a kernels of one progressive pass (Sec. 3, Alg. 1).
//
//   k_hist     material histogram of the batch (+ range check of material indices)
//   k_scan     per-material segment offsets, probe offsets and warp work items
//   k_scatter  groups the points by material into structure-of-arrays copies
//   k_lookup   probes of every (point, cacheable node) against the table as it was
//              when the pass started (Sec. 3.2, Fig. 3); several probes in flight per lane
//   k_scan_roots / k_eval_roots
//              the missed cacheable nodes, listed per node by k_lookup, evaluated 32 at a
//              time with each node's standalone program; values go back into the probe
//              records and become insert candidates (Sec. 3)
//   k_eval     warp-uniform interpreter of the material programs (Sec. 2); every cached
//              or computed block is skipped by the whole warp
//   k_insert   rounds of the insert in one cooperative launch: every live candidate
//              targets the first slot of its cell holding its hash2 (duplicate) or 0
//              (free, Alg. 1); the smallest (point index, node ID) per cell wins by
//              atomicMin and writes its slot
//   k_finish   advances the claim epoch and the batch counters
#include <algorithm>
#include <cstddef>
#include <cstdio>

#include "nodes.cuh"
#include "pmc_internal.h"

namespace pmc {

#define FULL_MASK 0xFFFFFFFFu

// =======================================================================================
// Small helpers
// =======================================================================================
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ void warp_add_u64(unsigned long long* dst, unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    if (lane_id() == 0 && v) atomicAdd(dst, v);
}

__device__ __forceinline__ void warp_add_u32(uint32_t* dst, uint32_t v) {
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
// Materials counted in shared memory per block; beyond this the counters are global.
constexpr uint32_t GROUP_SMEM_MATS = 4096;
// grouping kernels (k_hist, k_scatter): eight blocks of 256 threads per SM, the SM's full
// thread capacity, so that each block's range is short and the memory latency of its
// dependent count / reserve / scatter steps is hidden by the other blocks
constexpr int GROUP_BLOCKS_PER_SM = 8;

// Points of block b: the contiguous range [b * chunk, min(n, (b + 1) * chunk)).
__device__ __forceinline__ void block_range(uint32_t n, uint32_t* lo, uint32_t* hi) {
    const uint32_t chunk = ((n + gridDim.x - 1) / gridDim.x + 31u) & ~31u;
    *lo = min(n, blockIdx.x * chunk);
    *hi = min(n, *lo + chunk);
}

// Inclusive scan of one value per thread over the block (blockDim.x a multiple of 32, at
// most 1024) with warp shuffles and two block barriers; tmp holds 33 values of shared
// memory, *total receives the block's sum.  Every thread of the block must call it.
template <typename U>
__device__ __forceinline__ U block_incl_scan(U v, U* tmp, U* total) {
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    U x = v;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const U y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const U w = lane < nw ? tmp[lane] : U(0);
        U wi = w;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const U y = __shfl_up_sync(FULL_MASK, wi, o);
            if (lane >= o) wi += y;
        }
        tmp[lane] = wi - w;
        if (lane == 31) tmp[32] = wi;
    }
    __syncthreads();
    const U r = x + tmp[warp];
    *total = tmp[32];
    __syncthreads();   // tmp is free for the next call
    return r;
}

__global__ void __launch_bounds__(256) k_hist(BatchArgs a) {
    __shared__ uint32_t s_cnt[GROUP_SMEM_MATS];
    const bool local = a.n_mats <= GROUP_SMEM_MATS;
    if (local) {
        for (uint32_t m = threadIdx.x; m < a.n_mats; m += blockDim.x) s_cnt[m] = 0;
        __syncthreads();
    }
    uint32_t lo, hi;
    block_range(a.n, &lo, &hi);
    unsigned long long bad = 0;
    const uint32_t hi32 = (hi + 31u) & ~31u;
    // four material ids in flight per thread (a warp's indices are consecutive and 32-aligned,
    // so the bound checks are uniform over the warp)
    for (uint32_t i0 = lo + threadIdx.x; i0 < hi32 && lo < hi; i0 += 4u * blockDim.x) {
        uint32_t mm[4];
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t i = i0 + k * blockDim.x;
            mm[k] = i < hi ? a.mat[i] : 0u;
        }
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t i = i0 + k * blockDim.x;
            if (i >= hi32) break;
            const bool act = i < hi;
            const uint32_t m = mm[k];
            const bool ok = act && m < a.n_mats;
            if (act && !ok) bad++;
            const unsigned vmask = __ballot_sync(FULL_MASK, ok);
            if (ok) {
                const unsigned peers = __match_any_sync(vmask, m);
                const int leader = __ffs(peers) - 1;
                if ((int)lane_id() == leader) atomicAdd(local ? &s_cnt[m] : &a.counts[m], (uint32_t)__popc(peers));
            }
        }
    }
    if (local) {
        __syncthreads();
        for (uint32_t m = threadIdx.x; m < a.n_mats; m += blockDim.x)
            if (s_cnt[m]) atomicAdd(&a.counts[m], s_cnt[m]);
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
    __shared__ uint32_t s_tmp[33];
    const uint32_t T = blockDim.x, t = threadIdx.x;
    const uint32_t per = (a.n_mats + T - 1) / T;
    const uint32_t lo = min(t * per, a.n_mats), hi = min(lo + per, a.n_mats);
    // probes are laid out for every cacheable node (surrogate ones get their record from
    // the surrogate instead of a lookup)
    const bool surr = a.surr_slot != nullptr;
    uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    for (uint32_t m = lo; m < hi; ++m) {
        uint32_t c = a.counts[m];
        uint32_t k = (a.use_cache || surr) ? a.mats[m].n_roots : 0u;
        c0 += c;
        c1 += c * k;
        c2 += (c + 31u) >> 5;
        c3 += (surr && a.surr_slot[m] >= 0) ? (c + 127u) >> 7 : 0u;
    }
    uint32_t tot0, tot1, tot2, tot3;
    uint32_t b0 = block_incl_scan(c0, s_tmp, &tot0) - c0;
    uint32_t b1 = block_incl_scan(c1, s_tmp, &tot1) - c1;
    uint32_t b2 = block_incl_scan(c2, s_tmp, &tot2) - c2;
    uint32_t b3 = block_incl_scan(c3, s_tmp, &tot3) - c3;
    for (uint32_t m = lo; m < hi; ++m) {
        uint32_t c = a.counts[m];
        uint32_t k = (a.use_cache || surr) ? a.mats[m].n_roots : 0u;
        a.seg_start[m] = b0;
        a.cursor[m] = b0;
        a.probe_base[m] = b1;
        a.item_base[m] = b2;
        if (surr) a.surr_item_base[m] = b3;
        b0 += c;
        b1 += c * k;
        b2 += (c + 31u) >> 5;
        b3 += (surr && a.surr_slot[m] >= 0) ? (c + 127u) >> 7 : 0u;
    }
    if (t == T - 1) {
        a.seg_start[a.n_mats] = tot0;
        a.probe_base[a.n_mats] = tot1;
        a.item_base[a.n_mats] = tot2;
        if (surr) a.surr_item_base[a.n_mats] = tot3;
        a.ctl->n_surr_items = surr ? tot3 : 0u;
        a.ctl->n_items = tot2;
        a.ctl->total_probes = tot1;
        if (tot1 > a.probe_cap) {
            // more probe records than the scratch holds: the batch does no work and the
            // next synchronising call reports it
            a.ctl->n_items = 0;
            a.ctl->n_surr_items = 0;
            atomicOr(&a.ctl->err, ERR_CAPACITY);
        }
        atomicAdd(&a.stats[ST_POINTS], (unsigned long long)a.n);
    }
}

__device__ __forceinline__ void zero_output(const BatchArgs& a, uint32_t i) {
    // out-of-range material: zero output, no probes
    a.out_rgb[i] = 0.0f;
    a.out_rgb[(size_t)a.n + i] = 0.0f;
    a.out_rgb[2 * (size_t)a.n + i] = 0.0f;
    if (a.out_hits) a.out_hits[i] = 0;
}

// Groups the block's contiguous range of points by material.  With few materials the
// block counts its points per material in shared memory, reserves one range per
// material with a single global atomic, then hands out positions from shared counters.
__global__ void __launch_bounds__(256) k_scatter(BatchArgs a) {
    __shared__ uint32_t s_cnt[GROUP_SMEM_MATS];
    const bool local = a.n_mats <= GROUP_SMEM_MATS;
    uint32_t lo, hi;
    block_range(a.n, &lo, &hi);
    const uint32_t hi32 = (hi + 31u) & ~31u;
    if (local) {
        for (uint32_t m = threadIdx.x; m < a.n_mats; m += blockDim.x) s_cnt[m] = 0;
        __syncthreads();
        // four material ids in flight per thread; a warp's 32 indices are consecutive and
        // 32-aligned, so the bound checks are uniform over the warp
        for (uint32_t i0 = lo + threadIdx.x; i0 < hi32 && lo < hi; i0 += 4u * blockDim.x) {
            uint32_t mm[4];
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                const uint32_t i = i0 + k * blockDim.x;
                mm[k] = i < hi ? a.mat[i] : 0xFFFFFFFFu;
            }
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                if (i0 + k * blockDim.x >= hi32) break;
                const bool ok = mm[k] < a.n_mats;
                const unsigned vmask = __ballot_sync(FULL_MASK, ok);
                if (ok) {
                    const unsigned peers = __match_any_sync(vmask, mm[k]);
                    if ((int)lane_id() == __ffs(peers) - 1) atomicAdd(&s_cnt[mm[k]], (uint32_t)__popc(peers));
                }
            }
        }
        __syncthreads();
        // the block's first position in each material segment
        for (uint32_t m = threadIdx.x; m < a.n_mats; m += blockDim.x)
            if (s_cnt[m]) s_cnt[m] = atomicAdd(&a.cursor[m], s_cnt[m]);
        __syncthreads();
    }
    for (uint32_t i = lo + threadIdx.x; i < hi32 && lo < hi; i += blockDim.x) {
        const bool act = i < hi;
        const uint32_t m = act ? a.mat[i] : 0u;
        const bool ok = act && m < a.n_mats;
        // the point's fields are loaded before its position is known, so that the loads
        // overlap the match and the reservation
        PointIn p{0, 0, 0, 0, 0, 0, 0, 0};
        uint32_t lev = 0;
        if (ok) {
            p.u = a.u[i]; p.v = a.v[i];
            p.px = a.px[i]; p.py = a.py[i]; p.pz = a.pz[i];
            p.nx = a.nx[i]; p.ny = a.ny[i]; p.nz = a.nz[i];
            if (a.g1u) lev = d_level(a.g1u[i], a.g1v[i], a.g2u[i], a.g2v[i], a.level_offset);
        }
        const unsigned vmask = __ballot_sync(FULL_MASK, ok);
        if (ok) {
            const unsigned peers = __match_any_sync(vmask, m);
            const int leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if ((int)lane_id() == leader)
                base = atomicAdd(local ? &s_cnt[m] : &a.cursor[m], (uint32_t)__popc(peers));
            base = __shfl_sync(peers, base, leader);
            const uint32_t pos = base + __popc(peers & ((1u << lane_id()) - 1u));
            a.su[pos] = p.u; a.sv[pos] = p.v;
            a.spx[pos] = p.px; a.spy[pos] = p.py; a.spz[pos] = p.pz;
            a.snx[pos] = p.nx; a.sny[pos] = p.ny; a.snz[pos] = p.nz;
            a.sidx[pos] = i;
            if (a.g1u) a.slev[pos] = lev;
        } else if (act) {
            zero_output(a, i);
        }
    }
}

// =======================================================================================
// Lookup (Sec. 3.2).  Table cell c (16 * N_e bytes): N_e hash2 words, then N_e packed
// (r, g, b) values.  A probe reads the cell's hash2 words (one 32-byte sector for N_e = 8)
// and, on a hit, the 12 bytes of the matching value in the same line.
// =======================================================================================
__device__ __forceinline__ uint32_t* cell_h2(const BatchArgs& a, uint32_t cell) {
    return reinterpret_cast<uint32_t*>(a.table) + (size_t)cell * 4u * a.n_entries;
}
__device__ __forceinline__ float* cell_val(const BatchArgs& a, uint32_t cell, uint32_t j) {
    return reinterpret_cast<float*>(a.table) + (size_t)cell * 4u * a.n_entries + a.n_entries + 3u * j;
}
constexpr uint32_t PROBE_MISS = 0u;   // record {cell, hash2, first empty slot, 0}
constexpr uint32_t PROBE_HIT = 1u;    // record {r, g, b, 1}
constexpr uint32_t PROBE_FULL = 2u;   // record {cell, hash2, N_e, 2}: the cell cannot take the value

// Replacement by visibility class: a full cell whose entries all have classes at most q can
// never take a value of class q in this batch (a full cell's classes only decrease).
__device__ __forceinline__ bool cell_closed(const BatchArgs& a, uint32_t cell, uint32_t q) {
    const uint8_t* cc = a.slot_cls + (size_t)cell * a.n_entries;
    uint32_t mx = 0;
    for (uint32_t e = 0; e < a.n_entries; ++e) mx = max(mx, (uint32_t)__ldg(&cc[e]));
    return mx <= q;
}


// Scans the hash2 words of a cell held in registers: first slot holding h2 (hit) or 0.
template <int NQ>
__device__ __forceinline__ int scan_words(const uint4 (&w)[NQ], uint32_t h2, uint32_t ne, bool* hit) {
    int first = -1;
    *hit = false;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const uint32_t v[4] = {w[q].x, w[q].y, w[q].z, w[q].w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t idx = 4u * q + k;
            if (first < 0 && idx < ne && (v[k] == h2 || v[k] == 0u)) {
                first = (int)idx;
                *hit = v[k] == h2;
            }
        }
    }
    return first;
}

// NQ = 16-byte words of hash2 per cell (ceil(N_e / 4)); RB probes in flight per lane; POS:
// the cache has the world-position descriptor (a separate instantiation, so that caches
// without it keep the registers the position keys would take).
// Each group of RB probes takes two dependent round trips to memory, both fully
// overlapped across the group: first every probe's hash2 words, then the values of
// the hits.  Records and miss lists are written after both.
template <int NQ, int RB, bool POS>
__global__ void __launch_bounds__(256, 4) k_lookup(BatchArgs a) {
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t warps_total = gridDim.x * (blockDim.x >> 5);
    const uint32_t n_items = a.ctl->n_items;
    const uint32_t ne = a.n_entries;
    unsigned long long n_look = 0, n_hit = 0, n_slots = 0;
    for (uint32_t item = blockIdx.x * (blockDim.x >> 5) + warp; item < n_items; item += warps_total) {
        const uint32_t m = find_material(a.item_base, a.n_mats, item);
        const uint32_t cnt = __ldg(&a.counts[m]);
        const uint32_t j = (item - __ldg(&a.item_base[m])) * 32u + lane;
        const bool valid = j < cnt;
        const uint32_t s = __ldg(&a.seg_start[m]) + j;
        uint32_t iu = 0, iv = 0, lev = a.level;
        float px = 0.f, py = 0.f, pz = 0.f;
        if (valid) {
            if (a.g1u) lev = a.slev[s];
            iu = d_texel(a.su[s], lev);
            iv = d_texel(a.sv[s], lev);
            if (POS) {
                px = a.spx[s];
                py = a.spy[s];
                pz = a.spz[s];
            }
        }
        const MatInfo mi = a.mats[m];
        const int32_t surr = a.surr_ord ? a.surr_ord[m] : -1;   // a surrogate's node is not probed
        const size_t rec0 = (size_t)__ldg(&a.probe_base[m]) + j;
        // replacement: the point's visibility class decides whether a full cell is closed
        const uint32_t q = (a.slot_cls && a.vis && valid) ? (uint32_t)__ldg(&a.vis[a.sidx[s]]) : 0u;
        for (uint32_t r0 = 0; r0 < mi.n_roots; r0 += RB) {
            uint4 w[RB][NQ];
            uint32_t cell[RB], h2[RB];
            bool act[RB];
            // round trip 1: the hash2 words of every probe of the group
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                act[b] = valid && r0 + b < mi.n_roots && (int32_t)(r0 + b) != surr;
                cell[b] = 0;
                h2[b] = 0;
                if (act[b]) {
                    const uint32_t node = __ldg(&a.roots[mi.root_base + r0 + b]);
                    const uint64_t key = (POS && (node & ROOT_POS_BIT))
                                             ? d_key_pos(m, node & 0xFFFFu, (uint32_t)a.pos_level, px, py, pz)
                                             : d_key(m, node, lev, iu, iv);
                    d_address(key, a.n_cells, a.cells_pow2_mask, &cell[b], &h2[b]);
                }
                const uint4* hw = reinterpret_cast<const uint4*>(cell_h2(a, cell[b]));
                const bool ld = act[b] && !a.table_empty;   // an empty table misses at slot 0
#pragma unroll
                for (int q = 0; q < NQ; ++q) w[b][q] = ld ? __ldg(hw + q) : make_uint4(0, 0, 0, 0);
            }
            // round trip 2: the values of the hits
            int first[RB];
            bool hit[RB];
            float v[RB][3];
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                first[b] = scan_words<NQ>(w[b], h2[b], ne, &hit[b]);
                hit[b] = hit[b] && act[b];
                const float* val = cell_val(a, cell[b], hit[b] ? (uint32_t)first[b] : 0u);
                v[b][0] = hit[b] ? __ldg(val) : 0.0f;
                v[b][1] = hit[b] ? __ldg(val + 1) : 0.0f;
                v[b][2] = hit[b] ? __ldg(val + 2) : 0.0f;
            }
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                if (r0 + b >= mi.n_roots) break;                 // uniform in the warp
                if ((int32_t)(r0 + b) == surr) continue;          // uniform
                const size_t rec = rec0 + (size_t)(r0 + b) * cnt;
                if (valid) {
                    n_look++;
                    n_slots += first[b] >= 0 ? (uint32_t)first[b] + 1u : ne;
                    if (hit[b]) {
                        a.probes[rec] = make_float4(v[b][0], v[b][1], v[b][2], __uint_as_float(PROBE_HIT));
                        n_hit++;
                    } else {
                        bool full = first[b] < 0;
                        if (full && a.slot_cls) full = cell_closed(a, cell[b], q);
                        a.probes[rec] = make_float4(__uint_as_float(cell[b]), __uint_as_float(h2[b]),
                                                    __uint_as_float(first[b] >= 0 ? (uint32_t)first[b] : ne),
                                                    __uint_as_float(full ? PROBE_FULL : PROBE_MISS));
                    }
                }
                if (a.split) {
                    // list the misses of this cacheable node for the batched evaluation
                    const bool miss = valid && !hit[b];
                    const unsigned mm = __ballot_sync(FULL_MASK, miss);
                    if (mm) {
                        const int leader = __ffs(mm) - 1;
                        uint32_t base = 0;
                        if ((int)lane == leader) base = atomicAdd(&a.miss_cnt[mi.root_base + r0 + b], (uint32_t)__popc(mm));
                        base = __shfl_sync(FULL_MASK, base, leader);
                        if (miss)
                            a.misslist[rec0 - j + (size_t)(r0 + b) * cnt + base + __popc(mm & ((1u << lane) - 1u))] = j;
                    }
                }
            }
        }
    }
    warp_add_u64(&a.stats[ST_LOOKUPS], n_look);
    warp_add_u64(&a.stats[ST_HITS], n_hit);
    warp_add_u64(&a.stats[ST_MISSES], n_look - n_hit);
    warp_add_u64(&a.stats[ST_SLOTS], n_slots);
}

// =======================================================================================
// Evaluation (Sec. 2, Sec. 3)
// =======================================================================================
constexpr uint32_t PROBE_COMPUTED = 3u;   // record {r, g, b, 3}: a miss evaluated this pass
constexpr uint32_t EVAL_WARPS = 4;

size_t eval_smem_bytes(uint32_t max_slots) {
    return (size_t)EVAL_WARPS * max_slots * 3u * 32u * sizeof(float);
}

// Largest slot file (bytes per block) with which the two-points-per-lane evaluator runs:
// six blocks of its size fit an SM's shared memory.
constexpr size_t EVAL2_MAX_SMEM = 36 * 1024;

// Offers the lanes' freshly evaluated cacheable-node values to the table (Sec. 3).
// `full`: the cell cannot take the value in this batch, so it is counted as dropped
// without becoming a candidate.  Keep-first: the cell was full at lookup (nothing is
// evicted), and lanes carrying the same (cell, hash2) collapse onto the smallest point
// index; the others share its fate.  Replacement by visibility class: the cell was full
// at lookup of entries of classes at most the point's own; every other value becomes a
// candidate of its own, since copies of one key with different classes can meet different
// fates, and its dup scan starts at slot 0, since an eviction can put the key anywhere in
// the cell.  Must be called by all 32 lanes.
__device__ __forceinline__ void offer(const BatchArgs& a, bool act, uint32_t orig, uint32_t node, uint32_t cell,
                                      uint32_t h2, uint32_t start, bool full, float r, float g, float b,
                                      unsigned long long* n_cand, unsigned long long* n_full) {
    const bool replace = a.slot_cls != nullptr;   // uniform
    *n_cand += act ? 1u : 0u;
    *n_full += (act && full) ? 1u : 0u;
    const bool emit = act && !full;
    bool winner = false;
    uint32_t shadows = 0;
    const unsigned em = __ballot_sync(FULL_MASK, emit);
    if (emit && replace) {
        winner = true;
        start = 0;
    } else if (emit) {
        const unsigned long long k64 = ((unsigned long long)cell << 32) | h2;
        const unsigned grp = __match_any_sync(em, k64);
        const uint32_t mn = __reduce_min_sync(grp, orig);
        winner = orig == mn;
        shadows = (uint32_t)__popc(grp) - 1u;
    }
    const uint32_t idx = warp_append(&a.ctl->n_cand, winner);
    if (winner) {
        const uint32_t q = (replace && a.vis) ? (uint32_t)__ldg(&a.vis[orig]) : 0u;
        Candidate c;
        c.prio = ((unsigned long long)orig << 16) | node;
        c.cell = cell;
        c.h2 = h2;
        c.r = r;
        c.g = g;
        c.b = b;
        c.target = start | (q << 8) | (shadows << 16);
        if (idx < a.probe_cap) {
            a.cands[idx] = c;
            if (!a.insert_rounds) a.lists[0][idx] = cell;   // compact cells for the binning
        } else {
            atomicOr(&a.ctl->err, ERR_CAPACITY);
        }
    }
}

// EVAL_FILL: the pass on an empty table without surrogates.  Every probe would miss at slot
// 0, so every lane runs the whole program (as EVAL_PLAIN) and offers each cacheable node's
// value under its descriptor as it is computed; the counters of the skipped lookups are
// those of EVAL_GENERIC's inline descriptors (one lookup, one miss, one empty slot).
struct FillStats {
    unsigned long long n_cand = 0, n_full = 0, n_look = 0;
};

// Offers the value (r, g, b) of cacheable node `node` at grouped point s (act: a valid
// point); the point's level, texel and batch index are read here, where they are needed.
__device__ __forceinline__ void fill_offer(const BatchArgs& a, bool act, uint32_t s, uint32_t m, uint32_t node, bool pos,
                                           const PointIn& p, float r, float g, float b, FillStats* fs) {
    uint32_t cell = 0, h2 = 0, orig = 0;
    if (act) {
        uint64_t key;
        if (pos) {
            key = d_key_pos(m, node, (uint32_t)a.pos_level, p.px, p.py, p.pz);
        } else {
            const uint32_t lev = a.g1u ? (uint32_t)a.slev[s] : a.level;
            key = d_key(m, node, lev, d_texel(p.u, lev), d_texel(p.v, lev));
        }
        d_address(key, a.n_cells, a.cells_pow2_mask, &cell, &h2);
        orig = a.sidx[s];
        fs->n_look++;
    }
    offer(a, act, orig, node, cell, h2, 0u, false, r, g, b, &fs->n_cand, &fs->n_full);
}

// Per-point interpreter: one warp runs one material's program for 32 grouped points.
// EVAL_OUTER: every cacheable node already has its value in its probe record (a hit, a
//   value computed by k_eval_roots or a learned surrogate), so the outer program runs:
//   each block replaced by a load of its node's record.
// EVAL_PLAIN: the cache is off; the whole program runs for every point.
// EVAL_FILL: the first pass on an empty table without surrogates (two points per lane only;
//   see fill_offer).
// EVAL_GENERIC: the whole program with per-lane skipping: the first pass on an empty table
//   (descriptors formed here, every cacheable node offered), the inline evaluation of
//   misses (a lane whose lookup hit skips the block), learned surrogates on that pass.
// In the first two modes every lane runs every instruction: a lane past the end of its
// material's points shadows the segment's last point and stores nothing, and the node and
// operation counts come from the program's totals.
enum { EVAL_OUTER = 0, EVAL_PLAIN = 1, EVAL_GENERIC = 2, EVAL_FILL = 3 };

template <int MODE>
__global__ void __launch_bounds__(EVAL_WARPS * 32) k_eval(BatchArgs a, uint32_t* item_ctr) {
    extern __shared__ float s_val[];
    __shared__ float2 s_grad[8];
    init_gradients(s_grad);
    __syncthreads();
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    constexpr bool outer = MODE == EVAL_OUTER;
    char* Vb = reinterpret_cast<char*>(s_val + (size_t)warp * (outer ? a.max_slots_outer : a.max_slots) * 96u + lane);
    const uint32_t n_items = a.ctl->n_items;
    unsigned long long n_nodes = 0, n_flops = 0, n_cand = 0, n_full = 0, n_look = 0;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(item_ctr, 1u);
        item = __shfl_sync(FULL_MASK, item, 0);
        if (item >= n_items) break;
        const uint32_t m = find_material(a.item_base, a.n_mats, item);
        const uint32_t cnt = __ldg(&a.counts[m]);
        const uint32_t j = (item - __ldg(&a.item_base[m])) * 32u + lane;
        const bool valid = j < cnt;
        const uint32_t jj = valid ? j : cnt - 1u;   // an item holds at least one point
        const uint32_t s = __ldg(&a.seg_start[m]) + jj;
        PointIn pt;
        pt.u = a.su[s]; pt.v = a.sv[s];
        pt.px = a.spx[s]; pt.py = a.spy[s]; pt.pz = a.spz[s];
        pt.nx = a.snx[s]; pt.ny = a.sny[s]; pt.nz = a.snz[s];
        const uint32_t orig = a.sidx[s];
        const MatInfo mi = a.mats[m];
        const uint4* prog = a.prog + (outer ? mi.outer_start : mi.prog_start);
        const uint32_t out_off = (outer ? mi.outer_out_slot : mi.out_slot) * SLOT_BYTES;
        const uint32_t pbase = __ldg(&a.probe_base[m]);
        const int len = (int)(outer ? mi.outer_len : mi.prog_len);
        uint32_t hits = 0;
        if (outer) {
            // the point's cacheable-node records, read by the program's loads: fetched into
            // L1 now, so that the loads find them there instead of waiting on memory
            const float4* rec0 = a.probes + (size_t)pbase + jj;
            const uint32_t nr = min(mi.n_roots, 16u);
            for (uint32_t r = 0; r < nr; ++r)
                asm volatile("prefetch.global.L1 [%0];" ::"l"(rec0 + (size_t)r * cnt));
        }
        // the next instruction is fetched while the current one executes (the pool ends
        // with a padding instruction)
        uint4 nxt = __ldg(&prog[0]);
        if (MODE != EVAL_GENERIC) {
            for (int pc = 0; pc < len; ++pc) {
                const uint4 ins = nxt;
                nxt = __ldg(&prog[pc + 1]);
                const uint32_t op = ins.x & 0xFFu;
                if (outer && op == OP_LOAD_ROOT) {
                    const float4 rec = a.probes[(size_t)pbase + (size_t)(ins.y >> 16) * cnt + jj];
                    const uint32_t state = __float_as_uint(rec.w);
                    slot_store(Vb, ins.y & 0xFFFFu, rec.x, rec.y, rec.z);
                    hits += state == PROBE_HIT ? 1u : 0u;
                    // the batched evaluation or the surrogate must have given it a value
                    if (valid && state != PROBE_HIT && state != PROBE_COMPUTED) atomicOr(&a.ctl->err, ERR_BOUNDS);
                    continue;
                }
                if (!outer && op == OP_ROOT_BEGIN) continue;   // a block marker: nothing to skip
                exec_node(op, ins, Vb, pt, a.params, s_grad);
            }
            if (valid) {
                n_nodes += outer ? mi.outer_nodes : mi.full_nodes;
                n_flops += outer ? mi.outer_flops : mi.full_flops;
            }
        } else {
            int skip_end = -1;          // lane inactive while pc <= skip_end
            uint32_t cand_cell = 0, cand_h2 = 0, cand_node = 0, cand_start = 0;
            bool cand_full = false;
            uint32_t iu = 0, iv = 0, lev = a.level;
            if (a.keys_inline && valid) {
                if (a.g1u) lev = a.slev[s];
                iu = d_texel(pt.u, lev);
                iv = d_texel(pt.v, lev);
            }
            for (int pc = 0; pc < len; ++pc) {
                const uint4 ins = nxt;
                nxt = __ldg(&prog[pc + 1]);
                const uint32_t op = ins.x & 0xFFu;
                if (op == OP_ROOT_BEGIN) {
                    const uint32_t off = ins.y & 0xFFFFu, r = ins.y >> 16;
                    bool need = valid;
                    // the node's probe record: a hit, a miss, or a value computed this pass
                    float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (valid && ((a.use_cache && !a.keys_inline) || a.surr_ord))
                        rec = a.probes[(size_t)pbase + (size_t)r * cnt + j];
                    if (a.surr_ord && a.surr_ord[m] == (int32_t)r) {
                        // the learned surrogate already wrote this node's value
                        if (valid) slot_store(Vb, off, rec.x, rec.y, rec.z);
                        need = false;
                    } else if (a.keys_inline) {
                        // empty table: every probe misses at slot 0, so the descriptor is all
                        // the insert needs (no lookup kernel, no probe record)
                        if (valid) {
                            const uint64_t key = ((ins.x >> 8) & FLAG_POSROOT)
                                                     ? d_key_pos(m, ins.z, (uint32_t)a.pos_level, pt.px, pt.py, pt.pz)
                                                     : d_key(m, ins.z, lev, iu, iv);
                            d_address(key, a.n_cells, a.cells_pow2_mask, &cand_cell, &cand_h2);
                            cand_start = 0;
                            cand_full = false;
                            cand_node = ins.z;
                            n_look++;
                        }
                    } else if (a.use_cache && valid) {
                        const uint32_t state = __float_as_uint(rec.w);
                        if (state == PROBE_HIT || state == PROBE_COMPUTED) {
                            slot_store(Vb, off, rec.x, rec.y, rec.z);
                            hits += state == PROBE_HIT ? 1u : 0u;
                            need = false;
                        } else if (a.split) {
                            atomicOr(&a.ctl->err, ERR_BOUNDS);   // the batched evaluation missed it
                            need = false;
                        } else {
                            cand_cell = __float_as_uint(rec.x);
                            cand_h2 = __float_as_uint(rec.y);
                            cand_start = __float_as_uint(rec.z);
                            cand_full = state == PROBE_FULL;
                            cand_node = ins.z;
                        }
                    }
                    if (!need) skip_end = pc + (int)ins.w;
                    if (__all_sync(FULL_MASK, !need)) {
                        pc += (int)ins.w;
                        nxt = __ldg(&prog[pc + 1]);
                    }
                    continue;
                }
                const bool act = valid && pc > skip_end;
                if (act) {
                    exec_node(op, ins, Vb, pt, a.params, s_grad);
                    n_nodes++;
                    n_flops += ins.x >> 16;
                }
                if (a.use_cache && ((ins.x >> 8) & FLAG_ROOT)) {
                    const uint32_t out = ins.y & 0xFFFFu;
                    offer(a, act, orig, cand_node, cand_cell, cand_h2, cand_start, cand_full, slot_ch(Vb, out, 0),
                          slot_ch(Vb, out, 1), slot_ch(Vb, out, 2), &n_cand, &n_full);
                }
            }
        }
        if (valid) {
            a.out_rgb[orig] = slot_ch(Vb, out_off, 0);
            a.out_rgb[(size_t)a.n + orig] = slot_ch(Vb, out_off, 1);
            a.out_rgb[2 * (size_t)a.n + orig] = slot_ch(Vb, out_off, 2);
            if (a.out_hits) a.out_hits[orig] = (uint16_t)min(hits, 65535u);
        }
    }
    warp_add_u64(&a.stats[ST_NODES], n_nodes);
    warp_add_u64(&a.stats[ST_FLOPS], n_flops);
    if (MODE == EVAL_GENERIC) {
        warp_add_u64(&a.stats[ST_CANDIDATES], n_cand);
        warp_add_u64(&a.stats[ST_FULL], n_full);
        warp_add_u32(&a.ctl->w_cand, (uint32_t)(n_cand - n_full));
        if (a.keys_inline) {
            warp_add_u64(&a.stats[ST_LOOKUPS], n_look);
            warp_add_u64(&a.stats[ST_MISSES], n_look);
            warp_add_u64(&a.stats[ST_SLOTS], n_look);   // one (empty) slot examined per probe
        }
    }
}

// One 32-point item of the modes in which every lane runs every instruction (EVAL_OUTER,
// EVAL_PLAIN, EVAL_FILL), one point per lane (Vb: the lane's base in a [slot][channel][lane]
// file).
template <int MODE>
__device__ __forceinline__ void eval_item1(const BatchArgs& a, uint32_t item, uint32_t m, char* Vb, const float2* grad,
                                           unsigned long long* n_nodes, unsigned long long* n_flops, FillStats* fs) {
    constexpr bool outer = MODE == EVAL_OUTER;
    const uint32_t lane = lane_id();
    const uint32_t cnt = __ldg(&a.counts[m]);
    const uint32_t j = (item - __ldg(&a.item_base[m])) * 32u + lane;
    const bool valid = j < cnt;
    const uint32_t jj = valid ? j : cnt - 1u;   // an idle lane shadows the segment's last point
    const uint32_t s = __ldg(&a.seg_start[m]) + jj;
    PointIn pt;
    pt.u = a.su[s]; pt.v = a.sv[s];
    pt.px = a.spx[s]; pt.py = a.spy[s]; pt.pz = a.spz[s];
    pt.nx = a.snx[s]; pt.ny = a.sny[s]; pt.nz = a.snz[s];
    const uint32_t orig = a.sidx[s];
    const MatInfo mi = a.mats[m];
    const uint4* prog = a.prog + (outer ? mi.outer_start : mi.prog_start);
    const uint32_t out_off = (outer ? mi.outer_out_slot : mi.out_slot) * SLOT_BYTES;
    const uint32_t pbase = __ldg(&a.probe_base[m]);
    const int len = (int)(outer ? mi.outer_len : mi.prog_len);
    uint32_t hits = 0;
    if (outer) {
        const float4* rec0 = a.probes + (size_t)pbase + jj;
        const uint32_t nr = min(mi.n_roots, 16u);
        for (uint32_t r = 0; r < nr; ++r) asm volatile("prefetch.global.L1 [%0];" ::"l"(rec0 + (size_t)r * cnt));
    }
    uint32_t cnode = 0;
    bool cpos = false;
    uint4 nxt = __ldg(&prog[0]);   // the pool ends with a padding instruction
    for (int pc = 0; pc < len; ++pc) {
        const uint4 ins = nxt;
        nxt = __ldg(&prog[pc + 1]);
        const uint32_t op = ins.x & 0xFFu;
        if (outer && op == OP_LOAD_ROOT) {
            const float4 rec = a.probes[(size_t)pbase + (size_t)(ins.y >> 16) * cnt + jj];
            const uint32_t state = __float_as_uint(rec.w);
            slot_store(Vb, ins.y & 0xFFFFu, rec.x, rec.y, rec.z);
            hits += state == PROBE_HIT ? 1u : 0u;
            if (valid && state != PROBE_HIT && state != PROBE_COMPUTED) atomicOr(&a.ctl->err, ERR_BOUNDS);
            continue;
        }
        if (!outer && op == OP_ROOT_BEGIN) {
            if (MODE == EVAL_FILL) {
                cnode = ins.z;
                cpos = ((ins.x >> 8) & FLAG_POSROOT) != 0;
            }
            continue;
        }
        exec_node(op, ins, Vb, pt, a.params, grad);
        if (MODE == EVAL_FILL && ((ins.x >> 8) & FLAG_ROOT)) {
            const uint32_t o = ins.y & 0xFFFFu;
            fill_offer(a, valid, s, m, cnode, cpos, pt, slot_ch(Vb, o, 0), slot_ch(Vb, o, 1), slot_ch(Vb, o, 2), fs);
        }
    }
    if (valid) {
        a.out_rgb[orig] = slot_ch(Vb, out_off, 0);
        a.out_rgb[(size_t)a.n + orig] = slot_ch(Vb, out_off, 1);
        a.out_rgb[2 * (size_t)a.n + orig] = slot_ch(Vb, out_off, 2);
        if (a.out_hits) a.out_hits[orig] = (uint16_t)min(hits, 65535u);
        *n_nodes += outer ? mi.outer_nodes : mi.full_nodes;
        *n_flops += outer ? mi.outer_flops : mi.full_flops;
    }
}

// Two consecutive 32-point items of one material, two points per lane (A from the first
// item, B from the second; Vb: the lane's base in a [slot][channel][lane][2] file).
template <int MODE>
__device__ __forceinline__ void eval_item2(const BatchArgs& a, uint32_t item, uint32_t m, char* Vb, const float2* grad,
                                           unsigned long long* n_nodes, unsigned long long* n_flops, FillStats* fs) {
    constexpr bool outer = MODE == EVAL_OUTER;
    const uint32_t lane = lane_id();
    const uint32_t cnt = __ldg(&a.counts[m]);
    const uint32_t j = (item - __ldg(&a.item_base[m])) * 32u + lane;
    const bool vA = j < cnt, vB = j + 32u < cnt;
    const uint32_t jA = vA ? j : cnt - 1u, jB = vB ? j + 32u : cnt - 1u;
    const uint32_t s0 = __ldg(&a.seg_start[m]);
    const uint32_t sA = s0 + jA, sB = s0 + jB;
    PointIn A, B;
    A.u = a.su[sA]; A.v = a.sv[sA]; A.px = a.spx[sA]; A.py = a.spy[sA]; A.pz = a.spz[sA];
    A.nx = a.snx[sA]; A.ny = a.sny[sA]; A.nz = a.snz[sA];
    B.u = a.su[sB]; B.v = a.sv[sB]; B.px = a.spx[sB]; B.py = a.spy[sB]; B.pz = a.spz[sB];
    B.nx = a.snx[sB]; B.ny = a.sny[sB]; B.nz = a.snz[sB];
    const MatInfo mi = a.mats[m];
    const uint4* prog = a.prog + (outer ? mi.outer_start : mi.prog_start);
    const uint32_t out_off = (outer ? mi.outer_out_slot : mi.out_slot) * SLOT_BYTES;
    const uint32_t pbase = __ldg(&a.probe_base[m]);
    const int len = (int)(outer ? mi.outer_len : mi.prog_len);
    uint32_t hA = 0, hB = 0;
    if (outer) {
        const float4* ra = a.probes + (size_t)pbase + jA;
        const float4* rb = a.probes + (size_t)pbase + jB;
        const uint32_t nr = min(mi.n_roots, 16u);
        for (uint32_t r = 0; r < nr; ++r) {
            asm volatile("prefetch.global.L1 [%0];" ::"l"(ra + (size_t)r * cnt));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(rb + (size_t)r * cnt));
        }
    }
    uint32_t cnode = 0;
    bool cpos = false;
    uint4 nxt = __ldg(&prog[0]);
    for (int pc = 0; pc < len; ++pc) {
        const uint4 ins = nxt;
        nxt = __ldg(&prog[pc + 1]);
        const uint32_t op = ins.x & 0xFFu;
        if (outer && op == OP_LOAD_ROOT) {
            const size_t rb = (size_t)pbase + (size_t)(ins.y >> 16) * cnt;
            const float4 ra = a.probes[rb + jA], rc = a.probes[rb + jB];
            const uint32_t sa = __float_as_uint(ra.w), sc = __float_as_uint(rc.w);
            slot2_store(Vb, ins.y & 0xFFFFu, f2(ra.x, rc.x), f2(ra.y, rc.y), f2(ra.z, rc.z));
            hA += sa == PROBE_HIT ? 1u : 0u;
            hB += sc == PROBE_HIT ? 1u : 0u;
            if ((vA && sa != PROBE_HIT && sa != PROBE_COMPUTED) || (vB && sc != PROBE_HIT && sc != PROBE_COMPUTED))
                atomicOr(&a.ctl->err, ERR_BOUNDS);
            continue;
        }
        if (!outer && op == OP_ROOT_BEGIN) {
            if (MODE == EVAL_FILL) {
                cnode = ins.z;
                cpos = ((ins.x >> 8) & FLAG_POSROOT) != 0;
            }
            continue;
        }
        exec_node2(op, ins, Vb, A, B, a.params, grad);
        if (MODE == EVAL_FILL && ((ins.x >> 8) & FLAG_ROOT)) {
            const uint32_t o = ins.y & 0xFFFFu;
            const float2 c0 = slot2(Vb, o, 0), c1 = slot2(Vb, o, 1), c2 = slot2(Vb, o, 2);
            fill_offer(a, vA, sA, m, cnode, cpos, A, c0.x, c1.x, c2.x, fs);
            fill_offer(a, vB, sB, m, cnode, cpos, B, c0.y, c1.y, c2.y, fs);
        }
    }
    const float2 o0 = slot2(Vb, out_off, 0), o1 = slot2(Vb, out_off, 1), o2 = slot2(Vb, out_off, 2);
    const uint32_t nv = (vA ? 1u : 0u) + (vB ? 1u : 0u);
    if (vA) {
        const uint32_t oa = a.sidx[sA];
        a.out_rgb[oa] = o0.x;
        a.out_rgb[(size_t)a.n + oa] = o1.x;
        a.out_rgb[2 * (size_t)a.n + oa] = o2.x;
        if (a.out_hits) a.out_hits[oa] = (uint16_t)min(hA, 65535u);
    }
    if (vB) {
        const uint32_t ob = a.sidx[sB];
        a.out_rgb[ob] = o0.y;
        a.out_rgb[(size_t)a.n + ob] = o1.y;
        a.out_rgb[2 * (size_t)a.n + ob] = o2.y;
        if (a.out_hits) a.out_hits[ob] = (uint16_t)min(hB, 65535u);
    }
    *n_nodes += (unsigned long long)nv * (outer ? mi.outer_nodes : mi.full_nodes);
    *n_flops += (unsigned long long)nv * (outer ? mi.outer_flops : mi.full_flops);
}

// EVAL_OUTER and EVAL_PLAIN with two points per lane: a warp takes pairs of consecutive
// items; a pair that straddles two materials runs as two single items.  BLOCK: the block
// claims a tile of EVAL_WARPS consecutive pairs at a time (block-per-material work: the
// warps of a block run one material's program together and share its instruction and
// parameter lines in L1); else every warp claims its own pair.
template <int MODE, bool BLOCK>
__global__ void __launch_bounds__(EVAL_WARPS * 32, MODE == EVAL_FILL ? 6 : 7) k_eval2(BatchArgs a, uint32_t* item_ctr) {
    extern __shared__ float s_val[];
    __shared__ float2 s_grad[8];
    __shared__ uint32_t s_tile;
    init_gradients(s_grad);
    __syncthreads();
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t slots = MODE == EVAL_OUTER ? a.max_slots_outer : a.max_slots;
    FillStats fs;
    char* Vw = reinterpret_cast<char*>(s_val + (size_t)warp * slots * 192u);
    char* Vb2 = Vw + lane * 8u;
    char* Vb1 = Vw + lane * 4u;
    const uint32_t n_items = a.ctl->n_items;
    unsigned long long n_nodes = 0, n_flops = 0;
    for (;;) {
        uint32_t pr = 0;
        if (BLOCK) {
            if (threadIdx.x == 0) s_tile = atomicAdd(item_ctr, 1u);
            __syncthreads();
            const uint32_t tile = s_tile;
            __syncthreads();   // read by every warp before the next claim overwrites it
            if (2u * tile * EVAL_WARPS >= n_items) break;   // uniform over the block
            pr = tile * EVAL_WARPS + warp;
        } else {
            if (lane == 0) pr = atomicAdd(item_ctr, 1u);
            pr = __shfl_sync(FULL_MASK, pr, 0);
        }
        const uint32_t it = 2u * pr;
        if (it >= n_items) {
            if (BLOCK) continue;   // this warp's pair is past the end; the block's tile is not
            break;
        }
        const uint32_t m = find_material(a.item_base, a.n_mats, it);
        if (it + 1u < __ldg(&a.item_base[m + 1])) {
            eval_item2<MODE>(a, it, m, Vb2, s_grad, &n_nodes, &n_flops, &fs);
        } else {
            eval_item1<MODE>(a, it, m, Vb1, s_grad, &n_nodes, &n_flops, &fs);
            if (it + 1u < n_items)
                eval_item1<MODE>(a, it + 1u, find_material(a.item_base, a.n_mats, it + 1u), Vb1, s_grad, &n_nodes,
                                 &n_flops, &fs);
        }
    }
    warp_add_u64(&a.stats[ST_NODES], n_nodes);
    warp_add_u64(&a.stats[ST_FLOPS], n_flops);
    if (MODE == EVAL_FILL) {
        warp_add_u64(&a.stats[ST_CANDIDATES], fs.n_cand);
        warp_add_u64(&a.stats[ST_FULL], fs.n_full);
        warp_add_u32(&a.ctl->w_cand, (uint32_t)(fs.n_cand - fs.n_full));
        warp_add_u64(&a.stats[ST_LOOKUPS], fs.n_look);
        warp_add_u64(&a.stats[ST_MISSES], fs.n_look);
        warp_add_u64(&a.stats[ST_SLOTS], fs.n_look);   // one (empty) slot examined per probe
    }
}

// Scans cell `cell` for h2 (Alg. 1's entry loop read as a lookup): the first slot that
// holds h2 (hit) or 0 (miss), -1 if every slot holds another hash (full).
__device__ __forceinline__ int probe_cell(const BatchArgs& a, uint32_t cell, uint32_t h2, bool* hit) {
    const uint4* hw = reinterpret_cast<const uint4*>(cell_h2(a, cell));
    const uint32_t ne = a.n_entries;
    *hit = false;
    for (uint32_t q = 0; 4u * q < ne; q += 2) {
        // two 16-byte words per step; words past N_e are never compared
        const uint4 w0 = __ldg(hw + q);
        const uint4 w1 = 4u * (q + 1) < ne ? __ldg(hw + q + 1) : make_uint4(0, 0, 0, 0);
        const uint32_t v[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t idx = 4u * q + k;
            if (idx < ne && (v[k] == h2 || v[k] == 0u)) {
                *hit = v[k] == h2;
                return (int)idx;
            }
        }
    }
    return -1;
}

// ---- the paper's concurrent update (Alg. 1, Sec. 3.3): 8-byte slots {hash2 in the low word,
// the 32-bit encoded value in the high word}; a slot is empty iff it is 0 (hash2 is never 0).
__device__ __forceinline__ unsigned long long* alg1_cell(const BatchArgs& a, uint32_t cell) {
    return reinterpret_cast<unsigned long long*>(a.table) + (size_t)cell * a.n_entries;
}

// Alg. 1's entry loop over a cell: the first slot whose hash is h2 or that is empty, or -1
// (full); *word receives that slot.  The slots are read from L2 (other warps insert into
// them during the pass), all loads of a group of 8 in flight together.
__device__ __forceinline__ int alg1_scan(const BatchArgs& a, uint32_t cell, uint32_t h2, unsigned long long* word) {
    const unsigned long long* cw = alg1_cell(a, cell);
    const uint32_t ne = a.n_entries;
    for (uint32_t q = 0; q < ne; q += 8) {
        unsigned long long w[8];
        if ((ne & 1u) == 0 && q + 8 <= ne) {
            // 16-byte aligned pairs of slots, read as two 64-bit elements: each slot is read
            // in one access, so a slot being filled by a compare-and-swap is never seen torn
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const ulonglong2 x = __ldcg(reinterpret_cast<const ulonglong2*>(cw + q) + k);
                w[2 * k] = x.x;
                w[2 * k + 1] = x.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) w[k] = q + k < ne ? __ldcg(cw + q + k) : 0ull;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (q + k < ne && ((uint32_t)w[k] == h2 || w[k] == 0ull)) {
                *word = w[k];
                return (int)(q + k);
            }
    }
    return -1;
}

// round(c 2^k), ties up, exactly, for an FP32 c >= 0 whose scaled value is at most 512:
// c = M 2^E with a 24-bit integer M, so the rounding is an integer shift.
__device__ __forceinline__ uint32_t scaled_round(float c, int k) {
    const uint32_t b = __float_as_uint(c);
    const uint32_t be = b >> 23;
    uint32_t M = b & 0x7FFFFFu;
    int E = -149;
    if (be != 0) {
        M |= 0x800000u;
        E = (int)be - 150;
    }
    const int sh = E + k;
    if (sh >= 0) return M << sh;   // only c = 0 gets here within the format's range
    const int r = -sh;
    if (r > 25) return 0u;         // M < 2^24 <= 2^(r - 1): rounds to 0
    return (uint32_t)(((unsigned long long)M + (1ull << (r - 1))) >> r);
}

// The 32-bit encoding of a value (Alg. 1 "Encode"): shared-exponent RGB9E5 (the format of
// OpenGL's EXT_texture_shared_exponent): components clamped to [0, 511/512 * 2^16] (NaN to
// 0), exponent max(-16, floor(log2 max)) + 16, raised by one when the largest mantissa
// rounds to 512; mantissas rounded to nearest, ties up.  Bits: r 0-8, g 9-17, b 18-26,
// exponent 27-31.
__device__ __forceinline__ uint32_t rgb9e5_encode(float r, float g, float b) {
    float c[3] = {r, g, b};
    float mx = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        c[k] = c[k] > 0.0f ? fminf(c[k], 65408.0f) : 0.0f;
        mx = fmaxf(mx, c[k]);
    }
    const uint32_t be = __float_as_uint(mx) >> 23;
    const int fl = be != 0 ? max(-16, (int)be - 127) : -16;   // floor(log2 mx), at least -16
    int ex = fl + 16;
    if (scaled_round(mx, 24 - ex) == 512u) ex += 1;
    uint32_t code = (uint32_t)ex << 27;
#pragma unroll
    for (int k = 0; k < 3; ++k) code |= scaled_round(c[k], 24 - ex) << (9 * k);
    return code;
}

__device__ __forceinline__ void rgb9e5_decode(uint32_t code, float* r, float* g, float* b) {
    const float sc = __uint_as_float((uint32_t)((int)(code >> 27) - 24 + 127) << 23);   // 2^(e - 24)
    *r = (float)(code & 511u) * sc;
    *g = (float)((code >> 9) & 511u) * sc;
    *b = (float)((code >> 18) & 511u) * sc;
}

// Alg. 1 for one evaluated cacheable node: find the slot again, then one compare-and-swap
// of {hash2, encoded value} into it if it was empty; a lost race drops the value.
__device__ __forceinline__ void alg1_insert(const BatchArgs& a, uint32_t cell, uint32_t h2, float r, float g, float b,
                                            unsigned long long* n_ins, unsigned long long* n_dup,
                                            unsigned long long* n_full, unsigned long long* n_race) {
    unsigned long long cur = 0;
    const int j = alg1_scan(a, cell, h2, &cur);
    if (j < 0) { *n_full += 1; return; }
    if (cur != 0ull) { *n_dup += 1; return; }   // the key is present
    const unsigned long long word = ((unsigned long long)rgb9e5_encode(r, g, b) << 32) | h2;
    const unsigned long long old = atomicCAS(alg1_cell(a, cell) + j, 0ull, word);
    if (old == 0ull) *n_ins += 1;
    else if ((uint32_t)old == h2) *n_dup += 1;   // the same key, inserted meanwhile
    else *n_race += 1;                            // another key took the slot
}

// Unsorted evaluation: the in-shader form of Sec. 3.  A warp takes 32 consecutive
// shading points in batch order, runs each distinct material among them in turn (the
// other lanes idle) and probes the table when it reaches a cacheable node: a hit skips
// the node's block, a miss evaluates it and offers the value.  No grouping pass, no
// probe records; the table is read-only until the insert phase, so every probe sees the
// snapshot left by the previous batch, as in the grouped pipeline.
// GROUPED: the same evaluator over the material-grouped points (work items of 32 points
// of one material from the grouping pass), so a warp runs one program; a cacheable node
// replaced by a learned surrogate takes its value from the surrogate's record.
template <bool GROUPED>
__global__ void __launch_bounds__(EVAL_WARPS * 32) k_eval_fused(BatchArgs a, uint32_t* item_ctr) {
    extern __shared__ float s_val[];
    __shared__ float2 s_grad[8];
    init_gradients(s_grad);
    __syncthreads();
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    char* Vb = reinterpret_cast<char*>(s_val + (size_t)warp * a.max_slots * 96u + lane);
    const uint32_t n_chunks = GROUPED ? a.ctl->n_items : (a.n + 31u) >> 5;
    const uint32_t ne = a.n_entries;
    unsigned long long n_nodes = 0, n_flops = 0, n_cand = 0, n_full = 0;
    unsigned long long n_look = 0, n_hit = 0, n_slots = 0, n_bad = 0;
    unsigned long long n_ins = 0, n_dup = 0, n_race = 0;   // the paper's concurrent update
    uint32_t chunk = blockIdx.x * EVAL_WARPS + warp;
    for (;;) {
        if (GROUPED) {
            uint32_t item = 0;
            if (lane == 0) item = atomicAdd(item_ctr, 1u);
            chunk = __shfl_sync(FULL_MASK, item, 0);
        }
        if (chunk >= n_chunks) break;
        uint32_t i = 0, m = 0, cnt = 0, jj = 0;   // i: the point's index in the batch
        uint32_t lev = a.level;
        bool ok = false;
        PointIn pt{0, 0, 0, 0, 0, 0, 0, 0};
        if (GROUPED) {
            m = find_material(a.item_base, a.n_mats, chunk);
            cnt = __ldg(&a.counts[m]);
            jj = (chunk - __ldg(&a.item_base[m])) * 32u + lane;
            ok = jj < cnt;
            if (ok) {
                const uint32_t s = __ldg(&a.seg_start[m]) + jj;
                pt.u = a.su[s]; pt.v = a.sv[s];
                pt.px = a.spx[s]; pt.py = a.spy[s]; pt.pz = a.spz[s];
                pt.nx = a.snx[s]; pt.ny = a.sny[s]; pt.nz = a.snz[s];
                i = a.sidx[s];
                if (a.g1u) lev = a.slev[s];
            }
        } else {
            i = chunk * 32u + lane;
            const bool in = i < a.n;
            m = in ? a.mat[i] : 0u;
            ok = in && m < a.n_mats;
            if (in && !ok) {
                zero_output(a, i);
                n_bad++;
            }
            if (ok) {
                pt.u = a.u[i]; pt.v = a.v[i];
                pt.px = a.px[i]; pt.py = a.py[i]; pt.pz = a.pz[i];
                pt.nx = a.nx[i]; pt.ny = a.ny[i]; pt.nz = a.nz[i];
                if (a.g1u) lev = d_level(a.g1u[i], a.g1v[i], a.g2u[i], a.g2v[i], a.level_offset);
            }
        }
        uint32_t iu = 0, iv = 0;
        if (ok) {
            iu = d_texel(pt.u, lev);
            iv = d_texel(pt.v, lev);
        }
        const int32_t surr = (GROUPED && a.surr_ord) ? a.surr_ord[m] : -1;
        unsigned todo = __ballot_sync(FULL_MASK, ok);
        while (todo) {
            const uint32_t mg = __shfl_sync(FULL_MASK, m, __ffs(todo) - 1);
            const unsigned grp = __ballot_sync(FULL_MASK, ok && m == mg);
            todo &= ~grp;
            const bool mine = (grp >> lane) & 1u;
            const MatInfo mi = a.mats[mg];
            const uint4* prog = a.prog + mi.prog_start;
            int skip_end = -1;
            uint32_t hits = 0, cand_cell = 0, cand_h2 = 0, cand_node = 0, cand_start = 0;
            bool cand_full = false;
            const int len = (int)mi.prog_len;
            uint4 nxt = len > 0 ? __ldg(&prog[0]) : make_uint4(0, 0, 0, 0);
            for (int pc = 0; pc < len; ++pc) {
                const uint4 ins = nxt;
                if (pc + 1 < len) nxt = __ldg(&prog[pc + 1]);
                const uint32_t op = ins.x & 0xFFu;
                if (op == OP_ROOT_BEGIN) {
                    bool need = mine;
                    if (GROUPED && surr == (int32_t)(ins.y >> 16)) {
                        // the learned surrogate wrote this node's value
                        if (mine) {
                            const float4 rec = a.probes[(size_t)__ldg(&a.probe_base[mg]) + (size_t)(ins.y >> 16) * cnt + jj];
                            slot_store(Vb, ins.y & 0xFFFFu, rec.x, rec.y, rec.z);
                        }
                        need = false;
                    } else if (a.use_cache && mine && a.alg1) {
                        // the paper's scheme: the table as other warps are filling it
                        d_address(((ins.x >> 8) & FLAG_POSROOT) ? d_key_pos(mg, ins.z, (uint32_t)a.pos_level, pt.px, pt.py, pt.pz)
                                                                  : d_key(mg, ins.z, lev, iu, iv),
                                  a.n_cells, a.cells_pow2_mask, &cand_cell, &cand_h2);
                        unsigned long long w = 0;
                        const int first = alg1_scan(a, cand_cell, cand_h2, &w);
                        n_look++;
                        n_slots += first >= 0 ? (uint32_t)first + 1u : ne;
                        if (first >= 0 && w != 0ull) {
                            float r, g, b;
                            rgb9e5_decode((uint32_t)(w >> 32), &r, &g, &b);
                            slot_store(Vb, ins.y & 0xFFFFu, r, g, b);
                            hits++;
                            n_hit++;
                            need = false;
                        } else {
                            cand_full = first < 0;
                            cand_node = ins.z;
                        }
                    } else if (a.use_cache && mine) {
                        d_address(((ins.x >> 8) & FLAG_POSROOT) ? d_key_pos(mg, ins.z, (uint32_t)a.pos_level, pt.px, pt.py, pt.pz)
                                                                  : d_key(mg, ins.z, lev, iu, iv),
                                  a.n_cells, a.cells_pow2_mask, &cand_cell, &cand_h2);
                        bool hit = false;
                        const int first = a.table_empty ? 0 : probe_cell(a, cand_cell, cand_h2, &hit);
                        n_look++;
                        n_slots += first >= 0 ? (uint32_t)first + 1u : ne;
                        if (hit) {
                            const float* val = cell_val(a, cand_cell, (uint32_t)first);
                            slot_store(Vb, ins.y & 0xFFFFu, __ldg(val), __ldg(val + 1), __ldg(val + 2));
                            hits++;
                            n_hit++;
                            need = false;
                        } else {
                            cand_start = first >= 0 ? (uint32_t)first : ne;
                            cand_full = first < 0;
                            if (cand_full && a.slot_cls)
                                cand_full = cell_closed(a, cand_cell, a.vis ? (uint32_t)__ldg(&a.vis[i]) : 0u);
                            cand_node = ins.z;
                        }
                    }
                    if (!need) skip_end = pc + (int)ins.w;
                    if (__all_sync(FULL_MASK, !need)) {
                        pc += (int)ins.w;
                        if (pc + 1 < len) nxt = __ldg(&prog[pc + 1]);
                    }
                    continue;
                }
                const bool act = mine && pc > skip_end;
                if (act) {
                    exec_node(op, ins, Vb, pt, a.params, s_grad);
                    n_nodes++;
                    n_flops += ins.x >> 16;
                }
                if (a.use_cache && ((ins.x >> 8) & FLAG_ROOT)) {
                    const uint32_t out = ins.y & 0xFFFFu;
                    if (a.alg1) {
                        n_cand += act ? 1u : 0u;
                        n_full += (act && cand_full) ? 1u : 0u;   // a full cell stays full
                        if (act && !cand_full)
                            alg1_insert(a, cand_cell, cand_h2, slot_ch(Vb, out, 0), slot_ch(Vb, out, 1),
                                        slot_ch(Vb, out, 2), &n_ins, &n_dup, &n_full, &n_race);
                    } else {
                        offer(a, act, i, cand_node, cand_cell, cand_h2, cand_start, cand_full, slot_ch(Vb, out, 0),
                              slot_ch(Vb, out, 1), slot_ch(Vb, out, 2), &n_cand, &n_full);
                    }
                }
            }
            if (mine) {
                const uint32_t oo = mi.out_slot * SLOT_BYTES;
                a.out_rgb[i] = slot_ch(Vb, oo, 0);
                a.out_rgb[(size_t)a.n + i] = slot_ch(Vb, oo, 1);
                a.out_rgb[2 * (size_t)a.n + i] = slot_ch(Vb, oo, 2);
                if (a.out_hits) a.out_hits[i] = (uint16_t)min(hits, 65535u);
            }
        }
        if (!GROUPED) chunk += gridDim.x * EVAL_WARPS;
    }
    if (!GROUPED && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&a.stats[ST_POINTS], (unsigned long long)a.n);
    warp_add_u64(&a.stats[ST_NODES], n_nodes);
    warp_add_u64(&a.stats[ST_FLOPS], n_flops);
    warp_add_u64(&a.stats[ST_CANDIDATES], n_cand);
    warp_add_u64(&a.stats[ST_FULL], n_full);
    warp_add_u32(&a.ctl->w_cand, (uint32_t)(n_cand - n_full));
    warp_add_u64(&a.stats[ST_LOOKUPS], n_look);
    warp_add_u64(&a.stats[ST_HITS], n_hit);
    warp_add_u64(&a.stats[ST_MISSES], n_look - n_hit);
    warp_add_u64(&a.stats[ST_SLOTS], n_slots);
    if (a.alg1) {
        warp_add_u64(&a.stats[ST_INSERTED], n_ins);
        warp_add_u64(&a.stats[ST_DUP], n_dup);
        warp_add_u64(&a.stats[ST_RACE], n_race);
    }
    if (!GROUPED) {
        warp_add_u64(&a.stats[ST_BAD], n_bad);
        if (__any_sync(FULL_MASK, n_bad != 0) && lane == 0) atomicOr(&a.ctl->err, ERR_BAD_MAT);
    }
}

// Work items of the batched evaluation: ceil(misses / 32) per cacheable node, laid out in
// ascending nesting level (root_order), with the first item of each level after them.
__global__ void k_scan_roots(BatchArgs a) {
    __shared__ uint32_t s_tmp[33];
    const uint32_t T = blockDim.x, t = threadIdx.x, N = a.n_roots_total;
    const uint32_t per = (N + T - 1) / T;
    const uint32_t lo = min(t * per, N), hi = min(lo + per, N);
    uint32_t c = 0;
    for (uint32_t q = lo; q < hi; ++q) c += (a.miss_cnt[a.root_order[q]] + 31u) >> 5;
    uint32_t tot;
    uint32_t b = block_incl_scan(c, s_tmp, &tot) - c;
    for (uint32_t q = lo; q < hi; ++q) {
        a.root_item_base[q] = b;
        b += (a.miss_cnt[a.root_order[q]] + 31u) >> 5;
    }
    __syncthreads();
    if (t == T - 1) {
        a.root_item_base[N] = tot;
        a.ctl->n_root_items = tot;
    }
    __syncthreads();
    uint32_t* level_items = a.root_item_base + N + 1;
    for (uint32_t l = t; l <= MAX_LEVELS; l += T) level_items[l] = a.root_item_base[a.level_start[l]];
}

// Batched evaluation of the missed cacheable nodes (the "missed sub-graphs" of Sec. 3):
// a warp runs one cacheable node's standalone program for 32 of its misses, writes the
// values into their probe records and offers them to the table.  Every lane runs every
// instruction: a lane past the node's last miss shadows that miss and stores nothing.
struct RootStats {
    unsigned long long n_nodes = 0, n_flops = 0, n_cand = 0, n_full = 0;
};

// One item (32 misses of one cacheable node), one miss per lane (Vb: the lane's base in a
// [slot][channel][lane] file).
template <bool POS>
__device__ __forceinline__ void roots_item1(const BatchArgs& a, uint32_t item, uint32_t q, char* Vb, const float2* grad,
                                            RootStats* st) {
    const uint32_t lane = lane_id();
    const uint32_t g = __ldg(&a.root_order[q]);
    const RootInfo ri = a.rinfo[g];
    const uint32_t m = ri.mat, r = ri.ordinal;
    const uint32_t cnt = __ldg(&a.counts[m]);
    const uint32_t nm = a.miss_cnt[g];   // at least one: the item exists
    const uint32_t idx = (item - a.root_item_base[q]) * 32u + lane;
    const bool valid = idx < nm;
    const size_t pbase = __ldg(&a.probe_base[m]);
    const size_t base = pbase + (size_t)r * cnt;
    const uint32_t j = a.misslist[base + (valid ? idx : nm - 1u)];
    const uint32_t s = __ldg(&a.seg_start[m]) + j;
    PointIn pt{0, 0, 0, 0, 0, 0, 0, 0};
    pt.u = a.su[s];
    pt.v = a.sv[s];
    if (POS) {   // a position-class node reads the position
        pt.px = a.spx[s];
        pt.py = a.spy[s];
        pt.pz = a.spz[s];
    }
    const uint32_t orig = a.sidx[s];
    const float4 rec = a.probes[base + j];
    const uint4* prog = a.prog + ri.prog_start;
    uint4 nxt = __ldg(&prog[0]);   // the pool ends with a padding instruction
    for (uint32_t pc = 0; pc < ri.prog_len; ++pc) {
        const uint4 ins = nxt;
        nxt = __ldg(&prog[pc + 1]);
        const uint32_t op = ins.x & 0xFFu;
        if (op == OP_LOAD_ROOT) {
            const float4 v = a.probes[pbase + (size_t)(ins.y >> 16) * cnt + j];
            slot_store(Vb, ins.y & 0xFFFFu, v.x, v.y, v.z);
            continue;
        }
        exec_node(op, ins, Vb, pt, a.params, grad);
    }
    const uint32_t out_off = ri.out_slot * SLOT_BYTES;
    const float v0 = slot_ch(Vb, out_off, 0), v1 = slot_ch(Vb, out_off, 1), v2 = slot_ch(Vb, out_off, 2);
    if (valid) {
        a.probes[base + j] = make_float4(v0, v1, v2, __uint_as_float(PROBE_COMPUTED));
        st->n_nodes += ri.nodes;
        st->n_flops += ri.flops;
    }
    offer(a, valid, orig, ri.node, __float_as_uint(rec.x), __float_as_uint(rec.y), __float_as_uint(rec.z),
          __float_as_uint(rec.w) == PROBE_FULL, v0, v1, v2, &st->n_cand, &st->n_full);
}

// Two consecutive items of one cacheable node, two misses per lane (A from the first item,
// B from the second; Vb: the lane's base in a [slot][channel][lane][2] file).
template <bool POS>
__device__ __forceinline__ void roots_item2(const BatchArgs& a, uint32_t item, uint32_t q, char* Vb, const float2* grad,
                                            RootStats* st) {
    const uint32_t lane = lane_id();
    const uint32_t g = __ldg(&a.root_order[q]);
    const RootInfo ri = a.rinfo[g];
    const uint32_t m = ri.mat, r = ri.ordinal;
    const uint32_t cnt = __ldg(&a.counts[m]);
    const uint32_t nm = a.miss_cnt[g];
    const uint32_t iA = (item - a.root_item_base[q]) * 32u + lane, iB = iA + 32u;
    const bool vA = iA < nm, vB = iB < nm;
    const size_t pbase = __ldg(&a.probe_base[m]);
    const size_t base = pbase + (size_t)r * cnt;
    const uint32_t jA = a.misslist[base + (vA ? iA : nm - 1u)], jB = a.misslist[base + (vB ? iB : nm - 1u)];
    const uint32_t s0 = __ldg(&a.seg_start[m]);
    const uint32_t sA = s0 + jA, sB = s0 + jB;
    PointIn A{0, 0, 0, 0, 0, 0, 0, 0}, B{0, 0, 0, 0, 0, 0, 0, 0};
    A.u = a.su[sA]; A.v = a.sv[sA];
    B.u = a.su[sB]; B.v = a.sv[sB];
    if (POS) {
        A.px = a.spx[sA]; A.py = a.spy[sA]; A.pz = a.spz[sA];
        B.px = a.spx[sB]; B.py = a.spy[sB]; B.pz = a.spz[sB];
    }
    // the miss records and batch indices the offers need, loaded while the program runs
    const float4 recA = a.probes[base + jA], recB = a.probes[base + jB];
    const uint32_t oA = a.sidx[sA], oB = a.sidx[sB];
    const uint4* prog = a.prog + ri.prog_start;
    uint4 nxt = __ldg(&prog[0]);
    for (uint32_t pc = 0; pc < ri.prog_len; ++pc) {
        const uint4 ins = nxt;
        nxt = __ldg(&prog[pc + 1]);
        const uint32_t op = ins.x & 0xFFu;
        if (op == OP_LOAD_ROOT) {
            const size_t rb = pbase + (size_t)(ins.y >> 16) * cnt;
            const float4 ra = a.probes[rb + jA], rc = a.probes[rb + jB];
            slot2_store(Vb, ins.y & 0xFFFFu, f2(ra.x, rc.x), f2(ra.y, rc.y), f2(ra.z, rc.z));
            continue;
        }
        exec_node2(op, ins, Vb, A, B, a.params, grad);
    }
    const uint32_t out_off = ri.out_slot * SLOT_BYTES;
    const float2 o0 = slot2(Vb, out_off, 0), o1 = slot2(Vb, out_off, 1), o2 = slot2(Vb, out_off, 2);
    if (vA) {
        a.probes[base + jA] = make_float4(o0.x, o1.x, o2.x, __uint_as_float(PROBE_COMPUTED));
        st->n_nodes += ri.nodes;
        st->n_flops += ri.flops;
    }
    if (vB) {
        a.probes[base + jB] = make_float4(o0.y, o1.y, o2.y, __uint_as_float(PROBE_COMPUTED));
        st->n_nodes += ri.nodes;
        st->n_flops += ri.flops;
    }
    offer(a, vA, oA, ri.node, __float_as_uint(recA.x), __float_as_uint(recA.y), __float_as_uint(recA.z),
          __float_as_uint(recA.w) == PROBE_FULL, o0.x, o1.x, o2.x, &st->n_cand, &st->n_full);
    offer(a, vB, oB, ri.node, __float_as_uint(recB.x), __float_as_uint(recB.y), __float_as_uint(recB.z),
          __float_as_uint(recB.w) == PROBE_FULL, o0.y, o1.y, o2.y, &st->n_cand, &st->n_full);
}

__device__ __forceinline__ void roots_stats(const BatchArgs& a, const RootStats& st) {
    warp_add_u64(&a.stats[ST_NODES], st.n_nodes);
    warp_add_u64(&a.stats[ST_FLOPS], st.n_flops);
    warp_add_u64(&a.stats[ST_FLOPS_MISSED], st.n_flops);
    warp_add_u64(&a.stats[ST_CANDIDATES], st.n_cand);
    warp_add_u64(&a.stats[ST_FULL], st.n_full);
    warp_add_u32(&a.ctl->w_cand, (uint32_t)(st.n_cand - st.n_full));
}

template <bool POS>
__global__ void __launch_bounds__(EVAL_WARPS * 32) k_eval_roots(BatchArgs a, uint32_t level, uint32_t* item_ctr) {
    extern __shared__ float s_val[];
    __shared__ float2 s_grad[8];
    init_gradients(s_grad);
    __syncthreads();
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    char* Vb = reinterpret_cast<char*>(s_val + (size_t)warp * a.max_slots_roots * 96u + lane);
    // this level's items only: they are contiguous in the level-ordered item layout
    const uint32_t* level_items = a.root_item_base + a.n_roots_total + 1;
    const uint32_t first = level_items[level], end = level_items[level + 1];
    RootStats st;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = first + atomicAdd(item_ctr, 1u);
        item = __shfl_sync(FULL_MASK, item, 0);
        if (item >= end) break;
        roots_item1<POS>(a, item, find_material(a.root_item_base, a.n_roots_total, item), Vb, s_grad, &st);
    }
    roots_stats(a, st);
}

// The same with two misses per lane: a warp takes pairs of consecutive items (the item
// counter counts pairs); a pair whose items belong to two cacheable nodes runs as two
// single items.
template <bool POS>
__global__ void __launch_bounds__(EVAL_WARPS * 32, 6) k_eval_roots2(BatchArgs a, uint32_t level, uint32_t* item_ctr) {
    extern __shared__ float s_val[];
    __shared__ float2 s_grad[8];
    init_gradients(s_grad);
    __syncthreads();
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    char* Vw = reinterpret_cast<char*>(s_val + (size_t)warp * a.max_slots_roots * 192u);
    char* Vb2 = Vw + lane * 8u;
    char* Vb1 = Vw + lane * 4u;
    const uint32_t* level_items = a.root_item_base + a.n_roots_total + 1;
    const uint32_t first = level_items[level], end = level_items[level + 1];
    RootStats st;
    for (;;) {
        uint32_t pr = 0;
        if (lane == 0) pr = atomicAdd(item_ctr, 1u);
        pr = __shfl_sync(FULL_MASK, pr, 0);
        const uint32_t it = first + 2u * pr;
        if (it >= end) break;
        const uint32_t q = find_material(a.root_item_base, a.n_roots_total, it);
        if (it + 1u < end && it + 1u < a.root_item_base[q + 1]) {
            roots_item2<POS>(a, it, q, Vb2, s_grad, &st);
        } else {
            roots_item1<POS>(a, it, q, Vb1, s_grad, &st);
            if (it + 1u < end)
                roots_item1<POS>(a, it + 1u, find_material(a.root_item_base, a.n_roots_total, it + 1u), Vb1, s_grad,
                                 &st);
        }
    }
    roots_stats(a, st);
}

// =======================================================================================
// Insert (Alg. 1 semantics, deterministic): rounds of claim / resolve in one
// cooperative launch, separated by a grid barrier whose waits are bounded
// =======================================================================================
__device__ __forceinline__ unsigned long long claim_word(uint32_t epoch, unsigned long long prio) {
    return ((unsigned long long)(EPOCH_MAX - epoch) << 44) | prio;
}

constexpr uint32_t BARRIER_SPIN_LIMIT = 1u << 24;   // x >= 64 ns sleeps: about a second

// Grid-wide barrier for a cooperative launch (all blocks resident).  Returns false, with
// ERR_TIMEOUT set, if the other blocks did not arrive within the spin limit.
__device__ bool grid_barrier(Control* ctl) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t* gen = &ctl->bar_gen;
        const uint32_t g0 = *gen;
        __threadfence();
        const uint32_t arrived = atomicAdd(&ctl->bar_count, 1u);
        int ok = 1;
        if (arrived == gridDim.x - 1) {
            ctl->bar_count = 0;
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            uint32_t spins = 0;
            while (*gen == g0) {
                __nanosleep(64);
                if (++spins > BARRIER_SPIN_LIMIT) {
                    atomicOr(&ctl->err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__global__ void __launch_bounds__(256) k_insert(BatchArgs a) {
    const uint32_t ne = a.n_entries;
    const uint32_t stride = gridDim.x * blockDim.x;
    unsigned long long n_dup = 0, n_full = 0, n_ins = 0;
    for (uint32_t round = 0; round <= ne; ++round) {
        const uint32_t n_in = round == 0 ? min(__ldcg(&a.ctl->n_cand), a.probe_cap) : __ldcg(&a.ctl->out_count[round - 1]);
        if (n_in == 0) break;                         // same value in every block
        const uint32_t* list_in = round == 0 ? nullptr : a.lists[(round - 1) & 1u];
        const uint32_t epoch = __ldcg(&a.ctl->epoch) + round;
        const bool final_round = round == ne;
        // ---- claim: first slot holding the candidate's hash2 (duplicate) or 0 (free)
        const uint32_t n_r = (n_in + 31u) & ~31u;
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_r; i += stride) {
            const bool act = i < n_in;
            bool live = false;
            uint32_t idx = 0;
            if (act) {
                idx = list_in ? __ldcg(&list_in[i]) : i;
                const unsigned long long prio = __ldcg(&a.cands[idx].prio);
                const uint32_t cell = __ldcg(&a.cands[idx].cell), h2 = __ldcg(&a.cands[idx].h2);
                const uint32_t tgt = __ldcg(&a.cands[idx].target);
                const uint32_t* hw = cell_h2(a, cell);
                const uint32_t weight = 1u + (tgt >> 16);
                int target = -1;
                bool dup = false;
                // slots before the start held other keys when the pass began
                for (uint32_t e = tgt & 0xFFu; e < ne; ++e) {
                    const uint32_t h = __ldcg(&hw[e]);
                    if (h == h2) { dup = true; break; }
                    if (h == 0u) { target = (int)e; break; }
                }
                if (dup) n_dup += weight;
                else if (target < 0) n_full += weight;
                else if (final_round) atomicOr(&a.ctl->err, ERR_INSERT);
                else {
                    a.cands[idx].target = (uint32_t)target | (tgt & 0xFFFFFF00u);
                    atomicMin(&a.claims[cell], claim_word(epoch, prio));
                    live = true;
                }
            }
            const uint32_t pos = warp_append(&a.ctl->mid_count[round], live);
            if (live) a.lists[2][pos] = idx;
        }
        if (!grid_barrier(a.ctl)) return;
        if (final_round) break;
        // ---- resolve: the smallest (point, node) per cell writes its slot
        const uint32_t n_mid = __ldcg(&a.ctl->mid_count[round]);
        uint32_t* list_out = a.lists[round & 1u];
        const uint32_t n_m = (n_mid + 31u) & ~31u;
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_m; i += stride) {
            const bool act = i < n_mid;
            bool lose = false;
            uint32_t idx = 0;
            if (act) {
                idx = __ldcg(&a.lists[2][i]);
                const unsigned long long prio = __ldcg(&a.cands[idx].prio);
                const uint32_t cell = __ldcg(&a.cands[idx].cell);
                if (__ldcg(&a.claims[cell]) == claim_word(epoch, prio)) {
                    const uint32_t tgt = __ldcg(&a.cands[idx].target);
                    const uint32_t e = tgt & 0xFFu;
                    cell_h2(a, cell)[e] = __ldcg(&a.cands[idx].h2);
                    float* val = cell_val(a, cell, e);
                    val[0] = __ldcg(&a.cands[idx].r);
                    val[1] = __ldcg(&a.cands[idx].g);
                    val[2] = __ldcg(&a.cands[idx].b);
                    n_ins++;
                    n_dup += tgt >> 16;   // its shadows find it in the table
                } else {
                    lose = true;
                }
            }
            const uint32_t pos = warp_append(&a.ctl->out_count[round], lose);
            if (lose) list_out[pos] = idx;
        }
        if (!grid_barrier(a.ctl)) return;
    }
    warp_add_u64(&a.stats[ST_DUP], n_dup);
    warp_add_u64(&a.stats[ST_FULL], n_full);
    warp_add_u64(&a.stats[ST_INSERTED], n_ins);
}

// ---- cell-grouped insert: the same (point, node) order per cell, without rounds.
// Candidates are partitioned into bins of INS_CELLS consecutive cells (count, scan,
// scatter: coalesced), then one block per bin groups its candidates by cell in shared
// memory and one thread per cell inserts that cell's candidates in ascending order.
constexpr uint32_t INS_CELLS = INSERT_BIN_CELLS;   // cells per bin (a multiple of 256)
constexpr uint32_t INS_SMEM_BINS = 8192;  // bins counted in shared memory by the partition
constexpr uint32_t INS_WARP_MAX = 256;     // a bin with at most this many candidates: one warp
constexpr uint32_t INS_MID = 2048;         // at most this many: one block, staged in one pass

// Inserts one candidate into a cell owned by the calling thread (Alg. 1 scan).
__device__ __forceinline__ void insert_one(const BatchArgs& a, const Candidate& c, uint32_t ne,
                                           unsigned long long* n_ins, unsigned long long* n_dup,
                                           unsigned long long* n_full, unsigned long long* n_rep) {
    uint32_t* cw = cell_h2(a, c.cell);
    const uint32_t weight = 1u + (c.target >> 16);
    int target = -1;
    bool dup = false;
    // slots before the start held other keys when the pass began
    for (uint32_t e = c.target & 0xFFu; e < ne; ++e) {
        const uint32_t h = cw[e];
        if (h == c.h2) { dup = true; break; }
        if (h == 0u) { target = (int)e; break; }
    }
    if (!dup && target < 0 && a.slot_cls) {
        // replacement by visibility class: the first entry of the largest class, if larger
        // than the newcomer's
        const uint8_t* cc = a.slot_cls + (size_t)c.cell * ne;
        uint32_t worst = (c.target >> 8) & 0xFFu;
        int victim = -1;
        for (uint32_t e = 0; e < ne; ++e)
            if (cc[e] > worst) {
                worst = cc[e];
                victim = (int)e;
            }
        if (victim >= 0) {
            cw[victim] = c.h2;
            a.slot_cls[(size_t)c.cell * ne + victim] = (uint8_t)((c.target >> 8) & 0xFFu);
            float* val = cell_val(a, c.cell, (uint32_t)victim);
            val[0] = c.r;
            val[1] = c.g;
            val[2] = c.b;
            *n_rep += 1;
            return;
        }
    }
    if (dup) {
        *n_dup += weight;
    } else if (target < 0) {
        *n_full += weight;
    } else {
        cw[target] = c.h2;
        if (a.slot_cls) a.slot_cls[(size_t)c.cell * ne + target] = (uint8_t)((c.target >> 8) & 0xFFu);
        float* val = cell_val(a, c.cell, (uint32_t)target);
        val[0] = c.r;
        val[1] = c.g;
        val[2] = c.b;
        *n_ins += 1;
        *n_dup += c.target >> 16;   // its shadows find it in the table
    }
}

__device__ __forceinline__ uint32_t bin_of(uint32_t cell) { return cell / INS_CELLS; }

// Candidates per bin, counted from the compact cell array the evaluation wrote.
__global__ void __launch_bounds__(256) k_bin_count(BatchArgs a) {
    __shared__ uint32_t s_cnt[INS_SMEM_BINS];
    const uint32_t nb = a.n_bins;
    const uint32_t n_in = min(a.ctl->n_cand, a.probe_cap);
    if (blockIdx.x * blockDim.x >= n_in) return;   // uniform: this block has no candidates
    // few candidates per bin: global atomics are cheaper than clearing and flushing the
    // shared histogram
    const bool local = nb <= INS_SMEM_BINS && n_in / gridDim.x >= nb / 4u;
    if (local) {
        for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) s_cnt[b] = 0;
        __syncthreads();
    }
    const uint32_t* cc = a.lists[0];
    const uint32_t stride = gridDim.x * blockDim.x;
    // four independent loads in flight per thread
    for (uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n_in; i0 += 4 * stride) {
        uint32_t c[4];
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) c[k] = i0 + k * stride < n_in ? cc[i0 + k * stride] : 0u;
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k)
            if (i0 + k * stride < n_in) atomicAdd(local ? &s_cnt[bin_of(c[k])] : &a.bin_cnt[bin_of(c[k])], 1u);
    }
    if (local) {
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x)
            if (s_cnt[b]) atomicAdd(&a.bin_cnt[b], s_cnt[b]);
    }
}

// Exclusive scan of the bin counts (one block); bin_cnt becomes the fill cursor.  Also lists
// the non-empty bins by the kernel that resolves them: a warp (at most INS_WARP_MAX
// candidates), a block (at most INS_MID) or a block in ranges of cells (more).
__global__ void k_bin_scan(BatchArgs a) {
    __shared__ uint32_t s_tmp[33];
    __shared__ unsigned long long s_tmp64[33];
    constexpr uint32_t PER_MAX = 8;   // bins per thread held in registers
    const uint32_t T = blockDim.x, t = threadIdx.x, N = a.n_bins;
    const uint32_t per = (N + T - 1) / T;
    const uint32_t lo = min(t * per, N), hi = min(lo + per, N);
    // the class of a bin, as one of three 21-bit fields of a 64-bit counter
    auto cls = [](uint32_t x) -> unsigned long long {
        return x == 0 ? 0ull : x <= INS_WARP_MAX ? 1ull : x <= INS_MID ? (1ull << 21) : (1ull << 42);
    };
    uint32_t cv[PER_MAX];
    uint32_t c = 0;
    unsigned long long nc = 0;
    if (per <= PER_MAX) {
#pragma unroll
        for (uint32_t k = 0; k < PER_MAX; ++k) cv[k] = lo + k < hi ? a.bin_cnt[lo + k] : 0u;
#pragma unroll
        for (uint32_t k = 0; k < PER_MAX; ++k) {
            c += cv[k];
            nc += cls(cv[k]);
        }
    } else {
        for (uint32_t b = lo; b < hi; ++b) {
            const uint32_t x = a.bin_cnt[b];
            c += x;
            nc += cls(x);
        }
    }
    uint32_t tot;
    unsigned long long tcls;
    uint32_t base = block_incl_scan(c, s_tmp, &tot) - c;
    const unsigned long long pc = block_incl_scan(nc, s_tmp64, &tcls) - nc;
    const uint32_t M21 = (1u << 21) - 1u;
    const uint32_t tw = (uint32_t)tcls & M21, tm = (uint32_t)(tcls >> 21) & M21, tb = (uint32_t)(tcls >> 42) & M21;
    uint32_t pw = (uint32_t)pc & M21, pm = tw + ((uint32_t)(pc >> 21) & M21), pb = tw + tm + ((uint32_t)(pc >> 42) & M21);
    auto emit = [&](uint32_t b, uint32_t x) {
        a.bin_base[b] = base;
        a.bin_cnt[b] = base;
        base += x;
        if (x == 0) return;
        if (x <= INS_WARP_MAX) a.bin_list[pw++] = b;
        else if (x <= INS_MID) a.bin_list[pm++] = b;
        else a.bin_list[pb++] = b;
    };
    if (per <= PER_MAX) {
#pragma unroll
        for (uint32_t k = 0; k < PER_MAX; ++k)
            if (lo + k < hi) emit(lo + k, cv[k]);
    } else {
        for (uint32_t b = lo; b < hi; ++b) emit(b, a.bin_cnt[b]);
    }
    if (t == T - 1) {
        a.bin_base[N] = tot;
        a.ctl->bins_warp = tw;
        a.ctl->bins_mid = tm;
        a.ctl->bins_big = tb;
    }
}

// Copies every candidate into its bin's range.  A block takes a contiguous range of
// candidates: it counts them per bin in shared memory, reserves its part of every bin with
// one global atomic per bin, then places them.  The writes land at scattered positions;
// nothing else is written (a scattered 4-byte write costs nearly as much as a 32-byte one).
__global__ void __launch_bounds__(256) k_bin_scatter(BatchArgs a) {
    __shared__ uint32_t s_cnt[INS_SMEM_BINS];
    constexpr uint32_t U = 4;   // candidates in flight per thread
    const uint32_t nb = a.n_bins;
    const uint32_t n_in = min(a.ctl->n_cand, a.probe_cap);
    const uint32_t* cc = a.lists[0];
    const uint32_t T = blockDim.x;
    uint32_t lo, hi;
    block_range(n_in, &lo, &hi);
    if (lo >= hi) return;   // uniform: this block has no candidates
    // few candidates in this block per bin: take positions with global atomics instead of
    // clearing, filling and flushing the shared histogram
    const bool local = nb <= INS_SMEM_BINS && hi - lo >= nb / 4u;
    if (local) {
        for (uint32_t b = threadIdx.x; b < nb; b += T) s_cnt[b] = 0;
        __syncthreads();
        for (uint32_t i0 = lo + threadIdx.x; i0 < hi; i0 += U * T) {
            uint32_t c[U];
#pragma unroll
            for (uint32_t k = 0; k < U; ++k) c[k] = i0 + k * T < hi ? cc[i0 + k * T] : 0u;
#pragma unroll
            for (uint32_t k = 0; k < U; ++k)
                if (i0 + k * T < hi) atomicAdd(&s_cnt[bin_of(c[k])], 1u);
        }
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < nb; b += T)
            if (s_cnt[b]) s_cnt[b] = atomicAdd(&a.bin_cnt[b], s_cnt[b]);
        __syncthreads();
    }
    const uint4* src = reinterpret_cast<const uint4*>(a.cands);
    uint4* dst = reinterpret_cast<uint4*>(a.cands_binned);
    for (uint32_t i0 = lo + threadIdx.x; i0 < hi; i0 += U * T) {
        uint32_t c[U];
        uint4 x[U][2];
#pragma unroll
        for (uint32_t k = 0; k < U; ++k) {
            const uint32_t i = i0 + k * T;
            if (i < hi) {
                c[k] = cc[i];
                x[k][0] = __ldcs(src + 2 * (size_t)i);
                x[k][1] = __ldcs(src + 2 * (size_t)i + 1);
            }
        }
#pragma unroll
        for (uint32_t k = 0; k < U; ++k) {
            const uint32_t i = i0 + k * T;
            if (i < hi) {
                const uint32_t b = bin_of(c[k]);
                const uint32_t pos = atomicAdd(local ? &s_cnt[b] : &a.bin_cnt[b], 1u);
                dst[2 * (size_t)pos] = x[k][0];
                dst[2 * (size_t)pos + 1] = x[k][1];
            }
        }
    }
}

// ---- resolution of one bin: its candidates are grouped by cell and each cell is resolved
// in ascending (point, node) order by one thread holding the cell's hash2 words.  Bins are
// resolved by one of three kernels according to their number of candidates: a warp per bin
// (at most INS_WARP_MAX), a block per bin staged in one pass (at most INS_MID), or a block
// per bin staged in ranges of cells (more).
constexpr uint32_t INS_MID_T = INS_CELLS;               // one thread per cell of the bin
constexpr uint32_t INS_MID_PER = INS_MID / INS_MID_T;   // candidates per thread
constexpr uint8_t RES_NONE = 0xFFu;

// Resolves one cell (one thread).  order[x0 .. x0 + n) lists the cell's candidates in
// ascending priority as indices into the staged hash2 / target arrays; the slot each
// inserted candidate took is written to res[] (RES_NONE for the others).  Every candidate
// of a cell saw the same snapshot, so slots before its start held other keys and only the
// slots filled by this insert can hold its hash2.
template <typename IDX>
__device__ __forceinline__ void resolve_cell(const BatchArgs& a, uint32_t cell, const IDX* order, uint32_t x0,
                                             uint32_t n, const uint32_t* sh2, const uint32_t* stgt, uint8_t* res,
                                             uint32_t ne, unsigned long long* n_ins, unsigned long long* n_dup,
                                             unsigned long long* n_full) {
    uint32_t* cw = cell_h2(a, cell);
    uint32_t h[MAX_ENTRIES];
    uint32_t used = ne;
    for (uint32_t e = 0; e < ne; ++e) {
        h[e] = __ldcg(&cw[e]);
        if (h[e] == 0u && used == ne) used = e;
    }
    for (uint32_t x = x0; x < x0 + n; ++x) {
        const uint32_t j = order[x];
        const uint32_t hc = sh2[j], tg = stgt[j];
        const uint32_t shadows = tg >> 16;
        bool dup = false;
        for (uint32_t e = tg & 0xFFu; e < used; ++e)
            if (h[e] == hc) { dup = true; break; }
        if (dup) {
            *n_dup += 1u + shadows;
        } else if (used >= ne) {
            *n_full += 1u + shadows;
        } else {
            h[used] = hc;
            cw[used] = hc;
            res[j] = (uint8_t)used;
            used++;
            *n_ins += 1;
            *n_dup += shadows;   // its shadows find it in the table
        }
    }
}

// The same with replacement by visibility class (the prioritisation Sec. 5 proposes): a
// candidate whose hash2 is in the cell is a duplicate; otherwise it takes the first empty
// slot, or else overwrites the entry of the largest class if that class is larger than its
// own (the first such entry on ties), or is dropped.  An eviction can put a key anywhere,
// so every occupied slot is compared.  The slot file (hash2 words and classes) is written
// at once; a slot's value is written afterwards by the candidate left owning it, so a
// candidate that took a slot and was evicted within this resolution gives up its res[].
template <typename IDX>
__device__ __forceinline__ void resolve_cell_replace(const BatchArgs& a, uint32_t cell, const IDX* order, uint32_t x0,
                                                     uint32_t n, const uint32_t* sh2, const uint32_t* stgt,
                                                     uint8_t* res, uint32_t ne, unsigned long long* n_ins,
                                                     unsigned long long* n_dup, unsigned long long* n_full,
                                                     unsigned long long* n_rep) {
    uint32_t* cw = cell_h2(a, cell);
    uint8_t* cc = a.slot_cls + (size_t)cell * ne;
    uint32_t h[MAX_ENTRIES];
    uint32_t k[MAX_ENTRIES];
    uint32_t owner[MAX_ENTRIES];   // staged index of the candidate that took the slot here
    uint32_t used = ne;
    for (uint32_t e = 0; e < ne; ++e) {
        h[e] = __ldcg(&cw[e]);
        k[e] = h[e] ? (uint32_t)cc[e] : 0u;
        owner[e] = 0xFFFFFFFFu;
        if (h[e] == 0u && used == ne) used = e;
    }
    for (uint32_t x = x0; x < x0 + n; ++x) {
        const uint32_t j = order[x];
        const uint32_t hc = sh2[j], q = (stgt[j] >> 8) & 0xFFu;
        bool dup = false;
        for (uint32_t e = 0; e < used; ++e) dup |= h[e] == hc;
        if (dup) {
            *n_dup += 1;
            continue;
        }
        uint32_t slot = used;
        if (used < ne) {
            used++;
            *n_ins += 1;
        } else {
            uint32_t worst = q;
            slot = ne;
            for (uint32_t e = 0; e < ne; ++e)
                if (k[e] > worst) {
                    worst = k[e];
                    slot = e;
                }
            if (slot == ne) {
                *n_full += 1;
                continue;
            }
            if (owner[slot] != 0xFFFFFFFFu) res[owner[slot]] = RES_NONE;
            *n_rep += 1;
        }
        h[slot] = hc;
        k[slot] = q;
        owner[slot] = j;
        cw[slot] = hc;
        cc[slot] = (uint8_t)q;
        res[j] = (uint8_t)slot;
    }
}

// The same for N_e <= 8 with the cell's hash2 words held in registers (w0, w1: the cell's
// first 32 bytes, loaded by the caller).
template <typename IDX>
__device__ __forceinline__ void resolve_cell8(const BatchArgs& a, uint32_t cell, uint4 w0, uint4 w1, const IDX* order,
                                              uint32_t x0, uint32_t n, const uint32_t* sh2, const uint32_t* stgt,
                                              uint8_t* res, uint32_t ne, unsigned long long* n_ins,
                                              unsigned long long* n_dup, unsigned long long* n_full) {
    uint32_t h[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
    uint32_t used = ne;
#pragma unroll
    for (int e = 7; e >= 0; --e)
        if ((uint32_t)e < ne && h[e] == 0u) used = (uint32_t)e;   // the first empty slot
    uint32_t* cw = cell_h2(a, cell);
    for (uint32_t x = x0; x < x0 + n; ++x) {
        const uint32_t j = order[x];
        const uint32_t hc = sh2[j], tg = stgt[j];
        const uint32_t shadows = tg >> 16, st = tg & 0xFFu;
        bool dup = false;
#pragma unroll
        for (uint32_t e = 0; e < 8; ++e) dup |= e >= st && e < used && h[e] == hc;
        if (dup) {
            *n_dup += 1u + shadows;
        } else if (used >= ne) {
            *n_full += 1u + shadows;
        } else {
#pragma unroll
            for (uint32_t e = 0; e < 8; ++e)
                if (e == used) h[e] = hc;
            cw[used] = hc;
            res[j] = (uint8_t)used;
            used++;
            *n_ins += 1;
            *n_dup += shadows;   // its shadows find it in the table
        }
    }
}

// The first 32 bytes of a cell (its hash2 words for N_e <= 8; a cell is 16 * N_e bytes,
// so 16 bytes are read for N_e <= 4).
__device__ __forceinline__ void load_cell_words(const BatchArgs& a, uint32_t cell, uint4* w0, uint4* w1) {
    const uint4* hw = reinterpret_cast<const uint4*>(cell_h2(a, cell));
    *w0 = __ldcg(hw);
    *w1 = a.n_entries > 4 ? __ldcg(hw + 1) : make_uint4(0, 0, 0, 0);
}

// Writes the value of an inserted candidate (binned index i) into its slot.
__device__ __forceinline__ void write_value(const BatchArgs& a, uint32_t i, uint32_t cell, uint32_t slot) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(&a.cands_binned[i].r));   // r, g, b, target
    float* val = cell_val(a, cell, slot);
    val[0] = v.x;
    val[1] = v.y;
    val[2] = v.z;
}

// Bins of 1 .. INS_WARP_MAX candidates: one warp per bin, with its own stage in shared
// memory and no block barrier, so that many sparse bins are in flight per SM.  Lane l
// reads candidates l, l + 32, ... once; a count per cell and a warp scan stage the bin
// grouped by cell; each candidate's rank by priority within its cell orders the cell's segment;
// lane l resolves cells 8l .. 8l + 7; then the inserted candidates write their values.
constexpr uint32_t INS_WARP_PER = INS_WARP_MAX / 32;
constexpr uint32_t INS_WARPS = 4;   // warps (bins in flight) per block
static_assert(INS_CELLS == 8 * 32, "a lane resolves 8 consecutive cells of a bin");

struct WarpStage {
    unsigned long long key[INS_WARP_MAX];   // priority
    uint32_t h2[INS_WARP_MAX];
    uint32_t tgt[INS_WARP_MAX];
    uint32_t cnt[INS_CELLS];
    uint32_t off[INS_CELLS + 1];
    uint16_t ord[INS_WARP_MAX];
    uint8_t res[INS_WARP_MAX];
};

__global__ void __launch_bounds__(INS_WARPS * 32, 6) k_bin_insert_warp(BatchArgs a) {
    __shared__ WarpStage s_stage[INS_WARPS];
    const uint32_t w = threadIdx.x >> 5, lane = lane_id();
    WarpStage& st = s_stage[w];
    const uint32_t ne = a.n_entries;
    const Candidate* cb = a.cands_binned;
    unsigned long long n_dup = 0, n_full = 0, n_ins = 0, n_rep = 0;
    const uint32_t n_list = a.ctl->bins_warp;
    for (uint32_t x = blockIdx.x * INS_WARPS + w; x < n_list; x += gridDim.x * INS_WARPS) {
        const uint32_t bin = a.bin_list[x];
        const uint32_t lo = a.bin_base[bin], hi = a.bin_base[bin + 1];
        const uint32_t c0 = bin * INS_CELLS;
#pragma unroll
        for (uint32_t q = 0; q < 8; ++q) st.cnt[8 * lane + q] = 0;
        __syncwarp();
        // ---- one read of every candidate; count per cell, rank of arrival in its cell
        uint32_t cl[INS_WARP_PER], pos[INS_WARP_PER], hh[INS_WARP_PER], tg[INS_WARP_PER];
        unsigned long long pr[INS_WARP_PER];
#pragma unroll
        for (uint32_t k = 0; k < INS_WARP_PER; ++k) {
            const uint32_t i = lo + lane + 32 * k;
            cl[k] = 0;
            if (i < hi) {
                const uint4 q = __ldcg(reinterpret_cast<const uint4*>(&cb[i]));   // prio, cell, hash2
                tg[k] = __ldcg(&cb[i].target);
                pr[k] = ((unsigned long long)q.y << 32) | q.x;
                cl[k] = q.z - c0;
                hh[k] = q.w;
            }
        }
#pragma unroll
        for (uint32_t k = 0; k < INS_WARP_PER; ++k) {
            const uint32_t i = lo + lane + 32 * k;
            pos[k] = i < hi ? atomicAdd(&st.cnt[cl[k]], 1u) : 0u;
        }
        __syncwarp();
        // ---- exclusive scan of the counts: lane l holds cells 8l .. 8l + 7
        uint32_t v[8], sum = 0;
#pragma unroll
        for (uint32_t q = 0; q < 8; ++q) {
            v[q] = st.cnt[8 * lane + q];
            sum += v[q];
        }
        uint32_t incl = sum;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += y;
        }
        uint32_t run = incl - sum;
#pragma unroll
        for (uint32_t q = 0; q < 8; ++q) {
            st.off[8 * lane + q] = run;
            run += v[q];
        }
        if (lane == 31) st.off[INS_CELLS] = incl;
        __syncwarp();
        // ---- place: priority, hash2 and target, grouped by cell
#pragma unroll
        for (uint32_t k = 0; k < INS_WARP_PER; ++k) {
            const uint32_t i = lo + lane + 32 * k;
            pos[k] += st.off[cl[k]];
            if (i < hi) {
                st.key[pos[k]] = pr[k];
                st.h2[pos[k]] = hh[k];
                st.tgt[pos[k]] = tg[k];
                st.res[pos[k]] = RES_NONE;
            }
        }
        __syncwarp();
        // ---- order each cell's segment by priority
#pragma unroll
        for (uint32_t k = 0; k < INS_WARP_PER; ++k) {
            const uint32_t i = lo + lane + 32 * k;
            if (i < hi) {
                const uint32_t x0 = st.off[cl[k]], x1 = st.off[cl[k] + 1];
                const unsigned long long kv = st.key[pos[k]];
                uint32_t rank = 0;
                for (uint32_t y = x0; y < x1; ++y) rank += st.key[y] < kv ? 1u : 0u;
                st.ord[x0 + rank] = (uint16_t)pos[k];
            }
        }
        __syncwarp();
        // ---- resolve this lane's cells, two at a time so that their loads overlap
#pragma unroll
        for (uint32_t q = 0; q < 8; q += 2) {
            const uint32_t ca = 8 * lane + q, cbb = ca + 1;
            const uint32_t xa = st.off[ca], xb = st.off[cbb], xe = st.off[cbb + 1];
            if (a.slot_cls) {
                if (xb > xa)
                    resolve_cell_replace(a, c0 + ca, st.ord, xa, xb - xa, st.h2, st.tgt, st.res, ne, &n_ins, &n_dup,
                                         &n_full, &n_rep);
                if (xe > xb)
                    resolve_cell_replace(a, c0 + cbb, st.ord, xb, xe - xb, st.h2, st.tgt, st.res, ne, &n_ins, &n_dup,
                                         &n_full, &n_rep);
            } else if (ne <= 8) {
                uint4 a0 = make_uint4(0, 0, 0, 0), a1 = a0, b0 = a0, b1 = a0;
                if (xb > xa) load_cell_words(a, c0 + ca, &a0, &a1);
                if (xe > xb) load_cell_words(a, c0 + cbb, &b0, &b1);
                if (xb > xa)
                    resolve_cell8(a, c0 + ca, a0, a1, st.ord, xa, xb - xa, st.h2, st.tgt, st.res, ne, &n_ins, &n_dup,
                                  &n_full);
                if (xe > xb)
                    resolve_cell8(a, c0 + cbb, b0, b1, st.ord, xb, xe - xb, st.h2, st.tgt, st.res, ne, &n_ins, &n_dup,
                                  &n_full);
            } else {
                if (xb > xa) resolve_cell(a, c0 + ca, st.ord, xa, xb - xa, st.h2, st.tgt, st.res, ne, &n_ins, &n_dup, &n_full);
                if (xe > xb) resolve_cell(a, c0 + cbb, st.ord, xb, xe - xb, st.h2, st.tgt, st.res, ne, &n_ins, &n_dup, &n_full);
            }
        }
        __syncwarp();
        // ---- values of the inserted candidates
#pragma unroll
        for (uint32_t k = 0; k < INS_WARP_PER; ++k) {
            const uint32_t i = lo + lane + 32 * k;
            if (i < hi) {
                const uint8_t r = st.res[pos[k]];
                if (r != RES_NONE) write_value(a, i, c0 + cl[k], r);
            }
        }
        __syncwarp();
    }
    warp_add_u64(&a.stats[ST_DUP], n_dup);
    warp_add_u64(&a.stats[ST_FULL], n_full);
    warp_add_u64(&a.stats[ST_INSERTED], n_ins);
    warp_add_u64(&a.stats[ST_REPLACED], n_rep);
}

struct MidSmem {   // byte offsets into dynamic shared memory
    static constexpr uint32_t key = 0;                                // u64 [INS_MID] priority
    static constexpr uint32_t h2 = key + INS_MID * 8;                 // u32 [INS_MID]
    static constexpr uint32_t tgt = h2 + INS_MID * 4;                 // u32 [INS_MID]
    static constexpr uint32_t ord = tgt + INS_MID * 4;                // u16 [INS_MID]
    static constexpr uint32_t res = ord + INS_MID * 2;                // u8  [INS_MID]
    static constexpr uint32_t cnt = res + INS_MID;                    // u32 [INS_CELLS]
    static constexpr uint32_t off = cnt + INS_CELLS * 4;              // u32 [INS_CELLS + 4]
    static constexpr uint32_t wsum = off + (INS_CELLS + 4) * 4;       // u32 [32]
    static constexpr uint32_t end = wsum + 32 * 4;
};
static_assert(INS_MID <= 65536, "staged indices are 16-bit");
static_assert(INS_MID_T % 32 == 0 && INS_MID_T <= 1024, "one thread per cell of a bin");

size_t insert_mid_smem_bytes() { return MidSmem::end; }

// Bins of INS_WARP_MAX + 1 .. INS_MID candidates: a block per bin, one thread per cell.  Each
// thread takes up to INS_MID_PER candidates; a count per cell, a block scan and one
// placement stage the bin grouped by cell in a single read.  Each candidate's rank by
// priority within its cell orders the cell's segment (all candidates in parallel); one
// thread per cell resolves it with the cell's hash2 words, loaded while the bin is
// staged; then the inserted candidates write their values, all in parallel.
__global__ void __launch_bounds__(INS_MID_T, 4) k_bin_insert_mid(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char msm[];
    unsigned long long* s_key = reinterpret_cast<unsigned long long*>(msm + MidSmem::key);
    uint32_t* s_h2 = reinterpret_cast<uint32_t*>(msm + MidSmem::h2);
    uint32_t* s_tgt = reinterpret_cast<uint32_t*>(msm + MidSmem::tgt);
    uint16_t* s_ord = reinterpret_cast<uint16_t*>(msm + MidSmem::ord);
    uint8_t* s_res = reinterpret_cast<uint8_t*>(msm + MidSmem::res);
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(msm + MidSmem::cnt);
    uint32_t* s_off = reinterpret_cast<uint32_t*>(msm + MidSmem::off);
    uint32_t* s_wsum = reinterpret_cast<uint32_t*>(msm + MidSmem::wsum);
    const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;
    const uint32_t ne = a.n_entries;
    const Candidate* cb = a.cands_binned;
    unsigned long long n_dup = 0, n_full = 0, n_ins = 0, n_rep = 0;
    const uint32_t n_list = a.ctl->bins_mid, first = a.ctl->bins_warp;
    for (uint32_t x = blockIdx.x; x < n_list; x += gridDim.x) {
        const uint32_t bin = a.bin_list[first + x];
        const uint32_t lo = a.bin_base[bin], hi = a.bin_base[bin + 1];
        const uint32_t c0 = bin * INS_CELLS;
        s_cnt[t] = 0;
        __syncthreads();
        // ---- count per cell; each candidate's rank of arrival among its cell's
        uint32_t cl[INS_MID_PER], pos[INS_MID_PER];
#pragma unroll
        for (uint32_t k = 0; k < INS_MID_PER; ++k) {
            const uint32_t i = lo + t + k * INS_MID_T;
            cl[k] = i < hi ? __ldcg(&cb[i].cell) - c0 : 0u;
        }
#pragma unroll
        for (uint32_t k = 0; k < INS_MID_PER; ++k) {
            const uint32_t i = lo + t + k * INS_MID_T;
            pos[k] = i < hi ? atomicAdd(&s_cnt[cl[k]], 1u) : 0u;
        }
        __syncthreads();
        // ---- this thread's cell: start loading its hash2 words
        const uint32_t v = s_cnt[t];
        uint4 w0 = make_uint4(0, 0, 0, 0), w1 = w0;
        if (v && ne <= 8) load_cell_words(a, c0 + t, &w0, &w1);
        // ---- exclusive scan of the per-cell counts (thread t holds cell t)
        uint32_t incl = v;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t wv = lane < INS_MID_T / 32 ? s_wsum[lane] : 0u;
            uint32_t wi = wv;
#pragma unroll
            for (uint32_t o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL_MASK, wi, o);
                if (lane >= o) wi += y;
            }
            s_wsum[lane] = wi - wv;
        }
        __syncthreads();
        const uint32_t excl = incl - v + s_wsum[warp];
        s_off[t] = excl;
        __syncthreads();
        // ---- place: priority, hash2 and target, grouped by cell
#pragma unroll
        for (uint32_t k = 0; k < INS_MID_PER; ++k) pos[k] += s_off[cl[k]];
#pragma unroll
        for (uint32_t h = 0; h < INS_MID_PER; h += 4) {
            uint4 q[4];
            uint32_t tg[4];
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                const uint32_t i = lo + t + (h + k) * INS_MID_T;
                if (i < hi) {
                    q[k] = __ldcg(reinterpret_cast<const uint4*>(&cb[i]));   // prio, cell, hash2
                    tg[k] = __ldcg(&cb[i].target);
                }
            }
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                const uint32_t i = lo + t + (h + k) * INS_MID_T;
                if (i < hi) {
                    const uint32_t p = pos[h + k];
                    s_key[p] = ((unsigned long long)q[k].y << 32) | q[k].x;
                    s_h2[p] = q[k].w;
                    s_tgt[p] = tg[k];
                    s_res[p] = RES_NONE;
                }
            }
        }
        __syncthreads();
        // ---- order each cell's segment by priority: every candidate finds its rank
#pragma unroll
        for (uint32_t k = 0; k < INS_MID_PER; ++k) {
            const uint32_t i = lo + t + k * INS_MID_T;
            if (i < hi) {
                const uint32_t x0 = s_off[cl[k]], n = s_cnt[cl[k]];
                const unsigned long long kv = s_key[pos[k]];
                uint32_t rank = 0;
                for (uint32_t y = x0; y < x0 + n; ++y) rank += s_key[y] < kv ? 1u : 0u;
                s_ord[x0 + rank] = (uint16_t)pos[k];
            }
        }
        __syncthreads();
        // ---- resolve: one thread per cell
        if (v) {
            if (a.slot_cls)
                resolve_cell_replace(a, c0 + t, s_ord, excl, v, s_h2, s_tgt, s_res, ne, &n_ins, &n_dup, &n_full,
                                     &n_rep);
            else if (ne <= 8)
                resolve_cell8(a, c0 + t, w0, w1, s_ord, excl, v, s_h2, s_tgt, s_res, ne, &n_ins, &n_dup, &n_full);
            else
                resolve_cell(a, c0 + t, s_ord, excl, v, s_h2, s_tgt, s_res, ne, &n_ins, &n_dup, &n_full);
        }
        __syncthreads();
        // ---- values of the inserted candidates
#pragma unroll
        for (uint32_t k = 0; k < INS_MID_PER; ++k) {
            const uint32_t i = lo + t + k * INS_MID_T;
            if (i < hi) {
                const uint8_t r = s_res[pos[k]];
                if (r != RES_NONE) write_value(a, i, c0 + cl[k], r);
            }
        }
        __syncthreads();
    }
    warp_add_u64(&a.stats[ST_DUP], n_dup);
    warp_add_u64(&a.stats[ST_FULL], n_full);
    warp_add_u64(&a.stats[ST_INSERTED], n_ins);
    warp_add_u64(&a.stats[ST_REPLACED], n_rep);
}

// Bins of more than INS_MID candidates: one block per bin stages the candidates of a range
// of cells at a time in shared memory, grouped by cell: sort key (cell offset << 44 |
// priority), hash2, target and source index.  One thread per cell sorts its segment and inserts it with the cell's hash2
// words in registers; a range holding a cell with more than INS_CELL_SORT candidates is
// sorted by the whole block instead.  A single cell with more candidates than INS_STAGE is
// resolved by a block-wide selection.
constexpr uint32_t INS_STAGE = 1024;
constexpr uint32_t INS_CELL_SORT = 64;
static_assert(INS_CELLS % 256 == 0, "k_bin_insert scans INS_CELLS / 256 cells per thread");

struct InsSmem {   // byte offsets into dynamic shared memory
    static constexpr uint32_t key = 0;                                   // u64 [INS_STAGE]
    static constexpr uint32_t idx = key + INS_STAGE * 8;                 // u32 [INS_STAGE]
    static constexpr uint32_t h2 = idx + INS_STAGE * 4;                  // u32 [INS_STAGE]
    static constexpr uint32_t tgt = h2 + INS_STAGE * 4;                  // u32 [INS_STAGE]
    static constexpr uint32_t src = tgt + INS_STAGE * 4;                 // u32 [INS_STAGE]
    static constexpr uint32_t cnt = src + INS_STAGE * 4;                 // u32 [INS_CELLS]
    static constexpr uint32_t off = cnt + INS_CELLS * 4;                 // u32 [INS_CELLS + 1]
    static constexpr uint32_t cur = off + (INS_CELLS + 4) * 4;           // u32 [INS_CELLS]
    static constexpr uint32_t part = cur + INS_CELLS * 4;                // u32 [256]
    static constexpr uint32_t best = part + 256 * 4;                     // u64 [256]
    static constexpr uint32_t bidx = best + 256 * 8;                     // u32 [256]
    static constexpr uint32_t misc = bidx + 256 * 4;                     // u32 [4]
    static constexpr uint32_t end = misc + 16;
};

size_t insert_smem_bytes() { return InsSmem::end; }

// Resolves one cell from its staged, sorted segment [x0, x0 + n) (one thread).
__device__ __forceinline__ void insert_staged_cell(const BatchArgs& a, const Candidate* cb, uint32_t cell,
                                                   const uint32_t* idx, const uint32_t* sh2, const uint32_t* stgt,
                                                   const uint32_t* ssrc, uint32_t x0, uint32_t n, uint32_t ne,
                                                   unsigned long long* n_ins, unsigned long long* n_dup,
                                                   unsigned long long* n_full, unsigned long long* n_rep) {
    uint32_t* cw = cell_h2(a, cell);
    uint32_t h[MAX_ENTRIES];
    uint32_t used = ne;
    for (uint32_t e = 0; e < ne; ++e) {
        h[e] = __ldcg(&cw[e]);
        if (h[e] == 0u && used == ne) used = e;
    }
    if (a.slot_cls) {
        // replacement by visibility class, as in resolve_cell_replace; one thread handles
        // the cell's candidates in order and writes each value at once, so an entry
        // replaced later in the same resolution is simply overwritten
        uint8_t* cc = a.slot_cls + (size_t)cell * ne;
        for (uint32_t x = x0; x < x0 + n; ++x) {
            const uint32_t j = idx[x];
            const uint32_t hc = sh2[j], q = (stgt[j] >> 8) & 0xFFu;
            bool dup = false;
            for (uint32_t e = 0; e < used; ++e) dup |= h[e] == hc;
            if (dup) {
                *n_dup += 1;
                continue;
            }
            uint32_t slot = used;
            if (used < ne) {
                used++;
                *n_ins += 1;
            } else {
                uint32_t worst = q;
                slot = ne;
                for (uint32_t e = 0; e < ne; ++e)
                    if ((uint32_t)cc[e] > worst) {
                        worst = cc[e];
                        slot = e;
                    }
                if (slot == ne) {
                    *n_full += 1;
                    continue;
                }
                *n_rep += 1;
            }
            const float4 v = __ldcg(reinterpret_cast<const float4*>(&cb[ssrc[j]].r));   // r, g, b, target
            h[slot] = hc;
            cw[slot] = hc;
            cc[slot] = (uint8_t)q;
            float* val = cell_val(a, cell, slot);
            val[0] = v.x;
            val[1] = v.y;
            val[2] = v.z;
        }
        return;
    }
    for (uint32_t x = x0; x < x0 + n; ++x) {
        const uint32_t j = idx[x];
        const uint32_t hc = sh2[j], tg = stgt[j];
        const uint32_t shadows = tg >> 16;
        bool dup = false;
        // slots before the candidate's start held other keys when the pass began
        for (uint32_t e = tg & 0xFFu; e < used; ++e)
            if (h[e] == hc) { dup = true; break; }
        if (dup) {
            *n_dup += 1u + shadows;
        } else if (used >= ne) {
            *n_full += 1u + shadows;
        } else {
            const float4 v = __ldcg(reinterpret_cast<const float4*>(&cb[ssrc[j]].r));   // r, g, b, target
            h[used] = hc;
            cw[used] = hc;
            float* val = cell_val(a, cell, used);
            val[0] = v.x;
            val[1] = v.y;
            val[2] = v.z;
            used++;
            *n_ins += 1;
            *n_dup += shadows;   // its shadows find it in the table
        }
    }
}

__global__ void __launch_bounds__(256, 6) k_bin_insert(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char ism[];
    unsigned long long* s_key = reinterpret_cast<unsigned long long*>(ism + InsSmem::key);
    uint32_t* s_idx = reinterpret_cast<uint32_t*>(ism + InsSmem::idx);
    uint32_t* s_h2 = reinterpret_cast<uint32_t*>(ism + InsSmem::h2);
    uint32_t* s_tgt = reinterpret_cast<uint32_t*>(ism + InsSmem::tgt);
    uint32_t* s_src = reinterpret_cast<uint32_t*>(ism + InsSmem::src);
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(ism + InsSmem::cnt);
    uint32_t* s_off = reinterpret_cast<uint32_t*>(ism + InsSmem::off);
    uint32_t* s_cur = reinterpret_cast<uint32_t*>(ism + InsSmem::cur);
    uint32_t* s_part = reinterpret_cast<uint32_t*>(ism + InsSmem::part);
    unsigned long long* s_best = reinterpret_cast<unsigned long long*>(ism + InsSmem::best);
    uint32_t* s_bidx = reinterpret_cast<uint32_t*>(ism + InsSmem::bidx);
    uint32_t* s_misc = reinterpret_cast<uint32_t*>(ism + InsSmem::misc);
    const uint32_t ne = a.n_entries;
    const uint32_t t = threadIdx.x, T = blockDim.x;
    const Candidate* cb = a.cands_binned;
    unsigned long long n_dup = 0, n_full = 0, n_ins = 0, n_rep = 0;
    const uint32_t n_list = a.ctl->bins_big, first = a.ctl->bins_warp + a.ctl->bins_mid;
    for (uint32_t x = blockIdx.x; x < n_list; x += gridDim.x) {
        const uint32_t bin = a.bin_list[first + x];
        const uint32_t lo = a.bin_base[bin], hi = a.bin_base[bin + 1];
        const uint32_t c0 = bin * INS_CELLS;
        // ---- per-cell counts and their exclusive scan
        for (uint32_t k = t; k < INS_CELLS; k += T) s_cnt[k] = 0;
        __syncthreads();
        for (uint32_t i = lo + t; i < hi; i += T) atomicAdd(&s_cnt[__ldcg(&cb[i].cell) - c0], 1u);
        __syncthreads();
        const uint32_t per = INS_CELLS / T;
        uint32_t part = 0;
        for (uint32_t k = 0; k < per; ++k) part += s_cnt[t * per + k];
        s_part[t] = part;
        __syncthreads();
        for (uint32_t o = 1; o < T; o <<= 1) {
            const uint32_t v = t >= o ? s_part[t - o] : 0u;
            __syncthreads();
            s_part[t] += v;
            __syncthreads();
        }
        uint32_t run = s_part[t] - part;
        for (uint32_t k = 0; k < per; ++k) {
            s_off[t * per + k] = run;
            run += s_cnt[t * per + k];
        }
        if (t == T - 1) s_off[INS_CELLS] = run;
        __syncthreads();
        // ---- ranges of cells whose candidates fit the stage
        uint32_t s = 0;
        while (s < INS_CELLS) {
            if (t == 0) {
                uint32_t e = s + 1;
                if (s == 0 && s_off[INS_CELLS] <= INS_STAGE) e = INS_CELLS;   // the whole bin fits
                while (e < INS_CELLS && s_off[e + 1] - s_off[s] <= INS_STAGE) ++e;
                s_misc[0] = e;
            }
            __syncthreads();
            const uint32_t e = s_misc[0];
            const uint32_t base = s_off[s], R = s_off[e] - base;
            if (R <= INS_STAGE) {
                // stage the range grouped by cell
                for (uint32_t k = s + t; k < e; k += T) s_cur[k] = s_off[k] - base;
                __syncthreads();
                for (uint32_t i = lo + t; i < hi; i += T) {
                    const uint32_t k = __ldcg(&cb[i].cell) - c0;
                    if (k < s || k >= e) continue;
                    const uint32_t pos = atomicAdd(&s_cur[k], 1u);
                    s_key[pos] = ((unsigned long long)k << 44) | __ldcg(&cb[i].prio);
                    s_idx[pos] = pos;
                    s_h2[pos] = __ldcg(&cb[i].h2);
                    s_tgt[pos] = __ldcg(&cb[i].target);
                    s_src[pos] = i;
                }
                bool heavy = false;
                for (uint32_t k = s + t; k < e; k += T) heavy |= s_cnt[k] > INS_CELL_SORT;
                heavy = __syncthreads_or(heavy) != 0;
                if (heavy) {
                    // a crowded cell: sort the whole range by (cell, priority)
                    uint32_t N = 1;
                    while (N < R) N <<= 1;
                    for (uint32_t i = R + t; i < N; i += T) {
                        s_key[i] = ~0ull;
                        s_idx[i] = 0;
                    }
                    __syncthreads();
                    for (uint32_t kk = 2; kk <= N; kk <<= 1) {
                        for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
                            for (uint32_t i = t; i < N; i += T) {
                                const uint32_t ixj = i ^ j;
                                if (ixj > i) {
                                    const bool up = (i & kk) == 0;
                                    const unsigned long long ki = s_key[i], kj = s_key[ixj];
                                    if ((ki > kj) == up) {
                                        s_key[i] = kj;
                                        s_key[ixj] = ki;
                                        const uint32_t tmp = s_idx[i];
                                        s_idx[i] = s_idx[ixj];
                                        s_idx[ixj] = tmp;
                                    }
                                }
                            }
                            __syncthreads();
                        }
                    }
                }
                for (uint32_t k = s + t; k < e; k += T) {
                    const uint32_t n = s_cnt[k];
                    if (n == 0) continue;
                    const uint32_t x0 = s_off[k] - base;
                    if (!heavy) {
                        // insertion sort of the cell's own segment
                        for (uint32_t x = x0 + 1; x < x0 + n; ++x) {
                            const unsigned long long kv = s_key[x];
                            const uint32_t iv = s_idx[x];
                            uint32_t y = x;
                            while (y > x0 && s_key[y - 1] > kv) {
                                s_key[y] = s_key[y - 1];
                                s_idx[y] = s_idx[y - 1];
                                --y;
                            }
                            s_key[y] = kv;
                            s_idx[y] = iv;
                        }
                    }
                    insert_staged_cell(a, cb, c0 + k, s_idx, s_h2, s_tgt, s_src, x0, n, ne, &n_ins, &n_dup, &n_full,
                                       &n_rep);
                }
                __syncthreads();
            } else {
                // one cell with more candidates than the stage: the block selects them in order
                const uint32_t cell = c0 + s;
                const uint32_t cnt = s_cnt[s];
                unsigned long long last = 0;
                for (uint32_t step = 0; step < cnt; ++step) {
                    unsigned long long best = ~0ull;
                    uint32_t bi = 0;
                    for (uint32_t i = lo + t; i < hi; i += T) {
                        if (__ldcg(&cb[i].cell) != cell) continue;
                        const unsigned long long p = cb[i].prio;
                        if ((step == 0 || p > last) && p < best) { best = p; bi = i; }
                    }
                    s_best[t] = best;
                    s_bidx[t] = bi;
                    __syncthreads();
                    for (uint32_t o = T / 2; o > 0; o >>= 1) {
                        if (t < o && s_best[t + o] < s_best[t]) {
                            s_best[t] = s_best[t + o];
                            s_bidx[t] = s_bidx[t + o];
                        }
                        __syncthreads();
                    }
                    if (t == 0 && s_best[0] != ~0ull) insert_one(a, cb[s_bidx[0]], ne, &n_ins, &n_dup, &n_full, &n_rep);
                    last = s_best[0];
                    // keep-first: once the cell is full (its slots fill as a prefix) nothing
                    // changes it, so each remaining candidate is a duplicate or dropped as full
                    // whatever the order: they resolve in parallel
                    if (t == 0) s_misc[1] = (!a.slot_cls && __ldcg(&cell_h2(a, cell)[ne - 1]) != 0u) ? 1u : 0u;
                    __syncthreads();
                    if (s_misc[1]) {
                        const uint32_t* cw = cell_h2(a, cell);
                        for (uint32_t i = lo + t; i < hi; i += T) {
                            if (__ldcg(&cb[i].cell) != cell || cb[i].prio <= last) continue;
                            const uint32_t tg = __ldcg(&cb[i].target), hc = __ldcg(&cb[i].h2);
                            bool dup = false;
                            for (uint32_t e2 = tg & 0xFFu; e2 < ne; ++e2) dup |= __ldcg(&cw[e2]) == hc;
                            if (dup) n_dup += 1u + (tg >> 16);
                            else n_full += 1u + (tg >> 16);
                        }
                        __syncthreads();
                        break;
                    }
                    __syncthreads();
                }
            }
            s = e;
        }
    }
    warp_add_u64(&a.stats[ST_DUP], n_dup);
    warp_add_u64(&a.stats[ST_FULL], n_full);
    warp_add_u64(&a.stats[ST_INSERTED], n_ins);
    warp_add_u64(&a.stats[ST_REPLACED], n_rep);
}

// ---- insert through per-cell lists (keep-first, N_e <= 8): two launches and no staging.
// k_chain_link chains each candidate to the one that reached its cell before it
// (chain_head[cell] = the last arrival; candidate i's cell field becomes the one before i,
// CHAIN_END after the first, so that a step of a walk reads one 32-byte sector) and lists
// each cell once, when its first candidate arrives; k_chain_resolve then resolves each
// listed cell with one thread.
//
// The chain's order is arbitrary, but sequential resolution in ascending priority depends
// only on the set of the cell's candidates:
//   * they all saw the same snapshot of the cell, whose slots from the first empty one on
//     were empty, so only keys inserted by this resolution can make a duplicate;
//   * with F empty slots, the keys inserted are the F distinct hash2 values whose smallest
//     priority is smallest, in that order, each with the value of that candidate;
//   * a candidate with an inserted hash2 that is not its smallest is a duplicate; the
//     candidates of every other hash2 find the cell full.
// A first walk keeps the best F distinct keys seen so far in a buffer, each with the smallest
// priority seen for it; a new key pushes out the entry of largest priority when the buffer
// is full and its own priority is smaller.  A key that belongs to the final F is never pushed
// out (F better keys would have to exist) and enters at its smallest priority at the latest,
// so the buffer ends as the inserted keys.  A second walk (lists of two or more) writes each
// inserted key's candidate of smallest priority into the slot of its rank and sums the
// weights (1 + shadows) of the inserted keys' candidates.  The rest are dropped full: the
// evaluation counted the batch's emitted weight, which the resolution starts from, so a
// cell without an empty slot is not walked at all.
constexpr uint32_t CHAIN_END = 0xFFFFFFFFu;

__global__ void __launch_bounds__(256) k_chain_link(BatchArgs a) {
    const uint32_t n_in = min(a.ctl->n_cand, a.probe_cap);
    const uint32_t* cc = a.lists[0];
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, n_warps = (gridDim.x * blockDim.x) >> 5;
    // a warp takes 128 consecutive candidates per step: four independent atomics per lane
    for (uint32_t b = warp * 128u; b < n_in; b += n_warps * 128u) {
        uint32_t c[4];
        bool first[4];
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t i = b + 32u * k + lane;
            c[k] = i < n_in ? __ldcg(&cc[i]) : 0u;
        }
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t i = b + 32u * k + lane;
            first[k] = false;
            if (i < n_in) {
                const uint32_t prev = atomicExch(&a.chain_head[c[k]], i);
                a.cands[i].cell = prev;   // the successor replaces the cell, known from the list
                first[k] = prev == CHAIN_END;
            }
        }
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t x = warp_append(&a.ctl->n_lists, first[k]);
            if (first[k]) a.lists[1][x] = c[k];
        }
    }
}

__global__ void __launch_bounds__(256, 4) k_chain_resolve(BatchArgs a) {
    const uint32_t n_in = min(a.ctl->n_cand, a.probe_cap);
    const uint32_t n_cells = min(a.ctl->n_lists, n_in);
    const uint32_t ne = a.n_entries;
    const uint4* cb = reinterpret_cast<const uint4*>(a.cands);   // two 16-byte halves per candidate
    // every candidate counts as dropped full until its cell's resolution says otherwise
    // (modular arithmetic: the sum of the counter's updates is the non-negative count)
    unsigned long long n_dup = 0, n_ins = 0;
    unsigned long long n_full = (blockIdx.x == 0 && threadIdx.x == 0) ? (unsigned long long)a.ctl->w_cand : 0ull;
    bool bad = false;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_cells && !bad; t += stride) {
        const uint32_t cell = __ldcg(&a.lists[1][t]);
        const uint32_t head = atomicExch(&a.chain_head[cell], CHAIN_END);   // takes the list, leaves it empty
        uint4 w0, w1;
        load_cell_words(a, cell, &w0, &w1);
        uint32_t used = ne;
        {
            const uint32_t h[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int e = 7; e >= 0; --e)
                if ((uint32_t)e < ne && h[e] == 0u) used = (uint32_t)e;   // the first empty slot
        }
        const uint32_t F = ne - used;
        if (F == 0) continue;   // a full cell: every candidate is dropped, as counted
        // walk 1: the buffer (hash2 and the smallest priority seen for it, unordered)
        uint32_t hb[8];
        unsigned long long pb[8];
#pragma unroll
        for (uint32_t e = 0; e < 8; ++e) {
            hb[e] = 0u;
            pb[e] = 0ull;
        }
        uint32_t nb = 0, steps = 0;
        uint4 v = make_uint4(0, 0, 0, 0);   // r, g, b, target of the last candidate walked
        for (uint32_t j = head; j != CHAIN_END;) {
            if (j >= n_in || ++steps > n_in) {   // not a list of this batch's candidates
                bad = true;
                break;
            }
            // prio, successor (in place of the cell), hash2; the candidates are read-only here,
            // so the loads go through L1, where the second walk finds them
            const uint4 q = __ldg(cb + 2 * (size_t)j);
            v = __ldg(cb + 2 * (size_t)j + 1);
            const uint32_t nj = q.z;
            const unsigned long long pr = ((unsigned long long)q.y << 32) | q.x;
            const uint32_t hc = q.w;
            bool found = false;
#pragma unroll
            for (uint32_t e = 0; e < 8; ++e)
                if (e < nb && hb[e] == hc) {
                    found = true;
                    if (pr < pb[e]) pb[e] = pr;
                }
            if (!found) {
                uint32_t at = nb;   // the buffer entry it takes (8: none)
                if (nb < F) {
                    nb++;
                } else {
                    // a new key with the buffer full: it pushes out the entry of largest
                    // priority if its own is smaller
                    unsigned long long mx = 0ull;
#pragma unroll
                    for (uint32_t e = 0; e < 8; ++e)
                        if (e < nb && pb[e] > mx) {
                            mx = pb[e];
                            at = e;
                        }
                    if (pr >= mx) at = 8;
                }
#pragma unroll
                for (uint32_t e = 0; e < 8; ++e)
                    if (e == at) {
                        hb[e] = hc;
                        pb[e] = pr;
                    }
            }
            j = nj;
        }
        if (bad) break;
        uint32_t* cw = cell_h2(a, cell);
        if (steps == 1) {
            // one candidate: it takes the first empty slot; its shadows find it
            const uint32_t w = 1u + (v.w >> 16);
            cw[used] = hb[0];
            float* val = cell_val(a, cell, used);
            val[0] = __uint_as_float(v.x);
            val[1] = __uint_as_float(v.y);
            val[2] = __uint_as_float(v.z);
            n_ins += 1;
            n_dup += w - 1u;
            n_full -= w;
            continue;
        }
        // walk 2: the weight of the inserted keys' candidates; each key's candidate of
        // smallest priority writes the key and its value into the slot of its rank
        unsigned long long WI = 0;
        for (uint32_t j = head, k = 0; j != CHAIN_END && k < steps; ++k) {   // the list checked above
            const uint4 q = __ldg(cb + 2 * (size_t)j);
            const uint4 x = __ldg(cb + 2 * (size_t)j + 1);
            const uint32_t nj = q.z;
            const unsigned long long pr = ((unsigned long long)q.y << 32) | q.x;
            const uint32_t hc = q.w;
            bool in = false;
            unsigned long long best = 0ull;
#pragma unroll
            for (uint32_t e = 0; e < 8; ++e)
                if (e < nb && hb[e] == hc) {
                    in = true;
                    best = pb[e];
                }
            if (in) {
                WI += 1u + (x.w >> 16);
                if (pr == best) {
                    uint32_t slot = used;
#pragma unroll
                    for (uint32_t f = 0; f < 8; ++f) slot += (f < nb && pb[f] < best) ? 1u : 0u;
                    cw[slot] = hc;
                    float* val = cell_val(a, cell, slot);
                    val[0] = __uint_as_float(x.x);
                    val[1] = __uint_as_float(x.y);
                    val[2] = __uint_as_float(x.z);
                }
            }
            j = nj;
        }
        n_ins += nb;
        n_dup += WI - nb;
        n_full -= WI;
    }
    if (bad) atomicOr(&a.ctl->err, ERR_INSERT);
    warp_add_u64(&a.stats[ST_DUP], n_dup);
    warp_add_u64(&a.stats[ST_FULL], n_full);
    warp_add_u64(&a.stats[ST_INSERTED], n_ins);
}

__global__ void k_finish(BatchArgs a) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (a.use_cache) a.ctl->epoch += a.n_entries + 1u;
        a.stats[ST_BATCHES] += 1ull;
    }
}

// =======================================================================================
// Stand-alone mip levels (parity checks of Eq. 1)
// =======================================================================================
__global__ void k_levels(const float* g1u, const float* g1v, const float* g2u, const float* g2v, uint64_t n,
                         int32_t offset, uint32_t* level) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        level[i] = d_level(g1u[i], g1v[i], g2u[i], g2v[i], offset);
}

cudaError_t launch_levels(const float* g1u, const float* g1v, const float* g2u, const float* g2v, uint64_t n,
                          int32_t offset, uint32_t* level, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_levels<<<(unsigned)blocks, 256, 0, s>>>(g1u, g1v, g2u, g2v, n, offset, level);
    return cudaGetLastError();
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

cudaError_t launch_reset(uint4* table, size_t units, unsigned long long* claims, uint32_t* chain_head, size_t cells,
                         Control* ctl, unsigned long long* stats, cudaStream_t s, bool claim_words) {
    cudaError_t e;
    if (units && (e = cudaMemsetAsync(table, 0, (units + 16) * sizeof(uint4), s)) != cudaSuccess) return e;
    // all-ones: the largest claim word of the atomicMin rounds, and an empty list per cell
    // for the per-cell-list insert (which leaves every list empty after a batch; this only
    // repairs lists left by a batch that failed)
    (void)claim_words;
    if (cells && (e = cudaMemsetAsync(claims, 0xFF, cells * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if (cells && chain_head && (e = cudaMemsetAsync(chain_head, 0xFF, cells * sizeof(uint32_t), s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(ctl, 0, sizeof(Control), s)) != cudaSuccess) return e;
    return cudaMemsetAsync(stats, 0, ST_COUNT * sizeof(unsigned long long), s);
}

int insert_grid(int num_sms) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_insert, 256, 0) != cudaSuccess || v <= 0) v = 1;
        per_sm = v;
    }
    return per_sm * num_sms;
}

// Insert phase: the candidates of the batch into the table (Alg. 1 semantics).
static cudaError_t launch_insert(const BatchArgs& a, cudaStream_t s, int num_sms, uint64_t* nl) {
    cudaError_t e = cudaSuccess;
    const int gs_blocks = num_sms * 4;
    if (a.n > 0 && a.use_cache && a.insert_rounds) {
        BatchArgs arg = a;
        void* params[] = {&arg};
        if ((e = cudaLaunchCooperativeKernel((const void*)k_insert, dim3(insert_grid(num_sms)), dim3(256), params, 0, s)) !=
            cudaSuccess)
            return e;
        *nl += 1;
    } else if (a.n > 0 && a.use_cache && a.insert_lists) {
        static int per_sm = 0;
        if (per_sm == 0) {
            int v = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_chain_resolve, 256, 0) != cudaSuccess || v <= 0) v = 1;
            per_sm = v;
        }
        k_chain_link<<<num_sms * 8, 256, 0, s>>>(a);
        k_chain_resolve<<<num_sms * per_sm, 256, 0, s>>>(a);
        *nl += 2;
    } else if (a.n > 0 && a.use_cache) {
        if ((e = cudaMemsetAsync(a.bin_cnt, 0, (size_t)a.n_bins * sizeof(uint32_t), s)) != cudaSuccess) return e;
        k_bin_count<<<gs_blocks, 256, 0, s>>>(a);
        k_bin_scan<<<1, 1024, 0, s>>>(a);
        k_bin_scatter<<<num_sms * 8, 256, 0, s>>>(a);
        // each bin is resolved by exactly one of the three kernels, chosen by its size
        k_bin_insert_warp<<<std::min<uint32_t>((a.n_bins + INS_WARPS - 1) / INS_WARPS, (uint32_t)num_sms * 8u),
                            INS_WARPS * 32, 0, s>>>(a);
        const size_t msm = insert_mid_smem_bytes();
        if ((e = cudaFuncSetAttribute(k_bin_insert_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msm)) !=
            cudaSuccess)
            return e;
        k_bin_insert_mid<<<std::min<uint32_t>(a.n_bins, (uint32_t)num_sms * 4u), INS_MID_T, msm, s>>>(a);
        const size_t ism = insert_smem_bytes();
        if ((e = cudaFuncSetAttribute(k_bin_insert, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism)) != cudaSuccess)
            return e;
        k_bin_insert<<<std::min<uint32_t>(a.n_bins, (uint32_t)num_sms * 6u), 256, ism, s>>>(a);
        *nl += 6;
    }
    return e;
}

// The lookup instantiation for N_e (hash2 words per cell) and the probes in flight.
template <bool POS>
void launch_lookup(const BatchArgs& a, uint32_t ne, uint32_t rb, unsigned lb, cudaStream_t s) {
    if (ne <= 4) {
        if (rb >= 4) k_lookup<1, 4, POS><<<lb, 256, 0, s>>>(a);
        else if (rb >= 2) k_lookup<1, 2, POS><<<lb, 256, 0, s>>>(a);
        else k_lookup<1, 1, POS><<<lb, 256, 0, s>>>(a);
    } else if (ne <= 8) {
        if (rb >= 4) k_lookup<2, 4, POS><<<lb, 256, 0, s>>>(a);
        else if (rb >= 2) k_lookup<2, 2, POS><<<lb, 256, 0, s>>>(a);
        else k_lookup<2, 1, POS><<<lb, 256, 0, s>>>(a);
    } else if (ne <= 16) {
        if (rb >= 2) k_lookup<4, 2, POS><<<lb, 256, 0, s>>>(a);
        else k_lookup<4, 1, POS><<<lb, 256, 0, s>>>(a);
    } else {
        k_lookup<8, 1, POS><<<lb, 256, 0, s>>>(a);
    }
}

cudaError_t launch_batch(const BatchArgs& a, cudaStream_t s, int num_sms, cudaEvent_t* ev,
                         uint64_t* launches) {
    cudaError_t e;
    uint64_t nl = 0;
    auto mark = [&](int k) { return ev ? cudaEventRecord(ev[k], s) : cudaSuccess; };
    if ((e = mark(0)) != cudaSuccess) return e;
    // per-batch counters (epoch, errors and the barrier persist)
    if ((e = cudaMemsetAsync(a.ctl, 0, offsetof(Control, epoch), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.ctl->mid_count, 0, 2 * (MAX_ENTRIES + 2) * sizeof(uint32_t), s)) != cudaSuccess) return e;
    // counts has n_mats + 1 entries; the last one is the evaluation's work-item counter
    if ((e = cudaMemsetAsync(a.counts, 0, (a.n_mats + 1) * sizeof(uint32_t), s)) != cudaSuccess) return e;
    if (a.split && (e = cudaMemsetAsync(a.miss_cnt, 0, (a.n_roots_total + MAX_LEVELS) * sizeof(uint32_t), s)) != cudaSuccess)
        return e;
    uint32_t* item_ctr = a.counts + a.n_mats;
    if (a.alg1 && a.use_cache) {
        // the paper's concurrent update: lookups and inserts inside the evaluator, no
        // lookup kernel, no insert phase; grouped by material unless unsorted
        if (!a.unsorted && a.n > 0) {
            k_hist<<<num_sms * GROUP_BLOCKS_PER_SM, 256, 0, s>>>(a);
            nl++;
        }
        if (!a.unsorted) {
            k_scan<<<1, 1024, 0, s>>>(a);
            nl++;
        }
        if (!a.unsorted && a.n > 0) {
            k_scatter<<<num_sms * GROUP_BLOCKS_PER_SM, 256, 0, s>>>(a);
            nl++;
        }
        if ((e = mark(1)) != cudaSuccess) return e;
        if (!a.unsorted && a.n > 0 && a.surr_slot) {
            if ((e = launch_surrogate(a, num_sms, s)) != cudaSuccess) return e;
            nl++;
        }
        if ((e = mark(2)) != cudaSuccess) return e;
        if ((e = mark(3)) != cudaSuccess) return e;
        if (a.n > 0) {
            const size_t smem = eval_smem_bytes(a.max_slots);
            if (a.unsorted) {
                if (smem > 48 * 1024 &&
                    (e = cudaFuncSetAttribute(k_eval_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem)) != cudaSuccess)
                    return e;
                k_eval_fused<false><<<num_sms * 16, EVAL_WARPS * 32, smem, s>>>(a, nullptr);
            } else {
                if (smem > 48 * 1024 &&
                    (e = cudaFuncSetAttribute(k_eval_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem)) != cudaSuccess)
                    return e;
                k_eval_fused<true><<<num_sms * 16, EVAL_WARPS * 32, smem, s>>>(a, item_ctr);
            }
            nl++;
        }
        if ((e = mark(4)) != cudaSuccess) return e;
        if ((e = mark(5)) != cudaSuccess) return e;
        k_finish<<<1, 32, 0, s>>>(a);
        nl++;
        if ((e = mark(6)) != cudaSuccess) return e;
        if (launches) *launches += nl;
        return cudaGetLastError();
    }
    if (a.unsorted) {
        // one fused launch: probes inline, no grouping and no probe records
        if ((e = mark(1)) != cudaSuccess) return e;
        if ((e = mark(2)) != cudaSuccess) return e;
        if ((e = mark(3)) != cudaSuccess) return e;
        if (a.n > 0) {
            const size_t smem = eval_smem_bytes(a.max_slots);
            if (smem > 48 * 1024 &&
                (e = cudaFuncSetAttribute(k_eval_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                    cudaSuccess)
                return e;
            k_eval_fused<false><<<num_sms * 16, EVAL_WARPS * 32, smem, s>>>(a, nullptr);
            nl++;
        }
        if ((e = mark(4)) != cudaSuccess) return e;
        if ((e = launch_insert(a, s, num_sms, &nl)) != cudaSuccess) return e;
        if ((e = mark(5)) != cudaSuccess) return e;
        k_finish<<<1, 32, 0, s>>>(a);
        nl++;
        if ((e = mark(6)) != cudaSuccess) return e;
        if (launches) *launches += nl;
        return cudaGetLastError();
    }
    if (a.n > 0) {
        k_hist<<<num_sms * GROUP_BLOCKS_PER_SM, 256, 0, s>>>(a);
        nl++;
    }
    k_scan<<<1, 1024, 0, s>>>(a);
    nl++;
    if (a.n > 0) {
        k_scatter<<<num_sms * GROUP_BLOCKS_PER_SM, 256, 0, s>>>(a);
        nl++;
    }
    if ((e = mark(1)) != cudaSuccess) return e;
    // grouped schedule with the probes in the evaluator: no lookup kernel, no records
    const bool fused = a.probe_inline && a.use_cache;
    if (a.n > 0 && a.use_cache && !a.keys_inline && !fused && !a.all_surr) {
        const uint32_t ne = a.n_entries, rb = a.lookup_rb;
        const unsigned lb = (unsigned)num_sms * 8u;
        if (a.pos_level >= 0)
            launch_lookup<true>(a, ne, rb, lb, s);
        else
            launch_lookup<false>(a, ne, rb, lb, s);
        nl++;
    }
    if (a.n > 0 && a.surr_slot) {
        if ((e = launch_surrogate(a, num_sms, s)) != cudaSuccess) return e;
        nl++;
    }
    if ((e = mark(2)) != cudaSuccess) return e;
    if (a.n > 0 && fused) {
        const size_t smem = eval_smem_bytes(a.max_slots);
        if (smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(k_eval_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                cudaSuccess)
            return e;
        if ((e = mark(3)) != cudaSuccess) return e;
        k_eval_fused<true><<<num_sms * 16, EVAL_WARPS * 32, smem, s>>>(a, item_ctr);
        nl++;
    } else if (a.n > 0) {
        const bool outer = a.use_cache && a.split && !a.keys_inline;
        const bool plain = !a.use_cache && !a.surr_ord;
        const size_t smem = eval_smem_bytes(outer ? a.max_slots_outer : a.max_slots),
                     smem_roots = eval_smem_bytes(a.max_slots_roots);
        // the first pass on an empty table without surrogates: every lane runs every node
        const bool fill = a.use_cache && a.keys_inline && !a.surr_ord;
        auto keval = outer ? k_eval<EVAL_OUTER> : plain ? k_eval<EVAL_PLAIN> : k_eval<EVAL_GENERIC>;
        // two points per lane where every lane runs every instruction and the doubled slot
        // file leaves room for several blocks per SM; the item counter then counts pairs
        const bool two = (outer || plain || fill) && !a.one_point && 2 * smem <= EVAL2_MAX_SMEM;
        if (two && a.block_items)
            keval = outer ? k_eval2<EVAL_OUTER, true> : plain ? k_eval2<EVAL_PLAIN, true> : k_eval2<EVAL_FILL, true>;
        else if (two)
            keval = outer ? k_eval2<EVAL_OUTER, false> : plain ? k_eval2<EVAL_PLAIN, false> : k_eval2<EVAL_FILL, false>;
        const size_t smem_eval = two ? 2 * smem : smem;
        if (smem_eval > 48 * 1024 &&
            (e = cudaFuncSetAttribute(keval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_eval)) !=
                cudaSuccess)
            return e;
        // the batched misses: two misses per lane under the same conditions as the per-point
        // evaluator (the item counter then counts pairs)
        const bool two_roots = !a.one_point && 2 * smem_roots <= EVAL2_MAX_SMEM;
        auto kroots = a.pos_level >= 0 ? (two_roots ? k_eval_roots2<true> : k_eval_roots<true>)
                                       : (two_roots ? k_eval_roots2<false> : k_eval_roots<false>);
        const size_t smem_kroots = two_roots ? 2 * smem_roots : smem_roots;
        if (smem_kroots > 48 * 1024 &&
            (e = cudaFuncSetAttribute(kroots, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_kroots)) !=
                cudaSuccess)
            return e;
        if (a.use_cache && a.split && !a.keys_inline && !a.all_surr) {
            k_scan_roots<<<1, 1024, 0, s>>>(a);
            nl++;
            // the level counters live after the per-root miss counters
            for (uint32_t lv = 0; lv <= a.max_level; ++lv) {
                kroots<<<num_sms * 16, EVAL_WARPS * 32, smem_kroots, s>>>(a, lv, a.miss_cnt + a.n_roots_total + lv);
                nl++;
            }
        }
        if ((e = mark(3)) != cudaSuccess) return e;
        keval<<<num_sms * 16, EVAL_WARPS * 32, smem_eval, s>>>(a, item_ctr);
        nl++;
    } else if ((e = mark(3)) != cudaSuccess) {
        return e;
    }
    if ((e = mark(4)) != cudaSuccess) return e;
    // with every cacheable node a surrogate's there is nothing to insert
    if (!a.all_surr && (e = launch_insert(a, s, num_sms, &nl)) != cudaSuccess) return e;
    if ((e = mark(5)) != cudaSuccess) return e;
    k_finish<<<1, 32, 0, s>>>(a);
    nl++;
    if ((e = mark(6)) != cudaSuccess) return e;
    if (launches) *launches += nl;
    return cudaGetLastError();
}

}  // namespace pmc
