/*
 * pmc.h -- C ABI of the GB300 (sm_103a) Progressive Material Caching library.
 *
 * The library evaluates node-based material networks for wavefronts of shading
 * points and caches the outputs of cacheable nodes in a fixed-size hash table
 * (Fujieda & Harada, "Progressive Material Caching", SIGGRAPH Asia 2022 Technical
 * Communications):
 *   - Sec. 2: a material network is serialised into a linear program that a GPU
 *     interpreter runs in storage order;
 *   - Sec. 3: cacheable nodes are the highest nodes whose sub-graph depends on no
 *     shading-point information other than UV; a hit skips the sub-graph, a miss
 *     evaluates it and stores the value;
 *   - Sec. 3.1, Eq. 1: descriptor = (material ID, node ID, mip level, texel indices);
 *   - Sec. 3.2, Fig. 3: N_c cells x N_e entries, cell = Hash(desc) mod N_c, entry
 *     checked by Hash2(desc), first inserted value kept;
 *   - Alg. 1: an entry is taken at the first slot whose stored hash is Hash2(desc)
 *     or 0.  This library resolves concurrent inserts deterministically: a batch
 *     looks up against the table as it was when the batch started, then inserts
 *     its misses in ascending (point index, node ID) order, which it realises by
 *     grouping the candidates by cell (default: a list per cell for N_e <= 8
 *     keep-first tables, else bins of cells) or with rounds of atomicMin on a
 *     per-cell claim word (PMC_INSERT_ROUNDS).
 *
 * Conventions for every entry point:
 *   - All pointers to shading points and outputs are DEVICE pointers owned by the
 *     caller unless the name ends in _host.  The library never frees them.
 *   - The library owns the table, the compiled programs and all scratch memory.
 *   - Work is enqueued on the caller's CUDA stream (a cudaStream_t passed as void*;
 *     NULL = legacy default stream).  Argument errors are returned synchronously
 *     and enqueue nothing.  A CUDA launch error is recorded in the cache object and
 *     returned by this and every later call (PMC_ERR_CUDA, sticky).
 *   - Errors found on the device (a material ID out of range) are folded into the
 *     next pmc_sync / pmc_stats call.
 *   - A cache object is not thread-safe; distinct cache objects are independent.
 *   - The first pmc_eval_batch with a given batch size allocates scratch; later
 *     calls of the same or smaller size allocate nothing.
 */
#ifndef PMC_H
#define PMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PMC_OK = 0,
    PMC_ERR_INVALID_ARG = 1, /* malformed argument, network or shading point     */
    PMC_ERR_OOM = 2,         /* device or host allocation failed                  */
    PMC_ERR_CUDA = 3,        /* a CUDA call failed (sticky in the cache object)   */
    PMC_ERR_TIMEOUT = 4,     /* a bounded device wait ran out                     */
    PMC_ERR_UNSUPPORTED = 5  /* feature or size outside what this build supports */
} pmc_status;

/* Opaque cache object: compiled networks, the table and scratch; library-owned. */
typedef struct pmc_cache pmc_cache;

/* ---- material networks (Sec. 2, Fig. 2) -------------------------------------
 * A material is an array of nodes in topological order: in[k] names an earlier
 * node (0 <= in[k] < own index) or is -1.  The last node is the material output.
 * The node ID used in descriptors is the node's index in this array, as given
 * (Sec. 3.1), independent of any optimisation the library applies.
 * Every node value is 3 floats; single-valued nodes repeat their value.  All
 * outputs except UV, POSITION, NORMAL, CONST and UV_AFFINE are clamped to [0,1].
 *
 *  op              inputs          parameters
 *  PMC_OP_UV        -              -                     (u, v, 0)
 *  PMC_OP_POSITION  -              -                     (px, py, pz)
 *  PMC_OP_NORMAL    -              -                     (nx, ny, nz)
 *  PMC_OP_CONST     -              fp[0..2]              (fp0, fp1, fp2)
 *  PMC_OP_UV_AFFINE in0            fp[0..5]              (fp0 x + fp1 y + fp4, fp2 x + fp3 y + fp5, 0)
 *  PMC_OP_FBM       in0 (x, y)     fp0 scale, fp1 lacunarity, fp2 gain, ip0 octaves (1..16), ip1 seed
 *                                  0.5 + sum_k gain^k noise(scale lac^k (x,y); seed+k) / sum_k gain^k
 *  PMC_OP_VORONOI   in0 (x, y)     fp0 scale, ip1 seed   Worley F1 at scale (x, y)
 *  PMC_OP_CHECKER   in0 (x, y)     fp0 scale, fp1..3 colour A, fp4..6 colour B
 *                                  A if floor(x s) + floor(y s) is even, else B.
 *                                  The only discontinuous primitive; so that FP32 and
 *                                  wider arithmetic agree on the side of every cell edge,
 *                                  x s must be exact in FP32: in0 is the UV or POSITION
 *                                  node, or a UV_AFFINE of one of them with fp1 = fp2 =
 *                                  fp4 = fp5 = 0 and fp0, fp3 powers of two, and s is a
 *                                  power of two, every power in [2^-20, 2^20].  A network
 *                                  breaking this is rejected (PMC_ERR_INVALID_ARG)
 *  PMC_OP_RAMP      in0 (x)        ip0 stops (2..4), fp0..3 positions (ascending, in [0,1]),
 *                                  fp4.. colours (3 per stop); piecewise linear, constant outside
 *  PMC_OP_MIX       in0 a, in1 b, in2 f (optional; fp0 if -1)   a + (b - a) clamp(f.x, 0, 1)
 *  PMC_OP_ADD       in0, in1       -                     a + b
 *  PMC_OP_MUL       in0, in1       -                     a * b
 *  PMC_OP_POW       in0            fp0 exponent (> 0)    max(a, 0)^fp0
 *  PMC_OP_FACING    in0            fp0..2 direction      |dot(a, d)|
 */
enum {
    PMC_OP_UV = 0,
    PMC_OP_POSITION = 1,
    PMC_OP_NORMAL = 2,
    PMC_OP_CONST = 3,
    PMC_OP_UV_AFFINE = 4,
    PMC_OP_FBM = 5,
    PMC_OP_VORONOI = 6,
    PMC_OP_CHECKER = 7,
    PMC_OP_RAMP = 8,
    PMC_OP_MIX = 9,
    PMC_OP_ADD = 10,
    PMC_OP_MUL = 11,
    PMC_OP_POW = 12,
    PMC_OP_FACING = 13,
    PMC_NUM_OPS = 14
};

typedef struct {
    uint32_t op;
    int32_t in[4];
    int32_t ip[4];
    float fp[16];
} pmc_node; /* 100 bytes, host memory */

typedef struct {
    uint32_t n_nodes;      /* 1 .. 65535 */
    const pmc_node* nodes; /* host memory, copied by pmc_create_cache */
} pmc_material;

/* ---- cache description (Sec. 3.2, Fig. 3, Alg. 1 inputs N_c and N_e) --------- */
#define PMC_CACHE_OFF 0x1u        /* evaluate every node, no lookups, no inserts   */
#define PMC_SORT_BY_MATERIAL 0x2u /* accepted; grouping shading points by material
                                     is the default (see PMC_UNSORTED)             */
#define PMC_DEBUG_CHECKS 0x4u     /* extra device-side bounds checks               */
#define PMC_EVAL_INLINE 0x8u      /* evaluate missed cacheable nodes inside the
                                     per-point program (lanes that hit wait) instead of
                                     in batches of 32 misses of the same node          */
#define PMC_INSERT_ROUNDS 0x10u   /* resolve inserts by rounds of atomicMin on a claim
                                     word per cell instead of grouping the candidates
                                     by cell (same table either way)                   */
#define PMC_UNSORTED 0x20u        /* no grouping by material: a warp evaluates 32
                                     consecutive points, one material at a time, and
                                     probes the table inline (same results; not
                                     combinable with learned surrogates)               */
#define PMC_PROBE_INLINE 0x40u    /* grouped by material, the evaluator probes the
                                     table itself when it reaches a cacheable node: no
                                     lookup kernel and no probe records (same results) */
#define PMC_ALG1 0x80u            /* the paper's concurrent update (Sec. 3.3, Alg. 1)
                                     instead of the deterministic two-phase one: 8-byte
                                     slots {hash2, value encoded in 32 bits (shared-
                                     exponent RGB9E5)}; the evaluator looks a cacheable
                                     node up when it reaches it and, on a miss, inserts
                                     the value it evaluated at once with one 64-bit
                                     compare-and-swap into the first slot holding its
                                     hash2 or 0 (a lost race drops the value).  Entries
                                     inserted earlier in the same pass are visible, so
                                     hits, outputs and the table depend on thread timing;
                                     a hit returns the decoded value.  Only the grouped and
                                     unsorted schedules apply; pmc_last_hit_masks is not
                                     available */
#define PMC_REPLACE_VISIBILITY 0x100u /* replacement by visibility class instead of
                                     keep-first, the prioritisation of directly visible
                                     shading points that Sec. 5 proposes.  Each point may
                                     carry a class (pmc_points.vis: 0 = seen directly from
                                     the camera, k = reached after k bounces; NULL = all
                                     0) and each entry keeps its inserter's class.  Inserts
                                     are still resolved per cell in ascending (point
                                     index, node ID) order: a key already in the cell is
                                     a duplicate; else the first empty slot takes it;
                                     else the entry of the largest class is overwritten
                                     if that class is larger than the newcomer's (the
                                     first such entry on ties; counted in `replaced`);
                                     else the value is dropped.  Lookups do not change
                                     classes.  With every class 0 the table evolves as
                                     with keep-first.  The table is still deterministic.
                                     Not combinable with PMC_ALG1 or PMC_INSERT_ROUNDS
                                     (PMC_ERR_INVALID_ARG); one byte per slot more */
#define PMC_POSITION_DESCRIPTOR 0x200u /* world-position descriptor (Sec. 3.1 names a
                                     world-space position as a further descriptor; Sec. 5
                                     lists other shading-point information than UV as
                                     future work).  The position becomes a dependence
                                     class of its own: a node whose sub-graph depends on
                                     the position and on nothing else of the shading point
                                     (no UV, no normal) is cacheable by the same rule as a
                                     UV-only node, and is looked up under the descriptor
                                     (material, node, voxel of the position at pos_level):
                                     per axis floor(p 2^pos_level) clamped to [-512, 511]
                                     and offset by 512 (NaN -> 0), key = mat<<48 |
                                     node<<32 | 1<<31 | ix<<20 | iy<<10 | iz.  A node that
                                     joins UV and position is not cacheable.  Learned
                                     surrogates stay on UV-only nodes */
#define PMC_BLOCK_ITEMS 0x400u  /* schedule only (pmc_set_schedule): the per-point evaluator
                                     takes block-wide tiles of one material (the four warps of a
                                     block, 256 grouped points) per claim instead of one warp's
                                     64 points, so the warps of a block share the material's
                                     instruction and parameter lines (same results)          */
#define PMC_ONE_POINT 0x800u    /* schedule only: one point per lane in the per-point and
                                     batched-miss evaluators instead of two (same results)   */
#define PMC_INSERT_BINNED 0x1000u /* schedule only: group the candidates by bins of 256 cells
                                     (count, scan, scatter, then a warp or a block per bin)
                                     where the default would chain each cell's candidates in
                                     a list resolved by its first arrival (keep-first tables
                                     of N_e <= 8 without PMC_INSERT_ROUNDS); same table and
                                     counters either way                                     */
#define PMC_MAX_POS_LEVEL 20u

typedef struct {
    uint64_t n_cells;        /* N_c >= 1, < 2^32                                  */
    uint32_t n_entries;      /* N_e, 1 .. 32; a slot is 16 bytes {hash2, r, g, b} */
    uint32_t uv_level;       /* lambda of Eq. 1: 2^lambda texels per axis, 0 .. 13 */
    uint32_t flags;          /* PMC_* flags above                                  */
    uint32_t min_root_nodes; /* a cacheable node's sub-graph must hold at least this
                                many non-input nodes (0 is read as 2)              */
    int device;              /* CUDA device ordinal                                */
    uint64_t probe_capacity; /* (point, cacheable node) probes per batch that the
                                scratch is sized for; 0 = n times the largest number
                                of cacheable nodes of any material.  A batch that
                                needs more does no work and the next pmc_sync /
                                pmc_stats returns PMC_ERR_UNSUPPORTED            */
    int32_t level_offset;    /* -13 .. 13, added to the level of every point that
                                carries ray-cone gradients (pmc_points g1u ..);
                                positive values give finer texels (Sec. 4)      */
    uint32_t pos_level;      /* PMC_POSITION_DESCRIPTOR: voxels of 2^-pos_level world
                                units, 0 .. PMC_MAX_POS_LEVEL (else ignored)       */
    uint32_t min_root_cost;  /* a cacheable node's sub-graph (the node and every node it
                                reads, each once, in the network as given) must cost at
                                least this many FP32 operations of the node cost model
                                (pmc_node_cost); 0 = no threshold.  A lookup and an insert
                                cost the same whatever the sub-graph, so caching a cheap
                                one can cost more than evaluating it (Sec. 3 caches to save
                                evaluation).  Nodes below the threshold are evaluated
                                like any other node and never looked up            */
} pmc_cache_desc;

/* ---- shading points: structure of arrays, n entries each, DEVICE memory ----- *
 * g1u, g1v, g2u, g2v (optional): the texture-coordinate gradients along the two axes of
 * the point's ray-cone footprint (Sec. 3.1).  With them every point takes its own mip
 * level of the virtual texture (Eq. 1):
 *   level = clamp(floor(-log2(min(|g1|, |g2|))) + level_offset, 0, 13),
 * the squared norms formed in FP32 (each product and the sum rounded to nearest); a
 * zero footprint gives 13, an infinite or NaN one 0.  All four NULL: every point uses
 * the cache's uv_level.  Either all four or none must be given.
 * vis (optional): one byte per point, its visibility class for PMC_REPLACE_VISIBILITY
 * (0 = directly visible, k = after k bounces); NULL = class 0 for every point.  Read only
 * by caches created with that flag. */
typedef struct {
    const float* u;
    const float* v;
    const uint32_t* mat; /* material index < n_mats */
    const float* px;
    const float* py;
    const float* pz;
    const float* nx;
    const float* ny;
    const float* nz;
    uint64_t n; /* 0 .. 2^28 */
    const float* g1u;
    const float* g1v;
    const float* g2u;
    const float* g2v;
    const uint8_t* vis;
} pmc_points;

/* Cumulative counters since creation or pmc_reset. */
typedef struct {
    uint64_t lookups;         /* (point, cacheable node) probes                     */
    uint64_t hits;
    uint64_t misses;
    uint64_t candidates;      /* evaluated cacheable nodes offered for insertion     */
    uint64_t inserted;        /* = occupied slots (an entry is never removed; only
                                 PMC_REPLACE_VISIBILITY overwrites one)                */
    uint64_t dropped_dup;     /* an entry with the same (cell, hash2) was present    */
    uint64_t dropped_full;    /* the cell had no empty entry                         */
    uint64_t nodes_evaluated; /* node instructions executed, summed over points      */
    uint64_t batches;
    uint64_t flops;           /* FP32 operations of the executed nodes (FMA = 2)     */
    uint64_t slots_probed;    /* table slots examined by lookups                     */
    uint64_t points;
    uint64_t bad_points;      /* points whose material index was out of range        */
    uint64_t surrogate_evals; /* cacheable-node values produced by learned surrogates    */
    uint64_t flops_missed;    /* part of flops spent on missed cacheable nodes evaluated
                                 in batches (the batched-miss kernel)                  */
    uint64_t dropped_race;    /* PMC_ALG1: the compare-and-swap found its slot taken by
                                 another key (always 0 otherwise)                      */
    uint64_t replaced;        /* PMC_REPLACE_VISIBILITY: entries overwritten by a value of
                                 a smaller class (inserted counts only empty slots taken,
                                 so it still equals the occupied slots)                */
} pmc_stats_t;

/* Compiles the networks (cacheable-node analysis, constant folding, serialisation;
 * Sec. 2 and 3), uploads them to `desc->device` and allocates a zeroed table of
 * n_cells * n_entries 16-byte slots (8-byte slots with PMC_ALG1).  Returns PMC_ERR_INVALID_ARG for a malformed
 * network or description, PMC_ERR_OOM if the table does not fit. */
pmc_status pmc_create_cache(const pmc_cache_desc* desc, const pmc_material* mats,
                            uint32_t n_mats, pmc_cache** out);

/* One progressive pass (Sec. 3; Alg. 1 for the inserts) over `pts->n` shading points:
 * lookup of every cacheable node of every point against the table as it was when
 * the call was made, evaluation of the nodes still needed, deterministic insert of
 * the evaluated cacheable nodes.  out_rgb: DEVICE, 3*n floats, planar (r[0..n),
 * g[0..n), b[0..n)).  out_hits: DEVICE, n uint16 (cacheable nodes found in the
 * table per point, the Fig. 1d quantity) or NULL.  Asynchronous on `stream`. */
pmc_status pmc_eval_batch(pmc_cache* cache, const pmc_points* pts, float* out_rgb,
                          uint16_t* out_hits, void* stream);

/* Same pass with HOST buffers (the gradients too, if given): copies the points in, runs
 * pmc_eval_batch, copies rgb (and hits if non-NULL) out and waits for `stream`.  Pinned
 * host memory gives the fastest copies; pageable memory works. */
pmc_status pmc_eval_batch_host(pmc_cache* cache, const pmc_points* host_pts,
                               float* host_rgb, uint16_t* host_hits, void* stream);

/* n_passes consecutive passes from HOST buffers (host_passes[k] -> host_rgb[k], 3 * n
 * floats planar, and host_hits[k], n uint16, if host_hits and that entry are non-NULL), each
 * the same pass as pmc_eval_batch on `stream`.  The copies of a pass overlap the evaluation
 * of its neighbours: inputs go in on one library-owned stream and outputs come out on
 * another, through two device staging sets that the cache owns (grown, with a device
 * synchronisation, when a larger pass comes).  Returns when every output is in host memory.
 * Page-locked host buffers let the copies overlap; pageable ones work but copy
 * synchronously. */
pmc_status pmc_eval_passes_host(pmc_cache* cache, const pmc_points* host_passes, uint32_t n_passes,
                                float* const* host_rgb, uint16_t* const* host_hits, void* stream);

/* Waits for the last stream used with this cache and reports device-side errors
 * (PMC_ERR_INVALID_ARG for out-of-range material indices). */
pmc_status pmc_sync(pmc_cache* cache);

/* Synchronises (as pmc_sync) and copies the counters to `out` (host). */
pmc_status pmc_stats(pmc_cache* cache, pmc_stats_t* out);

/* Synchronises and copies the table to `host_dst`: n_cells * n_entries slots of
 * 16 bytes {uint32 hash2 (0 = empty); float r, g, b} (with PMC_ALG1 the values are the
 * decoded RGB9E5 codes).  `bytes` must be at least that size. */
pmc_status pmc_table_dump(pmc_cache* cache, void* host_dst, size_t bytes);

/* PMC_REPLACE_VISIBILITY only (else PMC_ERR_UNSUPPORTED): synchronises and copies the
 * visibility class of every slot's entry to `host_dst` (n_cells * n_entries bytes, slot
 * order as pmc_table_dump; 0 for an empty slot).  `bytes` must be at least that size. */
pmc_status pmc_slot_classes(pmc_cache* cache, uint8_t* host_dst, size_t bytes);

/* Synchronises and copies, for the last batch, one 64-bit mask per point (host
 * memory, n entries, original point order): bit r set when the point's r-th
 * cacheable node (ascending node ID, r < 64) was found in the table.  Returns
 * PMC_ERR_UNSUPPORTED after a batch that kept no probe records (PMC_UNSORTED or
 * PMC_PROBE_INLINE schedules) or a pmc_eval_batch_noalloc pass. */
pmc_status pmc_last_hit_masks(pmc_cache* cache, uint64_t* host_dst, uint64_t n);

/* Empties the table and clears the counters (enqueued on `stream`). */
pmc_status pmc_reset(pmc_cache* cache, void* stream);

/* Frees everything the cache owns (synchronises first).  NULL is ignored. */
void pmc_destroy_cache(pmc_cache* cache);

/* Cacheable nodes of a material (ascending node IDs, up to `cap` written) and the
 * size of its compiled program.  Any output pointer may be NULL. */
pmc_status pmc_material_info(const pmc_cache* cache, uint32_t mat, uint32_t* n_roots,
                             uint32_t* roots, uint32_t cap, uint32_t* n_instr,
                             uint32_t* n_slots);

/* Host-only: compiles one network as pmc_create_cache would (Sec. 2, Sec. 3) and
 * reports its cacheable nodes (ascending node IDs, up to `cap`), program length
 * and live-value slots.  Needs no GPU.  Any output pointer may be NULL. */
pmc_status pmc_analyze_material(const pmc_material* mat, uint32_t min_root_nodes,
                                uint32_t* n_roots, uint32_t* roots, uint32_t cap,
                                uint32_t* n_instr, uint32_t* n_slots);

/* The same with the cost threshold and creation flags of pmc_cache_desc: min_root_cost as
 * pmc_cache_desc.min_root_cost; PMC_POSITION_DESCRIPTOR adds the cacheable nodes of position
 * class.  kinds (may be NULL): per cacheable node 1 = UV descriptor, 2 = world-position
 * descriptor.  Needs no GPU. */
pmc_status pmc_analyze_material_ext(const pmc_material* mat, uint32_t min_root_nodes, uint32_t min_root_cost,
                                    uint32_t flags, uint32_t* n_roots, uint32_t* roots, uint8_t* kinds,
                                    uint32_t cap, uint32_t* n_instr, uint32_t* n_slots);

/* Node cost model: the FP32 operations of one evaluation of `node` (a fused multiply-add
 * counts 2), counted from the library's formulas: UV, POSITION, NORMAL, CONST 0; UV_AFFINE
 * 8; FBM 4 + 47 x octaves; VORONOI 99; CHECKER 4; RAMP 23; MIX 17; ADD, MUL 9; POW 18;
 * FACING 8.  It sets the cost threshold of pmc_cache_desc.min_root_cost and the FP32 work
 * counted in pmc_stats_t.flops.  Needs no GPU. */
uint32_t pmc_node_cost(const pmc_node* node);

/* Descriptor and table addressing for n (material, node, u, v) tuples, all DEVICE
 * arrays: key = mat<<48 | node<<32 | level<<26 | iu<<13 | iv with
 * iu = min(floor(clamp(u,0,1) 2^level), 2^level - 1) (Sec. 3.1, Eq. 1);
 * cell = Hash(key) mod n_cells, h2 = Hash2(key) (0 remapped to 1) (Alg. 1).
 * Hash is the SplitMix64 output function, Hash2 the upper half of MurmurHash3's
 * fmix64 of key xor 0x9E3779B97F4A7C15.  Asynchronous on `stream`. */
pmc_status pmc_compute_keys(const uint32_t* mat, const uint32_t* node, const float* u,
                            const float* v, uint64_t n, uint32_t level, uint64_t n_cells,
                            uint64_t* key, uint64_t* cell, uint32_t* h2, void* stream);

/* The per-point mip level of Eq. 1 (Sec. 3.1) for n gradient pairs, DEVICE arrays:
 * level[i] = clamp(floor(-log2(min(|g1_i|, |g2_i|))) + offset, 0, 13) as a pass computes
 * it (see pmc_points).  offset: -13 .. 13.  Asynchronous on `stream`. */
pmc_status pmc_compute_levels(const float* g1u, const float* g1v, const float* g2u, const float* g2v,
                              uint64_t n, int32_t offset, uint32_t* level, void* stream);

/* Per-phase device timing of later batches, measured with CUDA events recorded on
 * each batch's stream: 0 = grouping by material (histogram, scan, scatter),
 * 1 = lookup (and learned surrogates), 2 = batched evaluation of missed cacheable
 * nodes, 3 = evaluation of the per-point programs, 4 = insert, 5 = bookkeeping.
 * Timing adds one event record per phase boundary and is off by default; graph
 * replays are not timed. */
pmc_status pmc_set_timing(pmc_cache* cache, int enable);

/* Synchronises, then returns the milliseconds per phase summed over the batches
 * enqueued since the last read (ms[6], host), the number of kernels the library
 * launched in that time and the number of batches; clears the accumulators. */
pmc_status pmc_read_timing(pmc_cache* cache, double* ms, uint64_t* kernel_launches,
                           uint64_t* batches);

/* ---- learned surrogates --------------------------------------------------------------
 * A cacheable node's UV-only sub-graph (Sec. 3) can be replaced by a small network of
 * (u, v), trained on values of the exact evaluator:
 *   features = [sin pi k u, cos pi k u, sin pi k v, cos pi k v], k = 1..16 (64;
 *              half-range frequencies, so a network need not repeat from u = 0 to 1)
 *   h1 = relu(f W1 + b1) (64), h2 = relu(h1 W2 + b2) (64), y = h2 W3 + b3 (3),
 *   value = clamp(y, 0, 1).
 * Parameters: PMC_MLP_PARAMS floats, W1 [64][64], b1 [64], W2 [64][64], b2 [64],
 * W3 [64][3], b3 [3].  Products take BF16 operands and accumulate in FP32 on the
 * tcgen05 tensor cores (tensor-memory accumulators), in inference and in training (forward,
 * backward and the weight gradients); FP32 master weights take Adam steps.  Per material the candidate node is its
 * most expensive cacheable node with no cacheable node below it.  A node with an enabled
 * surrogate is not probed: every pass evaluates the network for it.  When every cacheable
 * node of every material has an enabled surrogate, a pass launches no lookup, no batched
 * evaluation of misses and no insert (nothing is probed, so nothing is missed or inserted). */
#define PMC_MLP_PARAMS 8515u

typedef struct {
    uint32_t n_train;   /* training pairs per material, a power of two >= 128          */
    uint32_t n_valid;   /* held-out pairs per material for the validation RMSE, >= 1   */
    uint32_t epochs;    /* passes over the training pairs, >= 1                        */
    float lr;           /* initial Adam step size (cosine decay to 5 %); 0 = 1e-2        */
    float rmse_max;     /* enable a network only if its validation RMSE <= this; 0 = 1.6e-3,
                           a margin under the accuracy bar of 2e-3 (RMSE against exact
                           values) so that points the validation did not see stay within it */
    uint64_t seed;      /* training and validation (u, v) come from SplitMix64(seed, ...) */
    const uint32_t* mats; /* host: materials to train; NULL = every material with a candidate */
    uint32_t n_mats;
} pmc_train_desc;

/* Generates pairs with the exact evaluator, trains one network per listed material on
 * the GPU, measures each one's RMSE on held-out pairs against the exact values and
 * enables those within rmse_max (others keep exact evaluation).  rmse: host, one per
 * listed material (NULL allowed; -1 for a material without a candidate node).
 * Synchronous; allocates its own temporary buffers. */
pmc_status pmc_train_surrogates(pmc_cache* cache, const pmc_train_desc* desc, float* rmse,
                                void* stream);

/* Installs (theta != NULL, host, PMC_MLP_PARAMS floats) and enables, or removes
 * (theta == NULL), the surrogate of a material's candidate node. */
pmc_status pmc_set_surrogate(pmc_cache* cache, uint32_t mat, const float* theta);

/* Copies a material's surrogate parameters (host, may be NULL), its candidate node ID
 * (UINT32_MAX if none) and whether it is enabled. */
pmc_status pmc_get_surrogate(pmc_cache* cache, uint32_t mat, float* theta, uint32_t* node,
                             int* enabled);

/* Whether later passes use the enabled surrogates (default on). */
pmc_status pmc_use_surrogates(pmc_cache* cache, int enable);

/* Stand-alone network, DEVICE arrays: values of n points (planar 3 x n), clamped to
 * [0, 1] if clamp != 0.  Evaluated like the in-pass inference on the tcgen05 tensor
 * cores (BF16 operands, FP32 accumulators in tensor memory).  Asynchronous on `stream`;
 * if a bounded wait for the tensor cores runs out, the affected outputs are NaN. */
pmc_status pmc_mlp_forward(const float* theta, const float* u, const float* v, uint64_t n,
                           float* out, int clamp, void* stream);

/* Gradient of the mean squared error over n rows (a multiple of 128) of `data` (DEVICE,
 * n x 5 floats: u, v, r, g, b) with respect to theta (DEVICE): grad (DEVICE,
 * PMC_MLP_PARAMS) is overwritten, *loss (DEVICE, 1 float) receives the sum of squared
 * errors over the 3n outputs.  The same kernel as training, without the Adam step.
 * Asynchronous on `stream`. */
pmc_status pmc_mlp_gradient(const float* theta, const float* data, uint64_t n, float* grad,
                            float* loss, void* stream);

/* Stand-alone training of one network on caller data (DEVICE): n rows (a power of two
 * >= 128) of `data` (u, v, r, g, b); theta (FP32, updated in place), adam_m and adam_v
 * (PMC_MLP_PARAMS each, zero before the first step) persist between calls; `steps`
 * minibatches of 128 rows, Adam steps numbered from step0 + 1, learning rate
 * lr * (0.05 + 0.95 * (1 + cos(pi * step / total_steps)) / 2).  *loss (DEVICE) receives
 * the sum of squared errors of the minibatches.  Asynchronous on `stream`. */
pmc_status pmc_mlp_train(float* theta, float* adam_m, float* adam_v, const float* data,
                         uint64_t n, uint32_t steps, uint32_t step0, uint32_t total_steps,
                         float lr, float* loss, void* stream);

/* ---- pass without device allocation ---------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that must not
 * allocate device memory while they run.  Examples: an application that hands all of
 * a GPU's memory to its own pool at start-up and forbids driver allocations after
 * that; code on a latency-critical thread, where cudaMalloc/cudaFree can synchronise
 * the device and stall it; a plug-in whose host process owns the device memory.
 *
 * pmc_eval_batch_noalloc runs the same pass as pmc_eval_batch (same arguments, same
 * results) but takes its per-batch scratch from one fixed array compiled into the
 * library's device image (PMC_NOALLOC_SCRATCH_BYTES, about 3.4 MiB), not from
 * cudaMalloc; it calls no cudaMalloc, cudaFree or other allocating routine.  Every
 * GPU that loads the library holds that array until the process exits.  The cache
 * object (table, programs, counters) must already exist (pmc_create_cache).
 *
 * Limits: n <= PMC_NOALLOC_MAX_POINTS; n times the largest number of cacheable nodes
 * of any material <= PMC_NOALLOC_MAX_PROBES; at most PMC_NOALLOC_MAX_MATERIALS
 * materials.  A larger request returns PMC_ERR_UNSUPPORTED (with a message on stderr)
 * and enqueues nothing.
 *
 * The first call on a device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream capture begins.
 * All calls, from every cache object, share the one array, which keeps the last
 * call's contents; each call clears what must start at zero.  Calls whose work can
 * overlap on the GPU (unordered streams, concurrent host threads) race on the array
 * and corrupt each other's results: order them on one stream.  pmc_set_timing does
 * not time these calls; pmc_last_hit_masks after one returns PMC_ERR_UNSUPPORTED.
 * pmc_cache_desc.probe_capacity binds as in pmc_eval_batch (a batch needing more probe
 * records than it does no work; the next pmc_sync reports PMC_ERR_UNSUPPORTED). */
#define PMC_NOALLOC_MAX_POINTS 8192u
#define PMC_NOALLOC_MAX_PROBES 32768u
#define PMC_NOALLOC_MAX_MATERIALS 4096u
#define PMC_NOALLOC_SCRATCH_BYTES 3555584u
pmc_status pmc_eval_batch_noalloc(pmc_cache* cache, const pmc_points* pts, float* out_rgb,
                                  uint16_t* out_hits, void* stream);

/* ---- schedule, graphs of passes, autotuning -------------------------------------
 * None of these change results: every schedule produces the same outputs, hit counts,
 * counters and table, bit for bit. */
typedef struct {
    uint32_t flags;     /* subset of PMC_EVAL_INLINE | PMC_INSERT_ROUNDS | PMC_UNSORTED |
                           PMC_PROBE_INLINE | PMC_BLOCK_ITEMS | PMC_ONE_POINT |
                           PMC_INSERT_BINNED                                          */
    uint32_t lookup_rb; /* probes in flight per lane in the lookup kernel: 1, 2 or 4    */
} pmc_schedule;

/* Reads / replaces the schedule of later passes.  pmc_set_schedule returns
 * PMC_ERR_UNSUPPORTED for PMC_UNSORTED while learned surrogates are in use and for a
 * batched evaluation of misses (no PMC_EVAL_INLINE) of networks whose cacheable nodes
 * nest deeper than this build handles (it then keeps PMC_EVAL_INLINE). */
pmc_status pmc_get_schedule(const pmc_cache* cache, pmc_schedule* out);
pmc_status pmc_set_schedule(pmc_cache* cache, const pmc_schedule* sched);

/* A CUDA graph of whole passes: the launches of n_passes consecutive pmc_eval_batch
 * calls (passes[k] -> out_rgb[k], out_hits[k]; out_hits may be NULL, or any entry of
 * it), preceded by pmc_reset if flags has PMC_GRAPH_RESET, recorded once by stream
 * capture and replayed by pmc_graph_launch with one launch call.  Nothing runs at
 * creation.  The points and outputs are bound by address: a replay reads whatever
 * the caller's buffers hold then.  A replay is the same work as the calls it
 * recorded: without PMC_GRAPH_RESET every pass looks up the table as it stands.
 * A graph holds the cache's scratch addresses: scratch growth (a larger batch), a
 * schedule change, or a change to learned surrogates makes it stale, and
 * pmc_graph_launch then returns PMC_ERR_INVALID_ARG without launching.  Graphs must
 * be destroyed before their cache. */
typedef struct pmc_graph pmc_graph;
#define PMC_GRAPH_RESET 0x1u
pmc_status pmc_graph_create(pmc_cache* cache, const pmc_points* passes, uint32_t n_passes,
                            float* const* out_rgb, uint16_t* const* out_hits, uint32_t flags,
                            pmc_graph** out);
/* Enqueues one replay on `stream` (asynchronous). */
pmc_status pmc_graph_launch(pmc_graph* graph, void* stream);
void pmc_graph_destroy(pmc_graph* graph);

/* Times the candidate schedules on one batch (DEVICE points, as pmc_eval_batch) and
 * keeps the fastest.  Each candidate runs `reps` times (1 .. 16) from the same table
 * state; the table, counters and hit history are restored afterwards, so the call
 * leaves the cache as it found it except for the schedule.  Tune on a table that has
 * seen a few passes: on an empty table every schedule takes the empty-table path.
 * Synchronous.  Allocates temporary device memory (a copy of the table and outputs).
 * out (host, may be NULL): per candidate its schedule and best time. */
#define PMC_TUNE_MAX 16
typedef struct {
    uint32_t n_tried;
    uint32_t best;                        /* index into tried[] of the kept schedule */
    pmc_schedule tried[PMC_TUNE_MAX];
    float ms[PMC_TUNE_MAX];
} pmc_tune_result;
pmc_status pmc_autotune(pmc_cache* cache, const pmc_points* sample, uint32_t reps,
                        pmc_tune_result* out);

/* ---- shading points from a ray caster ----------------------------------------------
 * The stage that feeds the material system in the paper's renderer: Sec. 3.1 takes each
 * shading point's UV, material and ray-cone texture-coordinate gradients from it.  A small
 * analytic scene (planes and spheres) and a pinhole camera; one primary ray per pixel per
 * pass, written as the planes of a pass's shading points (pmc_points with the gradients).
 *
 * Object (host memory, copied at each call): kind PMC_OBJ_PLANE: p = {n (unit), d}, the
 * points x with n.x = d, the scene on the side n.x >= d; kind PMC_OBJ_SPHERE: p = {centre,
 * radius > 0}.  mat: the material index written for its hits.  Texture coordinates are a
 * planar projection: u = frac(uv_scale x[a0]), v = frac(uv_scale x[a1]) with a0 = axes &
 * 0xFF, a1 = axes >> 8 (0 = x, 1 = y, 2 = z).
 * Camera: the ray of pixel (x, y) with sample offsets (jx, jy) in [0, 1) leaves eye along
 * normalize(fwd + sx right + sy up), sx = (2 (x + jx) / width - 1) tan_half_y width / height,
 * sy = (1 - 2 (y + jy) / height) tan_half_y.  The offsets come from the k-th output of
 * SplitMix64 seeded with `seed`, k = pass * 2^32 + y * width + x + 1 (the output function of
 * seed + k * 0x9E3779B97F4A7C15): jx = (r >> 40) 2^-24, jy = ((r >> 16) & 0xFFFFFF) 2^-24.
 * Hit: the closest object with distance t > 1e-4 (the first one on ties); a sphere's
 * discriminant is formed as r^2 - |oc - (d.oc) d|^2, oc = eye - centre.  Shading point:
 * P = eye + t d; N = n (plane) or (P - centre) / radius; the material and (u, v) above; the
 * ray cone of spread angle 2 tan_half_y / height has width w = t 2 tan_half_y / height at
 * the hit; the footprint's axes are A1 = w m1 with m1 = unit(N x d) (head-on, |N x d| <
 * 1e-6: unit(N x h), h = x axis if |N.x| < 0.9 else y axis) and A2 = w / max(|N.d|, 1e-3)
 * m2 with m2 = unit(d - (N.d) N) (head-on: unit(N x m1)); the gradients are
 * g1 = uv_scale (A1[a0], A1[a1]), g2 = uv_scale (A2[a0], A2[a1]).  A ray that hits nothing
 * writes material UINT32_MAX, which a pass reports as out of range: give a closed scene. */
#define PMC_MAX_SCENE_OBJECTS 64u
#define PMC_OBJ_PLANE 0u
#define PMC_OBJ_SPHERE 1u
typedef struct {
    uint32_t kind;
    uint32_t mat;
    uint32_t axes;
    float uv_scale;
    float p[4];
} pmc_scene_object; /* 32 bytes */

typedef struct {
    float eye[3];
    float fwd[3];
    float right[3];
    float up[3];
    float tan_half_y;
    uint32_t width;
    uint32_t height;
} pmc_camera;

/* Output planes, DEVICE memory owned by the caller, (row1 - row0) * width entries each,
 * scanline order from row row0. */
typedef struct {
    float* u;
    float* v;
    uint32_t* mat;
    float *px, *py, *pz;
    float *nx, *ny, *nz;
    float *g1u, *g1v, *g2u, *g2v;
} pmc_ray_hits;

/* Casts the primary rays of rows row0 .. row1 - 1 for pass `pass` (asynchronous on
 * `stream`).  PMC_ERR_INVALID_ARG for a malformed object or camera, more than
 * PMC_MAX_SCENE_OBJECTS objects, rows outside the image or a missing output plane;
 * PMC_ERR_UNSUPPORTED beyond 2^28 points. */
pmc_status pmc_cast_rays(const pmc_scene_object* objects, uint32_t n_objects, const pmc_camera* cam,
                         uint32_t row0, uint32_t row1, uint64_t seed, uint32_t pass,
                         const pmc_ray_hits* out, void* stream);

/* Human-readable name of a status code (static storage). */
const char* pmc_status_str(pmc_status s);

#ifdef __cplusplus
}
#endif
#endif
