/*
 * pmc_oracle.h -- CPU FP64 oracle of Progressive Material Caching
 * (Fujieda & Harada, SIGGRAPH Asia 2022 Technical Communications).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, sequential statement of
 * what the GPU path computes.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant with the CUDA library: every definition here is written again
 * from the paper and from the published descriptions of the primitives.
 *
 * What it follows:
 *   - Sec. 2: a material is a node network evaluated node by node in storage
 *     order (the "stack machine" form);
 *   - Sec. 3: cacheable nodes are the highest nodes whose sub-graph depends on
 *     no shading-point information other than UV; on a hit the sub-graph is
 *     skipped, on a miss it is evaluated and its value is stored;
 *   - Sec. 3.1 and Eq. 1: the descriptor is (material ID, node ID, mip level,
 *     texel indices) with a virtual texture of 2^lambda texels per axis;
 *   - Sec. 3.2 and Fig. 3: a fixed table of N_c cells x N_e entries, cell =
 *     Hash(desc) mod N_c, entry verified by Hash2(desc), first value kept;
 *   - Algorithm 1: an entry is taken at the first slot whose stored hash is
 *     either Hash2(desc) or 0.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   hash pair = SplitMix64 finalizer / MurmurHash3 fmix64 (Sec. 3.2 names
 *   none); Hash2 == 0 is remapped to 1 because 0 marks an empty entry
 *   (Alg. 1); the entry loop runs i = 0 .. N_e-1; a batch of shading points
 *   sees only entries inserted by earlier batches and inserts in ascending
 *   (point index, node ID) order (a serialisation of the concurrent CAS of
 *   Alg. 1); the stored value is the inserting point's own value rounded to
 *   FP32.
 */
#ifndef PMC_ORACLE_H
#define PMC_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One node of a material network (binary layout of the IR format).
 * in[k] is the index of an earlier node or -1; ip/fp are integer and float
 * parameters whose meaning depends on op. */
typedef struct {
    uint32_t op;
    int32_t in[4];
    int32_t ip[4];
    float fp[16];
} orc_node;

/* Node operators.  The numbering is part of the IR format. */
enum {
    ORC_UV = 0,        /* (u, v, 0)                                    */
    ORC_POSITION = 1,  /* (px, py, pz)         shading-point dependent */
    ORC_NORMAL = 2,    /* (nx, ny, nz)         shading-point dependent */
    ORC_CONST = 3,     /* (fp0, fp1, fp2)                              */
    ORC_UV_AFFINE = 4, /* 2-D affine map of in0.xy                     */
    ORC_FBM = 5,       /* fractal sum of 2-D gradient noise            */
    ORC_VORONOI = 6,   /* Worley F1 distance                           */
    ORC_CHECKER = 7,   /* two-colour checkerboard                      */
    ORC_RAMP = 8,      /* colour ramp of 2..4 stops                    */
    ORC_MIX = 9,       /* a + (b - a) f                                */
    ORC_ADD = 10,      /* a + b                                        */
    ORC_MUL = 11,      /* a * b                                        */
    ORC_POW = 12,      /* max(a,0)^e                                   */
    ORC_FACING = 13,   /* |dot(in0, d)|                                */
    ORC_NUM_OPS = 14
};

/* Dependence classes (Sec. 3): CONST < UV < SP; POS (position only) exists only with the
 * world-position descriptor. */
enum { ORC_CLS_CONST = 0, ORC_CLS_UV = 1, ORC_CLS_SP = 2, ORC_CLS_POS = 3 };

/* Status codes. */
enum {
    ORC_OK = 0,
    ORC_ERR_ARG = 1,     /* malformed network or argument */
    ORC_ERR_BADMAT = 2,  /* a shading point names a material that does not exist */
};

/* ---- published mixers ---------------------------------------------------- */
uint32_t orc_fmix32(uint32_t h);          /* MurmurHash3 32-bit finaliser     */
uint64_t orc_fmix64(uint64_t k);          /* MurmurHash3 64-bit finaliser     */
uint64_t orc_splitmix64_mix(uint64_t z);  /* SplitMix64 output function       */

/* ---- node primitives ------------------------------------------------------ */
uint32_t orc_lattice_hash(int64_t i, int64_t j, uint32_t seed);
double orc_fade(double t);
double orc_perlin(double x, double y, uint32_t seed);
double orc_fbm(double x, double y, double scale, int octaves, double lacunarity,
               double gain, uint32_t seed);
double orc_voronoi_f1(double x, double y, uint32_t seed);
/* Evaluate one node given its input values (3 doubles each, NULL if unused)
 * and the shading point sp = (u, v, px, py, pz, nx, ny, nz). */
void orc_eval_node(const orc_node* nd, const double* a, const double* b, const double* c,
                   const double sp[8], double out[3]);

/* ---- descriptor and hashes (Sec. 3.1, Eq. 1, Sec. 3.2) -------------------- */
uint32_t orc_texel(float u, uint32_t level);
/* Eq. 1: floor(-log2(min(|g1|, |g2|))) + offset, clamped to [0, 13] (squared norms in
 * FP32; a zero footprint gives 13, an infinite or NaN one 0). */
int32_t orc_level(float g1u, float g1v, float g2u, float g2v, int32_t offset);
/* The 32-bit encoding of a cached value (Alg. 1 "Encode"): shared-exponent RGB9E5. */
uint32_t orc_rgb9e5_encode(float r, float g, float b);
void orc_rgb9e5_decode(uint32_t code, float out[3]);
uint64_t orc_key(uint32_t mat, uint32_t node, uint32_t level, float u, float v);
/* World-position descriptor: voxel index floor(p 2^level) clamped to [-512, 511] + 512
 * per axis (NaN -> 0), key = mat<<48 | node<<32 | 1<<31 | ix<<20 | iy<<10 | iz. */
uint32_t orc_voxel(float p, uint32_t level);
uint64_t orc_key_pos(uint32_t mat, uint32_t node, uint32_t level, float px, float py, float pz);
uint64_t orc_hash1(uint64_t key);
uint32_t orc_hash2(uint64_t key);
/* Loops over the functions above: descriptor, cell (Hash mod n_cells) and check value of n
 * (material, node, u, v) tuples at one level; and the two 64-bit mixers (SplitMix64's
 * output function, fmix64 of key xor 0x9E3779B97F4A7C15) of n keys. */
void orc_address_batch(const uint32_t* mat, const uint32_t* node, const float* u, const float* v,
                       uint64_t n, uint32_t level, uint64_t n_cells, uint64_t* key, uint64_t* cell,
                       uint32_t* h2);
void orc_mix_batch(const uint64_t* key, uint64_t n, uint64_t* h1, uint64_t* m2);

/* ---- network analysis (Sec. 3) ------------------------------------------- */
/* Validates the network and fills cls[n] (ORC_CLS_*), is_root[n] (0/1).
 * Returns ORC_OK or ORC_ERR_ARG. */
int orc_validate(const orc_node* nodes, uint32_t n);
int orc_analyze(const orc_node* nodes, uint32_t n, uint32_t min_root_nodes,
                int32_t* cls, uint8_t* is_root, uint32_t* n_roots);
/* The same with the world-position descriptor if pos_desc != 0: nodes that depend on the
 * position and on nothing else of the shading point are cacheable too (is_root 2). */
int orc_analyze_desc(const orc_node* nodes, uint32_t n, uint32_t min_root_nodes, int pos_desc,
                     int32_t* cls, uint8_t* is_root, uint32_t* n_roots);
/* The same with a cost threshold: a root's sub-graph (the node and every node it reads,
 * each once) must cost at least min_root_cost FP32 operations by orc_node_cost. */
int orc_analyze_cost(const orc_node* nodes, uint32_t n, uint32_t min_root_nodes, uint32_t min_root_cost,
                     int pos_desc, int32_t* cls, uint8_t* is_root, uint32_t* n_roots);
/* The node cost model of the library's interface (FP32 operations, a multiply-add as 2). */
uint32_t orc_node_cost(const orc_node* nd);

/* ---- single shading point, no cache -------------------------------------- */
/* Plain evaluation of every node reachable from the output. */
int orc_eval_point_nocache(const orc_node* nodes, uint32_t n, const double sp[8],
                           double rgb[3]);

/* ---- progressive cache ----------------------------------------------------- */
typedef struct orc_cache orc_cache;

/* Optional test hook: replaces Hash/Hash2 for a descriptor. */
typedef void (*orc_hash_override_fn)(uint64_t key, uint64_t n_cells, uint64_t* cell,
                                     uint32_t* h2);

/* n_cells == 0 or cache_off != 0 gives plain evaluation (no lookups, no inserts). */
orc_cache* orc_cache_new(uint64_t n_cells, uint32_t n_entries, uint32_t level,
                         uint32_t min_root_nodes, int cache_off);
void orc_cache_free(orc_cache* c);
/* Copies the networks in (mat_nodes[m] points at n_nodes[m] nodes). */
int orc_cache_set_materials(orc_cache* c, uint32_t n_mats, const orc_node* const* mat_nodes,
                            const uint32_t* n_nodes);
void orc_cache_set_hash_override(orc_cache* c, orc_hash_override_fn fn);
/* Offset added to the ray-cone level of every point (default 0). */
void orc_cache_set_level_offset(orc_cache* c, int32_t offset);
/* on != 0: the paper's concurrent update (Alg. 1) serialised point by point: each point
 * looks up the table as the earlier points of its batch left it and inserts its evaluated
 * cacheable nodes at once, with values stored as their 32-bit encoding (RGB9E5). */
void orc_cache_set_alg1(orc_cache* c, int on);
/* on != 0: replacement by visibility class, the prioritisation of directly visible
 * shading points that Sec. 5 proposes.  Every point carries a class (0 = seen directly
 * from the camera, k = reached after k bounces; orc_run_batch's vis) and every entry
 * the class of the point that inserted it.  An insert into a full cell that holds no
 * entry of its descriptor overwrites the entry of the largest class, if that class is
 * larger than the newcomer's (the first such entry on ties), and counts it as replaced;
 * otherwise the value is dropped as with keep-first.  Lookups do not change classes.
 * A value whose cell, at lookup, is full of entries of classes at most its own can never
 * enter the cell in that batch (a full cell's classes only decrease), so it is dropped as
 * full there and then, even if a copy of its key with a smaller class enters the cell
 * earlier in the batch.  With every class 0 the table evolves exactly as with keep-first. */
void orc_cache_set_replacement(orc_cache* c, int on);
/* Replacement only: on (the default) = the rule above, a value whose full cell holds no
 * class larger than its own is dropped as full at lookup; off = every evaluated miss goes
 * to the sequential insert, where such a value is dropped as full or, if a copy of its key
 * with a smaller class entered the cell earlier in the batch, as a duplicate.  The two
 * rules leave the same table and classes; only that full/duplicate split differs. */
void orc_cache_set_close_at_lookup(orc_cache* c, int on);
/* The cost threshold of cacheable nodes (orc_analyze_cost); set it before the materials. */
void orc_cache_set_min_root_cost(orc_cache* c, uint32_t cost);
/* Host threads that orc_run_batch spreads the lookup and evaluation phase over (ranges of
 * points against the same snapshot of the table; the insert stays one candidate at a time
 * in ascending (point index, node ID) order, so the results are those of one thread).  The
 * paper's concurrent update (orc_cache_set_alg1) always runs on one thread. */
void orc_cache_set_threads(orc_cache* c, int threads);
/* level >= 0: the world-position descriptor (Sec. 3.1 names world-space position as a
 * further descriptor, Sec. 5 lists it as future work).  A node whose sub-graph depends on
 * the shading point's position and on nothing else of it is cacheable too; its key is
 * orc_key_pos at this level (voxels of 2^-level world units).  Must be called before
 * orc_cache_set_materials.  Default -1 (off). */
void orc_cache_set_position_level(orc_cache* c, int32_t level);
void orc_cache_reset(orc_cache* c);
uint32_t orc_cache_n_roots(const orc_cache* c, uint32_t mat);
/* Root node IDs of a material in ascending order (n_roots entries). */
void orc_cache_roots(const orc_cache* c, uint32_t mat, uint32_t* out);

/* One progressive pass over n shading points (SoA, FP32 as stored on the GPU).
 * Outputs: rgb (3*n doubles, SoA r[n] g[n] b[n]); hits (n), may be NULL;
 * evaluated (n; nodes evaluated per point), may be NULL;
 * probe_* arrays (sum over points of the point's root count, point-major,
 * roots in ascending node ID), each may be NULL.
 * g1u, g1v, g2u, g2v: per-point ray-cone texture-coordinate gradients (n each) that
 * give each point its own mip level (orc_level), or all NULL for the cache's level.
 * vis: per-point visibility class (n entries) for the replacement policy, or NULL for
 * class 0 everywhere.
 * Returns ORC_OK, or ORC_ERR_BADMAT if some mat[i] >= n_mats (those points
 * get rgb 0, hits 0 and no probes). */
int orc_run_batch(orc_cache* c, uint64_t n, const float* u, const float* v,
                  const uint32_t* mat, const float* px, const float* py, const float* pz,
                  const float* nx, const float* ny, const float* nz, double* rgb,
                  uint16_t* hits, uint32_t* evaluated, uint64_t* probe_key,
                  uint64_t* probe_cell, uint32_t* probe_h2, uint8_t* probe_hit,
                  const float* g1u, const float* g1v, const float* g2u, const float* g2v,
                  const uint8_t* vis);

/* Table contents: h2[N_c*N_e], rgb[3*N_c*N_e] (slot-major r,g,b). */
void orc_cache_table(const orc_cache* c, uint32_t* h2, float* rgb);
/* Visibility class of every slot's entry (N_c*N_e bytes; meaningful where h2 != 0). */
void orc_cache_classes(const orc_cache* c, uint8_t* cls);

/* ---- learned surrogate of a cacheable node -------------------------------------------
 * Network of (u, v): features [sin pi k u, cos pi k u, sin pi k v, cos pi k v], k=1..16,
 * -> relu(64) -> relu(64) -> 3; theta = W1[64][64], b1, W2[64][64], b2, W3[64][3], b3.
 * bf16 != 0 rounds features, weights and hidden activations to bfloat16 (nearest, ties to
 * even) where the tensor-core kernels round them; everything else is FP64. */
#define ORC_MLP_PARAMS 8515
void orc_mlp_forward(const double* theta, double u, double v, int bf16, double y[3]);
/* From the next batch on, node `node` of material `mat` takes clamp(network(u, v), 0, 1)
 * instead of a lookup and its sub-graph; theta == NULL removes it. */
int orc_cache_set_surrogate(orc_cache* c, uint32_t mat, uint32_t node, const double* theta, int bf16);

/* Counters, in this order:
 * 0 lookups, 1 hits, 2 misses, 3 candidates, 4 inserted, 5 dropped_dup,
 * 6 dropped_full, 7 nodes_evaluated, 8 batches, 9 replaced (entries overwritten by the
 * replacement policy; inserted counts only empty slots taken). */
#define ORC_NSTATS 10
void orc_cache_stats(const orc_cache* c, uint64_t out[ORC_NSTATS]);

#ifdef __cplusplus
}
#endif
#endif
