// pmc_internal.h -- data layouts shared by the library's host compiler, kernels and
// C-ABI layer.  Not installed; the public interface is include/pmc.h.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

#include "pmc.h"

namespace pmc {

// ---- compiled program ----------------------------------------------------------------
// A material is serialised (Sec. 2) into a linear program of 16-byte instructions run
// by one warp-uniform interpreter.  Node values live in per-lane "slots" (a register
// file in shared memory) assigned by linear-scan allocation.
//
//   x: op (bits 0-7) | flags (8-15) | cost in FP32 flops (16-31)
//   y: out slot (0-15) | in0 slot (16-31)         ROOT_BEGIN: out slot | root ordinal
//   z: in1 slot (0-15) | in2 slot (16-31)         ROOT_BEGIN: node ID
//   w: offset of the node's parameters in the parameter pool
//                                                 ROOT_BEGIN: number of instructions
//                                                 that follow up to the root itself
//
// A cacheable node r with the nodes only it needs (its exclusive sub-graph) forms a
// contiguous block: ROOT_BEGIN(r), the exclusive nodes, then r flagged FLAG_ROOT.  A
// lane whose lookup hit takes the cached value at ROOT_BEGIN and skips the block.
constexpr uint32_t OP_ROOT_BEGIN = 32;
constexpr uint32_t OP_LOAD_ROOT = 33;   // y: out slot | root ordinal; reads that node's probe record
constexpr uint32_t FLAG_ROOT = 1;
constexpr uint32_t FLAG_POSROOT = 2;    // ROOT_BEGIN of a node looked up under a position voxel
constexpr uint32_t FLAG_IN2 = 4;        // MIX: the factor comes from in2 (else from fp0)

// On the device, y and z of a node instruction hold byte offsets into the lane's slot
// file (slot x SLOT_BYTES: the file is [slot][channel][lane] per warp), so an operand is one
// add away from its address; 16-bit offsets allow MAX_DEVICE_SLOTS slots.
constexpr uint32_t SLOT_BYTES = 3u * 32u * 4u;
constexpr uint32_t MAX_DEVICE_SLOTS = 0xFFFFu / SLOT_BYTES;
constexpr uint32_t ROOT_POS_BIT = 1u << 31;   // device root table: node ID | this bit for such nodes

// Each cacheable node also gets a standalone program (its sub-graph, with any cacheable
// node below it read from its probe record) so that its misses can be evaluated 32 at
// a time.  Level 0 programs read no other cacheable node; level l reads levels < l.
struct RootInfo {
    uint32_t prog_start;  // in the shared program pool
    uint32_t prog_len;
    uint32_t mat;
    uint32_t ordinal;
    uint32_t level;
    uint32_t n_slots;
    uint32_t node;
    uint32_t out_slot;
    uint32_t nodes;       // nodes and FP32 operations one run of the program evaluates
    uint32_t flops;
};

struct MatInfo {
    uint32_t prog_start;  // first instruction in the program pool
    uint32_t prog_len;
    uint32_t root_base;   // first entry in the root-node table
    uint32_t n_roots;
    uint32_t out_slot;    // slot holding the material output after the program
    uint32_t n_slots;
    uint32_t n_nodes;
    uint32_t outer_start; // outer program: blocks replaced by loads of their node's record
    uint32_t outer_len;
    uint32_t outer_out_slot;
    uint32_t outer_slots;
    uint32_t pad;
    // nodes and FP32 operations one point evaluates with the whole program run (every
    // block evaluated) and with the outer program
    uint32_t full_nodes, full_flops, outer_nodes, outer_flops;
};

struct CompiledMaterial {
    std::vector<uint4> prog;
    std::vector<float> params;     // parameter offsets in prog are relative to this
    std::vector<uint32_t> roots;   // node IDs of cacheable nodes, ascending
    std::vector<uint8_t> root_pos; // per cacheable node: 1 = world-position descriptor
    std::vector<std::vector<uint4>> root_progs;  // standalone program per cacheable node
    std::vector<uint32_t> root_level;
    std::vector<uint32_t> root_slots;
    std::vector<uint32_t> root_out_slot;
    std::vector<uint4> outer_prog;    // the program with each block replaced by OP_LOAD_ROOT
    uint32_t outer_slots = 0;
    uint32_t outer_out_slot = 0;
    uint32_t out_slot = 0;
    uint32_t n_slots = 0;
    uint32_t n_nodes = 0;
};

// Compiles one network.  Returns false (with a reason) for a malformed network.
// min_root_cost: a cacheable node's sub-graph must cost at least this many FP32 operations
// of the node cost model (node_cost), summed over the network as given; 0 = no threshold.
bool compile_material(const pmc_node* nodes, uint32_t n, uint32_t min_root_nodes, uint32_t min_root_cost,
                      bool pos_desc, CompiledMaterial* out, const char** why);

// FP32 flops of one executed node (FMA counted as 2), from the device formulas: the node
// cost model of include/pmc.h (pmc_node_cost).
uint32_t node_cost(const pmc_node& nd);

// ---- insert candidates -----------------------------------------------------------------
struct __align__(16) Candidate {
    unsigned long long prio;  // (point index << 16) | node ID: the sequential order
    uint32_t cell;
    uint32_t h2;
    float r, g, b;
    uint32_t target;          // bits 0-7: first slot that can hold the key (the first empty
                              // slot at lookup; a round's choice in the claim-round insert);
                              // 8-15: the point's visibility class (replacement policy);
                              // 16-31: copies of the key merged into this candidate
};
static_assert(sizeof(Candidate) == 32, "candidate is one 32-byte sector");

constexpr uint32_t MAX_ENTRIES = 32;
constexpr uint32_t EPOCH_BITS = 20;
constexpr uint32_t EPOCH_MAX = (1u << EPOCH_BITS) - 1;
constexpr uint64_t MAX_POINTS = 1ull << 28;

constexpr uint32_t MAX_LEVELS = 16;    // nesting depth of cacheable nodes handled in batches
constexpr uint32_t MLP_PARAMS = 8515;  // learned surrogate: 64 -> 64 -> 64 -> 3
// A network's operand image: W1, W2 (64 x 64) and W3 (16 x 64, rows 3..15 zero) as BF16 in the
// inference kernel's shared-memory layout, then b1, b2, b3 and one zero as FP32 -- the bytes
// one bulk copy puts in place at a material boundary (a multiple of 16)
constexpr uint32_t SURR_IMG_BYTES = 8192 + 8192 + 2048 + 132 * 4;
static_assert(SURR_IMG_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");

// Device-side control block of one cache object.
struct Control {
    // cleared at the start of every batch
    uint32_t n_items;           // warp work items of the current batch
    uint32_t total_probes;
    uint32_t n_cand;            // candidates emitted by the evaluation
    uint32_t n_root_items;      // work items of the batched evaluation of misses
    uint32_t n_surr_items;      // work items of the surrogate inference
    uint32_t bins_warp;         // insert bins resolved by a warp, by a block, by ranges
    uint32_t bins_mid;
    uint32_t bins_big;
    uint32_t n_lists;           // cells with candidates (per-cell-list insert)
    uint32_t w_cand;            // candidates emitted for the insert, shadows included
    uint32_t pad1;
    // persistent
    uint32_t epoch;             // claim epoch of round 0 of the current batch
    uint32_t err;               // ERR_* bits
    uint32_t bar_count;         // grid barrier of the insert kernel
    uint32_t bar_gen;
    uint32_t mid_count[MAX_ENTRIES + 2];
    uint32_t out_count[MAX_ENTRIES + 2];
};

constexpr uint32_t ERR_BAD_MAT = 1;
constexpr uint32_t ERR_INSERT = 2;
constexpr uint32_t ERR_BOUNDS = 4;
constexpr uint32_t ERR_TIMEOUT = 8;
constexpr uint32_t ERR_CAPACITY = 16;   // the batch needs more probe records than the scratch holds

// Counter indices in the device stats array.
enum {
    ST_LOOKUPS = 0, ST_HITS, ST_MISSES, ST_CANDIDATES, ST_INSERTED, ST_DUP, ST_FULL,
    ST_NODES, ST_BATCHES, ST_FLOPS, ST_SLOTS, ST_POINTS, ST_BAD, ST_SURR, ST_FLOPS_MISSED, ST_RACE, ST_REPLACED,
    ST_COUNT = 17
};

// Everything a batch's kernels need, by value.
struct BatchArgs {
    // inputs (caller-owned device SoA)
    const float* u; const float* v; const uint32_t* mat;
    const float* px; const float* py; const float* pz;
    const float* nx; const float* ny; const float* nz;
    uint32_t n;
    // ray-cone gradients (caller-owned, optional): each point's own mip level (Eq. 1)
    const float* g1u; const float* g1v; const float* g2u; const float* g2v;
    int32_t level_offset;
    int32_t pos_level;         // world-position descriptor: voxels of 2^-pos_level; -1 = off
    // outputs
    float* out_rgb; uint16_t* out_hits;
    // materials
    const MatInfo* mats; uint32_t n_mats;
    const uint4* prog; const float* params; const uint32_t* roots;
    uint32_t max_slots;        // value slots of the largest per-point program
    uint32_t max_slots_roots;  // value slots of the largest standalone cacheable-node program
    uint32_t max_slots_outer;  // value slots of the largest outer program
    // sort / segments
    uint32_t* counts; uint32_t* seg_start; uint32_t* probe_base; uint32_t* item_base;
    uint32_t* cursor;
    float* su; float* sv; float* spx; float* spy; float* spz;
    float* snx; float* sny; float* snz; uint32_t* sidx;
    uint32_t* slev;            // grouped per-point mip levels (with ray-cone gradients)
    // cache: cell c = N_e hash2 words then N_e packed (r, g, b) values (16 * N_e bytes), or
    // with alg1 N_e 8-byte slots
    uint4* table; unsigned long long* claims;
    int table_empty;           // nothing inserted yet: every probe misses at slot 0
    int keys_inline;           // empty table: the evaluator forms descriptors itself and
                               // emits every cacheable node (no lookup pass)
    uint64_t n_cells; uint32_t n_entries; uint32_t level; uint32_t cells_pow2_mask;
    int use_cache; int debug;
    float4* probes; uint32_t probe_cap;
    Candidate* cands;
    // index lists of the claim-round insert; the cell-grouped insert uses lists[0] for
    // the cells of the candidates in emission order, and the per-cell-list insert lists[1]
    // for the cells that received candidates
    uint32_t* lists[3];
    Control* ctl; unsigned long long* stats;
    // batched evaluation of misses
    int split;
    const RootInfo* rinfo; uint32_t n_roots_total; uint32_t max_level;
    uint32_t* miss_cnt;        // n_roots_total counters, then MAX_LEVELS item counters
    // cacheable nodes in ascending nesting level (a permutation of the global root index),
    // and where each level starts in it (MAX_LEVELS + 1 entries): the batched evaluation of
    // one level visits only that level's work items
    const uint32_t* root_order; const uint32_t* level_start;
    uint32_t* root_item_base;  // n_roots_total + 1 item offsets in root_order's order, then
                               // MAX_LEVELS + 1 first items of each level
    uint32_t* misslist;        // probe_cap
    int insert_rounds;         // 1: atomicMin rounds (claims hold epoch words); 0: cell-grouped
    // learned surrogates: per material the surrogate's slot (-1 = none) and cacheable-node
    // ordinal; FP32 parameters per slot; work items of 128 points per material
    const int32_t* surr_slot; const int32_t* surr_ord; const float* surr_theta;
    const unsigned char* surr_img;   // per slot SURR_IMG_BYTES (16-byte aligned), or null
    uint32_t* surr_item_base;  // n_mats + 1 (computed by k_scan)
    int all_surr;              // 1: every cacheable node of every material is a surrogate's:
                               // no lookup, no batched misses, no insert
    uint32_t n_bins;           // cell-grouped insert: ceil(n_cells / INSERT_BIN_CELLS) bins
    uint32_t* bin_cnt;         // n_bins
    uint32_t* bin_base;        // n_bins + 1
    uint32_t* bin_list;        // n_bins: the non-empty bins by resolving kernel (warp, block,
                               // ranges), each class in ascending bin order
    Candidate* cands_binned;   // probe_cap
    // insert through per-cell lists (keep-first, N_e <= 8): the last candidate to reach
    // each cell (n_cells entries, CHAIN_END when none; every list is empty between
    // batches); a candidate's cell field then holds its predecessor in its cell's list
    int insert_lists;
    uint32_t* chain_head;
    // schedule (chosen by the caller's flags or by the autotuner)
    int unsorted;              // 1: no grouping; k_eval_fused probes inline in batch order
    int probe_inline;          // 1: grouped; k_eval_fused probes inline (no lookup kernel)
    uint32_t lookup_rb;        // k_lookup: probes in flight per lane (1, 2 or 4)
    int block_items;           // 1: the per-point evaluator claims block-wide tiles of items
    int one_point;             // 1: one point per lane in the per-point evaluator (else two)
    int alg1;                  // the paper's concurrent update: 8-byte slots {hash2, RGB9E5},
                               // looked up and inserted inside the evaluator (one 64-bit CAS)
    // replacement by visibility class (Sec. 5): per point its class (caller-owned, optional,
    // original order), per slot the class of its entry; slot_cls == nullptr = keep-first
    const uint8_t* vis;
    uint8_t* slot_cls;
};

constexpr uint32_t INSERT_BIN_CELLS = 256;


// Phases timed by the optional CUDA events of a batch.
enum { PH_SORT = 0, PH_LOOKUP, PH_MISSED, PH_EVAL, PH_INSERT, PH_FINISH, PH_COUNT };

// Launch sequence of one batch (kernels.cu).  `ev`, if not null, holds PH_COUNT + 1
// events recorded on `s` at the phase boundaries; `*launches` counts kernel launches.
cudaError_t launch_batch(const BatchArgs& a, cudaStream_t s, int num_sms, cudaEvent_t* ev,
                         uint64_t* launches);
cudaError_t launch_reset(uint4* table, size_t units, unsigned long long* claims, uint32_t* chain_head, size_t cells,
                         Control* ctl, unsigned long long* stats, cudaStream_t s, bool claim_words);
cudaError_t launch_levels(const float* g1u, const float* g1v, const float* g2u, const float* g2v, uint64_t n,
                          int32_t offset, uint32_t* level, cudaStream_t s);
cudaError_t launch_keys(const uint32_t* mat, const uint32_t* node, const float* u,
                        const float* v, uint64_t n, uint32_t level, uint64_t n_cells,
                        uint64_t* key, uint64_t* cell, uint32_t* h2, cudaStream_t s);
size_t eval_smem_bytes(uint32_t max_slots);

// Training of the learned surrogates on the tcgen05 tensor cores (mlp_tc.cu): `steps`
// minibatches of 128 rows per (split, material); mode 0 takes Adam steps, mode 1 adds the
// gradient into `grad`.  err (may be null) receives ERR_TIMEOUT if a bounded wait for the
// tensor cores ran out (that material's loss then reads NaN).
cudaError_t launch_mlp_train(float* theta, float* adam_m, float* adam_v, float* grad, const float* data, float* loss,
                             uint32_t* err, uint32_t n_mats, uint32_t n_data, uint32_t steps, uint64_t sample0,
                             uint32_t step0, uint32_t total_steps, float lr, float grad_scale, int mode, uint32_t splits,
                             cudaStream_t s);
// Tensor-core (tcgen05) inference (mlp_tc.cu); err may be null.
cudaError_t launch_mlp_forward_tc(const float* theta, const float* u, const float* v, uint32_t n, float* out, int clamp,
                                  uint32_t* err, int num_sms, cudaStream_t s);
cudaError_t launch_root_samples(const uint4* prog, const float* params, const RootInfo* rinfo, const uint32_t* groots,
                                uint32_t n_train_mats, uint32_t n_rows, uint64_t seed, float* data, uint32_t max_slots,
                                int num_sms, cudaStream_t s);
cudaError_t launch_surrogate(const BatchArgs& a, int num_sms, cudaStream_t s);
// Writes the operand images of slots 0 .. n_slots - 1 from their FP32 parameters.
cudaError_t launch_surrogate_images(const float* theta, uint32_t n_slots, unsigned char* img, cudaStream_t s);

}  // namespace pmc
