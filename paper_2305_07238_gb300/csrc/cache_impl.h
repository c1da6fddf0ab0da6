// cache_impl.h -- the library's definition of the opaque pmc_cache object.
#pragma once

#include <vector>

#include "pmc_internal.h"

struct pmc_cache {
    using MatInfo = pmc::MatInfo;
    using Control = pmc::Control;
    using Candidate = pmc::Candidate;

    pmc_cache_desc desc{};
    int use_cache = 1;
    uint32_t n_mats = 0;
    uint32_t max_roots = 0;
    uint32_t max_slots = 0;         // per-point programs (k_eval, k_eval_fused)
    uint32_t max_slots_roots = 0;   // standalone cacheable-node programs (k_eval_roots, sampling)
    uint32_t max_slots_outer = 0;   // outer programs (k_eval once every block has its value)
    int num_sms = 0;
    std::vector<MatInfo> mat_info;
    std::vector<uint32_t> roots;
    std::vector<uint32_t> roots_dev;      // the device root table: node ID | ROOT_POS_BIT
    std::vector<pmc::RootInfo> root_info;
    uint32_t max_level = 0;
    int split = 1;
    int unsorted = 0;                     // PMC_UNSORTED schedule
    int probe_inline = 0;                 // PMC_PROBE_INLINE schedule
    uint32_t lookup_rb = 4;               // probes in flight per lane in k_lookup
    int block_items = 0;                  // PMC_BLOCK_ITEMS schedule
    int one_point = 0;                    // PMC_ONE_POINT schedule
    int insert_binned = 0;                // PMC_INSERT_BINNED schedule
    uint64_t layout_gen = 1;              // bumped whenever a recorded graph would go stale
    uint32_t prog_len = 0;
    // device-resident, owned
    MatInfo* d_mats = nullptr;
    uint4* d_prog = nullptr;
    float* d_params = nullptr;
    uint32_t* d_roots = nullptr;
    uint4* d_table = nullptr;
    uint8_t* d_cls = nullptr;             // PMC_REPLACE_VISIBILITY: class of every slot's entry
    unsigned long long* d_claims = nullptr;
    uint32_t* d_chain_head = nullptr;     // n_cells list heads of the per-cell-list insert
    Control* d_ctl = nullptr;
    unsigned long long* d_stats = nullptr;
    pmc::RootInfo* d_rinfo = nullptr;
    uint32_t* d_miss_cnt = nullptr;       // roots + MAX_LEVELS
    uint32_t* d_root_items = nullptr;     // roots + 1, then MAX_LEVELS + 1 level item starts
    uint32_t* d_root_order = nullptr;     // roots by ascending level, then MAX_LEVELS + 1 starts
    uint32_t n_bins = 0;                  // cell-grouped insert bins
    bool table_empty = true;              // nothing inserted since creation or reset
    bool last_all_miss = false;           // the last batch ran on an empty table
    bool last_unsorted = false;           // the last batch kept no probe records
    bool last_noalloc = false;            // the last batch ran in the fixed no-alloc scratch
    // learned surrogates
    int use_surrogates = 1;
    std::vector<int32_t> surr_cand;       // per material: candidate node ordinal, -1 if none
    std::vector<int32_t> surr_slot;       // per material: parameter slot, -1 if none
    std::vector<uint8_t> surr_on;         // per material: enabled
    uint32_t n_surr_slots = 0, cap_surr_slots = 0;
    float* d_surr_theta = nullptr;        // cap_surr_slots x MLP_PARAMS
    unsigned char* d_surr_img = nullptr;  // cap_surr_slots x SURR_IMG_BYTES (operand images)
    int32_t* d_surr_slot = nullptr;       // n_mats: slot if enabled, else -1
    int32_t* d_surr_ord = nullptr;        // n_mats: ordinal if enabled, else -1
    uint32_t* d_surr_items = nullptr;     // n_mats + 1
    bool any_surr_on = false;
    bool all_roots_surr = false;   // every material's cacheable nodes are all surrogates' (>= one)
    uint32_t* d_bins = nullptr;           // counts (n_bins) | bases (n_bins + 1)
    // per-batch scratch, grown on demand
    uint64_t cap_points = 0;
    uint64_t cap_probes = 0;
    uint32_t* d_seg = nullptr;      // counts | seg_start | probe_base | item_base | cursor
    float* d_sorted = nullptr;      // 8 planes of cap_points
    uint32_t* d_sidx = nullptr;
    float4* d_probes = nullptr;
    Candidate* d_cands = nullptr;
    uint32_t* d_lists = nullptr;    // 3 lists of cap_probes
    uint32_t* d_misslist = nullptr; // cap_probes
    pmc::Candidate* d_cands_binned = nullptr;  // cap_probes
    // staging for the host-buffer entry point
    uint64_t cap_host = 0;
    float* d_hpts = nullptr;        // 8 float planes + 1 uint32 plane
    float* d_hrgb = nullptr;
    uint16_t* d_hhits = nullptr;
    // double-buffered staging of pmc_eval_passes_host: copies of one pass overlap the
    // evaluation of its neighbours, on two library-owned copy streams
    uint64_t cap_pipe = 0;
    float* d_pin[2] = {nullptr, nullptr};     // 13 float planes + one for the classes
    float* d_prgb[2] = {nullptr, nullptr};
    uint16_t* d_phits[2] = {nullptr, nullptr};
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
    // state
    cudaStream_t last_stream = nullptr;
    pmc_status sticky = PMC_OK;
    uint32_t epoch_host = 0;
    uint64_t last_n = 0;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> events;   // (PH_COUNT + 1) per timed batch, in order
    size_t events_used = 0;
    uint64_t launches = 0;
    uint64_t timed_batches = 0;
};

// The insert through per-cell lists applies to keep-first tables of N_e <= 8 resolved after
// the evaluation (not the claim rounds, the paper's concurrent update or replacement by
// visibility class), unless the PMC_INSERT_BINNED schedule asks for the binned insert.
inline bool insert_lists(const pmc_cache* c) {
    return c->use_cache && c->desc.n_entries <= 8 &&
           !(c->desc.flags & (PMC_INSERT_ROUNDS | PMC_ALG1 | PMC_REPLACE_VISIBILITY)) && !c->insert_binned;
}
