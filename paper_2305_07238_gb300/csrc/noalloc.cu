// noalloc.cu -- pmc_eval_batch_noalloc: the per-pass pipeline of pmc_eval_batch with its
// per-batch scratch in one fixed file-scope device array, so the call allocates nothing.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "cache_impl.h"
#include "pmc_internal.h"

using namespace pmc;

namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Regions of the array, each 256-byte aligned.
constexpr size_t NA_MATS1 = (size_t)PMC_NOALLOC_MAX_MATERIALS + 1;
constexpr size_t NA_POINTS = PMC_NOALLOC_MAX_POINTS;
constexpr size_t NA_PROBES = PMC_NOALLOC_MAX_PROBES;
constexpr size_t OFF_SEG = 0;                                          // 5 x (mats + 1) u32
constexpr size_t OFF_SORTED = OFF_SEG + align256(5 * NA_MATS1 * 4);     // 8 float planes, u32 levels
constexpr size_t OFF_SIDX = OFF_SORTED + align256(9 * NA_POINTS * 4);  // u32 point indices
constexpr size_t OFF_PROBES = OFF_SIDX + align256(NA_POINTS * 4);      // 16-B probe records
constexpr size_t OFF_CANDS = OFF_PROBES + align256(NA_PROBES * 16);    // 32-B candidates
constexpr size_t OFF_LISTS = OFF_CANDS + align256(NA_PROBES * 32);     // 3 u32 index lists
constexpr size_t OFF_MISS = OFF_LISTS + align256(3 * NA_PROBES * 4);   // u32 miss lists
constexpr size_t OFF_BINNED = OFF_MISS + align256(NA_PROBES * 4);    // 32-B binned candidates
constexpr size_t SCRATCH_BYTES = OFF_BINNED + align256(NA_PROBES * 32);
static_assert(SCRATCH_BYTES == PMC_NOALLOC_SCRATCH_BYTES, "pmc.h states the array size");

}  // namespace

// Present on every device that loads the library, for the life of the process.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[MAX_DEVICES] = {};

// The array's device address on the current device, looked up once per device.  In host
// code the name g_noalloc_scratch is only a host-side stand-in, never a device pointer.
pmc_status scratch_on_current_device(int dev, unsigned char** out) {
    if (dev < 0 || dev >= MAX_DEVICES) return PMC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            fprintf(stderr, "pmc: cudaGetSymbolAddress of the no-alloc scratch failed on device %d: %s\n",
                    dev, cudaGetErrorString(e));
            cudaGetLastError();
            return PMC_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[dev];
    return PMC_OK;
}

}  // namespace

extern "C" pmc_status pmc_eval_batch_noalloc(pmc_cache* c, const pmc_points* pts, float* out_rgb,
                                             uint16_t* out_hits, void* stream) {
    if (!c || !pts) return PMC_ERR_INVALID_ARG;
    if (c->sticky != PMC_OK) return c->sticky;
    const uint64_t n = pts->n;
    if (n > 0 && (!pts->u || !pts->v || !pts->mat || !pts->px || !pts->py || !pts->pz || !pts->nx ||
                  !pts->ny || !pts->nz || !out_rgb))
        return PMC_ERR_INVALID_ARG;
    const int ng = (pts->g1u != nullptr) + (pts->g1v != nullptr) + (pts->g2u != nullptr) + (pts->g2v != nullptr);
    if (ng != 0 && ng != 4) return PMC_ERR_INVALID_ARG;   // all four gradients or none
    const uint64_t probes = (c->use_cache || (c->use_surrogates && c->any_surr_on)) ? n * (uint64_t)c->max_roots : 0;
    if (n > PMC_NOALLOC_MAX_POINTS || c->n_mats > PMC_NOALLOC_MAX_MATERIALS || probes > PMC_NOALLOC_MAX_PROBES) {
        fprintf(stderr,
                "pmc_eval_batch_noalloc: %llu points x %u cacheable nodes over %u materials exceeds the fixed "
                "scratch (at most %u points, %u probes, %u materials)\n",
                (unsigned long long)n, c->max_roots, c->n_mats, PMC_NOALLOC_MAX_POINTS,
                PMC_NOALLOC_MAX_PROBES, PMC_NOALLOC_MAX_MATERIALS);
        return PMC_ERR_UNSUPPORTED;
    }
    if (c->unsorted && c->use_surrogates && c->any_surr_on) return PMC_ERR_UNSUPPORTED;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != c->desc.device && cudaSetDevice(c->desc.device) != cudaSuccess) return PMC_ERR_INVALID_ARG;
    struct Restore {
        int prev, dev;
        ~Restore() { if (prev >= 0 && prev != dev) cudaSetDevice(prev); }
    } restore{prev, c->desc.device};

    unsigned char* base = nullptr;
    pmc_status st = scratch_on_current_device(c->desc.device, &base);
    if (st != PMC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t ne = c->desc.n_entries;
    if (c->use_cache && (c->desc.flags & PMC_INSERT_ROUNDS) && c->epoch_host + 2 * (ne + 1) > EPOCH_MAX) {
        cudaError_t e = cudaMemsetAsync(c->d_claims, 0xFF, c->desc.n_cells * sizeof(unsigned long long), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(&c->d_ctl->epoch, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) {
            c->sticky = PMC_ERR_CUDA;
            return PMC_ERR_CUDA;
        }
        c->epoch_host = 0;
    }

    BatchArgs a{};
    a.u = pts->u; a.v = pts->v; a.mat = pts->mat;
    a.px = pts->px; a.py = pts->py; a.pz = pts->pz;
    a.nx = pts->nx; a.ny = pts->ny; a.nz = pts->nz;
    a.n = (uint32_t)n;
    a.g1u = pts->g1u; a.g1v = pts->g1v; a.g2u = pts->g2u; a.g2v = pts->g2v;
    a.level_offset = c->desc.level_offset;
    a.pos_level = (c->use_cache && (c->desc.flags & PMC_POSITION_DESCRIPTOR)) ? (int32_t)c->desc.pos_level : -1;
    a.out_rgb = out_rgb; a.out_hits = out_hits;
    a.mats = c->d_mats; a.n_mats = c->n_mats;
    a.prog = c->d_prog; a.params = c->d_params; a.roots = c->d_roots;
    a.max_slots = c->max_slots ? c->max_slots : 1;
    a.max_slots_roots = c->max_slots_roots ? c->max_slots_roots : 1;
    a.max_slots_outer = c->max_slots_outer ? c->max_slots_outer : 1;
    uint32_t* seg = reinterpret_cast<uint32_t*>(base + OFF_SEG);
    const size_t M1 = (size_t)c->n_mats + 1;
    a.counts = seg; a.seg_start = seg + M1; a.probe_base = seg + 2 * M1;
    a.item_base = seg + 3 * M1; a.cursor = seg + 4 * M1;
    float* sorted = reinterpret_cast<float*>(base + OFF_SORTED);
    a.su = sorted; a.sv = sorted + NA_POINTS; a.spx = sorted + 2 * NA_POINTS; a.spy = sorted + 3 * NA_POINTS;
    a.spz = sorted + 4 * NA_POINTS; a.snx = sorted + 5 * NA_POINTS; a.sny = sorted + 6 * NA_POINTS;
    a.snz = sorted + 7 * NA_POINTS;
    a.slev = reinterpret_cast<uint32_t*>(sorted + 8 * NA_POINTS);
    a.sidx = reinterpret_cast<uint32_t*>(base + OFF_SIDX);
    a.table = c->d_table; a.claims = c->d_claims;
    a.alg1 = (c->use_cache && (c->desc.flags & PMC_ALG1)) ? 1 : 0;
    a.table_empty = (c->table_empty && !a.alg1) ? 1 : 0;
    a.keys_inline = (c->use_cache && c->table_empty && !a.alg1) ? 1 : 0;
    a.n_cells = c->use_cache ? c->desc.n_cells : 1; a.n_entries = c->use_cache ? ne : 1;
    a.level = c->desc.uv_level;
    const uint64_t nc = a.n_cells;
    a.cells_pow2_mask = (nc > 1 && (nc & (nc - 1)) == 0) ? (uint32_t)(nc - 1) : 0u;
    a.use_cache = c->use_cache; a.debug = (c->desc.flags & PMC_DEBUG_CHECKS) != 0;
    a.probes = reinterpret_cast<float4*>(base + OFF_PROBES);
    // a stated probe capacity binds here as in pmc_eval_batch: a batch needing more
    // records does no work and the next synchronising call reports it
    a.probe_cap = (uint32_t)(c->desc.probe_capacity ? std::min<uint64_t>(c->desc.probe_capacity, NA_PROBES)
                                                    : NA_PROBES);
    a.cands = reinterpret_cast<Candidate*>(base + OFF_CANDS);
    uint32_t* lists = reinterpret_cast<uint32_t*>(base + OFF_LISTS);
    a.lists[0] = lists; a.lists[1] = lists + NA_PROBES; a.lists[2] = lists + 2 * NA_PROBES;
    a.ctl = c->d_ctl; a.stats = c->d_stats;
    a.split = c->use_cache && c->split;
    a.insert_rounds = (c->desc.flags & PMC_INSERT_ROUNDS) ? 1 : 0;
    a.n_bins = c->n_bins; a.bin_cnt = c->d_bins; a.bin_base = c->d_bins + c->n_bins;
    a.bin_list = c->d_bins + 2 * (size_t)c->n_bins + 1;
    a.cands_binned = reinterpret_cast<Candidate*>(base + OFF_BINNED);
    a.insert_lists = insert_lists(c) ? 1 : 0;
    a.chain_head = c->d_chain_head;
    if (c->use_surrogates && c->any_surr_on) {
        a.surr_slot = c->d_surr_slot; a.surr_ord = c->d_surr_ord; a.surr_theta = c->d_surr_theta;
        a.surr_item_base = c->d_surr_items;
        a.surr_img = c->d_surr_img;
        a.all_surr = c->all_roots_surr ? 1 : 0;
    }
    a.rinfo = c->d_rinfo; a.n_roots_total = (uint32_t)c->root_info.size(); a.max_level = c->max_level;
    a.miss_cnt = c->d_miss_cnt; a.root_item_base = c->d_root_items;
    a.root_order = c->d_root_order; a.level_start = c->d_root_order + c->root_info.size();
    a.misslist = reinterpret_cast<uint32_t*>(base + OFF_MISS);
    a.unsorted = c->unsorted;
    a.probe_inline = c->probe_inline;
    a.lookup_rb = c->lookup_rb;
    a.block_items = c->block_items;
    a.one_point = c->one_point;
    if (c->use_cache && (c->desc.flags & PMC_REPLACE_VISIBILITY)) {
        a.slot_cls = c->d_cls;
        a.vis = pts->vis;
    }
    // launch_batch clears the counters and offsets that must start at zero; every other
    // region is written before it is read within the pass.
    cudaError_t e = launch_batch(a, s, c->num_sms, nullptr, &c->launches);
    if (e != cudaSuccess) {
        fprintf(stderr, "pmc: CUDA error %d (%s)\n", (int)e, cudaGetErrorString(e));
        c->sticky = PMC_ERR_CUDA;
        return PMC_ERR_CUDA;
    }
    if (c->use_cache) c->epoch_host += ne + 1;
    if (n > 0) c->table_empty = false;
    c->last_stream = s;
    c->last_n = n;
    c->last_noalloc = true;   // pmc_last_hit_masks refuses this pass (PMC_ERR_UNSUPPORTED)
    return PMC_OK;
}
