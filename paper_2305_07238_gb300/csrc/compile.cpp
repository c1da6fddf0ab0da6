// compile.cpp -- host-side material compiler (Sec. 2 and Sec. 3).
//
//  1. validate the network;
//  2. dependence classes CONST < UV < SP and the cacheable nodes ("roots"): reachable
//     UV-class nodes, other than the bare UV input, that are the output or feed an
//     SP-class node, with at least min_root_nodes non-input nodes below them -- the
//     highest level at which the sub-graph depends on nothing but UV (Sec. 3).  With the
//     world-position descriptor the position is a class of its own (POS): a node joining
//     UV and POS inputs is SP, and POS-class nodes become roots by the same rule, looked
//     up under a voxel of the position instead of a texel;
//  3. constant folding of simple arithmetic on constants (Sec. 2);
//  4. for every other node, the set of roots through which all its uses pass: a node
//     used only under root r is skipped whenever r hits; such nodes and r form r's block;
//  5. emission in depth-first post-order over blocks and single nodes, each block
//     contiguous and ending with its root;
//  6. linear-scan slot allocation and encoding into 16-byte instructions.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>

#include "pmc_internal.h"

namespace pmc {
namespace {

enum { CLS_CONST = 0, CLS_UV = 1, CLS_SP = 2, CLS_POS = 3 };

// Class of a node with inputs of classes a and b: constants change nothing; two different
// shading-point dependences make it SP.
int join_class(int a, int b) {
    if (a == b || b == CLS_CONST) return a;
    if (a == CLS_CONST) return b;
    return CLS_SP;
}
constexpr uint32_t NO_SLOT = 0xFFFFu;

int required_inputs(uint32_t op, int* optional) {
    *optional = 0;
    switch (op) {
    case PMC_OP_UV: case PMC_OP_POSITION: case PMC_OP_NORMAL: case PMC_OP_CONST: return 0;
    case PMC_OP_UV_AFFINE: case PMC_OP_FBM: case PMC_OP_VORONOI: case PMC_OP_CHECKER:
    case PMC_OP_RAMP: case PMC_OP_POW: case PMC_OP_FACING: return 1;
    case PMC_OP_MIX: *optional = 1; return 2;
    case PMC_OP_ADD: case PMC_OP_MUL: return 2;
    default: return -1;
    }
}

uint32_t float_bits(float x) {
    uint32_t b;
    std::memcpy(&b, &x, sizeof(b));
    return b;
}

// A positive power of two 2^e, -20 <= e <= 20, read off the FP32 bits (no fraction).
bool pow2_scale(float x) {
    const uint32_t b = float_bits(x);
    const uint32_t ex = b >> 23;   // includes the sign bit: a negative x never matches
    return (b & 0x7FFFFFu) == 0 && ex >= 127 - 20 && ex <= 127 + 20;
}

// The checker flips colour where x s or y s crosses an integer (the only discontinuous
// primitive).  FP32 and wider arithmetic take the same side of every edge when the
// argument is exact in FP32: x and y from the UV or position input, directly or through
// an affine map that scales each axis by a power of two (no rotation or offset), and s a
// power of two.
bool exact_checker(const pmc_node* nodes, const pmc_node& nd) {
    if (!pow2_scale(nd.fp[0])) return false;
    const pmc_node& src = nodes[nd.in[0]];
    if (src.op == PMC_OP_UV || src.op == PMC_OP_POSITION) return true;
    if (src.op != PMC_OP_UV_AFFINE) return false;
    const uint32_t in = nodes[src.in[0]].op;
    return (in == PMC_OP_UV || in == PMC_OP_POSITION) && pow2_scale(src.fp[0]) && pow2_scale(src.fp[3]) &&
           src.fp[1] == 0.0f && src.fp[2] == 0.0f && src.fp[4] == 0.0f && src.fp[5] == 0.0f;
}

bool is_input_op(uint32_t op) {
    return op == PMC_OP_UV || op == PMC_OP_POSITION || op == PMC_OP_NORMAL || op == PMC_OP_CONST;
}

bool validate(const pmc_node* nodes, uint32_t n, const char** why) {
    if (n == 0 || n > 65535u) { *why = "node count must be 1..65535"; return false; }
    for (uint32_t i = 0; i < n; ++i) {
        const pmc_node& nd = nodes[i];
        int opt;
        int req = required_inputs(nd.op, &opt);
        if (req < 0) { *why = "unknown operator"; return false; }
        for (int k = 0; k < 4; ++k) {
            int32_t x = nd.in[k];
            if (k < req) {
                if (x < 0 || (uint32_t)x >= i) { *why = "missing or forward input"; return false; }
            } else if (k < req + opt) {
                if (x < -1 || (x >= 0 && (uint32_t)x >= i)) { *why = "forward input"; return false; }
            } else if (x != -1) {
                *why = "unused input slot must be -1";
                return false;
            }
        }
        if (nd.op == PMC_OP_FBM && (nd.ip[0] < 1 || nd.ip[0] > 16)) { *why = "octaves 1..16"; return false; }
        if (nd.op == PMC_OP_RAMP) {
            int ns = nd.ip[0];
            if (ns < 2 || ns > 4) { *why = "ramp stops 2..4"; return false; }
            for (int k = 0; k < ns; ++k) {
                if (!(nd.fp[k] >= 0.0f && nd.fp[k] <= 1.0f)) { *why = "ramp stop outside [0,1]"; return false; }
                if (k > 0 && nd.fp[k] < nd.fp[k - 1]) { *why = "ramp stops out of order"; return false; }
            }
        }
        if (nd.op == PMC_OP_POW && !(nd.fp[0] > 0.0f)) { *why = "exponent must be > 0"; return false; }
        if (nd.op == PMC_OP_CHECKER && !exact_checker(nodes, nd)) {
            *why = "a checker's argument must be exact in FP32: UV or position, directly or scaled per "
                   "axis by powers of two, times a power-of-two scale in [2^-20, 2^20]";
            return false;
        }
    }
    return true;
}

double clamp01d(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

// Folds ADD/MUL/MIX/POW whose inputs are all constants (Sec. 2: "pre-computing simple
// arithmetic nodes with constant inputs").  Arithmetic in double, rounded once to float.
bool fold(const pmc_node& nd, const std::vector<pmc_node>& g, pmc_node* out) {
    auto is_const = [&](int32_t x) { return x >= 0 && g[x].op == PMC_OP_CONST; };
    double r[3];
    switch (nd.op) {
    case PMC_OP_ADD: case PMC_OP_MUL:
        if (!is_const(nd.in[0]) || !is_const(nd.in[1])) return false;
        for (int i = 0; i < 3; ++i) {
            double a = g[nd.in[0]].fp[i], b = g[nd.in[1]].fp[i];
            r[i] = clamp01d(nd.op == PMC_OP_ADD ? a + b : a * b);
        }
        break;
    case PMC_OP_MIX: {
        if (!is_const(nd.in[0]) || !is_const(nd.in[1])) return false;
        if (nd.in[2] >= 0 && !is_const(nd.in[2])) return false;
        double f = clamp01d(nd.in[2] >= 0 ? (double)g[nd.in[2]].fp[0] : (double)nd.fp[0]);
        for (int i = 0; i < 3; ++i) {
            double a = g[nd.in[0]].fp[i], b = g[nd.in[1]].fp[i];
            r[i] = clamp01d(a + (b - a) * f);
        }
        break;
    }
    case PMC_OP_POW:
        if (!is_const(nd.in[0])) return false;
        for (int i = 0; i < 3; ++i) {
            double a = g[nd.in[0]].fp[i];
            r[i] = clamp01d(std::pow(a > 0.0 ? a : 0.0, (double)nd.fp[0]));
        }
        break;
    default:
        return false;
    }
    std::memset(out, 0, sizeof(*out));
    out->op = PMC_OP_CONST;
    for (int k = 0; k < 4; ++k) out->in[k] = -1;
    for (int i = 0; i < 3; ++i) out->fp[i] = (float)r[i];
    return true;
}

// Appends a node's parameters to the pool.  Every node's parameters start on a 16-byte
// boundary so that an interpreter can fetch the first eight with two vector loads.
void pack_params(const pmc_node& nd, std::vector<float>* pool) {
    auto bits = [](int32_t x) { float f; std::memcpy(&f, &x, 4); return f; };
    const float* p = nd.fp;
    switch (nd.op) {
    case PMC_OP_CONST: case PMC_OP_FACING:
        pool->insert(pool->end(), {p[0], p[1], p[2]});
        break;
    case PMC_OP_UV_AFFINE:
        pool->insert(pool->end(), {p[0], p[1], p[2], p[3], p[4], p[5]});
        break;
    case PMC_OP_FBM: {
        double norm = 0.0, amp = 1.0;
        for (int k = 0; k < nd.ip[0]; ++k) { norm += amp; amp *= (double)p[2]; }
        pool->insert(pool->end(), {p[0], p[1], p[2], (float)(1.0 / norm), bits(nd.ip[0]), bits(nd.ip[1])});
        break;
    }
    case PMC_OP_VORONOI:
        pool->insert(pool->end(), {p[0], bits(nd.ip[1])});
        break;
    case PMC_OP_CHECKER:
        pool->insert(pool->end(), {p[0], p[1], p[2], p[3], p[4], p[5], p[6]});
        break;
    case PMC_OP_RAMP: {
        // {first stop, last stop, second stop, third stop} (an absent interior stop reads 2,
        // above every clamped input), then (stop k, 1 / (stop k+1 - stop k)) of segments 0..2,
        // two floats of padding, the colours of stops 0..3 and of the last stop, each padded
        // to four floats; 32 floats, so every group is one aligned vector load
        const int ns = nd.ip[0];
        float q[32] = {};
        q[0] = p[0];
        q[1] = p[ns - 1];
        q[2] = ns > 2 ? p[1] : 2.0f;
        q[3] = ns > 3 ? p[2] : 2.0f;
        for (int k = 0; k + 1 < ns; ++k) {
            const double len = (double)p[k + 1] - (double)p[k];
            q[4 + 2 * k] = p[k];
            // an empty segment is never selected (no t lies in it); a tiny one saturates
            q[5 + 2 * k] = len > 0.0 ? (float)std::min(1.0 / len, 3.0e38) : 0.0f;
        }
        for (int k = 0; k < ns; ++k)
            for (int c = 0; c < 3; ++c) q[12 + 4 * k + c] = p[4 + 3 * k + c];
        for (int c = 0; c < 3; ++c) q[28 + c] = p[4 + 3 * (ns - 1) + c];
        pool->insert(pool->end(), q, q + 32);
        break;
    }
    case PMC_OP_MIX: case PMC_OP_POW:
        pool->push_back(p[0]);
        break;
    default:
        break;
    }
}


// Emits a linear program for `order` (nodes in topological order; entries flagged as
// loads take a cacheable node's value from its probe record instead of evaluating it)
// with linear-scan slot allocation.  `keep` is the node whose value must survive to the
// end.  Returns the number of slots; *out_slot receives keep's slot.
uint32_t emit_standalone(const std::vector<pmc_node>& g, const std::vector<std::pair<uint32_t, bool>>& order,
                         const std::vector<uint32_t>& ordinal, uint32_t keep, bool keep_is_root,
                         std::vector<uint4>* prog, std::vector<float>* params, uint32_t* out_slot) {
    const size_t L = order.size();
    std::vector<int64_t> last_use(g.size(), -1);
    std::vector<char> in_order(g.size(), 0);
    for (auto& e : order) in_order[e.first] = 1;
    for (size_t p = 0; p < L; ++p) {
        if (order[p].second) continue;  // loads read nothing
        uint32_t x = order[p].first;
        for (int k = 0; k < 4; ++k) {
            int32_t y = g[x].in[k];
            if (y >= 0) last_use[y] = std::max<int64_t>(last_use[y], (int64_t)p);
        }
    }
    last_use[keep] = (int64_t)L;
    std::vector<std::vector<uint32_t>> release_at(L + 1);
    for (uint32_t x = 0; x < g.size(); ++x)
        if (in_order[x] && last_use[x] >= 0 && last_use[x] < (int64_t)L) release_at[last_use[x]].push_back(x);
    std::vector<uint32_t> slot(g.size(), 0xFFFFu), free_slots;
    uint32_t n_slots = 0;
    auto take = [&]() {
        if (free_slots.empty()) return n_slots++;
        auto it = std::min_element(free_slots.begin(), free_slots.end());
        uint32_t s2 = *it;
        free_slots.erase(it);
        return s2;
    };
    for (size_t p = 0; p < L; ++p) {
        uint32_t x = order[p].first;
        uint4 ins;
        if (order[p].second) {
            for (uint32_t y : release_at[p]) free_slots.push_back(slot[y]);
            slot[x] = take();
            ins.x = OP_LOAD_ROOT;
            ins.y = slot[x] | (ordinal[x] << 16);
            ins.z = x;
            ins.w = 0;
            prog->push_back(ins);
            continue;
        }
        uint32_t in_slot[3] = {0xFFFFu, 0xFFFFu, 0xFFFFu};
        for (int k = 0; k < 3; ++k)
            if (g[x].in[k] >= 0) in_slot[k] = slot[g[x].in[k]];
        for (uint32_t y : release_at[p]) free_slots.push_back(slot[y]);
        slot[x] = take();
        const uint32_t flags = (x == keep && keep_is_root) ? FLAG_ROOT : 0u;
        const uint32_t cost = std::min<uint32_t>(node_cost(g[x]), 0xFFFFu);
        ins.x = g[x].op | (flags << 8) | (cost << 16);
        ins.y = slot[x] | (in_slot[0] << 16);
        ins.z = in_slot[1] | (in_slot[2] << 16);
        params->resize((params->size() + 3) & ~size_t(3), 0.0f);
        ins.w = (uint32_t)params->size();
        pack_params(g[x], params);
        prog->push_back(ins);
    }
    *out_slot = slot[keep];
    return n_slots;
}

}  // namespace

// FP32 operations per node, counted from the device formulas in kernels.cu with a
// fused multiply-add as 2: the figure the FP32 roofline of the evaluator uses.
uint32_t node_cost(const pmc_node& nd) {
    switch (nd.op) {
    case PMC_OP_UV: case PMC_OP_POSITION: case PMC_OP_NORMAL: case PMC_OP_CONST: return 0;
    case PMC_OP_UV_AFFINE: return 8;                      // 4 FMA
    // per octave: 2 mul (coordinates), noise 41 (2 floor, 4 sub, 4 x (mul + fma),
    // 2 fades of 2 fma + 3 mul, 3 lerps of sub + fma), 1 fma, 2 mul; then fma + clamp
    case PMC_OP_FBM: return 4 + 47 * (uint32_t)nd.ip[0];
    // 2 mul, 2 floor, 2 sub; per cell of 9: 2 fma + 2 sub + mul + fma + min = 10; sqrt, clamp
    case PMC_OP_VORONOI: return 6 + 9 * 10 + 3;
    case PMC_OP_CHECKER: return 4;                        // 2 mul, 2 floor
    case PMC_OP_RAMP: return 23;                          // clamp, compares, 2 sub, div, 3 lerps, 3 clamps
    case PMC_OP_MIX: return 17;                           // clamp f, 3 lerps (sub + fma), 3 clamps
    case PMC_OP_ADD: case PMC_OP_MUL: return 9;           // 3 ops + 3 clamps (2 each)
    case PMC_OP_POW: return 3 * 6;                        // max, pow (counted as log2/mul/exp2), clamp
    case PMC_OP_FACING: return 8;                         // dot (mul + 2 fma), abs, clamp
    default: return 0;
    }
}

bool compile_material(const pmc_node* nodes_in, uint32_t n, uint32_t min_root_nodes, uint32_t min_root_cost,
                      bool pos_desc, CompiledMaterial* out, const char** why) {
    if (!validate(nodes_in, n, why)) return false;
    std::vector<pmc_node> g(nodes_in, nodes_in + n);
    const uint32_t out_node = n - 1;

    // ---- reachability and classes on the network as given --------------------------
    std::vector<char> reach(n, 0);
    reach[out_node] = 1;
    for (int32_t i = (int32_t)n - 1; i >= 0; --i)
        if (reach[i])
            for (int k = 0; k < 4; ++k)
                if (g[i].in[k] >= 0) reach[g[i].in[k]] = 1;
    std::vector<int> cls(n);
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t op = g[i].op;
        if (op == PMC_OP_UV) cls[i] = CLS_UV;
        else if (op == PMC_OP_POSITION) cls[i] = pos_desc ? CLS_POS : CLS_SP;
        else if (op == PMC_OP_NORMAL) cls[i] = CLS_SP;
        else if (op == PMC_OP_CONST) cls[i] = CLS_CONST;
        else {
            int c = CLS_CONST;
            for (int k = 0; k < 4; ++k)
                if (g[i].in[k] >= 0) c = join_class(c, cls[g[i].in[k]]);
            cls[i] = c;
        }
    }
    std::vector<char> feeds_sp(n, 0);
    for (uint32_t i = 0; i < n; ++i)
        if (reach[i] && cls[i] == CLS_SP)
            for (int k = 0; k < 4; ++k)
                if (g[i].in[k] >= 0) feeds_sp[g[i].in[k]] = 1;

    // ---- cacheable nodes -------------------------------------------------------------
    std::vector<char> is_root(n, 0);
    std::vector<char> mark(n);
    for (uint32_t i = 0; i < n; ++i) {
        if (!reach[i] || (cls[i] != CLS_UV && cls[i] != CLS_POS)) continue;
        if (g[i].op == PMC_OP_UV || g[i].op == PMC_OP_POSITION) continue;
        if (!(i == out_node || feeds_sp[i])) continue;
        std::fill(mark.begin(), mark.end(), 0);
        mark[i] = 1;
        uint32_t work = 0;
        uint64_t cost = 0;   // what a hit saves at most: the FP32 operations of the sub-graph
        for (int32_t j = (int32_t)i; j >= 0; --j) {
            if (!mark[j]) continue;
            if (!is_input_op(g[j].op)) ++work;
            cost += node_cost(g[j]);
            for (int k = 0; k < 4; ++k)
                if (g[j].in[k] >= 0) mark[g[j].in[k]] = 1;
        }
        if (work >= min_root_nodes && cost >= min_root_cost) is_root[i] = 1;
    }
    out->roots.clear();
    out->root_pos.clear();
    for (uint32_t i = 0; i < n; ++i)
        if (is_root[i]) {
            out->roots.push_back(i);
            out->root_pos.push_back(cls[i] == CLS_POS ? 1 : 0);
        }
    std::vector<uint32_t> ordinal(n, 0);
    for (uint32_t r = 0; r < out->roots.size(); ++r) ordinal[out->roots[r]] = r;

    // ---- constant folding (roots are never CONST-class, so keys do not change) --------
    for (uint32_t i = 0; i < n; ++i) {
        if (!reach[i] || cls[i] != CLS_CONST) continue;
        pmc_node f;
        if (fold(g[i], g, &f)) g[i] = f;
    }
    // reachability again on the folded network
    std::fill(reach.begin(), reach.end(), 0);
    reach[out_node] = 1;
    for (int32_t i = (int32_t)n - 1; i >= 0; --i)
        if (reach[i])
            for (int k = 0; k < 4; ++k)
                if (g[i].in[k] >= 0) reach[g[i].in[k]] = 1;
    std::vector<std::vector<uint32_t>> consumers(n);
    for (uint32_t i = 0; i < n; ++i)
        if (reach[i])
            for (int k = 0; k < 4; ++k)
                if (g[i].in[k] >= 0) consumers[g[i].in[k]].push_back(i);

    // ---- skip sets: -1 = always evaluate, r = skipped whenever root r hits -----------
    const int32_t NEVER = -1;
    std::vector<int32_t> guard(n, NEVER);
    for (int32_t i = (int32_t)n - 1; i >= 0; --i) {
        if (!reach[i] || (uint32_t)i == out_node) continue;
        int32_t gset = -2;  // -2 = nothing seen yet
        for (uint32_t c : consumers[i]) {
            int32_t contrib = is_root[c] ? (int32_t)c : guard[c];
            if (contrib == NEVER) { gset = NEVER; break; }
            if (gset == -2) gset = contrib;
            else if (gset != contrib) { gset = NEVER; break; }  // shared by two roots
        }
        guard[i] = (gset == -2) ? NEVER : gset;
    }
    // block id of each node: the root whose block it belongs to, or -1
    std::vector<int32_t> block(n, -1);
    for (uint32_t i = 0; i < n; ++i) {
        if (!reach[i]) continue;
        if (is_root[i]) block[i] = (int32_t)i;
        else if (guard[i] >= 0) block[i] = guard[i];
    }
    auto unit_of = [&](uint32_t x) -> uint32_t { return block[x] >= 0 ? (uint32_t)block[x] : x; };

    // members of each block in post-order (iterative DFS inside the block)
    std::vector<std::vector<uint32_t>> members(n);
    for (uint32_t r : out->roots) {
        if (!reach[r]) continue;
        std::vector<std::pair<uint32_t, int>> st{{r, 0}};
        std::vector<uint32_t>& mem = members[r];
        std::vector<char> vis(n, 0);
        vis[r] = 1;
        while (!st.empty()) {
            auto& [x, k] = st.back();
            if (k < 4) {
                int32_t y = g[x].in[k++];
                if (y >= 0 && block[y] == (int32_t)r && !is_root[y] && !vis[y]) {
                    vis[y] = 1;
                    st.push_back({(uint32_t)y, 0});
                }
                continue;
            }
            mem.push_back(x);
            st.pop_back();
        }
    }
    // inputs of each unit, in the order its members read them
    auto unit_inputs = [&](uint32_t u, std::vector<uint32_t>* ins) {
        ins->clear();
        if (is_root[u]) {
            for (uint32_t x : members[u])
                for (int k = 0; k < 4; ++k) {
                    int32_t y = g[x].in[k];
                    if (y >= 0 && unit_of(y) != u) ins->push_back(unit_of(y));
                }
        } else {
            for (int k = 0; k < 4; ++k) {
                int32_t y = g[u].in[k];
                if (y >= 0) ins->push_back(unit_of(y));
            }
        }
    };

    // ---- emission order: post-order DFS over units from the output ---------------------
    struct Entry { uint32_t node; bool begin; };
    std::vector<Entry> order;
    {
        std::vector<char> vis(n, 0);
        std::vector<std::pair<uint32_t, size_t>> st;
        std::vector<std::vector<uint32_t>> ins_cache(n);
        uint32_t top = unit_of(out_node);
        vis[top] = 1;
        unit_inputs(top, &ins_cache[top]);
        st.push_back({top, 0});
        while (!st.empty()) {
            uint32_t u = st.back().first;
            size_t& k = st.back().second;
            if (k < ins_cache[u].size()) {
                uint32_t v = ins_cache[u][k++];
                if (!vis[v]) {
                    vis[v] = 1;
                    unit_inputs(v, &ins_cache[v]);
                    st.push_back({v, 0});
                }
                continue;
            }
            if (is_root[u]) {
                order.push_back({u, true});
                for (uint32_t x : members[u]) order.push_back({x, false});
            } else {
                order.push_back({u, false});
            }
            st.pop_back();
        }
    }

    // ---- linear-scan slot allocation -----------------------------------------------
    const size_t L = order.size();
    std::vector<int64_t> pos(n, -1), begin_pos(n, -1), last_use(n, -1);
    for (size_t p = 0; p < L; ++p) {
        if (order[p].begin) begin_pos[order[p].node] = (int64_t)p;
        else pos[order[p].node] = (int64_t)p;
    }
    for (size_t p = 0; p < L; ++p) {
        if (order[p].begin) continue;
        uint32_t x = order[p].node;
        for (int k = 0; k < 4; ++k) {
            int32_t y = g[x].in[k];
            if (y >= 0) last_use[y] = std::max<int64_t>(last_use[y], (int64_t)p);
        }
    }
    last_use[out_node] = (int64_t)L;  // the output stays live to the end
    std::vector<uint32_t> slot(n, NO_SLOT);
    std::vector<uint32_t> free_slots;
    uint32_t n_slots = 0;
    std::vector<std::vector<uint32_t>> release_at(L + 1);
    for (uint32_t x = 0; x < n; ++x)
        if (last_use[x] >= 0 && last_use[x] < (int64_t)L) release_at[last_use[x]].push_back(x);
    auto take = [&]() {
        if (free_slots.empty()) return n_slots++;
        auto it = std::min_element(free_slots.begin(), free_slots.end());
        uint32_t s = *it;
        free_slots.erase(it);
        return s;
    };

    out->prog.clear();
    out->params.clear();
    for (size_t p = 0; p < L; ++p) {
        const Entry& e = order[p];
        uint32_t x = e.node;
        if (e.begin) {
            slot[x] = take();
            uint4 ins;
            uint32_t skip = (uint32_t)members[x].size();  // exclusive nodes + the root itself
            ins.x = OP_ROOT_BEGIN | ((cls[x] == CLS_POS ? FLAG_POSROOT : 0u) << 8);
            ins.y = slot[x] | (ordinal[x] << 16);
            ins.z = x;
            ins.w = skip;
            out->prog.push_back(ins);
            continue;
        }
        // inputs whose last use is here are released before the output is placed
        uint32_t in_slot[3] = {NO_SLOT, NO_SLOT, NO_SLOT};
        for (int k = 0; k < 3; ++k)
            if (g[x].in[k] >= 0) in_slot[k] = slot[g[x].in[k]];
        for (uint32_t y : release_at[p]) free_slots.push_back(slot[y]);
        if (!is_root[x]) slot[x] = take();
        uint4 ins;
        uint32_t flags = is_root[x] ? FLAG_ROOT : 0;
        uint32_t cost = std::min<uint32_t>(node_cost(g[x]), 0xFFFFu);
        ins.x = g[x].op | (flags << 8) | (cost << 16);
        ins.y = slot[x] | (in_slot[0] << 16);
        ins.z = in_slot[1] | (in_slot[2] << 16);
        out->params.resize((out->params.size() + 3) & ~size_t(3), 0.0f);
        ins.w = (uint32_t)out->params.size();
        pack_params(g[x], &out->params);
        out->prog.push_back(ins);
    }
    if (n_slots >= NO_SLOT) { *why = "too many live values"; return false; }
    out->out_slot = slot[out_node];
    out->n_slots = n_slots;
    out->n_nodes = n;

    // ---- standalone program of each cacheable node ------------------------------------
    // its sub-graph in post-order, stopping at other cacheable nodes (read as loads)
    out->root_progs.assign(out->roots.size(), {});
    out->root_level.assign(out->roots.size(), 0);
    out->root_slots.assign(out->roots.size(), 0);
    out->root_out_slot.assign(out->roots.size(), 0);
    std::vector<uint32_t> level_of(n, 0);
    for (size_t ri = 0; ri < out->roots.size(); ++ri) {
        const uint32_t r = out->roots[ri];
        std::vector<std::pair<uint32_t, bool>> order_r;
        std::vector<char> vis(n, 0);
        std::vector<std::pair<uint32_t, int>> st{{r, 0}};
        vis[r] = 1;
        uint32_t lvl = 0;
        while (!st.empty()) {
            auto& [x, k] = st.back();
            if (x != r && is_root[x]) {          // another cacheable node: load its value
                order_r.push_back({x, true});
                lvl = std::max(lvl, level_of[x] + 1);
                st.pop_back();
                continue;
            }
            if (k < 4) {
                int32_t y = g[x].in[k++];
                if (y >= 0 && !vis[y]) {
                    vis[y] = 1;
                    st.push_back({(uint32_t)y, 0});
                }
                continue;
            }
            order_r.push_back({x, false});
            st.pop_back();
        }
        level_of[r] = lvl;
        out->root_level[ri] = lvl;
        uint32_t os = 0;
        out->root_slots[ri] = emit_standalone(g, order_r, ordinal, r, true, &out->root_progs[ri],
                                              &out->params, &os);
        out->root_out_slot[ri] = os;
        if (out->root_slots[ri] >= NO_SLOT) { *why = "too many live values"; return false; }
    }

    // ---- outer program: the per-point program with every block replaced by a load of
    // its cacheable node's value (used when all of them have values before evaluation)
    {
        std::vector<std::pair<uint32_t, bool>> order_o;
        for (size_t p = 0; p < order.size(); ++p) {
            if (order[p].begin) {
                order_o.push_back({order[p].node, true});
                p += members[order[p].node].size();   // the block: exclusive nodes + the node
                continue;
            }
            order_o.push_back({order[p].node, false});
        }
        // drop what only blocks consumed (every load stays: it also counts the node's hit)
        std::vector<char> need(n, 0);
        need[out_node] = 1;
        for (size_t p = order_o.size(); p-- > 0;) {
            if (order_o[p].second || !need[order_o[p].first]) continue;
            for (int k = 0; k < 4; ++k)
                if (g[order_o[p].first].in[k] >= 0) need[g[order_o[p].first].in[k]] = 1;
        }
        std::vector<std::pair<uint32_t, bool>> kept;
        for (auto& e : order_o)
            if (need[e.first] || e.second) kept.push_back(e);
        uint32_t os = 0;
        out->outer_slots = emit_standalone(g, kept, ordinal, out_node, false, &out->outer_prog, &out->params, &os);
        out->outer_out_slot = os;
        if (out->outer_slots >= NO_SLOT) { *why = "too many live values"; return false; }
    }
    return true;
}

}  // namespace pmc
