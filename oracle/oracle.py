"""ctypes wrapper of the CPU FP64 oracle (pmc_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may use it; the CUDA path never does.  It imports nothing from
the CUDA side except the seeded input generator's IR layout.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from paper_2305_07238_gb300.workload import CONE_FIELDS, NODE_DTYPE, POINT_FIELDS

from .build import build_oracle

_lib = None

NSTATS = 10
STAT_NAMES = ("lookups", "hits", "misses", "candidates", "inserted", "dropped_dup",
              "dropped_full", "nodes_evaluated", "batches", "replaced")

HASH_HOOK = C.CFUNCTYPE(None, C.c_uint64, C.c_uint64, C.POINTER(C.c_uint64),
                        C.POINTER(C.c_uint32))


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = C.CDLL(path)
        u32, u64, i64, f64, vp = C.c_uint32, C.c_uint64, C.c_int64, C.c_double, C.c_void_p
        L.orc_fmix32.restype = u32
        L.orc_fmix32.argtypes = [u32]
        L.orc_fmix64.restype = u64
        L.orc_fmix64.argtypes = [u64]
        L.orc_splitmix64_mix.restype = u64
        L.orc_splitmix64_mix.argtypes = [u64]
        L.orc_lattice_hash.restype = u32
        L.orc_lattice_hash.argtypes = [i64, i64, u32]
        L.orc_fade.restype = f64
        L.orc_fade.argtypes = [f64]
        L.orc_perlin.restype = f64
        L.orc_perlin.argtypes = [f64, f64, u32]
        L.orc_fbm.restype = f64
        L.orc_fbm.argtypes = [f64, f64, f64, C.c_int, f64, f64, u32]
        L.orc_voronoi_f1.restype = f64
        L.orc_voronoi_f1.argtypes = [f64, f64, u32]
        L.orc_eval_node.restype = None
        L.orc_eval_node.argtypes = [vp, vp, vp, vp, vp, vp]
        L.orc_texel.restype = u32
        L.orc_texel.argtypes = [C.c_float, u32]
        L.orc_key.restype = u64
        L.orc_key.argtypes = [u32, u32, u32, C.c_float, C.c_float]
        L.orc_hash1.restype = u64
        L.orc_hash1.argtypes = [u64]
        L.orc_hash2.restype = u32
        L.orc_hash2.argtypes = [u64]
        L.orc_address_batch.restype = None
        L.orc_address_batch.argtypes = [vp, vp, vp, vp, u64, u32, u64, vp, vp, vp]
        L.orc_mix_batch.restype = None
        L.orc_mix_batch.argtypes = [vp, u64, vp, vp]
        L.orc_validate.restype = C.c_int
        L.orc_validate.argtypes = [vp, u32]
        L.orc_analyze.restype = C.c_int
        L.orc_analyze.argtypes = [vp, u32, u32, vp, vp, vp]
        L.orc_analyze_desc.restype = C.c_int
        L.orc_analyze_desc.argtypes = [vp, u32, u32, C.c_int, vp, vp, vp]
        L.orc_analyze_cost.restype = C.c_int
        L.orc_analyze_cost.argtypes = [vp, u32, u32, u32, C.c_int, vp, vp, vp]
        L.orc_node_cost.restype = u32
        L.orc_node_cost.argtypes = [vp]
        L.orc_cache_set_min_root_cost.restype = None
        L.orc_cache_set_min_root_cost.argtypes = [vp, u32]
        L.orc_cache_set_threads.restype = None
        L.orc_cache_set_threads.argtypes = [vp, C.c_int]
        L.orc_voxel.restype = u32
        L.orc_voxel.argtypes = [C.c_float, u32]
        L.orc_key_pos.restype = u64
        L.orc_key_pos.argtypes = [u32, u32, u32, C.c_float, C.c_float, C.c_float]
        L.orc_cache_set_position_level.restype = None
        L.orc_cache_set_position_level.argtypes = [vp, C.c_int32]
        L.orc_eval_point_nocache.restype = C.c_int
        L.orc_eval_point_nocache.argtypes = [vp, u32, vp, vp]
        L.orc_cache_new.restype = vp
        L.orc_cache_new.argtypes = [u64, u32, u32, u32, C.c_int]
        L.orc_cache_free.restype = None
        L.orc_cache_free.argtypes = [vp]
        L.orc_cache_set_materials.restype = C.c_int
        L.orc_cache_set_materials.argtypes = [vp, u32, vp, vp]
        L.orc_cache_set_hash_override.restype = None
        L.orc_cache_set_hash_override.argtypes = [vp, HASH_HOOK]
        L.orc_cache_reset.restype = None
        L.orc_cache_reset.argtypes = [vp]
        L.orc_cache_n_roots.restype = u32
        L.orc_cache_n_roots.argtypes = [vp, u32]
        L.orc_cache_roots.restype = None
        L.orc_cache_roots.argtypes = [vp, u32, vp]
        L.orc_run_batch.restype = C.c_int
        L.orc_run_batch.argtypes = [vp, u64] + [vp] * 9 + [vp] * 7 + [vp] * 4 + [vp]
        L.orc_level.restype = C.c_int32
        L.orc_level.argtypes = [C.c_float] * 4 + [C.c_int32]
        L.orc_cache_set_level_offset.restype = None
        L.orc_cache_set_level_offset.argtypes = [vp, C.c_int32]
        L.orc_cache_set_alg1.restype = None
        L.orc_cache_set_alg1.argtypes = [vp, C.c_int]
        L.orc_cache_set_replacement.restype = None
        L.orc_cache_set_replacement.argtypes = [vp, C.c_int]
        L.orc_cache_set_close_at_lookup.restype = None
        L.orc_cache_set_close_at_lookup.argtypes = [vp, C.c_int]
        L.orc_cache_classes.restype = None
        L.orc_cache_classes.argtypes = [vp, vp]
        L.orc_rgb9e5_encode.restype = u32
        L.orc_rgb9e5_encode.argtypes = [C.c_float] * 3
        L.orc_rgb9e5_decode.restype = None
        L.orc_rgb9e5_decode.argtypes = [u32, vp]
        L.orc_cache_table.restype = None
        L.orc_cache_table.argtypes = [vp, vp, vp]
        L.orc_cache_stats.restype = None
        L.orc_cache_stats.argtypes = [vp, vp]
        L.orc_mlp_forward.restype = None
        L.orc_mlp_forward.argtypes = [vp, f64, f64, C.c_int, vp]
        L.orc_cache_set_surrogate.restype = C.c_int
        L.orc_cache_set_surrogate.argtypes = [vp, u32, u32, vp, C.c_int]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _nodes(nodes) -> np.ndarray:
    arr = np.ascontiguousarray(nodes, dtype=NODE_DTYPE)
    return arr


# ---- primitives ----------------------------------------------------------------------
def fmix32(h): return lib().orc_fmix32(h)
def fmix64(k): return lib().orc_fmix64(k)
def splitmix64_mix(z): return lib().orc_splitmix64_mix(z)
def lattice_hash(i, j, seed): return lib().orc_lattice_hash(i, j, seed)
def fade(t): return lib().orc_fade(t)
def perlin(x, y, seed): return lib().orc_perlin(x, y, seed)
def fbm(x, y, scale, octaves, lac, gain, seed): return lib().orc_fbm(x, y, scale, octaves, lac, gain, seed)
def voronoi_f1(x, y, seed): return lib().orc_voronoi_f1(x, y, seed)
def texel(u, level): return lib().orc_texel(u, level)
def key(mat, node, level, u, v): return lib().orc_key(mat, node, level, u, v)
def voxel(p, level): return lib().orc_voxel(p, level)
def key_pos(mat, node, level, px, py, pz): return lib().orc_key_pos(mat, node, level, px, py, pz)
def level(g1u, g1v, g2u, g2v, offset=0): return lib().orc_level(g1u, g1v, g2u, g2v, offset)
def rgb9e5_encode(r, g, b): return lib().orc_rgb9e5_encode(r, g, b)


def rgb9e5_decode(code):
    out = np.zeros(3, dtype=np.float32)
    lib().orc_rgb9e5_decode(code, _ptr(out))
    return out
def hash1(k): return lib().orc_hash1(k)
def hash2(k): return lib().orc_hash2(k)


def address_batch(mat, node, u, v, level, n_cells):
    """(key uint64[n], cell uint64[n], h2 uint32[n]) of n (material, node, u, v) tuples."""
    mat = np.ascontiguousarray(mat, dtype=np.uint32)
    node = np.ascontiguousarray(node, dtype=np.uint32)
    u = np.ascontiguousarray(u, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32)
    n = len(mat)
    key = np.zeros(max(n, 1), dtype=np.uint64)
    cell = np.zeros(max(n, 1), dtype=np.uint64)
    h2 = np.zeros(max(n, 1), dtype=np.uint32)
    lib().orc_address_batch(_ptr(mat), _ptr(node), _ptr(u), _ptr(v), n, level, n_cells,
                            _ptr(key), _ptr(cell), _ptr(h2))
    return key[:n], cell[:n], h2[:n]


def mix_batch(keys):
    """(SplitMix64 output function, fmix64 of key xor 0x9E3779B97F4A7C15) of n keys."""
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    h1 = np.zeros(max(len(k), 1), dtype=np.uint64)
    m2 = np.zeros(max(len(k), 1), dtype=np.uint64)
    lib().orc_mix_batch(_ptr(k), len(k), _ptr(h1), _ptr(m2))
    return h1[: len(k)], m2[: len(k)]


def eval_node(node_row, a=None, b=None, c=None, sp=(0.0,) * 8):
    """Evaluates one node (a structured NODE_DTYPE scalar/array of length 1)."""
    nd = np.ascontiguousarray(np.atleast_1d(node_row), dtype=NODE_DTYPE)
    def vec(x):
        return None if x is None else np.ascontiguousarray(x, dtype=np.float64)
    av, bv, cv = vec(a), vec(b), vec(c)
    spv = np.ascontiguousarray(sp, dtype=np.float64)
    out = np.zeros(3, dtype=np.float64)
    lib().orc_eval_node(_ptr(nd), _ptr(av), _ptr(bv), _ptr(cv), _ptr(spv), _ptr(out))
    return out


def validate(nodes) -> bool:
    arr = _nodes(nodes)
    return lib().orc_validate(_ptr(arr), len(arr)) == 0


def node_cost(node_row) -> int:
    """The node cost model: FP32 operations of one evaluation of the node."""
    nd = np.ascontiguousarray(np.atleast_1d(node_row), dtype=NODE_DTYPE)
    return int(lib().orc_node_cost(_ptr(nd)))


def analyze(nodes, min_root_nodes=2, pos_desc=False, kinds=False, min_root_cost=0):
    """Returns (classes int32[n], root node IDs) and, if kinds, the descriptor kind of each
    root (1 = UV, 2 = world position)."""
    arr = _nodes(nodes)
    n = len(arr)
    cls = np.zeros(n, dtype=np.int32)
    is_root = np.zeros(n, dtype=np.uint8)
    nr = np.zeros(1, dtype=np.uint32)
    rc = lib().orc_analyze_cost(_ptr(arr), n, min_root_nodes, min_root_cost, int(pos_desc), _ptr(cls),
                                _ptr(is_root), _ptr(nr))
    if rc != 0:
        raise ValueError("malformed network")
    roots = np.nonzero(is_root)[0].astype(np.uint32)
    return (cls, roots, is_root[roots]) if kinds else (cls, roots)


def eval_point_nocache(nodes, sp) -> np.ndarray:
    arr = _nodes(nodes)
    spv = np.ascontiguousarray(sp, dtype=np.float64)
    out = np.zeros(3, dtype=np.float64)
    if lib().orc_eval_point_nocache(_ptr(arr), len(arr), _ptr(spv), _ptr(out)) != 0:
        raise ValueError("malformed network")
    return out


def mlp_forward(theta, u, v, bf16=False) -> np.ndarray:
    """The surrogate network in C (FP64; bf16 rounds where the kernels round): (n, 3)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    uu = np.asarray(u, dtype=np.float64)
    vv = np.asarray(v, dtype=np.float64)
    out = np.zeros((len(uu), 3))
    y = np.zeros(3)
    for i in range(len(uu)):
        lib().orc_mlp_forward(_ptr(th), float(uu[i]), float(vv[i]), int(bf16), _ptr(y))
        out[i] = y
    return out


class Cache:
    """Sequential emulation of the progressive cache over a set of materials."""

    def __init__(self, materials, n_cells, n_entries, level=10, min_root_nodes=2,
                 cache_off=False, hash_hook=None, level_offset=0, alg1=False, replacement=False,
                 pos_level=-1, close_at_lookup=True, min_root_cost=0, threads=1):
        self._mats = [_nodes(m) for m in materials]
        self.n_cells, self.n_entries, self.level = n_cells, n_entries, level
        self.off = bool(cache_off) or n_cells == 0 or n_entries == 0
        self._h = lib().orc_cache_new(n_cells, n_entries, level, min_root_nodes, int(cache_off))
        if not self._h:
            raise ValueError("bad cache description")
        lib().orc_cache_set_position_level(self._h, int(pos_level))
        lib().orc_cache_set_min_root_cost(self._h, int(min_root_cost))
        ptrs = (C.c_void_p * len(self._mats))(*[m.ctypes.data for m in self._mats])
        counts = np.array([len(m) for m in self._mats], dtype=np.uint32)
        if lib().orc_cache_set_materials(self._h, len(self._mats), ptrs, _ptr(counts)) != 0:
            raise ValueError("malformed network")
        lib().orc_cache_set_level_offset(self._h, int(level_offset))
        lib().orc_cache_set_alg1(self._h, int(alg1))
        lib().orc_cache_set_replacement(self._h, int(replacement))
        lib().orc_cache_set_close_at_lookup(self._h, int(close_at_lookup))
        lib().orc_cache_set_threads(self._h, int(threads))
        self._hook = None
        if hash_hook is not None:
            def _cb(k, nc, cell, h2):
                c_, h_ = hash_hook(k, nc)
                cell[0] = c_
                h2[0] = h_
            self._hook = HASH_HOOK(_cb)
            lib().orc_cache_set_hash_override(self._h, self._hook)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_cache_free(self._h)
            self._h = None

    def reset(self):
        lib().orc_cache_reset(self._h)

    def set_surrogate(self, mat, node, theta, bf16=True):
        th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
        self._surr = getattr(self, "_surr", {})
        self._surr[mat] = th
        if lib().orc_cache_set_surrogate(self._h, mat, node, _ptr(th), int(bf16)) != 0:
            raise ValueError("bad surrogate")

    def n_roots(self, m):
        return lib().orc_cache_n_roots(self._h, m)

    def roots(self, m):
        out = np.zeros(max(1, self.n_roots(m)), dtype=np.uint32)
        lib().orc_cache_roots(self._h, m, _ptr(out))
        return out[: self.n_roots(m)]

    def run_batch(self, pts: dict, probes: bool = False):
        """One progressive pass.  Returns a dict with rgb (3, n) float64, hits,
        evaluated, status and (if probes) key/cell/h2/hit per (point, root).  If pts holds
        the ray-cone gradients (CONE_FIELDS), each point takes its own mip level; if it holds
        "vis", that is each point's visibility class for the replacement policy."""
        arrs = [np.ascontiguousarray(pts[k], dtype=np.uint32 if k == "mat" else np.float32)
                for k in POINT_FIELDS]
        cones = [np.ascontiguousarray(pts[k], dtype=np.float32) for k in CONE_FIELDS] \
            if all(k in pts for k in CONE_FIELDS) else [None] * 4
        vis = np.ascontiguousarray(pts["vis"], dtype=np.uint8) if "vis" in pts else None
        n = len(arrs[0])
        rgb = np.zeros(3 * n, dtype=np.float64)
        hits = np.zeros(n, dtype=np.uint16)
        ev = np.zeros(n, dtype=np.uint32)
        pk = pc = ph = phit = None
        if probes:
            mat = arrs[2]
            nr = np.array([self.n_roots(m) for m in range(len(self._mats))] + [0], dtype=np.int64)
            m_idx = np.where(mat < len(self._mats), mat, len(self._mats))
            total = int(nr[m_idx].sum()) if not self.off else 0
            pk = np.zeros(max(total, 1), dtype=np.uint64)
            pc = np.zeros(max(total, 1), dtype=np.uint64)
            ph = np.zeros(max(total, 1), dtype=np.uint32)
            phit = np.zeros(max(total, 1), dtype=np.uint8)
        st = lib().orc_run_batch(self._h, n, *[_ptr(a) for a in arrs], _ptr(rgb), _ptr(hits),
                                 _ptr(ev), _ptr(pk), _ptr(pc), _ptr(ph), _ptr(phit),
                                 *[_ptr(g) for g in cones], _ptr(vis))
        out = {"rgb": rgb.reshape(3, n), "hits": hits, "evaluated": ev, "status": st}
        if probes:
            out.update(key=pk[:total], cell=pc[:total], h2=ph[:total], hit=phit[:total])
        return out

    def table(self):
        slots = 0 if self.off else self.n_cells * self.n_entries
        h2 = np.zeros(max(slots, 1), dtype=np.uint32)
        rgb = np.zeros(max(3 * slots, 1), dtype=np.float32)
        lib().orc_cache_table(self._h, _ptr(h2), _ptr(rgb))
        return h2[:slots], rgb[: 3 * slots].reshape(slots, 3)

    def classes(self):
        """Visibility class of every slot's entry (meaningful where the slot's h2 != 0)."""
        slots = 0 if self.off else self.n_cells * self.n_entries
        cls = np.zeros(max(slots, 1), dtype=np.uint8)
        lib().orc_cache_classes(self._h, _ptr(cls))
        return cls[:slots]

    def stats(self) -> dict:
        out = np.zeros(NSTATS, dtype=np.uint64)
        lib().orc_cache_stats(self._h, _ptr(out))
        return {k: int(v) for k, v in zip(STAT_NAMES, out)}
