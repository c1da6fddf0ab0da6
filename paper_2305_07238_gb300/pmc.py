"""Thin ctypes binding of libpmc.so (include/pmc.h): argument marshalling only.

Every step of the pass runs in the library's CUDA kernels.  Device buffers are torch
tensors (PyTorch supplies device memory and streams); host buffers are numpy arrays.
Loading fails loudly when the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .workload import CONE_FIELDS, NODE_DTYPE, POINT_FIELDS

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpmc.so")

PMC_OK, PMC_ERR_INVALID_ARG, PMC_ERR_OOM, PMC_ERR_CUDA, PMC_ERR_TIMEOUT, PMC_ERR_UNSUPPORTED = range(6)
PMC_CACHE_OFF = 0x1
PMC_SORT_BY_MATERIAL = 0x2
PMC_DEBUG_CHECKS = 0x4
PMC_EVAL_INLINE = 0x8
PMC_INSERT_ROUNDS = 0x10
PMC_UNSORTED = 0x20
PMC_PROBE_INLINE = 0x40
PMC_ALG1 = 0x80
PMC_REPLACE_VISIBILITY = 0x100
PMC_POSITION_DESCRIPTOR = 0x200
PMC_BLOCK_ITEMS = 0x400
PMC_ONE_POINT = 0x800
PMC_INSERT_BINNED = 0x1000
PMC_GRAPH_RESET = 0x1
TUNE_MAX = 16

EXPORTED = (
    "pmc_create_cache", "pmc_eval_batch", "pmc_eval_batch_host", "pmc_sync", "pmc_stats",
    "pmc_table_dump", "pmc_last_hit_masks", "pmc_reset", "pmc_destroy_cache",
    "pmc_material_info", "pmc_analyze_material", "pmc_compute_keys", "pmc_compute_levels", "pmc_set_timing",
    "pmc_read_timing", "pmc_eval_batch_noalloc", "pmc_train_surrogates", "pmc_set_surrogate",
    "pmc_get_surrogate", "pmc_use_surrogates", "pmc_mlp_forward", "pmc_mlp_gradient", "pmc_mlp_train",
    "pmc_get_schedule", "pmc_set_schedule", "pmc_graph_create", "pmc_graph_launch", "pmc_graph_destroy",
    "pmc_autotune", "pmc_status_str", "pmc_slot_classes", "pmc_analyze_material_ext", "pmc_cast_rays",
    "pmc_node_cost", "pmc_eval_passes_host",
)
NOALLOC_MAX_POINTS, NOALLOC_MAX_PROBES, NOALLOC_MAX_MATERIALS = 8192, 32768, 4096
PHASES = ("sort", "lookup", "missed", "eval", "insert", "finish")


class PmcError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: {status_str(status)} ({status})")
        self.status = status


class _Node(C.Structure):
    _fields_ = [("op", C.c_uint32), ("inp", C.c_int32 * 4), ("ip", C.c_int32 * 4), ("fp", C.c_float * 16)]


class _Material(C.Structure):
    _fields_ = [("n_nodes", C.c_uint32), ("nodes", C.c_void_p)]


class _Desc(C.Structure):
    _fields_ = [("n_cells", C.c_uint64), ("n_entries", C.c_uint32), ("uv_level", C.c_uint32),
                ("flags", C.c_uint32), ("min_root_nodes", C.c_uint32), ("device", C.c_int),
                ("probe_capacity", C.c_uint64), ("level_offset", C.c_int32), ("pos_level", C.c_uint32),
                ("min_root_cost", C.c_uint32)]


class _Schedule(C.Structure):
    _fields_ = [("flags", C.c_uint32), ("lookup_rb", C.c_uint32)]


class _TuneResult(C.Structure):
    _fields_ = [("n_tried", C.c_uint32), ("best", C.c_uint32), ("tried", _Schedule * TUNE_MAX),
                ("ms", C.c_float * TUNE_MAX)]


class _Points(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in POINT_FIELDS] + [("n", C.c_uint64)] + \
        [(k, C.c_void_p) for k in CONE_FIELDS] + [("vis", C.c_void_p)]


STAT_FIELDS = ("lookups", "hits", "misses", "candidates", "inserted", "dropped_dup", "dropped_full",
               "nodes_evaluated", "batches", "flops", "slots_probed", "points", "bad_points",
               "surrogate_evals", "flops_missed", "dropped_race", "replaced")
MLP_PARAMS = 8515


class _TrainDesc(C.Structure):
    _fields_ = [("n_train", C.c_uint32), ("n_valid", C.c_uint32), ("epochs", C.c_uint32), ("lr", C.c_float),
                ("rmse_max", C.c_float), ("seed", C.c_uint64), ("mats", C.c_void_p), ("n_mats", C.c_uint32)]


class _Stats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in STAT_FIELDS]


assert C.sizeof(_Node) == NODE_DTYPE.itemsize == 100

_lib = None


def load():
    """Loads libpmc.so; raises if it was not built (call __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libpmc.so is not built ({LIB_PATH}); run paper_2305_07238_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, u32, u64, st = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
    L.pmc_create_cache.argtypes = [vp, vp, u32, vp]
    L.pmc_create_cache.restype = st
    L.pmc_eval_batch.argtypes = [vp, vp, vp, vp, vp]
    L.pmc_eval_batch.restype = st
    L.pmc_eval_batch_host.argtypes = [vp, vp, vp, vp, vp]
    L.pmc_eval_batch_host.restype = st
    L.pmc_sync.argtypes = [vp]
    L.pmc_sync.restype = st
    L.pmc_stats.argtypes = [vp, vp]
    L.pmc_stats.restype = st
    L.pmc_table_dump.argtypes = [vp, vp, C.c_size_t]
    L.pmc_table_dump.restype = st
    L.pmc_slot_classes.argtypes = [vp, vp, C.c_size_t]
    L.pmc_slot_classes.restype = st
    L.pmc_last_hit_masks.argtypes = [vp, vp, u64]
    L.pmc_last_hit_masks.restype = st
    L.pmc_reset.argtypes = [vp, vp]
    L.pmc_reset.restype = st
    L.pmc_destroy_cache.argtypes = [vp]
    L.pmc_destroy_cache.restype = None
    L.pmc_material_info.argtypes = [vp, u32, vp, vp, u32, vp, vp]
    L.pmc_material_info.restype = st
    L.pmc_analyze_material.argtypes = [vp, u32, vp, vp, u32, vp, vp]
    L.pmc_analyze_material.restype = st
    L.pmc_analyze_material_ext.argtypes = [vp, u32, u32, u32, vp, vp, vp, u32, vp, vp]
    L.pmc_eval_passes_host.argtypes = [vp, vp, u32, vp, vp, vp]
    L.pmc_eval_passes_host.restype = st
    L.pmc_node_cost.argtypes = [vp]
    L.pmc_node_cost.restype = u32
    L.pmc_analyze_material_ext.restype = st
    L.pmc_compute_keys.argtypes = [vp, vp, vp, vp, u64, u32, u64, vp, vp, vp, vp]
    L.pmc_compute_keys.restype = st
    L.pmc_compute_levels.argtypes = [vp, vp, vp, vp, u64, C.c_int32, vp, vp]
    L.pmc_compute_levels.restype = st
    L.pmc_cast_rays.argtypes = [vp, u32, vp, u32, u32, u64, u32, vp, vp]
    L.pmc_cast_rays.restype = st
    L.pmc_set_timing.argtypes = [vp, C.c_int]
    L.pmc_set_timing.restype = st
    L.pmc_read_timing.argtypes = [vp, vp, vp, vp]
    L.pmc_read_timing.restype = st
    L.pmc_eval_batch_noalloc.argtypes = [vp, vp, vp, vp, vp]
    L.pmc_eval_batch_noalloc.restype = st
    L.pmc_train_surrogates.argtypes = [vp, vp, vp, vp]
    L.pmc_train_surrogates.restype = st
    L.pmc_set_surrogate.argtypes = [vp, u32, vp]
    L.pmc_set_surrogate.restype = st
    L.pmc_get_surrogate.argtypes = [vp, u32, vp, vp, vp]
    L.pmc_get_surrogate.restype = st
    L.pmc_use_surrogates.argtypes = [vp, C.c_int]
    L.pmc_use_surrogates.restype = st
    L.pmc_mlp_forward.argtypes = [vp, vp, vp, u64, vp, C.c_int, vp]
    L.pmc_mlp_forward.restype = st
    L.pmc_mlp_gradient.argtypes = [vp, vp, u64, vp, vp, vp]
    L.pmc_mlp_gradient.restype = st
    L.pmc_mlp_train.argtypes = [vp, vp, vp, vp, u64, u32, u32, u32, C.c_float, vp, vp]
    L.pmc_mlp_train.restype = st
    L.pmc_get_schedule.argtypes = [vp, vp]
    L.pmc_get_schedule.restype = st
    L.pmc_set_schedule.argtypes = [vp, vp]
    L.pmc_set_schedule.restype = st
    L.pmc_graph_create.argtypes = [vp, vp, u32, vp, vp, u32, vp]
    L.pmc_graph_create.restype = st
    L.pmc_graph_launch.argtypes = [vp, vp]
    L.pmc_graph_launch.restype = st
    L.pmc_graph_destroy.argtypes = [vp]
    L.pmc_graph_destroy.restype = None
    L.pmc_autotune.argtypes = [vp, vp, u32, vp]
    L.pmc_autotune.restype = st
    L.pmc_status_str.argtypes = [st]
    L.pmc_status_str.restype = C.c_char_p
    _lib = L
    return L


def status_str(s: int) -> str:
    try:
        return load().pmc_status_str(s).decode()
    except Exception:  # library missing: still report the number
        return f"status {s}"


def _check(s, what):
    if s != PMC_OK:
        raise PmcError(s, what)


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _has_cones(pts) -> bool:
    return all(pts.get(k) is not None for k in CONE_FIELDS)


def _points(pts, n, ptr):
    """The pmc_points struct of a point dict; ptr maps an array to its address.  The
    gradients present are passed as they are (the library rejects a partial set)."""
    cones = [ptr(pts[k]) if pts.get(k) is not None else None for k in CONE_FIELDS]
    vis = ptr(pts["vis"]) if pts.get("vis") is not None else None
    return _Points(*[ptr(pts[k]) for k in POINT_FIELDS], n, *cones, vis)


def points_to_device(pts: dict, device="cuda"):
    """Copies a host point batch (numpy SoA, with or without the ray-cone gradients and
    the visibility classes "vis") into torch device tensors."""
    import torch
    out = {}
    for k in POINT_FIELDS + (CONE_FIELDS if _has_cones(pts) else ()):
        a = np.ascontiguousarray(pts[k])
        t = torch.from_numpy(a.view(np.int32) if k == "mat" else a)
        out[k] = t.to(device)
    if pts.get("vis") is not None:
        out["vis"] = torch.from_numpy(np.ascontiguousarray(pts["vis"], dtype=np.uint8)).to(device)
    return out


class Cache:
    """A cache object of libpmc: compiled materials + a table of n_cells x n_entries slots."""

    def __init__(self, materials, n_cells, n_entries, uv_level=10, flags=0, min_root_nodes=2, device=0,
                 probe_capacity=0, level_offset=0, pos_level=0, min_root_cost=0):
        L = load()
        self._mats = [np.ascontiguousarray(m, dtype=NODE_DTYPE) for m in materials]
        arr = (_Material * len(self._mats))()
        for i, m in enumerate(self._mats):
            arr[i].n_nodes = len(m)
            arr[i].nodes = m.ctypes.data
        desc = _Desc(n_cells, n_entries, uv_level, flags, min_root_nodes, device, probe_capacity, level_offset,
                     pos_level, min_root_cost)
        h = C.c_void_p()
        _check(L.pmc_create_cache(C.byref(desc), arr, len(self._mats), C.byref(h)), "pmc_create_cache")
        self._h = h
        self.n_cells, self.n_entries, self.uv_level = n_cells, n_entries, uv_level
        self.flags, self.device = flags, device
        self.n_mats = len(self._mats)

    def close(self):
        if getattr(self, "_h", None):
            load().pmc_destroy_cache(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def cache_off(self):
        return bool(self.flags & PMC_CACHE_OFF)

    # ---- the pass --------------------------------------------------------------------
    def eval_batch(self, pts, out_rgb, out_hits=None, stream=None):
        """pts: dict of device tensors (float32; mat int32/uint32; optionally the ray-cone
        gradients g1u, g1v, g2u, g2v); out_rgb: float32 (3, n) device tensor; out_hits:
        int16/uint16 (n,) device tensor or None."""
        n = int(pts["u"].numel())
        p = _points(pts, n, _dptr)
        _check(load().pmc_eval_batch(self._h, C.byref(p), _dptr(out_rgb), _dptr(out_hits),
                                     _stream_handle(stream)), "pmc_eval_batch")

    def eval_batch_noalloc(self, pts, out_rgb, out_hits=None, stream=None):
        """Same pass as eval_batch with the library's fixed scratch array instead of device
        allocations (for callers that must not allocate; see include/pmc.h for the limits)."""
        n = int(pts["u"].numel())
        p = _points(pts, n, _dptr)
        _check(load().pmc_eval_batch_noalloc(self._h, C.byref(p), _dptr(out_rgb), _dptr(out_hits),
                                             _stream_handle(stream)), "pmc_eval_batch_noalloc")

    def eval_batch_host(self, pts: dict, out_rgb: np.ndarray, out_hits: np.ndarray | None = None,
                        stream=None):
        """Host buffers in and out; returns once the results are in out_rgb/out_hits."""
        keep = {k: np.ascontiguousarray(pts[k]) for k in POINT_FIELDS + (CONE_FIELDS if _has_cones(pts) else ())}
        if pts.get("vis") is not None:
            keep["vis"] = np.ascontiguousarray(pts["vis"], dtype=np.uint8)
        n = len(keep["u"])
        p = _points(keep, n, lambda a: a.ctypes.data)
        _check(load().pmc_eval_batch_host(self._h, C.byref(p), out_rgb.ctypes.data,
                                          None if out_hits is None else out_hits.ctypes.data,
                                          _stream_handle(stream)), "pmc_eval_batch_host")

    def eval_passes_host(self, passes, out_rgb, out_hits=None, stream=None):
        """Consecutive passes from host buffers (dicts of numpy arrays) into out_rgb[k] (and
        out_hits[k]), copies overlapped with the evaluation; returns when all are done."""
        keep = []
        for pts in passes:
            d = {k: np.ascontiguousarray(pts[k]) for k in POINT_FIELDS + (CONE_FIELDS if _has_cones(pts) else ())}
            if pts.get("vis") is not None:
                d["vis"] = np.ascontiguousarray(pts["vis"], dtype=np.uint8)
            keep.append(d)
        arr = (_Points * max(1, len(keep)))()
        for i, d in enumerate(keep):
            arr[i] = _points(d, len(d["u"]), lambda a: a.ctypes.data)
        rgb_p = (C.c_void_p * max(1, len(keep)))(*[o.ctypes.data for o in out_rgb])
        hits_p = None
        if out_hits is not None:
            hits_p = (C.c_void_p * max(1, len(keep)))(*[None if h is None else h.ctypes.data for h in out_hits])
        _check(load().pmc_eval_passes_host(self._h, arr, len(keep), rgb_p, hits_p, _stream_handle(stream)),
               "pmc_eval_passes_host")

    def sync(self):
        _check(load().pmc_sync(self._h), "pmc_sync")

    # ---- schedule, graphs of passes, autotuning ----------------------------------------
    def schedule(self) -> dict:
        sc = _Schedule()
        _check(load().pmc_get_schedule(self._h, C.byref(sc)), "pmc_get_schedule")
        return {"flags": int(sc.flags), "lookup_rb": int(sc.lookup_rb)}

    def set_schedule(self, flags: int, lookup_rb: int = 4):
        sc = _Schedule(flags, lookup_rb)
        _check(load().pmc_set_schedule(self._h, C.byref(sc)), "pmc_set_schedule")

    def graph(self, passes, out_rgb, out_hits=None, reset=False) -> "Graph":
        """Records len(passes) passes (dicts of device tensors) writing out_rgb[k] (and
        out_hits[k]) as one CUDA graph; see Graph.launch."""
        return Graph(self, passes, out_rgb, out_hits, reset)

    def autotune(self, pts, reps=3) -> dict:
        """Times the candidate schedules on one device batch and keeps the fastest."""
        n = int(pts["u"].numel())
        p = _points(pts, n, _dptr)
        r = _TuneResult()
        _check(load().pmc_autotune(self._h, C.byref(p), reps, C.byref(r)), "pmc_autotune")
        tried = [{"flags": int(r.tried[k].flags), "lookup_rb": int(r.tried[k].lookup_rb), "ms": float(r.ms[k])}
                 for k in range(r.n_tried)]
        return {"tried": tried, "best": int(r.best), "schedule": self.schedule()}

    def reset(self, stream=None):
        _check(load().pmc_reset(self._h, _stream_handle(stream)), "pmc_reset")

    # ---- inspection ------------------------------------------------------------------
    def stats(self, check=True) -> dict:
        s = _Stats()
        rc = load().pmc_stats(self._h, C.byref(s))
        if check:
            _check(rc, "pmc_stats")
        return {k: int(getattr(s, k)) for k in STAT_FIELDS}

    def table(self):
        """(h2 uint32[slots], rgb float32[slots, 3]) copied from the device."""
        slots = 0 if self.cache_off else self.n_cells * self.n_entries
        buf = np.zeros((max(slots, 1), 4), dtype=np.uint32)
        _check(load().pmc_table_dump(self._h, buf.ctypes.data, buf.nbytes), "pmc_table_dump")
        buf = buf[:slots]
        return buf[:, 0].copy(), buf[:, 1:].view(np.float32).copy()

    def classes(self) -> np.ndarray:
        """Visibility class of every slot's entry (uint8[slots]; 0 for an empty slot), for a
        cache created with PMC_REPLACE_VISIBILITY."""
        slots = self.n_cells * self.n_entries
        buf = np.zeros(max(slots, 1), dtype=np.uint8)
        _check(load().pmc_slot_classes(self._h, buf.ctypes.data, buf.nbytes), "pmc_slot_classes")
        return buf[:slots].copy()

    def last_hit_masks(self, n: int) -> np.ndarray:
        out = np.zeros(max(n, 1), dtype=np.uint64)
        _check(load().pmc_last_hit_masks(self._h, out.ctypes.data, n), "pmc_last_hit_masks")
        return out[:n]

    def set_timing(self, on: bool):
        _check(load().pmc_set_timing(self._h, int(bool(on))), "pmc_set_timing")

    def read_timing(self) -> dict:
        """Per-phase milliseconds (CUDA events) since the last read, kernel launches, batches."""
        ms = np.zeros(len(PHASES), dtype=np.float64)
        nl, nb = C.c_uint64(), C.c_uint64()
        _check(load().pmc_read_timing(self._h, ms.ctypes.data, C.byref(nl), C.byref(nb)), "pmc_read_timing")
        return {"ms": dict(zip(PHASES, ms.tolist())), "launches": nl.value, "batches": nb.value}

    # ---- learned surrogates ------------------------------------------------------------
    def train_surrogates(self, n_train=1 << 16, n_valid=8192, epochs=4, lr=0.0, rmse_max=0.0, seed=1,
                         mats=None, stream=None) -> np.ndarray:
        """Trains and validates surrogates; returns the validation RMSE per listed material."""
        ml = None if mats is None else np.ascontiguousarray(mats, dtype=np.uint32)
        n = self.n_mats if ml is None else len(ml)
        d = _TrainDesc(n_train, n_valid, epochs, lr, rmse_max, seed,
                       None if ml is None else ml.ctypes.data, 0 if ml is None else len(ml))
        out = np.zeros(max(n, 1), dtype=np.float32)
        _check(load().pmc_train_surrogates(self._h, C.byref(d), out.ctypes.data, _stream_handle(stream)),
               "pmc_train_surrogates")
        return out[:n]

    def set_surrogate(self, m: int, theta):
        th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float32)
        _check(load().pmc_set_surrogate(self._h, m, None if th is None else th.ctypes.data), "pmc_set_surrogate")

    def get_surrogate(self, m: int, with_theta=True) -> dict:
        node, en = C.c_uint32(), C.c_int()
        th = np.zeros(MLP_PARAMS, dtype=np.float32) if with_theta else None
        _check(load().pmc_get_surrogate(self._h, m, None if th is None else th.ctypes.data, C.byref(node),
                                        C.byref(en)), "pmc_get_surrogate")
        return {"theta": th, "node": node.value, "enabled": bool(en.value)}

    def use_surrogates(self, on: bool):
        _check(load().pmc_use_surrogates(self._h, int(bool(on))), "pmc_use_surrogates")

    def material_info(self, m: int) -> dict:
        nr, ni, ns = C.c_uint32(), C.c_uint32(), C.c_uint32()
        roots = np.zeros(65536, dtype=np.uint32)
        _check(load().pmc_material_info(self._h, m, C.byref(nr), roots.ctypes.data, 65536,
                                        C.byref(ni), C.byref(ns)), "pmc_material_info")
        return {"roots": roots[: nr.value].copy(), "n_instr": ni.value, "n_slots": ns.value}


def compute_levels(g1u, g1v, g2u, g2v, offset=0, stream=None):
    """Mip level of Eq. 1 for device tensors of ray-cone gradients (float32): uint32 levels
    as int32 tensor."""
    import torch
    n = int(g1u.numel())
    level = torch.empty(n, dtype=torch.int32, device=g1u.device)
    _check(load().pmc_compute_levels(_dptr(g1u), _dptr(g1v), _dptr(g2u), _dptr(g2v), n, offset, _dptr(level),
                                     _stream_handle(stream)), "pmc_compute_levels")
    return level


class _Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("fwd", C.c_float * 3), ("right", C.c_float * 3), ("up", C.c_float * 3),
                ("tan_half_y", C.c_float), ("width", C.c_uint32), ("height", C.c_uint32)]


RAY_HIT_FIELDS = ("u", "v", "mat", "px", "py", "pz", "nx", "ny", "nz", "g1u", "g1v", "g2u", "g2v")


class _RayHits(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in RAY_HIT_FIELDS]


def cast_rays(objects, camera: dict, seed: int, pass_index: int, rows=None, device="cuda", stream=None,
              out=None) -> dict:
    """Shading points of one pass from the library's ray caster: objects is a
    workload.OBJECT_DTYPE array (host), camera a dict with eye, fwd, right, up (3 floats),
    tan_half_y, width, height.  Returns device tensors u, v, mat (int32), px .. nz and the
    ray-cone gradients g1u .. g2v, one entry per pixel of rows (y0, y1) (all rows if None),
    ready for Cache.eval_batch.  `out`: the dict of a previous call of the same size, to
    write into instead of allocating."""
    import torch
    from .workload import OBJECT_DTYPE
    objs = np.ascontiguousarray(objects, dtype=OBJECT_DTYPE)
    W, H = int(camera["width"]), int(camera["height"])
    y0, y1 = rows if rows is not None else (0, H)
    n = max(0, (y1 - y0) * W)
    cam = _Camera((C.c_float * 3)(*camera["eye"]), (C.c_float * 3)(*camera["fwd"]),
                  (C.c_float * 3)(*camera["right"]), (C.c_float * 3)(*camera["up"]),
                  float(camera["tan_half_y"]), W, H)
    if out is None or any(int(out[k].numel()) != n for k in RAY_HIT_FIELDS):
        out = {k: torch.empty(n, dtype=torch.int32 if k == "mat" else torch.float32, device=device)
               for k in RAY_HIT_FIELDS}
    hits = _RayHits(*[_dptr(out[k]) for k in RAY_HIT_FIELDS])
    _check(load().pmc_cast_rays(objs.ctypes.data, len(objs), C.byref(cam), y0, y1, seed & ((1 << 64) - 1),
                                pass_index, C.byref(hits), _stream_handle(stream)), "pmc_cast_rays")
    return out


class Graph:
    """A CUDA graph of consecutive passes of one cache (pmc_graph_create).  The tensors
    are bound by address and kept alive here."""

    def __init__(self, cache: Cache, passes, out_rgb, out_hits=None, reset=False):
        L = load()
        k = len(passes)
        self._keep = (passes, out_rgb, out_hits, cache)
        pts = (_Points * max(k, 1))()
        for i, pp in enumerate(passes):
            pts[i] = _points(pp, int(pp["u"].numel()), _dptr)
        rgb = (C.c_void_p * max(k, 1))(*[t.data_ptr() for t in out_rgb])
        hits = None
        if out_hits is not None:
            hits = (C.c_void_p * max(k, 1))(*[None if t is None else t.data_ptr() for t in out_hits])
        h = C.c_void_p()
        _check(L.pmc_graph_create(cache._h, pts, k, rgb, hits, PMC_GRAPH_RESET if reset else 0, C.byref(h)),
               "pmc_graph_create")
        self._h = h

    def launch(self, stream=None):
        _check(load().pmc_graph_launch(self._h, _stream_handle(stream)), "pmc_graph_launch")

    def close(self):
        if getattr(self, "_h", None):
            load().pmc_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_forward(theta, u, v, clamp=True, stream=None):
    """The surrogate network on device tensors: theta (8515 float32), u, v -> (3, n)."""
    import torch
    n = int(u.numel())
    out = torch.empty((3, n), dtype=torch.float32, device=u.device)
    _check(load().pmc_mlp_forward(_dptr(theta), _dptr(u), _dptr(v), n, _dptr(out), int(clamp),
                                  _stream_handle(stream)), "pmc_mlp_forward")
    return out


def mlp_gradient(theta, data, stream=None):
    """Gradient (8515) and summed squared error of the mean-squared loss over data (n x 5)."""
    import torch
    n = int(data.shape[0])
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=data.device)
    loss = torch.empty(1, dtype=torch.float32, device=data.device)
    _check(load().pmc_mlp_gradient(_dptr(theta), _dptr(data), n, _dptr(grad), _dptr(loss),
                                   _stream_handle(stream)), "pmc_mlp_gradient")
    return grad, loss


def mlp_train(theta, adam_m, adam_v, data, steps, step0, total_steps, lr, stream=None):
    """Adam steps of the surrogate network on data (n x 5, n a power of two) in place."""
    import torch
    loss = torch.zeros(1, dtype=torch.float32, device=data.device)
    _check(load().pmc_mlp_train(_dptr(theta), _dptr(adam_m), _dptr(adam_v), _dptr(data), int(data.shape[0]),
                                steps, step0, total_steps, lr, _dptr(loss), _stream_handle(stream)),
           "pmc_mlp_train")
    return loss


def node_cost(node_row) -> int:
    """The library's node cost model: FP32 operations of one evaluation of the node."""
    m = np.ascontiguousarray(np.atleast_1d(node_row), dtype=NODE_DTYPE)
    return int(load().pmc_node_cost(m.ctypes.data))


def analyze_material(nodes, min_root_nodes=2, flags=0, min_root_cost=0) -> dict:
    """Host-only compile of one network: cacheable nodes (and their descriptor kinds, 1 = UV,
    2 = world position), program length, slots."""
    m = np.ascontiguousarray(nodes, dtype=NODE_DTYPE)
    mat = _Material(len(m), m.ctypes.data)
    nr, ni, ns = C.c_uint32(), C.c_uint32(), C.c_uint32()
    roots = np.zeros(65536, dtype=np.uint32)
    kinds = np.zeros(65536, dtype=np.uint8)
    _check(load().pmc_analyze_material_ext(C.byref(mat), min_root_nodes, min_root_cost, flags, C.byref(nr),
                                           roots.ctypes.data,
                                           kinds.ctypes.data, 65536, C.byref(ni), C.byref(ns)),
           "pmc_analyze_material_ext")
    return {"roots": roots[: nr.value].copy(), "kinds": kinds[: nr.value].copy(), "n_instr": ni.value,
            "n_slots": ns.value}


def compute_keys(mat, node, u, v, level, n_cells, stream=None):
    """Descriptor, cell and hash2 for device tensors mat/node (int32), u/v (float32)."""
    import torch
    n = int(u.numel())
    dev = u.device
    key = torch.empty(n, dtype=torch.int64, device=dev)
    cell = torch.empty(n, dtype=torch.int64, device=dev)
    h2 = torch.empty(n, dtype=torch.int32, device=dev)
    _check(load().pmc_compute_keys(_dptr(mat), _dptr(node), _dptr(u), _dptr(v), n, level, n_cells,
                                   _dptr(key), _dptr(cell), _dptr(h2), _stream_handle(stream)),
           "pmc_compute_keys")
    return key, cell, h2
