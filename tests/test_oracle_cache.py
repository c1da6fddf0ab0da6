"""Pins of the oracle's progressive cache (Sec. 3, Sec. 3.2, Alg. 1).

Each test checks the batch emulation against something it does not share code
with: plain evaluation without a cache, a direct serial transcription of Alg. 1 with
a compare-and-swap on the whole entry, hand-built tables, exhaustive counting, or
structural invariants of a keep-first table.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_07238_gb300 import workload as W

from .test_oracle_analysis import g_nested, g_two_roots


def _pts(n, seed, n_mats=1):
    return W.points_uniform(n, seed=seed, n_mats=n_mats)


def _sp(p, i):
    return [float(p[k][i]) for k in W.POINT_FIELDS if k != "mat"]


def _nocache(mat_nodes, pts):
    n = len(pts["u"])
    out = np.zeros((3, n))
    for i in range(n):
        out[:, i] = O.eval_point_nocache(mat_nodes[int(pts["mat"][i])], _sp(pts, i))
    return out


# ---- (i) cache off / first pass == plain evaluation ------------------------------------
def test_cache_off_equals_plain_evaluation():
    mats = W.random_materials(4, 20, 80, 0.2, seed=1)
    pts = _pts(300, 5, n_mats=4)
    c = O.Cache(mats, 0, 8, cache_off=True)
    for _ in range(2):
        r = c.run_batch(pts)
        assert np.array_equal(r["rgb"], _nocache(mats, pts))
        assert not r["hits"].any()
    st = c.stats()
    assert st["lookups"] == 0 and st["inserted"] == 0


def test_first_pass_on_empty_table_equals_plain_evaluation():
    mats = W.random_materials(4, 20, 80, 0.2, seed=2)
    pts = _pts(300, 6, n_mats=4)
    c = O.Cache(mats, 1024, 8)
    r = c.run_batch(pts)
    assert np.array_equal(r["rgb"], _nocache(mats, pts))
    st = c.stats()
    assert st["hits"] == 0 and st["lookups"] == st["misses"]
    assert st["candidates"] == st["misses"]


# ---- (ii) one point per batch == serial Alg. 1 -------------------------------------------
class SerialAlg1:
    """Alg. 1 as printed, run for one shading point at a time: scan the cell for an
    entry whose hash is Hash2(desc) or 0, then CAS(entry, 0, {hash2, value}); the CAS
    only succeeds on an all-zero (empty) entry.  Lookup scans the same way."""

    def __init__(self, mats, n_cells, n_entries, level=10):
        self.mats = mats
        self.nc, self.ne, self.level = n_cells, n_entries, level
        self.h2 = [0] * (n_cells * n_entries)
        self.val = [(0.0, 0.0, 0.0)] * (n_cells * n_entries)
        self.roots = [list(O.analyze(m)[1]) for m in mats]

    def _cell(self, key):
        return O.hash1(key) % self.nc, O.hash2(key)

    def lookup(self, key):
        cell, hv = self._cell(key)
        for i in range(self.ne):
            e = cell * self.ne + i
            if self.h2[e] == hv:
                return self.val[e]
            if self.h2[e] == 0:
                return None
        return None

    def insert(self, key, v):
        cell, hv = self._cell(key)
        idx = -1
        for i in range(self.ne):
            e = cell * self.ne + i
            if self.h2[e] == hv or self.h2[e] == 0:
                idx = e
                break
        if idx != -1:
            if self.h2[idx] == 0 and self.val[idx] == (0.0, 0.0, 0.0):   # CAS(entry, 0, new)
                self.h2[idx] = hv
                self.val[idx] = v

    def shade(self, m, sp, u, v):
        nodes = self.mats[m].copy()
        hits = 0
        for r in self.roots[m]:
            key = O.key(m, int(r), self.level, np.float32(u), np.float32(v))
            got = self.lookup(key)
            if got is not None:
                hits += 1
                nodes[r]["op"] = W.OP_CONST          # use the cached value ...
                nodes[r]["inp"][:] = -1
                nodes[r]["fp"][:3] = got
            else:
                val = O.eval_point_nocache(self.mats[m][: r + 1], sp)   # ... or evaluate
                self.insert(key, tuple(float(np.float32(x)) for x in val))
        # nodes no longer read by anyone are harmless for plain evaluation
        return O.eval_point_nocache(nodes, sp), hits


def test_single_point_batches_match_serial_alg1():
    mats = W.random_materials(3, 15, 60, 0.2, seed=4)
    # few distinct texels so that hits happen: UV on a 6x6 grid of texel centres
    rng = np.random.default_rng(7)
    n = 120
    pts = _pts(n, 8, n_mats=3)
    pts["u"] = ((rng.integers(0, 6, n) + 0.5) / 1024).astype(np.float32)
    pts["v"] = ((rng.integers(0, 6, n) + 0.5) / 1024).astype(np.float32)
    nc, ne = 16, 4                                   # small table: collisions and full cells
    oc = O.Cache(mats, nc, ne)
    ser = SerialAlg1(mats, nc, ne)
    for i in range(n):
        one = W.slice_points(pts, i, i + 1)
        r = oc.run_batch(one)
        m = int(pts["mat"][i])
        exp_rgb, exp_hits = ser.shade(m, _sp(pts, i), pts["u"][i], pts["v"][i])
        assert r["hits"][0] == exp_hits
        assert np.allclose(r["rgb"][:, 0], exp_rgb, atol=1e-12)
    h2, rgb = oc.table()
    assert list(h2) == ser.h2
    assert np.array_equal(rgb, np.array(ser.val, dtype=np.float32))
    assert oc.stats()["hits"] > 0


# ---- (iii) hand tables -----------------------------------------------------------------
def _distinct_texel_points(n):
    pts = _pts(n, 9)
    pts["u"] = ((np.arange(n) + 0.5) / 1024).astype(np.float32)
    pts["v"] = np.full(n, 0.5 / 1024, dtype=np.float32)
    return pts


def test_one_cell_two_entries_third_key_dropped():
    mat = W.material_tiny()
    c = O.Cache([mat], 1, 2)                         # N_c = 1, N_e = 2
    r = c.run_batch(_distinct_texel_points(3))
    st = c.stats()
    assert (st["inserted"], st["dropped_full"], st["dropped_dup"]) == (2, 1, 0)
    h2, rgb = c.table()
    # keep-first: slots hold points 0 and 1 (ascending point index), point 2 is dropped
    keys = [O.key(0, 7, 10, np.float32((i + 0.5) / 1024), np.float32(0.5 / 1024)) for i in range(3)]
    assert list(h2) == [O.hash2(keys[0]), O.hash2(keys[1])]
    assert np.allclose(rgb[0], r["rgb"][:, 0], atol=1e-7)
    assert np.allclose(rgb[1], r["rgb"][:, 1], atol=1e-7)
    # next pass: the dropped key still misses, the kept ones hit
    r2 = c.run_batch(_distinct_texel_points(3))
    assert list(r2["hits"]) == [1, 1, 0]


def test_fig3_table_geometry_forced_cell():
    # 10 cells x 5 entries (Fig. 3); every key forced into cell 3 with its own hash2.
    mat = W.material_tiny()
    hook = lambda k, nc: (3, (k & 0xFFFFFF) + 1)
    c = O.Cache([mat], 10, 5, hash_hook=hook)
    c.run_batch(_distinct_texel_points(12))
    st = c.stats()
    assert (st["inserted"], st["dropped_full"]) == (5, 7)
    h2, _ = c.table()
    assert np.count_nonzero(h2) == 5 and np.all(h2[15:20] != 0)
    assert np.all(h2[:15] == 0) and np.all(h2[20:] == 0)


# ---- (iv) forced hash2 collision: a false hit returns the first key's value ---------------
def test_forced_hash2_collision_false_hit():
    mat = W.material_tiny()
    hook = lambda k, nc: (0, 42)
    c = O.Cache([mat], 4, 2, hash_hook=hook)
    pts = _distinct_texel_points(3)
    r1 = c.run_batch(pts)
    st = c.stats()
    assert (st["inserted"], st["dropped_dup"]) == (1, 2)     # same (cell, hash2) = same key
    first = r1["rgb"][:, 0].astype(np.float32).astype(np.float64)
    other = W.slice_points(_distinct_texel_points(5), 4, 5)   # a texel never seen
    r2 = c.run_batch(other)
    assert r2["hits"][0] == 1
    assert np.array_equal(r2["rgb"][:, 0], first)           # the tiny material's root is its output


# ---- (v) invariants of a keep-first table ---------------------------------------------------
def _check_invariants(c, st):
    h2, _ = c.table()
    cells = h2.reshape(c.n_cells, c.n_entries)
    occ = cells != 0
    for row, o in zip(cells, occ):
        k = int(o.sum())
        assert o[:k].all() and not o[k:].any()          # occupied slots form a prefix
        assert len(set(row[:k].tolist())) == k           # unique hash2 per cell
    assert st["inserted"] == int(occ.sum())
    assert st["hits"] <= st["lookups"] and st["hits"] + st["misses"] == st["lookups"]
    assert st["candidates"] == st["inserted"] + st["dropped_dup"] + st["dropped_full"]


def test_invariants_over_frame_passes():
    spec = W.FrameSpec(width=64, height=48, n_mats=6, seed=1)
    frame = W.Frame(spec)
    mats = W.random_materials(6, 20, 60, 0.2, seed=5)
    c = O.Cache(mats, 512, 8)
    hits_per_pass = []
    for p in range(4):
        before = c.stats()["hits"]
        c.run_batch(frame.points(p))
        st = c.stats()
        _check_invariants(c, st)
        hits_per_pass.append(st["hits"] - before)
    assert hits_per_pass[0] == 0 and hits_per_pass[-1] > 0


def test_same_texel_twice_in_one_batch_both_miss():
    mat = W.material_tiny()
    c = O.Cache([mat], 64, 4)
    pts = _distinct_texel_points(2)
    pts["u"][1] = pts["u"][0]                            # same texel, same batch
    r = c.run_batch(pts)
    assert list(r["hits"]) == [0, 0]
    st = c.stats()
    assert (st["inserted"], st["dropped_dup"]) == (1, 1)


# ---- (vi) a sub-graph constant on every texel caches exactly ------------------------------
def test_texel_constant_subgraph_caches_exactly():
    b = W.Builder()
    uv = b.add(W.OP_UV)
    c1 = b.add(W.OP_CHECKER, [uv], fp=[256.0, 0.5, 0.25, 0.75, 1.0, 0.125, 0.5])
    c2 = b.add(W.OP_CHECKER, [uv], fp=[1024.0, 0.5, 0.5, 0.5, 0.25, 1.0, 0.75])
    m3 = b.add(W.OP_MUL, [c1, c2])                       # dyadic products: exact in FP32
    nrm = b.add(W.OP_NORMAL)
    f5 = b.add(W.OP_FACING, [nrm], fp=[0.0, 0.0, 1.0])
    b.add(W.OP_MIX, [m3, b.add(W.OP_CONST, fp=[0.3, 0.6, 0.9]), f5])
    mat = b.build()
    assert list(O.analyze(mat)[1]) == [3]
    pts = _pts(2000, 11)
    pts["u"] = (np.floor(pts["u"] * 16) / 1024).astype(np.float32)   # 16x16 texels: many repeats
    pts["v"] = (np.floor(pts["v"] * 16) / 1024).astype(np.float32)
    c = O.Cache([mat], 4096, 8)
    off = O.Cache([mat], 0, 8, cache_off=True)
    tot_hits = 0
    for p in range(4):
        part = W.slice_points(pts, 500 * p, 500 * (p + 1))
        r = c.run_batch(part)
        assert np.array_equal(r["rgb"], off.run_batch(part)["rgb"])
        tot_hits += int(r["hits"].sum())
    assert tot_hits > 1000


# ---- (vii) hit count == exhaustive count of earlier keys --------------------------------
def test_tiny_hit_count_equals_brute_force():
    mat = W.material_tiny()
    pts = W.points_uniform(16384, seed=0)
    c = O.Cache([mat], 8192, 8)                         # 2^16 slots, N_e = 8
    seen = set()
    for p in range(4):
        part = W.slice_points(pts, 4096 * p, 4096 * (p + 1))
        keys = [O.key(0, 7, 10, part["u"][i], part["v"][i]) for i in range(4096)]
        expected = sum(k in seen for k in keys)
        before = c.stats()["dropped_full"]
        r = c.run_batch(part)
        assert int(r["hits"].sum()) == expected
        if c.stats()["dropped_full"] == before:
            seen.update(keys)
        else:  # a full cell dropped some key: stop comparing
            break


# ---- needed set: a hit root's sub-graph is not evaluated -----------------------------------
@pytest.mark.parametrize("graph,total,after", [(g_two_roots, 12, 6), (g_nested, 9, 4)])
def test_hit_roots_skip_their_subgraph(graph, total, after):
    mat = graph()
    pts = _pts(1, 12)
    c = O.Cache([mat], 64, 4)
    r1 = c.run_batch(pts)
    assert r1["evaluated"][0] == total and r1["hits"][0] == 0
    r2 = c.run_batch(pts)
    assert r2["hits"][0] == 2
    assert r2["evaluated"][0] == after


def test_bad_material_id_reported():
    mat = W.material_tiny()
    pts = _pts(4, 13)
    pts["mat"][2] = 5
    c = O.Cache([mat], 64, 4)
    r = c.run_batch(pts)
    assert r["status"] == 2
    assert r["hits"][2] == 0 and np.all(r["rgb"][:, 2] == 0)


@pytest.mark.parametrize("kw", [{}, {"replacement": True}, {"pos_level": 4}, {"cones": True},
                                {"cache_off": True}, {"alg1": True}])
def test_all_core_form_equals_one_thread(kw):
    """The all-core form of a pass (ranges of points in parallel against the same snapshot,
    then one sequential insert) gives the one-thread results bit for bit."""
    kw = dict(kw)
    cones = kw.pop("cones", False)
    mats = W.random_materials(12, 10, 80, 0.3, seed=31)
    frame = W.Frame(W.FrameSpec(width=640, height=48, n_mats=12, seed=31))
    caches = [O.Cache(mats, 512, 4, threads=t, **kw) for t in (1, 4)]
    for p in range(3):
        pts = frame.points(p, cones=cones) if cones else frame.points(p)
        if kw.get("replacement"):
            pts["vis"] = (np.arange(len(pts["u"])) % 3).astype(np.uint8)
        pts["mat"][::997] = 99                    # a few bad material indices
        r = [c.run_batch(pts, probes=True) for c in caches]
        for k in ("rgb", "hits", "evaluated", "key", "cell", "h2", "hit"):
            assert np.array_equal(r[0][k], r[1][k]), k
        assert r[0]["status"] == r[1]["status"] != 0
        assert caches[0].stats() == caches[1].stats()
        for a, b in zip(caches[0].table(), caches[1].table()):
            assert np.array_equal(a, b)
