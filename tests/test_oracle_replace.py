"""Pins of the oracle's replacement policy by visibility class (Sec. 5 proposes
prioritising directly visible materials over indirectly visible ones; keep-first is the
method of Sec. 3.2 and Alg. 1).

A point's class is 0 when the camera sees it directly and k after k bounces.  A full cell
that lacks the newcomer's descriptor gives up its entry of the largest class if that class
is larger than the newcomer's (the first such entry on ties); otherwise the value is
dropped as with keep-first.  Every expected table below is worked out by hand.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_07238_gb300 import workload as W

ROOT = 7   # the tiny material's only cacheable node (its output)


def _texel_points(texels, vis):
    """One point per entry: texel (t, 0) of the 1024-texel level, class vis[k]."""
    n = len(texels)
    pts = W.points_uniform(n, seed=9)
    pts["u"] = ((np.asarray(texels, dtype=np.float64) + 0.5) / 1024).astype(np.float32)
    pts["v"] = np.full(n, 0.5 / 1024, dtype=np.float32)
    pts["vis"] = np.asarray(vis, dtype=np.uint8)
    return pts


def _h2(t):
    # descriptor of texel (t, 0): iu = t sits at bits 13.. of the key; the hook below
    # keeps the low 24 bits, so every texel gets its own check value
    return (t << 13) + 1


def _one_cell(n_entries, replacement=True, close_at_lookup=True):
    mat = W.material_tiny()
    hook = lambda k, nc: (0, (k & 0xFFFFFF) + 1)
    return O.Cache([mat], 1, n_entries, hash_hook=hook, replacement=replacement,
                   close_at_lookup=close_at_lookup)


def _cell(c):
    h2, _ = c.table()
    return list(h2), list(c.classes())


def test_hand_sequence_one_cell_two_entries():
    c = _one_cell(2)
    c.run_batch(_texel_points([0, 1], [2, 1]))                 # fills the cell
    assert _cell(c) == ([_h2(0), _h2(1)], [2, 1])
    c.run_batch(_texel_points([2], [0]))                       # evicts class 2 (slot 0)
    assert _cell(c) == ([_h2(2), _h2(1)], [0, 1])
    c.run_batch(_texel_points([3], [1]))                       # nothing of class > 1: dropped
    assert _cell(c) == ([_h2(2), _h2(1)], [0, 1])
    c.run_batch(_texel_points([4], [0]))                       # evicts class 1 (slot 1)
    assert _cell(c) == ([_h2(2), _h2(4)], [0, 0])
    r = c.run_batch(_texel_points([0], [0]))                   # texel 0 was evicted: a miss
    assert r["hits"][0] == 0
    assert _cell(c) == ([_h2(2), _h2(4)], [0, 0])              # all class 0: dropped
    r = c.run_batch(_texel_points([2], [3]))                   # a hit whatever its class
    assert r["hits"][0] == 1
    st = c.stats()
    assert (st["inserted"], st["replaced"], st["dropped_full"], st["dropped_dup"]) == (2, 2, 2, 0)
    assert st["candidates"] == 6


def test_same_batch_order_and_classes():
    c = _one_cell(1)
    c.run_batch(_texel_points([0], [1]))
    # ascending point order: class 2 cannot evict class 1; class 0 can; the next class 0
    # finds only class 0
    c.run_batch(_texel_points([1, 2, 3], [2, 0, 0]))
    assert _cell(c) == ([_h2(2)], [0])
    st = c.stats()
    assert (st["inserted"], st["replaced"], st["dropped_full"]) == (1, 1, 2)


def test_same_descriptor_two_classes_in_one_batch():
    # the first copy (class 3) is dropped, the second (class 0) of the SAME texel then
    # evicts: no deduplication may tie the second copy's fate to the first's
    c = _one_cell(1)
    c.run_batch(_texel_points([0], [1]))
    c.run_batch(_texel_points([5, 5], [3, 0]))
    assert _cell(c) == ([_h2(5)], [0])
    st = c.stats()
    assert (st["replaced"], st["dropped_full"], st["dropped_dup"]) == (1, 1, 0)
    # a copy after an eviction in the same batch is a duplicate if its cell, at lookup, held
    # an entry it could have evicted (class 3 > 2) ...
    c2 = _one_cell(1)
    c2.run_batch(_texel_points([0], [3]))
    c2.run_batch(_texel_points([6, 6], [0, 2]))
    assert _cell(c2) == ([_h2(6)], [0])
    st = c2.stats()
    assert (st["replaced"], st["dropped_dup"], st["dropped_full"]) == (1, 1, 0)
    # ... and is dropped as full at lookup if every entry there was of its class or smaller
    # (class 1 <= 2): it could never have entered the cell in this batch
    c3 = _one_cell(1)
    c3.run_batch(_texel_points([0], [1]))
    c3.run_batch(_texel_points([6, 6], [0, 2]))
    assert _cell(c3) == ([_h2(6)], [0])
    st = c3.stats()
    assert (st["replaced"], st["dropped_dup"], st["dropped_full"]) == (1, 0, 1)


def test_ties_evict_the_first_entry_of_the_largest_class():
    c = _one_cell(4)
    c.run_batch(_texel_points([0, 1, 2, 3], [1, 3, 2, 3]))
    c.run_batch(_texel_points([4], [2]))                       # largest class 3: slots 1, 3
    assert _cell(c) == ([_h2(0), _h2(4), _h2(2), _h2(3)], [1, 2, 2, 3])
    c.run_batch(_texel_points([5], [2]))                       # slot 3 is the only class > 2
    assert _cell(c) == ([_h2(0), _h2(4), _h2(2), _h2(5)], [1, 2, 2, 2])
    c.run_batch(_texel_points([6], [2]))                       # nothing > 2 left
    assert c.stats()["dropped_full"] == 1


def test_replaced_entry_holds_the_newcomers_value():
    c = _one_cell(1)
    c.run_batch(_texel_points([0], [2]))
    pts = _texel_points([7], [0])
    r1 = c.run_batch(pts)
    _, rgb = c.table()
    assert np.array_equal(rgb[0], r1["rgb"][:, 0].astype(np.float32))
    r2 = c.run_batch(pts)                                      # hit on the new entry
    assert r2["hits"][0] == 1
    assert np.array_equal(r2["rgb"][:, 0], rgb[0].astype(np.float64))


def _frame_passes(n_passes, n, seed, n_mats=4):
    out = []
    for p in range(n_passes):
        pts = W.points_uniform(n, seed=seed + p, n_mats=n_mats)
        # coherent direct points re-visit a small UV window; indirect ones land anywhere
        rng = np.random.Generator(np.random.PCG64([seed, p]))
        vis = rng.choice(4, size=n, p=[0.5, 0.25, 0.15, 0.10]).astype(np.uint8)
        direct = vis == 0
        pts["u"][direct] = (pts["u"][direct] * 0.05).astype(np.float32)
        pts["v"][direct] = (pts["v"][direct] * 0.05).astype(np.float32)
        pts["vis"] = vis
        out.append(pts)
    return out


def test_all_class_zero_equals_keep_first():
    mats = W.random_materials(4, 8, 30, 0.2, seed=3)
    a = O.Cache(mats, 16, 4, replacement=True)
    b = O.Cache(mats, 16, 4, replacement=False)
    for pts in _frame_passes(3, 600, 11):
        pts["vis"][:] = 0
        ra, rb = a.run_batch(pts), b.run_batch(pts)
        assert np.array_equal(ra["rgb"], rb["rgb"]) and np.array_equal(ra["hits"], rb["hits"])
    assert np.array_equal(a.table()[0], b.table()[0])
    assert np.array_equal(a.table()[1], b.table()[1])
    assert a.stats() == b.stats() and a.stats()["replaced"] == 0


def test_invariants_over_passes():
    mats = W.random_materials(4, 8, 30, 0.2, seed=3)
    c = O.Cache(mats, 16, 4, replacement=True)
    ne = 4
    prev_h2 = prev_cls = None
    for pts in _frame_passes(5, 800, 21):
        c.run_batch(pts)
        h2, _ = c.table()
        cls = c.classes()
        H, K = h2.reshape(-1, ne), cls.reshape(-1, ne)
        occ = H != 0
        # occupied slots form a prefix of every cell; hash2 unique within a cell
        assert np.all(np.diff(occ.astype(np.int8), axis=1) <= 0)
        for row, o in zip(H, occ):
            assert len(set(row[o].tolist())) == int(o.sum())
        st = c.stats()
        assert st["inserted"] == int(occ.sum())
        assert st["candidates"] == st["inserted"] + st["replaced"] + st["dropped_dup"] + st["dropped_full"]
        assert set(K[occ].tolist()) <= {0, 1, 2, 3}
        if prev_h2 is not None:
            PH, PK = prev_h2.reshape(-1, ne), prev_cls.reshape(-1, ne)
            # an entry of class 0 is never evicted
            keep = (PH != 0) & (PK == 0)
            assert np.array_equal(H[keep], PH[keep]) and np.all(K[keep] == 0)
            # a full cell's classes only move toward the camera
            full = (PH != 0).all(axis=1)
            assert np.all(K[full].astype(int).sum(axis=1) <= PK[full].astype(int).sum(axis=1))
        prev_h2, prev_cls = h2.copy(), cls.copy()
    assert c.stats()["replaced"] > 0


def test_direct_points_hit_more_with_replacement():
    mats = W.random_materials(4, 8, 30, 0.2, seed=3)
    rates = {}
    for rep in (False, True):
        c = O.Cache(mats, 16, 4, replacement=rep)
        hits = looks = 0
        for p, pts in enumerate(_frame_passes(6, 800, 31)):
            r = c.run_batch(pts)
            if p >= 2:
                d = pts["vis"] == 0
                hits += int(r["hits"][d].sum())
                looks += int(sum(c.n_roots(int(m)) for m in pts["mat"][d]))
        rates[rep] = hits / looks
    assert rates[True] > rates[False]


def test_replacement_off_ignores_classes():
    mat = W.material_tiny()
    hook = lambda k, nc: (0, (k & 0xFFFFFF) + 1)
    c = O.Cache([mat], 1, 1, hash_hook=hook)
    c.run_batch(_texel_points([0], [3]))
    c.run_batch(_texel_points([1], [0]))
    assert list(c.table()[0]) == [_h2(0)]
    assert c.stats()["replaced"] == 0 and c.stats()["dropped_full"] == 1


@pytest.mark.parametrize("n_entries", [1, 3, 8])
def test_cache_off_and_first_pass_outputs_unchanged(n_entries):
    # the policy only decides what the table keeps: a pass's outputs depend on the
    # table it starts from, so the first pass equals keep-first exactly
    mats = W.random_materials(3, 8, 30, 0.2, seed=5)
    pts = _frame_passes(1, 500, 41, n_mats=3)[0]
    a = O.Cache(mats, 8, n_entries, replacement=True).run_batch(pts)
    b = O.Cache(mats, 8, n_entries).run_batch(pts)
    assert np.array_equal(a["rgb"], b["rgb"])


def test_closing_a_full_cell_at_lookup_changes_only_the_full_duplicate_split():
    """Dropping a value as full at lookup when its full cell holds no class larger than its
    own (the rule the CUDA path uses) against sending every evaluated miss to the sequential
    insert: the same cells, values and classes after every pass, hand cases where the
    accounting differs, and random passes where nothing but that split may differ."""
    # hand case: the cell holds class 1; the first copy (class 0) of texel 6 evicts it, the
    # second copy (class 1, later point) finds its key there.  Closed at lookup it is a full
    # drop (class 1 <= 1 at lookup); sent to the insert it is a duplicate.
    split = {}
    for close in (True, False):
        c = _one_cell(1, close_at_lookup=close)
        c.run_batch(_texel_points([0], [1]))
        c.run_batch(_texel_points([6, 6], [0, 1]))
        assert _cell(c) == ([_h2(6)], [0])
        st = c.stats()
        split[close] = (st["replaced"], st["dropped_dup"], st["dropped_full"])
    assert split[True] == (1, 0, 1) and split[False] == (1, 1, 0)
    # a value closed at lookup whose key never enters the cell: a full drop either way
    for close in (True, False):
        c = _one_cell(2, close_at_lookup=close)
        c.run_batch(_texel_points([0, 1], [0, 1]))
        c.run_batch(_texel_points([2], [1]))
        assert _cell(c) == ([_h2(0), _h2(1)], [0, 1])
        assert c.stats()["dropped_full"] == 1 and c.stats()["dropped_dup"] == 0
    # random passes: identical tables, classes, outputs and hits after every pass; the
    # counters agree except for the split between duplicates and full drops
    mats = W.random_materials(4, 8, 30, 0.2, seed=3)
    a = O.Cache(mats, 16, 4, replacement=True, close_at_lookup=True)
    b = O.Cache(mats, 16, 4, replacement=True, close_at_lookup=False)
    moved = 0
    for pts in _frame_passes(6, 800, 51):
        ra, rb = a.run_batch(pts), b.run_batch(pts)
        assert np.array_equal(ra["rgb"], rb["rgb"]) and np.array_equal(ra["hits"], rb["hits"])
        assert np.array_equal(a.table()[0], b.table()[0])
        assert np.array_equal(a.table()[1], b.table()[1])
        assert np.array_equal(a.classes(), b.classes())
        sa, sb = a.stats(), b.stats()
        for k in ("lookups", "hits", "misses", "candidates", "inserted", "replaced"):
            assert sa[k] == sb[k], k
        assert sa["dropped_dup"] + sa["dropped_full"] == sb["dropped_dup"] + sb["dropped_full"]
        moved = sb["dropped_dup"] - sa["dropped_dup"]
        assert moved >= 0
    assert a.stats()["replaced"] > 0
