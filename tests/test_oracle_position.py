"""Pins of the oracle's world-position descriptor (Sec. 3.1 names a world-space position as
a further descriptor of a cacheable node; Sec. 5 lists other shading-point information
than UV as future work).

With it, a node whose sub-graph depends on the shading point's position and on nothing
else of the point is cacheable too; its descriptor is (material, node, voxel of the
position on a grid of 2^-level world units).  Expected values are worked out by hand.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_07238_gb300 import workload as W


@pytest.mark.parametrize("p,level,expected", [
    (0.0, 6, 512), (0.01, 6, 512), (-1.0 / 64, 6, 511), (-0.001, 6, 511),
    (7.99, 6, 1023), (8.0, 6, 1023), (100.0, 6, 1023), (-8.0, 6, 0), (-9.0, 6, 0),
    (3.7, 0, 515), (-0.5, 0, 511), (0.5, 1, 513), (0.49, 1, 512),
    (float("nan"), 6, 0), (float("inf"), 6, 1023), (float("-inf"), 6, 0),
])
def test_voxel_by_hand(p, level, expected):
    assert O.voxel(p, level) == expected


def test_position_key_packing_by_hand():
    k = O.key_pos(3, 17, 6, 0.0, -1.0 / 64, 8.0)
    assert k == (3 << 48) | (17 << 32) | (1 << 31) | (512 << 20) | (511 << 10) | 1023
    # bit 31 tells a position key from a UV key of the same (material, node)
    assert O.key(3, 17, 13, 1.0, 1.0) >> 31 & 1 == 0


def g_position():
    """0 UV; 1 POSITION; 2 UV_AFFINE(1); 3 FBM(2); 4 RAMP(3); 5 FBM(0); 6 RAMP(5);
    7 NORMAL; 8 FACING(7); 9 MIX(6, 4, 8); 10 VORONOI(2); 11 MUL(9, 10) = output."""
    b = W.Builder()
    uv = b.add(W.OP_UV)
    pos = b.add(W.OP_POSITION)
    a2 = b.add(W.OP_UV_AFFINE, [pos], fp=[0.5, 0.0, 0.0, 0.5, 0.25, 0.25])
    f3 = b.add(W.OP_FBM, [a2], ip=[2, 3], fp=[4.0, 2.0, 0.5])
    r4 = b.add(W.OP_RAMP, [f3], ip=[2], fp=[0.0, 1.0, 0, 0, 0.1, 0.2, 0.3, 0.9, 0.8, 0.7])
    f5 = b.add(W.OP_FBM, [uv], ip=[1, 4], fp=[8.0, 2.0, 0.5])
    r6 = b.add(W.OP_RAMP, [f5], ip=[2], fp=[0.0, 1.0, 0, 0, 0.3, 0.3, 0.3, 0.6, 0.9, 0.2])
    nrm = b.add(W.OP_NORMAL)
    f8 = b.add(W.OP_FACING, [nrm], fp=[0.0, 0.0, 1.0])
    m9 = b.add(W.OP_MIX, [r6, r4, f8])
    v10 = b.add(W.OP_VORONOI, [a2], ip=[0, 9], fp=[3.0])
    b.add(W.OP_MUL, [m9, v10])
    return b.build()


def test_analysis_by_hand():
    g = g_position()
    cls, roots, kinds = O.analyze(g, pos_desc=True, kinds=True)
    # classes: CONST 0, UV 1, SP 2, POS 3
    assert list(cls) == [1, 3, 3, 3, 3, 1, 1, 2, 2, 2, 3, 2]
    # node 2 feeds only position-class nodes: not maximal; node 4 (3 nodes of work) and 10
    # (affine + Worley) feed SP nodes; node 6 is the UV root
    assert list(roots) == [4, 6, 10] and list(kinds) == [2, 1, 2]
    # without the descriptor the position is plain shading-point information
    cls0, roots0 = O.analyze(g)
    assert list(roots0) == [6] and cls0[1] == 2 and cls0[4] == 2


def test_mixed_and_bare_inputs_are_not_roots():
    b = W.Builder()
    uv = b.add(W.OP_UV)
    pos = b.add(W.OP_POSITION)
    f2 = b.add(W.OP_FBM, [uv], ip=[1, 1], fp=[4.0, 2.0, 0.5])
    f3 = b.add(W.OP_FBM, [pos], ip=[1, 2], fp=[4.0, 2.0, 0.5])
    b.add(W.OP_MUL, [f2, f3])              # UV with position: SP
    g = b.build()
    assert list(O.analyze(g, pos_desc=True)[1]) == []                        # 1 node of work each
    _, roots, kinds = O.analyze(g, min_root_nodes=1, pos_desc=True, kinds=True)
    assert list(roots) == [2, 3] and list(kinds) == [1, 2]
    # the output itself of position class is a root; the bare POSITION never is
    b = W.Builder()
    pos = b.add(W.OP_POSITION)
    f1 = b.add(W.OP_FBM, [pos], ip=[2, 1], fp=[2.0, 2.0, 0.5])
    b.add(W.OP_RAMP, [f1], ip=[2], fp=[0.0, 1.0, 0, 0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
    _, roots, kinds = O.analyze(b.build(), pos_desc=True, kinds=True)
    assert list(roots) == [2] and list(kinds) == [2]


def _voxel_checker(level):
    """CHECKER of (px, py) at scale 2^level: constant on every voxel of that level."""
    b = W.Builder()
    pos = b.add(W.OP_POSITION)
    a1 = b.add(W.OP_UV_AFFINE, [pos], fp=[1.0, 0.0, 0.0, 1.0, 0.0, 0.0])
    c2 = b.add(W.OP_CHECKER, [a1], fp=[float(2 ** level), 0.1, 0.2, 0.3, 0.9, 0.8, 0.7])
    nrm = b.add(W.OP_NORMAL)
    f4 = b.add(W.OP_FACING, [nrm], fp=[0.0, 1.0, 0.0])
    b.add(W.OP_MIX, [c2, b.add(W.OP_CONST, fp=[0.5, 0.5, 0.5]), f4])
    return b.build()


def test_subgraph_constant_per_voxel_caches_exactly():
    L = 1
    mat = _voxel_checker(L)
    c = O.Cache([mat], 4096, 8, pos_level=L)
    plain = O.Cache([mat], 4096, 8, cache_off=True)
    assert list(c.roots(0)) == [2]
    hits = 0
    for p in range(4):
        pts = W.points_uniform(2000, seed=70 + p)
        r, r0 = c.run_batch(pts), plain.run_batch(pts)
        assert np.array_equal(r["rgb"], r0["rgb"])
        hits += int(r["hits"].sum())
    assert hits > 1000


def test_hit_count_equals_exhaustive_count():
    L = 2
    mat = _voxel_checker(L)
    c = O.Cache([mat], 1 << 14, 8, pos_level=L)
    seen = set()
    for p in range(4):
        pts = W.points_uniform(3000, seed=90 + p)
        keys = [O.key_pos(0, 2, L, pts["px"][i], pts["py"][i], pts["pz"][i]) for i in range(3000)]
        r = c.run_batch(pts)
        assert c.stats()["dropped_full"] == 0
        assert int(r["hits"].sum()) == sum(k in seen for k in keys)
        seen.update(keys)


def test_off_is_the_uv_method():
    mats = W.random_materials(4, 10, 60, 0.3, seed=8)
    a, b = O.Cache(mats, 64, 4), O.Cache(mats, 64, 4, pos_level=-1)
    for p in range(2):
        pts = W.points_uniform(800, seed=110 + p, n_mats=4)
        ra, rb = a.run_batch(pts), b.run_batch(pts)
        assert np.array_equal(ra["rgb"], rb["rgb"]) and np.array_equal(ra["hits"], rb["hits"])
    assert a.stats() == b.stats()


def test_position_roots_add_lookups_on_generated_networks():
    # the generator's position noise (single FBM, Worley or checker nodes, hence a minimum
    # of one node of work) becomes cacheable: more roots, every UV root kept
    mats = W.random_materials(16, 20, 200, 0.2, seed=0)
    extra = 0
    for m in mats:
        _, r_uv = O.analyze(m, min_root_nodes=1)
        _, r_all, kinds = O.analyze(m, min_root_nodes=1, pos_desc=True, kinds=True)
        assert set(r_all[kinds == 1].tolist()) == set(r_uv.tolist())
        extra += int((kinds == 2).sum())
    assert extra > 0
