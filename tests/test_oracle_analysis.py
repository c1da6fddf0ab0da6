"""Cacheable-node analysis (Sec. 3) on hand-built networks with hand-derived roots."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_07238_gb300 import workload as W

CONST, UV, SP = 0, 1, 2


def g_two_roots():
    """0 UV; 1 FBM(0); 2 RAMP(1); 3 VORONOI(0); 4 MUL(2,3); 5 NORMAL; 6 FACING(5);
    7 CHECKER(0); 8 MIX(4,7,6); 9 FBM(0); 10 POW(9); 11 MUL(8,10) = output."""
    b = W.Builder()
    uv = b.add(W.OP_UV)
    n1 = b.add(W.OP_FBM, [uv], ip=[2, 3], fp=[4.0, 2.0, 0.5])
    r2 = b.add(W.OP_RAMP, [n1], ip=[2], fp=[0.0, 1.0, 0, 0, 0.1, 0.2, 0.3, 0.9, 0.8, 0.7])
    v3 = b.add(W.OP_VORONOI, [uv], ip=[0, 5], fp=[6.0])
    m4 = b.add(W.OP_MUL, [r2, v3])
    nrm = b.add(W.OP_NORMAL)
    f6 = b.add(W.OP_FACING, [nrm], fp=[0.0, 0.0, 1.0])
    c7 = b.add(W.OP_CHECKER, [uv], fp=[8.0, 0.2, 0.2, 0.2, 0.9, 0.9, 0.9])
    x8 = b.add(W.OP_MIX, [m4, c7, f6])
    n9 = b.add(W.OP_FBM, [uv], ip=[1, 8], fp=[3.0, 2.0, 0.5])
    p10 = b.add(W.OP_POW, [n9], fp=[1.5])
    b.add(W.OP_MUL, [x8, p10])
    return b.build()


def g_nested():
    """0 UV; 1 FBM(0); 2 RAMP(1); 3 POSITION; 4 FBM(3); 5 MUL(2,4); 6 POW(2);
    7 ADD(6,0); 8 MIX(5,7,4) = output.  Node 2 feeds the SP node 5 and the UV node 6."""
    b = W.Builder()
    uv = b.add(W.OP_UV)
    n1 = b.add(W.OP_FBM, [uv], ip=[2, 3], fp=[4.0, 2.0, 0.5])
    r2 = b.add(W.OP_RAMP, [n1], ip=[2], fp=[0.0, 1.0, 0, 0, 0.1, 0.2, 0.3, 0.9, 0.8, 0.7])
    pos = b.add(W.OP_POSITION)
    f4 = b.add(W.OP_FBM, [pos], ip=[1, 2], fp=[1.0, 2.0, 0.5])
    m5 = b.add(W.OP_MUL, [r2, f4])
    p6 = b.add(W.OP_POW, [r2], fp=[2.0])
    a7 = b.add(W.OP_ADD, [p6, uv])
    b.add(W.OP_MIX, [m5, a7, f4])
    return b.build()


def test_tiny_material_single_root_is_output():
    cls, roots = O.analyze(W.material_tiny())
    assert list(cls) == [UV, UV, UV, CONST, CONST, UV, CONST, UV]
    assert list(roots) == [7]


def test_two_roots_and_min_size():
    cls, roots = O.analyze(g_two_roots())
    assert list(cls) == [UV, UV, UV, UV, UV, SP, SP, UV, SP, UV, UV, SP]
    assert list(roots) == [4, 10]           # checker 7 has a one-node sub-graph
    _, roots1 = O.analyze(g_two_roots(), min_root_nodes=1)
    assert list(roots1) == [4, 7, 10]
    _, roots5 = O.analyze(g_two_roots(), min_root_nodes=5)
    assert list(roots5) == []


def test_nested_roots():
    cls, roots = O.analyze(g_nested())
    assert list(cls) == [UV, UV, UV, SP, SP, SP, UV, UV, SP]
    assert list(roots) == [2, 7]            # 2 feeds SP node 5 and sits under root 7


def test_bare_uv_never_root_and_dead_nodes_ignored():
    b = W.Builder()
    uv = b.add(W.OP_UV)
    pos = b.add(W.OP_POSITION)
    dead_uv = b.add(W.OP_FBM, [uv], ip=[1, 1], fp=[2.0, 2.0, 0.5])
    dead_uv2 = b.add(W.OP_POW, [dead_uv], fp=[2.0])
    b.add(W.OP_MUL, [dead_uv2, pos])         # dead: not the output, nobody reads it
    b.add(W.OP_MIX, [uv, pos], fp=[0.5])     # output reads the bare UV node
    cls, roots = O.analyze(b.build(), min_root_nodes=1)
    assert list(roots) == []


def test_constant_and_sp_outputs():
    b = W.Builder()
    c0 = b.add(W.OP_CONST, fp=[0.1, 0.2, 0.3])
    c1 = b.add(W.OP_CONST, fp=[0.5, 0.5, 0.5])
    b.add(W.OP_MUL, [c0, c1])
    cls, roots = O.analyze(b.build(), min_root_nodes=1)
    assert list(cls) == [CONST, CONST, CONST] and list(roots) == []


def test_malformed_networks_rejected():
    good = W.material_tiny()
    assert O.validate(good)
    bad = good.copy()
    bad[5]["inp"][0] = 6                     # forward reference
    assert not O.validate(bad)
    bad = good.copy()
    bad[1]["ip"][0] = 0                      # zero octaves
    assert not O.validate(bad)
    bad = good.copy()
    bad[2]["fp"][1] = 0.9                    # ramp stops out of order (0, .9, .66, 1)
    assert not O.validate(bad)
    bad = good.copy()
    bad[0]["op"] = 99
    assert not O.validate(bad)
    bad = good.copy()
    bad[3]["inp"][0] = 0                     # a constant with an input
    assert not O.validate(bad)
    with pytest.raises(ValueError):
        O.analyze(bad)


def test_generated_networks_have_roots_and_sp_share():
    mats = W.random_materials(16, 20, 200, 0.2, seed=3)
    for m in mats:
        assert O.validate(m)
        cls, roots = O.analyze(m)
        assert len(roots) >= 1
        assert cls[-1] == SP
        sp_share = np.mean(cls == SP)
        assert 0.05 < sp_share < 0.5


def _checker_net(src_op, scale):
    b = W.Builder()
    uv = b.add(W.OP_UV)
    pos = b.add(W.OP_POSITION)
    src = {"uv": uv, "pos": pos,
           "affine": b.add(W.OP_UV_AFFINE, [uv], fp=[1.0, 0.1, -0.1, 1.0, 0.3, 0.7]),
           "offset": b.add(W.OP_UV_AFFINE, [uv], fp=[2.0, 0.0, 0.0, 2.0, 0.5, 0.0]),
           "scale2": b.add(W.OP_UV_AFFINE, [uv], fp=[4.0, 0.0, 0.0, 0.25, 0.0, 0.0]),
           "scale3": b.add(W.OP_UV_AFFINE, [uv], fp=[3.0, 0.0, 0.0, 1.0, 0.0, 0.0]),
           "posid": b.add(W.OP_UV_AFFINE, [pos], fp=[1.0, 0.0, 0.0, 1.0, 0.0, 0.0]),
           "noise": b.add(W.OP_FBM, [uv], ip=[2, 3], fp=[4.0, 2.0, 0.5])}[src_op]
    b.add(W.OP_CHECKER, [src], fp=[scale, 1, 0, 0, 0, 1, 0])
    return b.build()


@pytest.mark.parametrize("src,scale,ok", [
    ("uv", 8.0, True), ("uv", 1.0, True), ("pos", 0.5, True), ("uv", 2.0 ** 20, True),
    ("uv", 2.0 ** -20, True),
    ("uv", 3.0, False),            # x s rounds in FP32: a point near an edge may flip
    ("uv", 2.0 ** 21, False), ("uv", 2.0 ** -21, False), ("uv", -8.0, False), ("uv", 0.0, False),
    ("scale2", 8.0, True), ("posid", 4.0, True),   # per-axis power-of-two scalings are exact
    ("affine", 8.0, False),        # a rotated, offset image of UV is rounded in FP32
    ("offset", 8.0, False),        # so is an offset one
    ("scale3", 8.0, False),        # and one scaled by 3
    ("noise", 8.0, False),         # and a noise value
])
def test_checker_argument_must_be_exact(src, scale, ok):
    """The checker flips colour where x s or y s crosses an integer, so FP32 and FP64 can
    disagree by a whole colour near an edge unless x s is exact in both: x from the UV or
    position input itself and s a power of two (within a range where x s cannot leave
    FP32's exponent range for a UV or a position)."""
    assert O.validate(_checker_net(src, scale)) == ok


# ---- cost threshold of cacheable nodes --------------------------------------------------
def test_node_cost_model_hand_values():
    """The cost model of the interface: FP32 operations per evaluation, FMA = 2."""
    b = W.Builder()
    uv = b.add(W.OP_UV)
    rows = {
        "uv": (uv, 0), "const": (b.add(W.OP_CONST, fp=[1, 2, 3]), 0),
        "affine": (b.add(W.OP_UV_AFFINE, [uv], fp=[1, 0, 0, 1, 0, 0]), 8),
        "fbm1": (b.add(W.OP_FBM, [uv], ip=[1, 1], fp=[4.0, 2.0, 0.5]), 51),
        "fbm3": (b.add(W.OP_FBM, [uv], ip=[3, 1], fp=[4.0, 2.0, 0.5]), 145),
        "fbm16": (b.add(W.OP_FBM, [uv], ip=[16, 1], fp=[4.0, 2.0, 0.5]), 756),
        "voronoi": (b.add(W.OP_VORONOI, [uv], ip=[0, 1], fp=[4.0]), 99),
        "checker": (b.add(W.OP_CHECKER, [uv], fp=[4.0, 0, 0, 0, 1, 1, 1]), 4),
        "ramp": (b.add(W.OP_RAMP, [uv], ip=[2], fp=[0, 1, 0, 0, 0, 0, 0, 1, 1, 1]), 23),
        "mix": (b.add(W.OP_MIX, [uv, uv], fp=[0.5]), 17),
        "add": (b.add(W.OP_ADD, [uv, uv]), 9), "mul": (b.add(W.OP_MUL, [uv, uv]), 9),
        "pow": (b.add(W.OP_POW, [uv], fp=[2.0]), 18),
        "facing": (b.add(W.OP_FACING, [uv], fp=[0, 0, 1]), 8),
    }
    net = b.build()
    for name, (i, cost) in rows.items():
        assert O.node_cost(net[i]) == cost, name


def test_cost_threshold_two_roots():
    # root 4 = MUL(RAMP(FBM2(uv)), VORONOI(uv)): 98 + 23 + 99 + 9 = 229
    # root 10 = POW(FBM1(uv)): 51 + 18 = 69
    g = g_two_roots()
    for thr, want in ((0, [4, 10]), (69, [4, 10]), (70, [4]), (229, [4]), (230, [])):
        assert list(O.analyze(g, min_root_cost=thr)[1]) == want, thr


def test_cost_threshold_nested_roots():
    # root 2 = RAMP(FBM2(uv)): 98 + 23 = 121; root 7 = ADD(POW(node 2), uv): 121 + 18 + 9 = 148
    g = g_nested()
    for thr, want in ((121, [2, 7]), (122, [7]), (148, [7]), (149, [])):
        assert list(O.analyze(g, min_root_cost=thr)[1]) == want, thr


def test_cost_threshold_counts_a_shared_node_once():
    # 0 UV; 1 FBM1(0); 2 POW(1); 3 RAMP(1); 4 MUL(2, 3) = output: 51 + 18 + 23 + 9 = 101, the
    # noise counted once although both branches read it
    b = W.Builder()
    uv = b.add(W.OP_UV)
    n1 = b.add(W.OP_FBM, [uv], ip=[1, 2], fp=[4.0, 2.0, 0.5])
    p2 = b.add(W.OP_POW, [n1], fp=[2.0])
    r3 = b.add(W.OP_RAMP, [n1], ip=[2], fp=[0, 1, 0, 0, 0, 0, 0, 1, 1, 1])
    b.add(W.OP_MUL, [p2, r3])
    g = b.build()
    assert list(O.analyze(g, min_root_cost=101)[1]) == [4]
    assert list(O.analyze(g, min_root_cost=102)[1]) == []


def test_cost_threshold_zero_is_the_plain_rule_and_thresholds_only_remove_roots():
    mats = W.random_materials(24, 20, 200, 0.2, seed=13)
    for m in mats:
        base = set(O.analyze(m)[1].tolist())
        assert set(O.analyze(m, min_root_cost=0)[1].tolist()) == base
        prev = base
        for thr in (100, 300, 600, 1000):
            cur = set(O.analyze(m, min_root_cost=thr)[1].tolist())
            assert cur <= prev
            prev = cur


def test_cost_threshold_in_the_cache_emulation():
    """Nodes below the threshold are evaluated like any other node and never looked up:
    lookups = points x kept cacheable nodes; the first pass equals plain evaluation; a
    threshold above every node leaves a cache that never looks anything up."""
    g = g_two_roots()
    pts = W.points_uniform(300, seed=4)
    plain = np.array([O.eval_point_nocache(g, [pts[k][i] for k in ("u", "v", "px", "py", "pz", "nx", "ny", "nz")])
                      for i in range(300)]).T
    for thr, kept in ((0, 2), (70, 1), (230, 0)):
        c = O.Cache([g], 1 << 12, 4, min_root_cost=thr)
        assert list(c.roots(0)) == list(O.analyze(g, min_root_cost=thr)[1])
        r = c.run_batch(pts)
        assert np.abs(r["rgb"] - plain).max() <= 1e-12
        assert c.stats()["lookups"] == 300 * kept
        r2 = c.run_batch(pts)                        # same points: every kept node hits
        assert c.stats()["hits"] == 300 * kept
        assert np.abs(r2["rgb"] - plain).max() <= 1e-6
