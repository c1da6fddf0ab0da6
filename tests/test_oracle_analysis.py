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
