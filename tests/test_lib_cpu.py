"""CPU-side checks of the C-ABI library: it loads, exports what include/pmc.h declares,
agrees with the oracle on the IR numbering and on which nodes are cacheable.  No call
here touches a GPU."""
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_07238_gb300 import build as B
from paper_2305_07238_gb300 import pmc as P
from paper_2305_07238_gb300 import workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.load()


def _declared(header):
    text = open(os.path.join(ROOT, header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pmc_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = _declared("include/pmc.h")
    assert "pmc_eval_batch" in names and "pmc_create_cache" in names and "pmc_stats" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(P.EXPORTED) <= set(names)


def test_binding_flag_values_match_the_header():
    """Every PMC_* flag or limit the Python binding names has the header's value."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include/pmc.h")).read(), flags=re.S)
    header = {m.group(1): int(m.group(2), 0) for m in re.finditer(r"#define\s+(PMC_[A-Z_0-9]+)\s+(0x[0-9A-Fa-f]+|\d+)u?\b", text)}
    named = {k: v for k, v in vars(P).items() if k.startswith("PMC_") and isinstance(v, int)}
    assert {"PMC_CACHE_OFF", "PMC_INSERT_ROUNDS", "PMC_ONE_POINT", "PMC_INSERT_BINNED"} <= set(named)
    for k, v in named.items():
        if k in header:
            assert header[k] == v, k


def _enum(path, prefix):
    text = open(os.path.join(ROOT, path)).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(rf"\b{prefix}([A-Z_]+)\s*=\s*(\d+)", text)}


def test_ir_numbering_agrees_everywhere():
    lib_ops = _enum("include/pmc.h", "PMC_OP_")
    orc_ops = _enum("oracle/pmc_oracle.h", "ORC_")
    for code, name in W.OP_NAMES.items():
        assert lib_ops[name] == code, name
        assert orc_ops[name] == code, name
    assert _enum("include/pmc.h", "PMC_")["NUM_OPS"] == W.NUM_OPS == orc_ops["NUM_OPS"]


def test_cacheable_nodes_match_oracle(lib):
    mats = W.random_materials(40, 5, 400, 0.25, seed=11) + [W.material_tiny()]
    for m in mats:
        for mr in (1, 2, 3):
            got = P.analyze_material(m, min_root_nodes=mr)
            _, exp = O.analyze(m, min_root_nodes=mr)
            assert np.array_equal(got["roots"], exp)
            assert got["n_slots"] >= 1 and got["n_instr"] >= 1


def test_hand_built_networks_roots(lib):
    from .test_oracle_analysis import g_nested, g_two_roots
    assert list(P.analyze_material(g_two_roots())["roots"]) == [4, 10]
    assert list(P.analyze_material(g_nested())["roots"]) == [2, 7]
    assert list(P.analyze_material(W.material_tiny())["roots"]) == [7]


def test_malformed_networks_rejected(lib):
    good = W.material_tiny()
    for mutate in (lambda b: b[5]["inp"].__setitem__(0, 6), lambda b: b[1]["ip"].__setitem__(0, 0),
                   lambda b: b[2]["fp"].__setitem__(1, 0.9), lambda b: b[0].__setitem__("op", 99),
                   lambda b: b[3]["inp"].__setitem__(0, 0)):
        bad = good.copy()
        mutate(bad)
        with pytest.raises(P.PmcError) as ei:
            P.analyze_material(bad)
        assert ei.value.status == P.PMC_ERR_INVALID_ARG


def test_constant_folding_keeps_node_ids(lib):
    # MUL(CONST, CONST) folds; the cacheable node above it keeps its original ID.
    b = W.Builder()
    uv = b.add(W.OP_UV)
    c1 = b.add(W.OP_CONST, fp=[0.5, 0.5, 0.5])
    c2 = b.add(W.OP_CONST, fp=[0.25, 1.0, 0.0])
    k = b.add(W.OP_MUL, [c1, c2])
    n = b.add(W.OP_FBM, [uv], ip=[2, 1], fp=[4.0, 2.0, 0.5])
    r = b.add(W.OP_MUL, [n, k])
    nrm = b.add(W.OP_NORMAL)
    f = b.add(W.OP_FACING, [nrm], fp=[0, 0, 1])
    b.add(W.OP_MIX, [r, k, f])
    m = b.build()
    info = P.analyze_material(m)
    assert list(info["roots"]) == list(O.analyze(m)[1]) == [5]


def test_generated_programs_are_small(lib):
    mats = W.random_materials(64, 20, 200, 0.2, seed=0)
    slots = [P.analyze_material(m)["n_slots"] for m in mats]
    assert max(slots) <= 64


def test_replacement_rejects_concurrent_and_round_inserts(lib):
    # checked before any device work: the replacement policy needs the per-cell insert
    for extra in (P.PMC_ALG1, P.PMC_INSERT_ROUNDS):
        with pytest.raises(P.PmcError) as ei:
            P.Cache([W.material_tiny()], 64, 4, flags=P.PMC_REPLACE_VISIBILITY | extra)
        assert ei.value.status == P.PMC_ERR_INVALID_ARG


def test_position_descriptor_roots_match_oracle(lib):
    from .test_oracle_position import g_position
    mats = W.random_materials(30, 5, 400, 0.3, seed=12) + [g_position()]
    for m in mats:
        for mr in (1, 2):
            got = P.analyze_material(m, min_root_nodes=mr, flags=P.PMC_POSITION_DESCRIPTOR)
            _, roots, kinds = O.analyze(m, min_root_nodes=mr, pos_desc=True, kinds=True)
            assert np.array_equal(got["roots"], roots)
            assert np.array_equal(got["kinds"], kinds)
    assert list(P.analyze_material(g_position(), flags=P.PMC_POSITION_DESCRIPTOR)["kinds"]) == [2, 1, 2]


def test_cast_rays_rejects_bad_arguments(lib):
    # checked before any device work
    import ctypes as C
    sc = W.Scene(W.SceneSpec(width=16, height=8))
    cam = sc.camera
    mk = lambda w, h: P._Camera((C.c_float * 3)(*cam["eye"]), (C.c_float * 3)(*cam["fwd"]),
                                (C.c_float * 3)(*cam["right"]), (C.c_float * 3)(*cam["up"]),
                                float(cam["tan_half_y"]), w, h)
    hits = P._RayHits()   # no output planes
    objs = np.ascontiguousarray(sc.objects)
    call = lambda o, n, c, r0, r1: lib.pmc_cast_rays(o.ctypes.data, n, C.byref(c), r0, r1, 0, 0, C.byref(hits), None)
    assert call(objs, 0, mk(16, 8), 0, 8) == P.PMC_ERR_INVALID_ARG                 # no objects
    assert call(objs, 65, mk(16, 8), 0, 8) == P.PMC_ERR_INVALID_ARG                # too many
    assert call(objs, len(objs), mk(0, 8), 0, 0) == P.PMC_ERR_INVALID_ARG          # empty image
    assert call(objs, len(objs), mk(16, 8), 4, 9) == P.PMC_ERR_INVALID_ARG         # rows outside
    assert call(objs, len(objs), mk(16, 8), 0, 8) == P.PMC_ERR_INVALID_ARG         # no outputs
    bad = objs.copy()
    bad[7]["p"][3] = 0.0                                                            # zero radius
    assert call(bad, len(bad), mk(16, 8), 0, 0) == P.PMC_ERR_INVALID_ARG
    assert call(objs, len(objs), mk(16, 8), 3, 3) == 0                              # nothing to do


def test_checker_exactness_rule_matches_oracle(lib):
    from .test_oracle_analysis import _checker_net
    for src, scale in (("uv", 8.0), ("pos", 0.5), ("uv", 3.0), ("uv", 2.0 ** 21), ("affine", 8.0),
                       ("noise", 8.0), ("uv", 2.0 ** -20), ("scale2", 8.0), ("posid", 4.0), ("offset", 8.0),
                       ("scale3", 8.0)):
        net = _checker_net(src, scale)
        if O.validate(net):
            P.analyze_material(net)
        else:
            with pytest.raises(P.PmcError) as ei:
                P.analyze_material(net)
            assert ei.value.status == P.PMC_ERR_INVALID_ARG


def test_node_cost_model_matches_oracle(lib):
    for m in W.random_materials(8, 20, 200, 0.2, seed=5) + [W.material_tiny()]:
        for row in m:
            assert P.node_cost(row) == O.node_cost(row)


def test_cost_threshold_roots_match_oracle(lib):
    mats = W.random_materials(16, 20, 200, 0.2, seed=9)
    for m in mats:
        for thr in (0, 100, 300, 600):
            got = P.analyze_material(m, min_root_cost=thr)["roots"]
            want = O.analyze(m, min_root_cost=thr)[1]
            assert list(got) == list(want), thr
