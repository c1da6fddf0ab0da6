"""GPU parity of the replacement policy by visibility class (PMC_REPLACE_VISIBILITY; the
prioritisation of directly visible shading points that Sec. 5 proposes) against the CPU
FP64 oracle.

Bit-exact: hits, table hash2 and classes per slot, counters (replaced included).  Outputs
and table values within max-abs 1e-4.  Every insert kernel is reached: bins resolved by a
warp (sparse), by a block (up to 2048 candidates), by cell ranges, and a single cell with
more candidates than the block's stage.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_07238_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
EXACT_STATS = ("lookups", "hits", "misses", "candidates", "inserted", "dropped_dup", "dropped_full", "replaced")
SCHEDULES = {"grouped": 0x0, "inline": 0x8, "unsorted": 0x28, "probe_inline": 0x40}


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_07238_gb300 import pmc
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return pmc


def _passes(n_passes, n, seed, n_mats=4, window=0.05):
    """Direct points (half of them) re-visit a small UV window; indirect ones land anywhere."""
    out = []
    for p in range(n_passes):
        pts = W.points_uniform(n, seed=seed + p, n_mats=n_mats)
        rng = np.random.Generator(np.random.PCG64([seed, p]))
        vis = rng.choice(4, size=n, p=[0.5, 0.25, 0.15, 0.10]).astype(np.uint8)
        d = vis == 0
        pts["u"][d] = (pts["u"][d] * window).astype(np.float32)
        pts["v"][d] = (pts["v"][d] * window).astype(np.float32)
        pts["vis"] = vis
        out.append(pts)
    return out


def _run(cache, P, part):
    n = len(part["u"])
    d = P.points_to_device(part)
    rgb = torch.full((3, n), -7.0, dtype=torch.float32, device="cuda")
    hits = torch.full((n,), -1, dtype=torch.int16, device="cuda")
    cache.eval_batch(d, rgb, hits)
    cache.sync()
    return rgb.cpu().numpy(), hits.cpu().numpy().astype(np.uint16)


def _compare(gpu, ref, P, part):
    g_rgb, g_hits = _run(gpu, P, part)
    r = ref.run_batch(part)
    assert float(np.abs(g_rgb - r["rgb"]).max()) <= TOL
    assert np.array_equal(g_hits, r["hits"])
    gs, rs = gpu.stats(), ref.stats()
    for k in EXACT_STATS:
        assert gs[k] == rs[k], (k, gs[k], rs[k])
    gh, gv = gpu.table()
    rh, rv = ref.table()
    assert np.array_equal(gh, rh)
    occ = rh != 0
    if occ.any():
        assert float(np.abs(gv[occ] - rv[occ]).max()) <= TOL
    assert np.array_equal(gpu.classes()[occ], ref.classes()[occ])
    return gs


@pytest.mark.parametrize("sched", list(SCHEDULES))
@pytest.mark.parametrize("n_cells,n_entries", [(16, 4), (64, 8), (7, 13)])
def test_replacement_matches_oracle(P, sched, n_cells, n_entries):
    mats = W.random_materials(4, 8, 30, 0.2, seed=3)
    gpu = P.Cache(mats, n_cells, n_entries, flags=P.PMC_REPLACE_VISIBILITY)
    gpu.set_schedule(SCHEDULES[sched])
    ref = O.Cache(mats, n_cells, n_entries, replacement=True)
    for pts in _passes(4, 1500, 17):
        _compare(gpu, ref, P, pts)
    assert gpu.stats()["replaced"] > 0


@pytest.mark.parametrize("n_cells,n_pts", [(4096, 3000), (256, 1200), (256, 9000)])
def test_bins_of_every_size(P, n_cells, n_pts):
    # 4096 cells: sparse bins (one warp each); 256 cells = one bin of a few hundred to 2048
    # candidates (one block) or more (cell ranges)
    mats = W.random_materials(2, 10, 40, 0.2, seed=7)
    gpu = P.Cache(mats, n_cells, 4, flags=P.PMC_REPLACE_VISIBILITY)
    ref = O.Cache(mats, n_cells, 4, replacement=True)
    for pts in _passes(3, n_pts, 29, n_mats=2, window=0.5):
        _compare(gpu, ref, P, pts)


def test_one_crowded_cell(P):
    # one cell, several thousand candidates: more than a block stages at once
    mat = W.material_tiny()
    gpu = P.Cache([mat], 1, 8, flags=P.PMC_REPLACE_VISIBILITY)
    ref = O.Cache([mat], 1, 8, replacement=True)
    rng = np.random.Generator(np.random.PCG64(5))
    for p in range(3):
        pts = W.points_uniform(3000, seed=40 + p)
        pts["vis"] = rng.integers(0, 6, 3000).astype(np.uint8)
        _compare(gpu, ref, P, pts)
    assert gpu.stats()["replaced"] > 0


def test_all_class_zero_is_keep_first(P):
    mats = W.random_materials(4, 8, 30, 0.2, seed=3)
    a = P.Cache(mats, 16, 4, flags=P.PMC_REPLACE_VISIBILITY)
    b = P.Cache(mats, 16, 4)
    for pts in _passes(3, 1500, 51):
        pts["vis"][:] = 0
        ra, rb = _run(a, P, pts), _run(b, P, pts)
        assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
    assert np.array_equal(a.table()[0], b.table()[0]) and np.array_equal(a.table()[1], b.table()[1])
    sa, sb = a.stats(), b.stats()
    assert sa["replaced"] == 0
    for k in EXACT_STATS[:-1]:
        assert sa[k] == sb[k], k


def test_path_traced_frame_band(P):
    # direct samples of a band of the 1080p frame plus two bounces of indirect points
    mats = W.random_materials(64, 20, 200, 0.2, seed=0)
    frame = W.Frame(W.FrameSpec(seed=0))
    # 2^13 cells: the direct points of the first pass leave room that indirect ones fill,
    # so later direct misses find full cells holding classes 1 and 2 (a smaller table is
    # filled by class 0 alone and never replaces)
    gpu = P.Cache(mats, 1 << 13, 8, flags=P.PMC_REPLACE_VISIBILITY)
    ref = O.Cache(mats, 1 << 13, 8, replacement=True)
    for p in range(3):
        _compare(gpu, ref, P, frame.points_paths(p, rows=(100, 104)))
    assert gpu.stats()["replaced"] > 0


def test_graph_noalloc_and_autotune_agree(P):
    mats = W.random_materials(4, 8, 30, 0.2, seed=3)
    passes = _passes(3, 1500, 61)
    eager = P.Cache(mats, 16, 4, flags=P.PMC_REPLACE_VISIBILITY)
    outs = []
    for pts in passes:
        outs.append(_run(eager, P, pts))
    # the same passes as one CUDA graph
    g = P.Cache(mats, 16, 4, flags=P.PMC_REPLACE_VISIBILITY)
    dev = [P.points_to_device(p) for p in passes]
    rgbs = [torch.empty((3, 1500), dtype=torch.float32, device="cuda") for _ in passes]
    hits = [torch.empty(1500, dtype=torch.int16, device="cuda") for _ in passes]
    graph = g.graph(dev, rgbs, hits, reset=True)
    graph.launch()
    g.sync()
    for k in range(len(passes)):
        assert np.array_equal(rgbs[k].cpu().numpy(), outs[k][0])
        assert np.array_equal(hits[k].cpu().numpy().astype(np.uint16), outs[k][1])
    graph.close()
    assert np.array_equal(g.table()[0], eager.table()[0]) and np.array_equal(g.classes(), eager.classes())
    # the fixed-scratch entry point
    na = P.Cache(mats, 16, 4, flags=P.PMC_REPLACE_VISIBILITY)
    for k, d in enumerate(dev):
        rgb = torch.empty((3, 1500), dtype=torch.float32, device="cuda")
        h = torch.empty(1500, dtype=torch.int16, device="cuda")
        na.eval_batch_noalloc(d, rgb, h)
        na.sync()
        assert np.array_equal(rgb.cpu().numpy(), outs[k][0])
    assert np.array_equal(na.table()[0], eager.table()[0]) and np.array_equal(na.classes(), eager.classes())
    # autotuning leaves table, classes and counters as it found them
    h0, c0, s0 = eager.table()[0].copy(), eager.classes().copy(), eager.stats()
    tune = eager.autotune(dev[0], reps=2)
    assert all(t["flags"] & P.PMC_INSERT_ROUNDS == 0 for t in tune["tried"])
    assert np.array_equal(eager.table()[0], h0) and np.array_equal(eager.classes(), c0)
    assert eager.stats() == s0
