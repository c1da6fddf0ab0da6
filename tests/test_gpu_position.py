"""GPU parity of the world-position descriptor (PMC_POSITION_DESCRIPTOR; Sec. 3.1 names a
world-space position as a further descriptor, Sec. 5 lists it as future work) against the
CPU FP64 oracle.

Bit-exact: hits and hit masks per (point, cacheable node), table hash2, counters.  Outputs
and table values within max-abs 1e-4.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_07238_gb300 import workload as W

from .test_oracle_position import _voxel_checker, g_position

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
EXACT_STATS = ("lookups", "hits", "misses", "candidates", "inserted", "dropped_dup", "dropped_full")
SCHEDULES = {"grouped": 0x0, "inline": 0x8, "unsorted": 0x28, "probe_inline": 0x40, "rounds": 0x10}


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_07238_gb300 import pmc
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return pmc


def _run(cache, P, part, noalloc=False):
    n = len(part["u"])
    d = P.points_to_device(part)
    rgb = torch.full((3, n), -7.0, dtype=torch.float32, device="cuda")
    hits = torch.full((n,), -1, dtype=torch.int16, device="cuda")
    (cache.eval_batch_noalloc if noalloc else cache.eval_batch)(d, rgb, hits)
    cache.sync()
    return rgb.cpu().numpy(), hits.cpu().numpy().astype(np.uint16)


def _masks(ref, part, r):
    n = len(part["u"])
    masks = np.zeros(n, dtype=np.uint64)
    k = 0
    for i in range(n):
        nr = ref.n_roots(int(part["mat"][i]))
        for j in range(nr):
            if r["hit"][k + j] and j < 64:
                masks[i] |= np.uint64(1) << np.uint64(j)
        k += nr
    return masks


def _compare(gpu, ref, P, part, masks=False):
    g_rgb, g_hits = _run(gpu, P, part)
    r = ref.run_batch(part, probes=masks)
    assert float(np.abs(g_rgb - r["rgb"]).max()) <= TOL
    assert np.array_equal(g_hits, r["hits"])
    if masks:
        assert np.array_equal(gpu.last_hit_masks(len(part["u"])), _masks(ref, part, r))
    gs, rs = gpu.stats(), ref.stats()
    for k in EXACT_STATS:
        assert gs[k] == rs[k], (k, gs[k], rs[k])
    gh, gv = gpu.table()
    rh, rv = ref.table()
    assert np.array_equal(gh, rh)
    occ = rh != 0
    if occ.any():
        assert float(np.abs(gv[occ] - rv[occ]).max()) <= TOL


def _local_points(n, seed, n_mats, span=0.25):
    """Points whose positions stay in a small box, so that position voxels repeat."""
    pts = W.points_uniform(n, seed=seed, n_mats=n_mats)
    for k in ("px", "py", "pz"):
        pts[k] = (pts[k] * (span / 4.0)).astype(np.float32)
    return pts


@pytest.mark.parametrize("sched", list(SCHEDULES))
def test_position_roots_match_oracle(P, sched):
    mats = W.random_materials(5, 10, 80, 0.3, seed=21) + [g_position()]
    level = 5
    gpu = P.Cache(mats, 256, 8, flags=P.PMC_POSITION_DESCRIPTOR, pos_level=level, min_root_nodes=1)
    gpu.set_schedule(SCHEDULES[sched])
    ref = O.Cache(mats, 256, 8, min_root_nodes=1, pos_level=level)
    for m in range(len(mats)):
        assert gpu.material_info(m)["roots"].tolist() == ref.roots(m).tolist()
    for p in range(4):
        _compare(gpu, ref, P, _local_points(2000, 300 + p, len(mats)), masks=sched in ("grouped", "inline", "rounds"))
    assert gpu.stats()["hits"] > 0


def test_voxel_constant_subgraph_matches_uncached_exactly(P):
    L = 1
    mat = _voxel_checker(L)
    gpu = P.Cache([mat], 4096, 8, flags=P.PMC_POSITION_DESCRIPTOR, pos_level=L)
    plain = P.Cache([mat], 4096, 8, flags=P.PMC_CACHE_OFF)
    hits = 0
    for p in range(4):
        pts = W.points_uniform(4000, seed=70 + p)
        a, b = _run(gpu, P, pts), _run(plain, P, pts)
        assert np.array_equal(a[0], b[0])
        hits += int(a[1].sum())
    assert hits > 2000


def test_frame_band_with_position_descriptor(P):
    mats = W.random_materials(64, 20, 200, 0.2, seed=0)
    frame = W.Frame(W.FrameSpec(seed=0))
    gpu = P.Cache(mats, 1 << 12, 8, flags=P.PMC_POSITION_DESCRIPTOR, pos_level=6, min_root_nodes=1)
    ref = O.Cache(mats, 1 << 12, 8, min_root_nodes=1, pos_level=6)
    for p in range(3):
        _compare(gpu, ref, P, frame.points(p, rows=(200, 204)), masks=True)
    assert gpu.stats()["hits"] > 0


def test_noalloc_and_replacement_with_positions(P):
    mats = W.random_materials(4, 10, 60, 0.3, seed=23)
    flags = P.PMC_POSITION_DESCRIPTOR | P.PMC_REPLACE_VISIBILITY
    a = P.Cache(mats, 64, 4, flags=flags, pos_level=4, min_root_nodes=1)
    b = P.Cache(mats, 64, 4, flags=flags, pos_level=4, min_root_nodes=1)
    ref = O.Cache(mats, 64, 4, min_root_nodes=1, pos_level=4, replacement=True)
    rng = np.random.Generator(np.random.PCG64(9))
    for p in range(3):
        pts = _local_points(1500, 500 + p, 4)
        pts["vis"] = rng.integers(0, 3, 1500).astype(np.uint8)
        ra, rb = _run(a, P, pts), _run(b, P, pts, noalloc=True)
        r = ref.run_batch(pts)
        assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
        assert float(np.abs(ra[0] - r["rgb"]).max()) <= TOL and np.array_equal(ra[1], r["hits"])
    assert np.array_equal(a.table()[0], ref.table()[0]) and np.array_equal(b.table()[0], ref.table()[0])
    assert a.stats()["replaced"] == ref.stats()["replaced"]
