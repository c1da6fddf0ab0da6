"""GPU checks of the paper's concurrent update (PMC_ALG1; Sec. 3.3, Alg. 1).

With several shading points in flight the table depends on thread timing, so whole
passes are checked by what must hold in any interleaving: a keep-first table (occupied
slots form a prefix of their cell, hash2 unique per cell), every occupied (cell, hash2)
one of the batch's descriptors, counters that add up.  Where nothing can race the result
is unique and compared with the serialised oracle: batches of one shading point, and
cacheable nodes whose value is exact in FP32 (a checker of stored colours), whose table
is the same set of entries per cell in any interleaving, with bit-identical RGB9E5 codes.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_07238_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEP = 2.0 ** -8   # one RGB9E5 mantissa step for values in [0.5, 1]


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
    rgb = torch.empty((3, n), dtype=torch.float32, device="cuda")
    hits = torch.empty(n, dtype=torch.int16, device="cuda")
    (cache.eval_batch_noalloc if noalloc else cache.eval_batch)(d, rgb, hits)
    cache.sync()
    return rgb.cpu().numpy(), hits.cpu().numpy().astype(np.uint16)


def _keep_first(cache, st):
    h2, _ = cache.table()
    cells = h2.reshape(cache.n_cells, cache.n_entries)
    occ = cells != 0
    k = occ.sum(axis=1)
    prefix = np.arange(cache.n_entries)[None, :] < k[:, None]
    assert np.array_equal(occ, prefix)
    for row, kk in zip(cells, k):
        assert len(set(row[:kk].tolist())) == kk
    assert st["inserted"] == int(occ.sum())
    assert st["hits"] + st["misses"] == st["lookups"]
    assert st["candidates"] == st["inserted"] + st["dropped_dup"] + st["dropped_full"] + st["dropped_race"]


def _checker_materials(k, seed):
    rng = np.random.default_rng(seed)
    mats = []
    for _ in range(k):
        b = W.Builder()
        uv = b.add(W.OP_UV)
        s = float(2.0 ** rng.integers(1, 5))
        aff = b.add(W.OP_UV_AFFINE, [uv], fp=[s, 0.0, 0.0, s, 0.0, 0.0])
        col = rng.random(6).astype(np.float32)
        b.add(W.OP_CHECKER, [aff], fp=[1.0] + col.tolist())
        mats.append(b.build())
    return mats


def _cell_sets(cache):
    h2, rgb = cache.table()
    cells = h2.reshape(cache.n_cells, cache.n_entries)
    vals = rgb.reshape(cache.n_cells, cache.n_entries, 3)
    out = {}
    for c in np.nonzero(cells[:, 0])[0]:
        k = int((cells[c] != 0).sum())
        order = np.argsort(cells[c, :k])
        out[int(c)] = (cells[c, :k][order].tolist(), vals[c, :k][order].tolist())
    return out


@pytest.mark.parametrize("flags", [0, 0x20])   # grouped, unsorted
def test_exact_values_give_a_unique_table(P, flags):
    # two halves of the points, then all of them again: a key whose compare-and-swap lost a
    # race to another key of its cell is inserted by the last pass
    mats = _checker_materials(16, seed=3)
    pts = W.points_uniform(60000, seed=3, n_mats=16)
    gpu = P.Cache(mats, 1 << 16, 8, flags=P.PMC_ALG1 | flags)
    ref = O.Cache(mats, 1 << 16, 8, alg1=True)
    plain = O.Cache(mats, 1 << 16, 8, cache_off=True)
    parts = [W.slice_points(pts, 0, 30000), W.slice_points(pts, 30000, 60000), pts]
    for part in parts:
        races = gpu.stats()["dropped_race"]
        g_rgb, g_hits = _run(gpu, P, part)
        ref.run_batch(part)
        exact = np.float32(plain.run_batch(part)["rgb"])   # the checker colour: a miss returns it
        enc = np.array([O.rgb9e5_decode(O.rgb9e5_encode(*map(float, exact[:, i]))) for i in range(len(part["u"]))]).T
        ok = np.all(g_rgb == exact, axis=0) | np.all(g_rgb == enc, axis=0)
        assert ok.all()
        assert np.all(g_hits <= 1)
        _keep_first(gpu, gpu.stats())
        races = gpu.stats()["dropped_race"] - races
    assert gpu.stats()["dropped_full"] == 0 == ref.stats()["dropped_full"]
    g, r = _cell_sets(gpu), _cell_sets(ref)
    for c, (h, v) in g.items():   # every entry is one of the oracle's, with the same code
        rh, rv = r[c]
        for x, y in zip(h, v):
            assert x in rh and rv[rh.index(x)] == y
    if races == 0:
        assert g == r


def test_one_point_batches_match_the_serialised_oracle(P):
    mats = W.random_materials(4, 12, 50, 0.2, seed=8)
    pts = W.points_uniform(240, seed=8, n_mats=4)
    pts["u"] = (np.floor(pts["u"] * 32) / 32 + 1 / 64).astype(np.float32)   # texels repeat
    pts["v"] = (np.floor(pts["v"] * 32) / 32 + 1 / 64).astype(np.float32)
    gpu = P.Cache(mats, 61, 4, flags=P.PMC_ALG1)
    ref = O.Cache(mats, 61, 4, alg1=True)
    for i in range(240):
        part = W.slice_points(pts, i, i + 1)
        g_rgb, g_hits = _run(gpu, P, part)
        r = ref.run_batch(part)
        assert np.array_equal(g_hits, r["hits"])
        assert float(np.abs(g_rgb - r["rgb"]).max()) <= 2 * STEP + 1e-4
    gh, gv = gpu.table()
    rh, rv = ref.table()
    assert np.array_equal(gh, rh)
    occ = rh != 0
    assert float(np.abs(gv[occ] - rv[occ]).max()) <= STEP + 1e-4
    gs, rs = gpu.stats(), ref.stats()
    for k in ("lookups", "hits", "misses", "candidates", "inserted", "dropped_dup", "dropped_full"):
        assert gs[k] == rs[k], k
    assert gs["dropped_race"] == 0


@pytest.mark.parametrize("flags,cones,noalloc", [(0, False, False), (0x20, False, False), (0, True, False),
                                                 (0, False, True)])
def test_frame_passes_keep_first_table(P, flags, cones, noalloc):
    frame = W.Frame(W.FrameSpec(seed=5))
    mats = W.random_materials(64, 20, 200, 0.2, seed=5)
    rows = (0, 4) if noalloc else (0, 24)
    gpu = P.Cache(mats, 1 << 10 if noalloc else 1 << 14, 8, flags=P.PMC_ALG1 | flags)
    ref = O.Cache(mats, 1 << 10 if noalloc else 1 << 14, 8)
    seen = set()
    for p in range(3):
        part = frame.points(p, rows=rows, cones=cones)
        if noalloc:
            part = W.slice_points(part, 0, 2000)   # within the fixed scratch (16 probes a point)
        _run(gpu, P, part, noalloc=noalloc)
        r = ref.run_batch(part, probes=True)
        seen |= set(zip(r["cell"].tolist(), r["h2"].tolist()))
        _keep_first(gpu, gpu.stats())
    h2, _ = gpu.table()
    cells = h2.reshape(gpu.n_cells, gpu.n_entries)
    occupied = {(int(c), int(h)) for c, row in enumerate(cells) for h in row if h}
    assert occupied <= seen
    st = gpu.stats()
    assert st["hits"] > 0 and st["inserted"] > 0
    with pytest.raises(P.PmcError):
        gpu.last_hit_masks(len(part["u"]))
