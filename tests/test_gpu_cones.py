"""GPU parity of the per-point mip level from ray-cone gradients (Sec. 3.1, Eq. 1).

Bit-exact: the level of every gradient pair, and with it the descriptors, hit/miss of
every (point, cacheable node), counters and table hash2 of whole passes.  Floating point:
outputs and table values within max-abs 1e-4 of the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_07238_gb300 import workload as W

from .test_gpu_parity import MODES, _compare_pass, _compare_tables, _run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_07238_gb300 import pmc
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return pmc


def _gradients(n, seed):
    rng = np.random.default_rng(seed)
    mag = np.exp2(rng.uniform(-16.0, 2.0, (2, n)))
    th = rng.uniform(0.0, 2.0 * np.pi, n)
    b = np.exp2(rng.uniform(0.0, 2.0, n))
    g = np.stack([mag[0] * np.cos(th), mag[0] * np.sin(th), -mag[1] * b * np.sin(th), mag[1] * b * np.cos(th)])
    g = g.astype(np.float32)
    # edge cases: zero, subnormal, infinite, NaN, exact powers of four and their neighbours
    e = np.float32(2.0 ** -10)
    edge = [(0, 0, 0, 0), (1e-40, 0, 0, 1e-40), (np.inf, 0, 1e-3, 0), (np.inf, 0, np.inf, 0),
            (np.nan, 0, 0, 1e-3), (e, 0, 0, e), (np.nextafter(e, np.float32(1)), 0, 0, 1),
            (np.nextafter(e, np.float32(0)), 0, 0, 1), (1, 0, 0, 1), (2, 0, 0, 3), (-e, 0, 0, -e)]
    g[:, :len(edge)] = np.array(edge, dtype=np.float32).T
    return g


@pytest.mark.parametrize("offset", [0, 2, -3, 13, -13])
def test_levels_bit_exact(P, offset):
    g = _gradients(20000, seed=offset + 20)
    dg = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in g]
    lv = P.compute_levels(*dg, offset=offset).cpu().numpy()
    ref = np.array([O.level(*(float(x) for x in g[:, i]), offset) for i in range(g.shape[1])])
    assert np.array_equal(lv, ref)


def test_bad_offset_and_partial_gradients_rejected(P):
    mats = [W.material_tiny()]
    with pytest.raises(P.PmcError):
        P.Cache(mats, 64, 8, level_offset=14)
    with pytest.raises(P.PmcError):
        P.compute_levels(*[torch.zeros(4, device="cuda")] * 4, offset=-14)
    c = P.Cache(mats, 64, 8)
    pts = P.points_to_device(W.points_uniform(64, seed=1))
    pts["g1u"] = torch.zeros(64, device="cuda")   # one of the four: invalid
    rgb = torch.empty((3, 64), device="cuda")
    with pytest.raises(P.PmcError):
        c.eval_batch(pts, rgb)


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("n_cells,n_entries,offset", [(1 << 21, 8, 0), (1 << 10, 8, -1), (97, 32, 1)])
def test_frame_band_parity_cones(P, n_cells, n_entries, offset, mode):
    spec = W.FrameSpec(width=1920, height=1080, n_mats=64, seed=2)
    frame = W.Frame(spec)
    mats = W.random_materials(64, 20, 200, 0.2, seed=2)
    gpu = P.Cache(mats, n_cells, n_entries, flags=MODES[mode], level_offset=offset)
    ref = O.Cache(mats, n_cells, n_entries, level_offset=offset)
    rows = (0, 9) if n_cells >= 1024 else (0, 3)
    for p in range(3):
        _compare_pass(gpu, ref, P, frame.points(p, rows=rows, cones=True))
    _compare_tables(gpu, ref)


def test_uniform_footprint_equals_fixed_level(P):
    # every footprint gives level 9: the same results as a cache fixed at level 9, bit for bit
    frame = W.Frame(W.FrameSpec(seed=4))
    mats = W.random_materials(64, 20, 200, 0.2, seed=4)
    a = P.Cache(mats, 1 << 12, 8, uv_level=9)
    b = P.Cache(mats, 1 << 12, 8, uv_level=2)
    g = np.float32(2.0 ** -9)
    for p in range(3):
        part = frame.points(p, rows=(100, 110))
        n = len(part["u"])
        q = dict(part, g1u=np.full(n, g), g1v=np.zeros(n, np.float32), g2u=np.zeros(n, np.float32),
                 g2v=np.full(n, g))
        ra, ha = _run_gpu(a, P, part)
        rb, hb = _run_gpu(b, P, q)
        assert np.array_equal(ra, rb) and np.array_equal(ha, hb)
    assert np.array_equal(a.table()[0], b.table()[0])
    assert a.stats() == b.stats()


def test_host_entry_and_graph_with_cones(P):
    frame = W.Frame(W.FrameSpec(seed=6))
    mats = W.random_materials(64, 20, 200, 0.2, seed=6)
    parts = [frame.points(p, rows=(40, 48), cones=True) for p in range(3)]
    dev = P.Cache(mats, 1 << 14, 8, level_offset=1)
    host = P.Cache(mats, 1 << 14, 8, level_offset=1)
    graph_cache = P.Cache(mats, 1 << 14, 8, level_offset=1)
    n = len(parts[0]["u"])
    dparts = [P.points_to_device(q) for q in parts]
    outs = [torch.empty((3, n), device="cuda") for _ in parts]
    g = graph_cache.graph(dparts, outs)
    g.launch()
    graph_cache.sync()
    for k, q in enumerate(parts):
        r1, h1 = _run_gpu(dev, P, q)
        rgb = np.zeros((3, n), np.float32)
        hits = np.zeros(n, np.uint16)
        host.eval_batch_host(q, rgb, hits)
        assert np.array_equal(r1, rgb) and np.array_equal(h1, hits)
        assert np.array_equal(r1, outs[k].cpu().numpy())
    g.close()
    assert np.array_equal(dev.table()[0], host.table()[0])
    assert np.array_equal(dev.table()[0], graph_cache.table()[0])


def test_noalloc_with_cones_matches(P):
    frame = W.Frame(W.FrameSpec(width=256, height=64, n_mats=8, seed=7))
    mats = W.random_materials(8, 20, 60, 0.2, seed=7)
    a = P.Cache(mats, 4096, 8)
    b = P.Cache(mats, 4096, 8)
    for p in range(3):
        part = frame.points(p, rows=(0, 8), cones=True)
        d = P.points_to_device(part)
        n = len(part["u"])
        ra, rb = torch.empty((3, n), device="cuda"), torch.empty((3, n), device="cuda")
        ha = torch.empty(n, dtype=torch.int16, device="cuda")
        hb = torch.empty(n, dtype=torch.int16, device="cuda")
        a.eval_batch(d, ra, ha)
        b.eval_batch_noalloc(d, rb, hb)
        torch.cuda.synchronize()
        assert torch.equal(ra, rb) and torch.equal(ha, hb)
    assert np.array_equal(a.table()[0], b.table()[0])
