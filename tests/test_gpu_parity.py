"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Bit-exact: descriptors, cells, hash2, hit/miss of every (point, cacheable node), table
hash2 per slot, counters.  Floating point: every output and table value within max-abs
1e-4 of the FP64 oracle (FP32 evaluation of bounded networks; see the design notes for
the derivation of the tolerance).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_07238_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
EXACT_STATS = ("lookups", "hits", "misses", "candidates", "inserted", "dropped_dup", "dropped_full")


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_07238_gb300 import pmc
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return pmc


def _run_gpu(cache, P, part):
    n = len(part["u"])
    d = P.points_to_device(part)
    rgb = torch.full((3, max(n, 1)), -7.0, dtype=torch.float32, device="cuda")[:, :n]
    rgb = rgb.contiguous()
    hits = torch.full((max(n, 1),), -1, dtype=torch.int16, device="cuda")[:n]
    cache.eval_batch(d, rgb, hits)
    cache.sync()
    return rgb.cpu().numpy(), hits.cpu().numpy().astype(np.uint16)


def _oracle_masks(ref, part, r):
    n = len(part["u"])
    masks = np.zeros(n, dtype=np.uint64)
    k = 0
    for i in range(n):
        m = int(part["mat"][i])
        nr = ref.n_roots(m) if m < len(ref._mats) else 0
        for j in range(nr):
            if r["hit"][k + j] and j < 64:
                masks[i] |= np.uint64(1) << np.uint64(j)
        k += nr
    return masks


def _compare_pass(gpu, ref, P, part, check_masks=True):
    g_rgb, g_hits = _run_gpu(gpu, P, part)
    r = ref.run_batch(part, probes=check_masks)
    err = float(np.abs(g_rgb - r["rgb"]).max()) if len(part["u"]) else 0.0
    assert err <= TOL, f"max-abs error {err}"
    assert np.array_equal(g_hits, r["hits"])
    if check_masks and not ref.off and not gpu.flags & 0x60:   # these schedules keep no probe records
        assert np.array_equal(gpu.last_hit_masks(len(part["u"])), _oracle_masks(ref, part, r))
    gs, rs = gpu.stats(), ref.stats()
    for k in EXACT_STATS:
        assert gs[k] == rs[k], (k, gs[k], rs[k])
    return err


def _compare_tables(gpu, ref):
    gh, gv = gpu.table()
    rh, rv = ref.table()
    assert np.array_equal(gh, rh)
    occ = rh != 0
    if occ.any():
        assert float(np.abs(gv[occ] - rv[occ]).max()) <= TOL
    assert np.all(gv[~occ] == 0)


# ---- descriptors and addressing -----------------------------------------------------------
@pytest.mark.parametrize("n_cells", [1, 10, 8192, 12345, 1 << 21, 10**7, (1 << 32) - 5])
@pytest.mark.parametrize("level", [0, 10, 13])
def test_keys_cells_hash2_bit_exact(P, n_cells, level):
    rng = np.random.default_rng(level + n_cells % 1000)
    n = 5000
    mat = rng.integers(0, 65536, n).astype(np.uint32)
    node = rng.integers(0, 65536, n).astype(np.uint32)
    u = rng.uniform(-0.2, 1.2, n).astype(np.float32)
    v = rng.uniform(-0.2, 1.2, n).astype(np.float32)
    edge = np.array([0.0, 1.0, 0.5, 511 / 1024, np.nextafter(np.float32(0.5), np.float32(0)), -0.0,
                     np.nan, 1.0 - 2**-24], dtype=np.float32)
    u[: len(edge)] = edge
    v[-len(edge):] = edge
    t = lambda a: torch.from_numpy(a.view(np.int32) if a.dtype == np.uint32 else a).cuda()
    key, cell, h2 = P.compute_keys(t(mat), t(node), t(u), t(v), level, n_cells)
    torch.cuda.synchronize()
    key = key.cpu().numpy().view(np.uint64)
    cell = cell.cpu().numpy().view(np.uint64)
    h2 = h2.cpu().numpy().view(np.uint32)
    for i in range(n):
        k = O.key(int(mat[i]), int(node[i]), level, float(u[i]), float(v[i]))
        assert int(key[i]) == k
        assert int(cell[i]) == O.hash1(k) % n_cells
        assert int(h2[i]) == O.hash2(k)


@pytest.mark.parametrize("n_cells", [1 << 21, 10**7])
def test_keys_cells_hash2_bit_exact_on_2_24_tuples(P, n_cells):
    """CPU == GPU on 2^24 (material, node, u, v) tuples: descriptor, cell and check value
    bit for bit (the oracle's loop over its scalar definition against pmc_compute_keys)."""
    rng = np.random.default_rng(29)
    n = 1 << 24
    mat = rng.integers(0, 65536, n, dtype=np.uint32)
    node = rng.integers(0, 65536, n, dtype=np.uint32)
    u = rng.uniform(-0.05, 1.05, n).astype(np.float32)
    v = rng.uniform(-0.05, 1.05, n).astype(np.float32)
    t = lambda a: torch.from_numpy(a.view(np.int32) if a.dtype == np.uint32 else a).cuda()
    key, cell, h2 = P.compute_keys(t(mat), t(node), t(u), t(v), 10, n_cells)
    torch.cuda.synchronize()
    rk, rc, rh = O.address_batch(mat, node, u, v, 10, n_cells)
    assert np.array_equal(key.cpu().numpy().view(np.uint64), rk)
    assert np.array_equal(cell.cpu().numpy().view(np.uint64), rc)
    assert np.array_equal(h2.cpu().numpy().view(np.uint32), rh)


# ---- the tiny 8-node material, 4 passes of 4096 ---------------------------------------------
def test_tiny_config_cache_on(P):
    mat = W.material_tiny()
    pts = W.points_uniform(16384, seed=0)
    gpu = P.Cache([mat], 8192, 8, uv_level=10)
    ref = O.Cache([mat], 8192, 8, level=10)
    for p in range(4):
        _compare_pass(gpu, ref, P, W.slice_points(pts, 4096 * p, 4096 * (p + 1)))
    _compare_tables(gpu, ref)
    assert gpu.stats()["hits"] > 0


def test_tiny_config_cache_off(P):
    mat = W.material_tiny()
    pts = W.points_uniform(4096, seed=0)
    gpu = P.Cache([mat], 8192, 8, flags=P.PMC_CACHE_OFF)
    ref = O.Cache([mat], 8192, 8, cache_off=True)
    for _ in range(2):
        _compare_pass(gpu, ref, P, pts)
    assert gpu.stats()["lookups"] == 0


# ---- frame-shaped streams: a band of the 1920-wide frame, several table geometries ----------
# PMC_EVAL_INLINE, PMC_INSERT_ROUNDS, PMC_UNSORTED, PMC_PROBE_INLINE, PMC_INSERT_BINNED (the
# default insert of N_e <= 8 tables chains each cell's candidates; "binned" groups them by
# bins of cells, as the default does for N_e > 8)
MODES = {"grouped": 0, "inline": 0x8, "rounds": 0x10, "unsorted": 0x20, "unsorted_rounds": 0x30,
         "probe_inline": 0x40, "probe_inline_rounds": 0x50, "binned": 0x1000, "unsorted_binned": 0x1020}


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("n_cells,n_entries", [(1 << 21, 8), (1 << 10, 8), (10, 5), (1000, 16), (97, 32), (3, 1)])
def test_frame_band_parity(P, n_cells, n_entries, mode):
    spec = W.FrameSpec(width=1920, height=1080, n_mats=64, seed=0)
    frame = W.Frame(spec)
    mats = W.random_materials(64, 20, 200, 0.2, seed=0)
    gpu = P.Cache(mats, n_cells, n_entries, flags=MODES[mode])
    ref = O.Cache(mats, n_cells, n_entries)
    rows = (0, 9) if n_cells >= 1024 else (0, 3)       # 17,280 / 5,760 points: ragged warps
    for p in range(3):
        _compare_pass(gpu, ref, P, frame.points(p, rows=rows))
    _compare_tables(gpu, ref)


@pytest.mark.parametrize("mode", ["grouped", "unsorted", "probe_inline", "inline"])
@pytest.mark.parametrize("min_root_cost", [300, 600])
def test_frame_band_parity_with_cost_threshold(P, min_root_cost, mode):
    """Only cacheable nodes whose sub-graph costs at least min_root_cost FP32 operations
    are looked up and inserted; the rest are evaluated every time.  Same bar as without it."""
    frame = W.Frame(W.FrameSpec(width=1920, height=1080, n_mats=64, seed=0))
    mats = W.random_materials(64, 20, 200, 0.2, seed=0)
    gpu = P.Cache(mats, 1 << 12, 8, flags=MODES[mode], min_root_cost=min_root_cost)
    ref = O.Cache(mats, 1 << 12, 8, min_root_cost=min_root_cost)
    for m in range(0, 64, 7):
        assert list(gpu.material_info(m)["roots"]) == list(ref.roots(m))
    for p in range(3):
        _compare_pass(gpu, ref, P, frame.points(p, rows=(0, 9)))
    _compare_tables(gpu, ref)
    full = P.Cache(mats, 1 << 12, 8)
    full.eval_batch(P.points_to_device(frame.points(0, rows=(0, 9))),
                    torch.empty((3, 9 * 1920), device="cuda"))
    assert gpu.stats()["lookups"] < 3 * full.stats()["lookups"]


@pytest.fixture(scope="module")
def scale_mats():
    # the scale configuration: 4096 networks of 10-2000 nodes, 40 % shading-point dependent
    return W.random_materials(4096, 10, 2000, 0.4, seed=5)


@pytest.mark.parametrize("n_cells", [1 << 17, 1 << 12])
def test_scale_config_band_parity(P, scale_mats, n_cells):
    # a band of the 2048x2048 stream (2^22 points per batch), materials Zipf(0.9) over 4096
    frame = W.Frame(W.FrameSpec(width=2048, height=2048, n_mats=4096, zipf_s=0.9, seed=5))
    gpu = P.Cache(scale_mats, n_cells, 8)
    ref = O.Cache(scale_mats, n_cells, 8)
    for p in range(3):
        _compare_pass(gpu, ref, P, frame.points(p, rows=(1000, 1008)))
    _compare_tables(gpu, ref)


def test_frame_band_cache_off(P):
    frame = W.Frame(W.FrameSpec(seed=3))
    mats = W.random_materials(64, 20, 200, 0.2, seed=3)
    gpu = P.Cache(mats, 1 << 16, 8, flags=P.PMC_CACHE_OFF)
    ref = O.Cache(mats, 1 << 16, 8, cache_off=True)
    _compare_pass(gpu, ref, P, frame.points(0, rows=(500, 506)))


@pytest.mark.parametrize("n", [0, 1, 31, 33, 4097])
def test_ragged_batch_sizes(P, n):
    mats = W.random_materials(5, 20, 120, 0.2, seed=9)
    pts = W.points_uniform(max(n, 1), seed=n, n_mats=5)
    pts = W.slice_points(pts, 0, n)
    flags = (MODES["rounds"] if n % 2 else 0) | (MODES["unsorted"] if n in (1, 33) else 0)
    gpu = P.Cache(mats, 256, 8, flags=flags)
    ref = O.Cache(mats, 256, 8)
    for _ in range(2):
        _compare_pass(gpu, ref, P, pts)
    _compare_tables(gpu, ref)


def test_deep_and_wide_networks(P):
    # 1000-2000 node networks with long UV-only chains (the learned-surrogate workload shape)
    rng = np.random.default_rng(4)
    mats = [W.random_material(rng, int(n), 0.05, n_trees=1) for n in (600, 1500, 2000)]
    mats += [W.random_material(rng, 800, 0.4)]
    pts = W.points_uniform(3000, seed=5, n_mats=len(mats))
    gpu = P.Cache(mats, 4096, 8)
    ref = O.Cache(mats, 4096, 8)
    for p in range(2):
        _compare_pass(gpu, ref, P, W.slice_points(pts, 1500 * p, 1500 * (p + 1)))
    _compare_tables(gpu, ref)


@pytest.mark.parametrize("mode", sorted(MODES))
def test_hand_built_nested_roots(P, mode):
    from .test_oracle_analysis import g_nested, g_two_roots
    mats = [g_nested(), g_two_roots()]
    pts = W.points_uniform(600, seed=6, n_mats=2)
    pts["u"] = (np.floor(pts["u"] * 8) / 1024 + 0.3).astype(np.float32)   # few texels: many hits
    pts["v"] = (np.floor(pts["v"] * 8) / 1024 + 0.6).astype(np.float32)
    gpu = P.Cache(mats, 64, 4, flags=MODES[mode])
    ref = O.Cache(mats, 64, 4)
    for p in range(3):
        _compare_pass(gpu, ref, P, W.slice_points(pts, 200 * p, 200 * (p + 1)))
    _compare_tables(gpu, ref)
    assert gpu.stats()["hits"] > 100


# ---- errors, determinism, host entry point ----------------------------------------------------
@pytest.mark.parametrize("mode", ["grouped", "unsorted"])
def test_bad_material_index_reported(P, mode):
    mat = W.material_tiny()
    pts = W.points_uniform(100, seed=7)
    pts["mat"][17] = 3
    gpu = P.Cache([mat], 64, 8, flags=MODES[mode])
    d = P.points_to_device(pts)
    rgb = torch.full((3, 100), 5.0, device="cuda")
    gpu.eval_batch(d, rgb)
    with pytest.raises(P.PmcError) as ei:
        gpu.sync()
    assert ei.value.status == P.PMC_ERR_INVALID_ARG
    out = rgb.cpu().numpy()
    assert np.all(out[:, 17] == 0)
    assert gpu.stats()["bad_points"] == 1
    ref = O.Cache([mat], 64, 8)
    r = ref.run_batch(pts)
    ok = np.arange(100) != 17
    assert float(np.abs(out[:, ok] - r["rgb"][:, ok]).max()) <= TOL


@pytest.mark.parametrize("insert", ["lists", "binned"])
@pytest.mark.parametrize("n_cells", [2, 16])
def test_cells_with_more_candidates_than_a_stage(P, n_cells, insert):
    """A table of a few cells takes thousands of candidates per cell in the first pass.  The
    large-bin insert selects a crowded cell's candidates in order until the cell is full,
    then settles the rest (duplicates or dropped) at once; the per-cell lists are walked
    thousands of steps, with keys pushed out of the walk's buffer.  The table and every
    counter equal the oracle's sequential insert."""
    mats = W.random_materials(4, 20, 80, 0.2, seed=31)
    frame = W.Frame(W.FrameSpec(width=1920, height=1080, n_mats=4, seed=31))
    gpu = P.Cache(mats, n_cells, 8, flags=P.PMC_INSERT_BINNED if insert == "binned" else 0)
    ref = O.Cache(mats, n_cells, 8)
    for p in range(2):
        _compare_pass(gpu, ref, P, frame.points(p, rows=(0, 8)), check_masks=False)   # 15,360 points
    assert gpu.stats()["dropped_full"] > 1024 * n_cells
    _compare_tables(gpu, ref)


def test_two_runs_identical(P):
    frame = W.Frame(W.FrameSpec(seed=2))
    mats = W.random_materials(64, 20, 200, 0.2, seed=2)
    outs, tables = [], []
    for _ in range(2):
        gpu = P.Cache(mats, 1 << 12, 8)
        rgbs = [_run_gpu(gpu, P, frame.points(p, rows=(40, 60)))[0] for p in range(3)]
        outs.append(np.stack(rgbs))
        tables.append(gpu.table())
        gpu.close()
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(tables[0][0], tables[1][0]) and np.array_equal(tables[0][1], tables[1][1])


def test_host_entry_point_matches_device_entry(P):
    frame = W.Frame(W.FrameSpec(seed=1))
    mats = W.random_materials(64, 20, 200, 0.2, seed=1)
    a = P.Cache(mats, 1 << 14, 8)
    b = P.Cache(mats, 1 << 14, 8)
    for p in range(2):
        part = frame.points(p, rows=(100, 110))
        n = len(part["u"])
        g_rgb, g_hits = _run_gpu(a, P, part)
        h_rgb = np.zeros(3 * n, dtype=np.float32)
        h_hits = np.zeros(n, dtype=np.uint16)
        b.eval_batch_host(part, h_rgb, h_hits)
        assert np.array_equal(h_rgb.reshape(3, n), g_rgb)
        assert np.array_equal(h_hits, g_hits)
    assert np.array_equal(a.table()[0], b.table()[0])


@pytest.mark.parametrize("mode", sorted(MODES))
def test_reset_empties_table(P, mode):
    mat = W.material_tiny()
    pts = W.points_uniform(512, seed=8)
    gpu = P.Cache([mat], 64, 8, flags=MODES[mode])
    _run_gpu(gpu, P, pts)
    assert gpu.stats()["inserted"] > 0
    gpu.reset()
    gpu.sync()
    assert gpu.stats()["inserted"] == 0 and not gpu.table()[0].any()
    _, hits = _run_gpu(gpu, P, pts)
    assert not hits.any()


def test_pipelined_host_passes_equal_device_passes(P):
    """pmc_eval_passes_host (copies overlapped with evaluation, two staging sets) gives the
    device entry point's outputs, hits, counters and table, pass by pass, with a ragged last
    pass and a pass without hit output."""
    frame = W.Frame(W.FrameSpec(width=1920, height=1080, n_mats=16, seed=4))
    mats = W.random_materials(16, 20, 120, 0.2, seed=4)
    passes = [frame.points(p, rows=(100, 130)) for p in range(5)]
    passes[-1] = W.slice_points(passes[-1], 0, 40000 - 17)
    dev = P.Cache(mats, 1 << 14, 8)
    host = P.Cache(mats, 1 << 14, 8)
    want = []
    for pts in passes:
        n = len(pts["u"])
        rgb = torch.empty((3, n), device="cuda")
        hits = torch.empty(n, dtype=torch.int16, device="cuda")
        dev.eval_batch(P.points_to_device(pts), rgb, hits)
        want.append((rgb.cpu().numpy(), hits.cpu().numpy().astype(np.uint16)))
    out_rgb = [np.full(3 * len(p["u"]), -1.0, dtype=np.float32) for p in passes]
    out_hits = [np.zeros(len(p["u"]), dtype=np.uint16) for p in passes]
    out_hits[2] = None
    host.eval_passes_host(passes, out_rgb, out_hits)
    for k, (rgb, hits) in enumerate(want):
        assert np.array_equal(out_rgb[k].reshape(3, -1), rgb), k
        if out_hits[k] is not None:
            assert np.array_equal(out_hits[k], hits), k
    assert dev.stats() == host.stats()
    assert np.array_equal(dev.table()[0], host.table()[0])
    assert np.array_equal(dev.table()[1], host.table()[1])
