"""GPU tests of schedules, CUDA graphs of passes, autotuning and the probe capacity.

* every schedule (grouped with 4/2/1 probes in flight, inline misses, unsorted inline
  probing, claim-round insert) gives the same outputs, hit counts, counters and table;
* a graph of passes replays exactly the calls it recorded (with and without the reset),
  and both match the FP64 oracle;
* a graph goes stale when the scratch or the schedule changes;
* autotuning leaves the table and counters as it found them;
* a batch that needs more probe records than the declared capacity does no work and is
  reported.
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


@pytest.fixture(scope="module")
def band():
    """Four passes over a 12-row band of the 1080p frame, 64 materials."""
    frame = W.Frame(W.FrameSpec(seed=4))
    mats = W.random_materials(64, 20, 200, 0.2, seed=4)
    return mats, [frame.points(p, rows=(300, 312)) for p in range(4)]


def _outputs(P, parts):
    rgb = [torch.zeros((3, len(p["u"])), device="cuda") for p in parts]
    hits = [torch.zeros(len(p["u"]), dtype=torch.int16, device="cuda") for p in parts]
    return rgb, hits


def _eager(P, cache, dparts, rgb, hits):
    for d, r, h in zip(dparts, rgb, hits):
        cache.eval_batch(d, r, h)
    cache.sync()


def _host(ts):
    return [t.cpu().numpy() for t in ts]


# ... plus the evaluator's work distribution: block-wide tiles of one material (0x400) and one
# point per lane (0x800), and the binned insert instead of per-cell lists (0x1000)
SCHEDULES = [(0, 4), (0, 2), (0, 1), (0x8, 4), (0x28, 4), (0x10, 4), (0x30, 2), (0x40, 4), (0x50, 4),
             (0x400, 2), (0x800, 2), (0x410, 4), (0x840, 4), (0x1000, 4), (0x1028, 4), (0x1040, 1),
             (0x1800, 2)]


def test_every_schedule_same_results(P, band):
    mats, parts = band
    dparts = [P.points_to_device(p) for p in parts]
    base = None
    for flags, rb in SCHEDULES:
        c = P.Cache(mats, 1 << 12, 8)
        c.set_schedule(flags, rb)
        assert c.schedule() == {"flags": flags, "lookup_rb": rb}
        rgb, hits = _outputs(P, parts)
        _eager(P, c, dparts, rgb, hits)
        got = (_host(rgb), _host(hits), c.table(), {k: c.stats()[k] for k in EXACT_STATS})
        c.close()
        if base is None:
            base = got
            continue
        for a, b in zip(got[0], base[0]):
            assert np.array_equal(a, b), (flags, rb, float(np.abs(a - b).max()))
        for a, b in zip(got[1], base[1]):
            assert np.array_equal(a, b), (flags, rb)
        assert np.array_equal(got[2][0], base[2][0]) and np.array_equal(got[2][1], base[2][1])
        assert got[3] == base[3], (flags, rb)


@pytest.mark.parametrize("flags", [0, 0x20, 0x10, 0x40, 0x1000])
def test_graph_with_reset_replays_the_frame(P, band, flags):
    mats, parts = band
    dparts = [P.points_to_device(p) for p in parts]
    eager = P.Cache(mats, 1 << 12, 8, flags=flags)
    e_rgb, e_hits = _outputs(P, parts)
    _eager(P, eager, dparts, e_rgb, e_hits)

    g = P.Cache(mats, 1 << 12, 8, flags=flags)
    g_rgb, g_hits = _outputs(P, parts)
    graph = g.graph(dparts, g_rgb, g_hits, reset=True)
    for rep in range(2):                       # each replay renders the frame from scratch
        for t in g_rgb:
            t.fill_(-1.0)
        graph.launch()
        g.sync()
        for a, b in zip(_host(g_rgb), _host(e_rgb)):
            assert np.array_equal(a, b)
        for a, b in zip(_host(g_hits), _host(e_hits)):
            assert np.array_equal(a, b)
        gs, es = g.stats(), eager.stats()
        for k in EXACT_STATS:
            assert gs[k] == es[k], (rep, k)
        assert np.array_equal(g.table()[0], eager.table()[0])

    ref = O.Cache(mats, 1 << 12, 8)
    for p, r_gpu, h_gpu in zip(parts, _host(g_rgb), _host(g_hits)):
        r = ref.run_batch(p)
        assert float(np.abs(r_gpu - r["rgb"]).max()) <= TOL
        assert np.array_equal(h_gpu.astype(np.uint16), r["hits"])
    assert np.array_equal(g.table()[0], ref.table()[0])
    # the cache keeps working eagerly after a replay
    more = P.points_to_device(parts[0])
    rgb = torch.zeros((3, len(parts[0]["u"])), device="cuda")
    g.eval_batch(more, rgb)
    g.sync()
    r = ref.run_batch(parts[0])
    assert float(np.abs(rgb.cpu().numpy() - r["rgb"]).max()) <= TOL
    graph.close()


def test_graph_without_reset_continues_the_table(P, band):
    mats, parts = band
    dparts = [P.points_to_device(p) for p in parts]
    a = P.Cache(mats, 1 << 12, 8)
    b = P.Cache(mats, 1 << 12, 8)
    rgb_a, hits_a = _outputs(P, parts)
    rgb_b, hits_b = _outputs(P, parts)
    _eager(P, a, dparts[:2], rgb_a[:2], hits_a[:2])
    _eager(P, b, dparts[:2], rgb_b[:2], hits_b[:2])
    _eager(P, a, dparts[2:], rgb_a[2:], hits_a[2:])
    graph = b.graph(dparts[2:], rgb_b[2:], hits_b[2:], reset=False)
    graph.launch()
    b.sync()
    for x, y in zip(_host(rgb_a), _host(rgb_b)):
        assert np.array_equal(x, y)
    for x, y in zip(_host(hits_a), _host(hits_b)):
        assert np.array_equal(x, y)
    assert all(a.stats()[k] == b.stats()[k] for k in EXACT_STATS)
    assert np.array_equal(a.table()[0], b.table()[0])


def test_graph_goes_stale(P, band):
    mats, parts = band
    dparts = [P.points_to_device(p) for p in parts[:1]]
    c = P.Cache(mats, 1 << 12, 8)
    rgb, hits = _outputs(P, parts[:1])
    graph = c.graph(dparts, rgb, hits, reset=True)
    graph.launch()
    c.sync()
    c.set_schedule(0x8, 4)
    with pytest.raises(P.PmcError) as ei:
        graph.launch()
    assert ei.value.status == P.PMC_ERR_INVALID_ARG
    graph2 = c.graph(dparts, rgb, hits, reset=True)
    big = P.points_to_device(W.points_uniform(4 * len(parts[0]["u"]), seed=3, n_mats=len(mats)))
    c.eval_batch(big, torch.zeros((3, int(big["u"].numel())), device="cuda"))   # scratch grows
    c.sync()
    with pytest.raises(P.PmcError):
        graph2.launch()


def test_autotune_leaves_cache_unchanged(P, band):
    mats, parts = band
    dparts = [P.points_to_device(p) for p in parts]
    a = P.Cache(mats, 1 << 12, 8)
    b = P.Cache(mats, 1 << 12, 8)
    rgb, hits = _outputs(P, parts)
    for c in (a, b):
        _eager(P, c, dparts[:2], rgb[:2], hits[:2])
    res = b.autotune(dparts[2], reps=2)
    assert len(res["tried"]) >= 5 and 0 <= res["best"] < len(res["tried"])
    assert all(t["ms"] > 0 for t in res["tried"])
    assert res["schedule"] == {k: res["tried"][res["best"]][k] for k in ("flags", "lookup_rb")}
    # the fastest schedule is tried again with the binned insert
    assert res["tried"][-1]["flags"] & P.PMC_INSERT_BINNED
    assert a.stats() == b.stats()
    assert np.array_equal(a.table()[0], b.table()[0]) and np.array_equal(a.table()[1], b.table()[1])
    ra, ha = _outputs(P, parts[2:])
    rb_, hb = _outputs(P, parts[2:])
    _eager(P, a, dparts[2:], ra, ha)
    _eager(P, b, dparts[2:], rb_, hb)
    for x, y in zip(_host(ra), _host(rb_)):
        assert np.array_equal(x, y)
    assert np.array_equal(a.table()[0], b.table()[0])


def test_probe_capacity_exceeded_is_reported(P, band):
    mats, parts = band
    d = P.points_to_device(parts[0])
    n = int(d["u"].numel())
    c = P.Cache(mats, 1 << 12, 8, probe_capacity=n)          # one probe per point: too few
    c.eval_batch(d, torch.zeros((3, n), device="cuda"))
    with pytest.raises(P.PmcError) as ei:
        c.sync()
    assert ei.value.status == P.PMC_ERR_UNSUPPORTED
    roots = np.array([len(c.material_info(m)["roots"]) for m in range(len(mats))])
    need = int(roots[parts[0]["mat"]].sum())
    ok = P.Cache(mats, 1 << 12, 8, probe_capacity=need)        # exactly enough
    ref = O.Cache(mats, 1 << 12, 8)
    rgb = torch.zeros((3, n), device="cuda")
    ok.eval_batch(d, rgb)
    ok.sync()
    assert float(np.abs(rgb.cpu().numpy() - ref.run_batch(parts[0])["rgb"]).max()) <= TOL


def test_unsorted_refused_with_surrogates(P):
    mats = W.surrogate_materials(2, 200, 300, seed=1)
    c = P.Cache(mats, 1 << 10, 8)
    theta = np.zeros(P.MLP_PARAMS, dtype=np.float32)
    c.set_surrogate(0, theta)
    with pytest.raises(P.PmcError) as ei:
        c.set_schedule(0x20, 4)
    assert ei.value.status == P.PMC_ERR_UNSUPPORTED
    c.use_surrogates(False)
    c.set_schedule(0x20, 4)


@pytest.mark.parametrize("flags", [0, 0x400, 0x800])
def test_uncached_work_distributions_same_results(P, band, flags):
    """With the cache off every point runs its whole program: two points per lane in warp
    pairs or block tiles, and one point per lane, give the same outputs bit for bit (and
    match the FP64 oracle)."""
    mats, parts = band
    ref = O.Cache(mats, 1 << 12, 8, cache_off=True)
    c = P.Cache(mats, 1 << 12, 8, flags=P.PMC_CACHE_OFF)
    c.set_schedule(flags, 4)
    base = P.Cache(mats, 1 << 12, 8, flags=P.PMC_CACHE_OFF)
    for p in parts[:2]:
        d = P.points_to_device(p)
        rgb, hits = _outputs(P, [p])
        _eager(P, c, [d], rgb, hits)
        rgb0, hits0 = _outputs(P, [p])
        _eager(P, base, [d], rgb0, hits0)
        assert np.array_equal(rgb[0].cpu().numpy(), rgb0[0].cpu().numpy())
        assert float(np.abs(rgb[0].cpu().numpy() - ref.run_batch(p)["rgb"]).max()) <= TOL
    for k in ("flops", "nodes_evaluated", "points"):
        assert c.stats()[k] == base.stats()[k], k
