"""pmc_eval_batch_noalloc, the pass for callers that must not allocate device memory
(an application that owns all device memory through its own pool, a latency-critical
thread where cudaMalloc/cudaFree could stall the device, a plug-in whose host owns the
memory).  It must give the same results as pmc_eval_batch; this file is collected last
so that a stop-at-first-failure run has already run every other test."""
import numpy as np
import pytest

from paper_2305_07238_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2305_07238_gb300 import pmc
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return pmc


def _pass(fn, pts, P):
    n = len(pts["u"])
    d = P.points_to_device(pts)
    rgb = torch.full((3, n), -1.0, dtype=torch.float32, device="cuda")
    hits = torch.full((n,), -1, dtype=torch.int16, device="cuda")
    fn(d, rgb, hits)
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), hits.cpu().numpy()


def test_noalloc_matches_allocating_pass_on_two_calls(P):
    mats = W.random_materials(12, 20, 150, 0.2, seed=21)
    frame = W.Frame(W.FrameSpec(width=1920, height=1080, n_mats=12, seed=21))
    alloc = P.Cache(mats, 1 << 12, 8)
    noalloc = P.Cache(mats, 1 << 12, 8)
    max_roots = max(len(alloc.material_info(m)["roots"]) for m in range(len(mats)))
    n = min(P.NOALLOC_MAX_POINTS, P.NOALLOC_MAX_PROBES // max(1, max_roots)) // 1920 * 1920
    assert n >= 1920
    rows = (300, 300 + n // 1920)
    for p in range(2):                      # the second call sees the first call's inserts
        pts = frame.points(p, rows=rows)
        a_rgb, a_hits = _pass(alloc.eval_batch, pts, P)
        b_rgb, b_hits = _pass(noalloc.eval_batch_noalloc, pts, P)
        alloc.sync()
        noalloc.sync()
        assert float(np.abs(a_rgb - b_rgb).max()) <= TOL
        assert np.array_equal(a_hits, b_hits)
    assert alloc.stats()["hits"] > 0
    sa, sb = alloc.stats(), noalloc.stats()
    for k in ("lookups", "hits", "misses", "candidates", "inserted", "dropped_dup", "dropped_full"):
        assert sa[k] == sb[k], k
    assert np.array_equal(alloc.table()[0], noalloc.table()[0])


def test_noalloc_rejects_batches_beyond_the_fixed_scratch(P):
    mat = W.material_tiny()
    cache = P.Cache([mat], 64, 8)
    big = W.points_uniform(P.NOALLOC_MAX_POINTS + 1, seed=3)
    d = P.points_to_device(big)
    rgb = torch.empty((3, P.NOALLOC_MAX_POINTS + 1), dtype=torch.float32, device="cuda")
    with pytest.raises(P.PmcError) as ei:
        cache.eval_batch_noalloc(d, rgb)
    assert ei.value.status == P.PMC_ERR_UNSUPPORTED
    assert cache.stats()["batches"] == 0


def test_hit_masks_are_refused_after_a_noalloc_pass(P):
    """The probe records of a no-alloc pass live in the shared fixed array, so the masks
    of that pass cannot be read back from the cache; the call says so instead of reading
    the records of an older pass."""
    mats = W.random_materials(4, 20, 60, 0.2, seed=5)
    cache = P.Cache(mats, 1 << 10, 8)
    n = 2048
    d = P.points_to_device(W.points_uniform(n, seed=5, n_mats=4))
    rgb = torch.empty((3, n), dtype=torch.float32, device="cuda")
    cache.eval_batch(d, rgb)
    cache.eval_batch(d, rgb)
    assert cache.last_hit_masks(n).any()
    cache.eval_batch_noalloc(d, rgb)
    with pytest.raises(P.PmcError) as ei:
        cache.last_hit_masks(n)
    assert ei.value.status == P.PMC_ERR_UNSUPPORTED
    cache.eval_batch(d, rgb)                # an allocating pass makes them available again
    assert cache.last_hit_masks(n).any()


def test_noalloc_honours_the_probe_capacity(P):
    """A cache created with a probe capacity below a batch's needs refuses that batch in
    both entry points alike: no work, PMC_ERR_UNSUPPORTED at the next synchronising call."""
    mats = W.random_materials(4, 20, 60, 0.2, seed=6)
    n = 2048
    d = P.points_to_device(W.points_uniform(n, seed=6, n_mats=4))
    rgb = torch.empty((3, n), dtype=torch.float32, device="cuda")
    for fn in ("eval_batch", "eval_batch_noalloc"):
        cache = P.Cache(mats, 1 << 10, 8, probe_capacity=64)
        getattr(cache, fn)(d, rgb)
        with pytest.raises(P.PmcError) as ei:
            cache.sync()
        assert ei.value.status == P.PMC_ERR_UNSUPPORTED, fn
        assert cache.stats(check=False)["lookups"] == 0, fn
