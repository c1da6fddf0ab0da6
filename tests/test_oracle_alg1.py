"""Pins of the paper's concurrent update (Sec. 3.3, Alg. 1) in the oracle.

The value is stored as a 32-bit code so that hash2 and value fit one 64-bit
compare-and-swap; the paper names no format, the reading is shared-exponent RGB9E5.
The encoding is checked against hand-worked codes and against an independent derivation
(the smallest exponent whose rounded largest mantissa fits 9 bits, found by search); the
serialised Alg. 1 against the bulk-synchronous cache, which it must equal batch for batch
when every batch holds one point, and against hand-worked intra-batch hits.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_07238_gb300 import workload as W

from .test_oracle_cache import _check_invariants


@pytest.mark.parametrize("rgb,code", [
    ((0.0, 0.0, 0.0), 0x00000000),
    ((1.0, 1.0, 1.0), (16 << 27) | (256 << 18) | (256 << 9) | 256),      # 1 = 256 * 2^(16-24)
    ((0.5, 0.25, 0.125), (15 << 27) | (64 << 18) | (128 << 9) | 256),    # 2^-1 = 256 * 2^(15-24)
    ((0.75, 0.0, 0.0), (15 << 27) | 384),
    ((65408.0, 0.0, 0.0), (31 << 27) | 511),                             # the largest value
    ((1e9, 0.0, 0.0), (31 << 27) | 511),                                 # clamped
    ((-1.0, 0.5, float("nan")), (15 << 27) | (256 << 9)),                # negative and NaN -> 0
    ((2.0 ** -20, 0.0, 0.0), (0 << 27) | 16),                            # exponent floor -16: 16 steps
    ((2.0 ** -26, 0.0, 0.0), (0 << 27) | 0),                             # below half a step: 0
    ((2.0 ** -24, 0.0, 0.0), (0 << 27) | 1),                             # the smallest step
    ((511.5 / 512, 0.0, 0.0), (16 << 27) | 256),                         # rounds up to 512: exponent + 1
])
def test_rgb9e5_hand_worked(rgb, code):
    assert O.rgb9e5_encode(*rgb) == code


def _by_search(c):
    """Code of (r, g, b) found by searching the exponent: the smallest e in [0, 31] with
    round(max 2^(24-e)) <= 511, ties up, after clamping to [0, 511/512 2^16]."""
    f = [min(max(float(x), 0.0), 65408.0) if x == x else 0.0 for x in np.float32(c)]
    mx = max(f)
    for e in range(32):
        if math.floor(mx * 2.0 ** (24 - e) + 0.5) <= 511:
            break
    m = [int(math.floor(x * 2.0 ** (24 - e) + 0.5)) for x in f]
    return (e << 27) | (m[2] << 18) | (m[1] << 9) | m[0]


def test_rgb9e5_matches_exponent_search():
    rng = np.random.default_rng(9)
    for _ in range(4000):
        scale = 2.0 ** rng.uniform(-20, 16)
        c = (rng.random(3) * scale).astype(np.float32)
        c[rng.random(3) < 0.1] = 0.0
        assert O.rgb9e5_encode(*map(float, c)) == _by_search(c), c


def test_rgb9e5_error_bound_and_round_trip():
    rng = np.random.default_rng(2)
    for _ in range(2000):
        c = rng.random(3).astype(np.float32)
        code = O.rgb9e5_encode(*map(float, c))
        d = O.rgb9e5_decode(code)
        step = 2.0 ** ((code >> 27) - 24)
        assert np.all(np.abs(d - c) <= step / 2 + 1e-12)
        assert O.rgb9e5_encode(*map(float, d)) == code          # decoded values are fixed points


def _one_point_batches(pts, n):
    return [W.slice_points(pts, i, i + 1) for i in range(n)]


def test_alg1_one_point_batches_equal_bulk_cache():
    # with one shading point per batch the concurrent update has nothing to race with: the
    # table holds the same keys as the bulk-synchronous cache, values are their encodings
    mats = W.random_materials(3, 12, 40, 0.2, seed=4)
    pts = W.points_uniform(300, seed=4, n_mats=3)
    pts["u"] = (np.floor(pts["u"] * 64) / 64).astype(np.float32)   # repeated texels
    pts["v"] = (np.floor(pts["v"] * 64) / 64).astype(np.float32)
    bulk = O.Cache(mats, 97, 4)
    alg1 = O.Cache(mats, 97, 4, alg1=True)
    for b in _one_point_batches(pts, 300):
        rb, ra = bulk.run_batch(b), alg1.run_batch(b)
        assert np.array_equal(rb["hits"], ra["hits"])
    hb, vb = bulk.table()
    ha, va = alg1.table()
    assert np.array_equal(hb, ha)
    for k in np.nonzero(hb)[0]:
        assert np.array_equal(va[k], O.rgb9e5_decode(O.rgb9e5_encode(*map(float, vb[k]))))
    sb, sa = bulk.stats(), alg1.stats()
    for k in ("lookups", "hits", "misses", "inserted", "dropped_dup", "dropped_full"):
        assert sb[k] == sa[k]
    _check_invariants(alg1, alg1.stats())


def test_alg1_hits_within_a_batch():
    # two points in one texel in one batch: the bulk cache misses twice, the concurrent
    # update (serialised) lets the second point hit the first point's encoded value
    mats = [W.material_tiny()]
    pts = W.points_uniform(2, seed=1)
    pts["u"][:] = 0.3
    pts["v"][:] = 0.6
    bulk = O.Cache(mats, 64, 4)
    alg1 = O.Cache(mats, 64, 4, alg1=True)
    rb = bulk.run_batch(pts)
    ra = alg1.run_batch(pts)
    assert list(rb["hits"]) == [0, 0] and list(ra["hits"]) == [0, 1]
    # the tiny network's only cacheable node is the output: the hit returns the decoding
    want = O.rgb9e5_decode(O.rgb9e5_encode(*map(float, np.float32(ra["rgb"][:, 0]))))
    assert np.array_equal(np.float32(ra["rgb"][:, 1]), want)
    assert alg1.stats()["inserted"] == 1 and bulk.stats()["inserted"] == 1


def test_alg1_invariants_on_a_frame_band():
    mats = W.random_materials(8, 20, 80, 0.2, seed=1)
    fr = W.Frame(W.FrameSpec(width=512, height=32, n_mats=8, seed=1))
    c = O.Cache(mats, 211, 8, alg1=True)
    for p in range(3):
        c.run_batch(fr.points(p, rows=(0, 8)))
        _check_invariants(c, c.stats())
