"""Pins of the per-point mip level from ray-cone gradients (Sec. 3.1, Eq. 1).

Eq. 1 gives lambda = -log2(min(|g1|, |g2|)) for the texture-coordinate gradients g1, g2
along the axes of the footprint ellipse; the virtual texture then has 2^lambda texels
per axis.  The readings pinned here: the squared norms are formed in FP32, the level is
the floor of Eq. 1 plus the offset of the discussion (Sec. 4), clamped to [0, 13]; a zero
footprint gives 13, an infinite or NaN one 0.

The checks do not restate the oracle's formula: hand-worked values, the defining
inequality of the floor decided with exact rationals (a texel is at least as wide as the
footprint and less than twice as wide), the halving law, and the reduction of the
per-point cache to the fixed-level cache when every point's level is the same.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_07238_gb300 import workload as W


@pytest.mark.parametrize("g,offset,expected", [
    ((2.0 ** -10, 0.0, 0.0, 2.0 ** -10), 0, 10),          # isotropic, footprint = one 1024th
    ((0.75 * 2 ** -10, 0.0, 0.0, 1.0), 0, 10),            # -log2(0.75/1024) = 10.415
    ((1.5 * 2 ** -10, 0.0, 0.0, 1.0), 0, 9),              # -log2(1.5/1024) = 9.415
    ((2.0 ** -8, 0.0, 0.0, 2.0 ** -11), 0, 11),           # the minor axis decides
    ((3 * 2.0 ** -12, 4 * 2.0 ** -12, 1.0, 1.0), 0, 9),   # |g1| = 5/4096: -log2 = 9.678
    ((0.0, 2.0 ** -10, 2.0 ** -10, 0.0), 0, 10),          # axes swapped
    ((2.0 ** -10, 0.0, 0.0, 2.0 ** -10), 1, 11),          # offset towards finer texels
    ((2.0 ** -10, 0.0, 0.0, 2.0 ** -10), -3, 7),
    ((2.0 ** -12, 0.0, 0.0, 2.0 ** -12), 5, 13),          # clamped at the finest level
    ((0.0, 0.0, 1.0, 1.0), 0, 13),                        # zero footprint: finest
    ((2.0, 0.0, 0.0, 3.0), 0, 0),                         # wider than the texture: 0
    ((0.5, 0.0, 0.0, 0.5), 0, 1),
    ((1.0, 0.0, 0.0, 1.0), 0, 0),
    ((float("nan"), 0.0, 0.0, 1e-3), 0, 0),               # NaN: coarsest
    ((float("inf"), 0.0, 1e-3, 0.0), 0, 9),               # the finite axis decides
    ((float("inf"), 0.0, float("inf"), 0.0), 0, 0),
    ((1e-30, 0.0, 0.0, 1e-30), -13, 13),                  # squared norm underflows to 0
])
def test_level_hand_worked(g, offset, expected):
    assert O.level(*g, offset) == expected


def _exact_level(g1u, g1v, g2u, g2v, offset):
    """The floor of Eq. 1 characterised without logarithms: the integer L with
    4^-(L+1) < s <= 4^-L for the FP32 squared norm s of the minor axis."""
    f = np.float32
    s1 = f(f(f(g1u) * f(g1u)) + f(f(g1v) * f(g1v)))
    s2 = f(f(f(g2u) * f(g2u)) + f(f(g2v) * f(g2v)))
    s = Fraction(float(min(s1, s2)))
    assert s > 0
    q = Fraction(1, 4)
    L = 0
    while s > q ** L:
        L -= 1
    while s <= q ** (L + 1):
        L += 1
    assert q ** (L + 1) < s <= q ** L
    return min(13, max(0, L + offset))


def test_level_defining_inequality():
    rng = np.random.default_rng(11)
    for _ in range(3000):
        mag = np.exp2(rng.uniform(-15.0, 1.5, 2))
        th = rng.uniform(0.0, 2.0 * math.pi)
        b = np.exp2(rng.uniform(0.0, 2.0))
        g = (float(np.float32(mag[0] * math.cos(th))), float(np.float32(mag[0] * math.sin(th))),
             float(np.float32(-mag[1] * b * math.sin(th))), float(np.float32(mag[1] * b * math.cos(th))))
        off = int(rng.integers(-2, 3))
        assert O.level(*g, off) == _exact_level(*g, off), g


def test_level_boundaries_between_powers_of_four():
    # squared norm exactly 4^-10 is level 10; one FP32 step above it is level 9
    e = 2.0 ** -10
    assert O.level(e, 0.0, e, 0.0) == 10
    up = float(np.nextafter(np.float32(e), np.float32(1.0)))
    assert O.level(up, 0.0, up, 0.0) == 9
    dn = float(np.nextafter(np.float32(e), np.float32(0.0)))
    assert O.level(dn, 0.0, dn, 0.0) == 10


def test_level_halving_law():
    rng = np.random.default_rng(3)
    for _ in range(500):
        g = rng.uniform(0.2, 1.0, 4) * 2.0 ** -6
        lv = O.level(*g)
        assert O.level(*(g * 0.5)) == lv + 1
        assert O.level(*(g * 2.0)) == lv - 1


def _frame_band(seed=0, rows=(0, 4)):
    mats = W.random_materials(6, 12, 40, 0.2, seed=seed)
    fr = W.Frame(W.FrameSpec(width=256, height=16, n_mats=6, seed=seed))
    return mats, [fr.points(p, rows=rows, cones=True) for p in range(3)]


def test_uniform_level_reduces_to_fixed_level_cache():
    # every point's footprint gives level 9: the per-point cache is the fixed-level cache
    mats, passes = _frame_band()
    g = np.float32(2.0 ** -9)
    a = O.Cache(mats, 509, 4, level=9)
    b = O.Cache(mats, 509, 4, level=3)   # the fixed level must not be used
    for p in passes:
        q = dict(p)
        n = len(q["u"])
        q.update(g1u=np.full(n, g), g1v=np.zeros(n, np.float32), g2u=np.zeros(n, np.float32),
                 g2v=np.full(n, g))
        ra = a.run_batch({k: p[k] for k in W.POINT_FIELDS}, probes=True)
        rb = b.run_batch(q, probes=True)
        assert np.array_equal(ra["rgb"], rb["rgb"])
        assert np.array_equal(ra["hits"], rb["hits"])
        assert np.array_equal(ra["key"], rb["key"])
    assert np.array_equal(a.table()[0], b.table()[0])
    assert a.stats() == b.stats()


def test_levels_partition_the_keys():
    # the same UV at two levels is two descriptors: no hit across levels
    mats = [W.material_tiny()]
    pt = {"u": np.array([0.3], np.float32), "v": np.array([0.6], np.float32),
          "mat": np.zeros(1, np.uint32)}
    for k in ("px", "py", "pz", "nx", "ny", "nz"):
        pt[k] = np.zeros(1, np.float32)
    def at(level):
        q = dict(pt)
        g = np.float32(2.0 ** -level)
        q.update(g1u=np.array([g]), g1v=np.zeros(1, np.float32), g2u=np.zeros(1, np.float32),
                 g2v=np.array([g]))
        return q
    c = O.Cache(mats, 64, 4)
    r0 = c.run_batch(at(10), probes=True)
    r1 = c.run_batch(at(9), probes=True)
    r2 = c.run_batch(at(10), probes=True)
    r3 = c.run_batch(at(9), probes=True)
    assert list(r0["hit"]) == [0] and list(r1["hit"]) == [0]
    assert list(r2["hit"]) == [1] and list(r3["hit"]) == [1]
    assert (int(r0["key"][0]) >> 26) & 63 == 10 and (int(r1["key"][0]) >> 26) & 63 == 9


def test_cone_stream_levels_span_the_frame_recipe():
    # the synthetic footprints (minor axis delta * 2^U(-1/2, 1/2), delta in [2^-12, 2^-8])
    # give levels 7 .. 12
    fr = W.Frame(W.FrameSpec(width=512, height=64, n_mats=4, seed=1))
    p = fr.points(0, cones=True)
    lv = np.array([O.level(p["g1u"][i], p["g1v"][i], p["g2u"][i], p["g2v"][i]) for i in range(0, len(p["u"]), 7)])
    assert lv.min() >= 7 and lv.max() <= 12
    assert len(np.unique(lv)) >= 4
