"""Pins of the oracle's primitives against published vectors, closed forms and brute force.

Nothing here compares the oracle with itself: each expected value comes from a
published test vector, a mathematical property of the primitive, or an exhaustive
search on a tiny input.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_07238_gb300 import workload as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


def _vectors():
    out = []
    with open(os.path.join(GOLDEN, "hash_vectors.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                parts = line.split()
                out.append((parts[0], [int(x, 16) for x in parts[1:]]))
    return out


# ---- mixers: published vectors --------------------------------------------------------
def test_splitmix64_reference_stream():
    rows = [v for k, v in _vectors() if k == "splitmix64"]
    assert len(rows) == 3
    state = 0
    for st, expected in rows:
        state = (state + 0x9E3779B97F4A7C15) & M64
        assert state == st
        assert O.splitmix64_mix(state) == expected


def test_fmix32_via_murmur3_empty_input():
    rows = [v for k, v in _vectors() if k == "murmur3_x86_32_empty"]
    assert rows
    for seed, expected in rows:
        assert O.fmix32(seed) == expected


def test_fmix64_via_murmur3_x64_128_empty_input():
    rows = [v for k, v in _vectors() if k == "murmur3_x64_128_empty"]
    assert rows
    for seed, e1, e2 in rows:
        h1 = h2 = seed
        h1 = (h1 + h2) & M64
        h2 = (h2 + h1) & M64
        h1 = O.fmix64(h1)
        h2 = O.fmix64(h2)
        h1 = (h1 + h2) & M64
        h2 = (h2 + h1) & M64
        assert (h1, h2) == (e1, e2)


def test_hash_pair_is_injective_on_random_keys():
    # Both 64-bit finalisers are bijections: 2^16 random keys give 2^16 distinct outputs.
    rng = np.random.default_rng(1)
    keys = rng.integers(0, 2**63, 1 << 16, dtype=np.int64).astype(np.uint64)
    keys = np.unique(keys)
    h1 = {O.hash1(int(k)) for k in keys}
    assert len(h1) == len(keys)


def test_hash2_never_zero_and_avalanche():
    # hash2 = 0 is reserved for "empty"; single-bit key changes flip about half the bits.
    assert O.hash2(0) != 0
    rng = np.random.default_rng(2)
    flips = []
    for _ in range(200):
        k = int(rng.integers(0, 2**62))
        b = int(rng.integers(0, 64))
        flips.append(bin(O.hash2(k) ^ O.hash2(k ^ (1 << b))).count("1"))
    assert 14.0 < np.mean(flips) < 18.0


def test_lattice_hash_uniform_gradient_choice():
    # The 8 gradient directions are chosen with equal frequency (chi-square, 7 dof).
    counts = np.zeros(8)
    for i in range(-40, 40):
        for j in range(-40, 40):
            counts[O.lattice_hash(i, j, 7) & 7] += 1
    exp = counts.sum() / 8
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 24.3  # p = 0.001 for 7 degrees of freedom


# ---- fade and gradient noise ----------------------------------------------------------
def test_fade_closed_form_properties():
    assert O.fade(0.0) == 0.0
    assert O.fade(1.0) == pytest.approx(1.0, abs=1e-15)
    assert O.fade(0.5) == pytest.approx(0.5, abs=1e-15)
    h = 1e-5
    for t0 in (0.0, 1.0):
        d1 = (O.fade(t0 + h) - O.fade(t0 - h)) / (2 * h)
        d2 = (O.fade(t0 + h) - 2 * O.fade(t0) + O.fade(t0 - h)) / (h * h)
        assert abs(d1) < 1e-8 and abs(d2) < 1e-3
    ts = np.linspace(0, 1, 101)
    vals = [O.fade(t) for t in ts]
    assert all(b >= a for a, b in zip(vals, vals[1:]))
    # symmetric: fade(1 - t) = 1 - fade(t)
    for t in ts:
        assert O.fade(1 - t) == pytest.approx(1 - O.fade(t), abs=1e-14)


def _grad(i, j, seed):
    k = O.lattice_hash(i, j, seed) & 7
    a = k * math.pi / 4
    return math.cos(a), math.sin(a)


def test_perlin_zero_on_lattice():
    rng = np.random.default_rng(3)
    for _ in range(200):
        i, j = (int(x) for x in rng.integers(-1000, 1000, 2))
        assert O.perlin(float(i), float(j), 11) == 0.0


def test_perlin_gradient_at_lattice_points():
    # The derivative of the noise at a lattice point is that point's gradient vector.
    h = 1e-6
    for (i, j, s) in [(0, 0, 1), (3, -2, 5), (-7, 9, 123), (100, 50, 77), (-1, -1, 0)]:
        gx = (O.perlin(i + h, j, s) - O.perlin(i - h, j, s)) / (2 * h)
        gy = (O.perlin(i, j + h, s) - O.perlin(i, j - h, s)) / (2 * h)
        ex, ey = _grad(i, j, s)
        assert gx == pytest.approx(ex, abs=1e-6)
        assert gy == pytest.approx(ey, abs=1e-6)


def test_perlin_cell_centre_is_mean_of_corner_dots():
    # At the cell centre fade = 1/2, so the noise is the mean of the four corner dots.
    for (i, j, s) in [(0, 0, 1), (4, -3, 9), (-10, 2, 31)]:
        tot = 0.0
        for cx in (0, 1):
            for cy in (0, 1):
                gx, gy = _grad(i + cx, j + cy, s)
                tot += gx * (0.5 - cx) + gy * (0.5 - cy)
        assert O.perlin(i + 0.5, j + 0.5, s) == pytest.approx(tot / 4, abs=1e-15)


def test_perlin_bound_and_continuity():
    rng = np.random.default_rng(4)
    xs = rng.uniform(-50, 50, (4000, 2))
    vals = np.array([O.perlin(x, y, 3) for x, y in xs])
    assert np.all(np.abs(vals) <= math.sqrt(0.5) + 1e-12)
    assert vals.std() > 0.1
    eps = 1e-9
    for i in range(-5, 5):
        y = float(rng.uniform(0, 1))
        assert O.perlin(i - eps, y + 3, 2) == pytest.approx(O.perlin(i + eps, y + 3, 2), abs=1e-7)


def test_fbm_reduces_to_noise():
    for (x, y) in [(0.1, 0.7), (0.33, 0.9), (0.5, 0.5)]:
        s = 8.0
        one = O.fbm(x, y, s, 1, 2.0, 0.5, 9)
        assert one == pytest.approx(min(1.0, max(0.0, 0.5 + O.perlin(x * s, y * s, 9))), abs=1e-15)
        two = O.fbm(x, y, s, 2, 2.0, 0.5, 9)
        n0 = O.perlin(x * s, y * s, 9)
        n1 = O.perlin(x * s * 2, y * s * 2, 10)
        assert two == pytest.approx(min(1.0, max(0.0, 0.5 + (n0 + 0.5 * n1) / 1.5)), abs=1e-15)


# ---- Worley F1 ------------------------------------------------------------------------
def _feature(i, j, seed):
    h = O.lattice_hash(i, j, seed)
    return i + 0.25 + 0.5 * (h & 0xFFFF) / 65536.0, j + 0.25 + 0.5 * (h >> 16) / 65536.0


def test_voronoi_zero_at_feature_points():
    for (i, j) in [(0, 0), (5, -3), (-8, 12)]:
        fx, fy = _feature(i, j, 17)
        assert O.voronoi_f1(fx, fy, 17) == pytest.approx(0.0, abs=1e-12)


def test_voronoi_equals_brute_force_7x7():
    rng = np.random.default_rng(5)
    for _ in range(300):
        x, y = rng.uniform(-20, 20, 2)
        ix, iy = math.floor(x), math.floor(y)
        best = min(math.dist((x, y), _feature(ix + a, iy + b, 4))
                   for a in range(-3, 4) for b in range(-3, 4))
        assert O.voronoi_f1(x, y, 4) == pytest.approx(best, abs=1e-12)
        assert best <= math.sqrt(2) * 0.75 + 1e-12


# ---- node operators -----------------------------------------------------------------
def _node(op, fp=(), ip=(), nin=0):
    b = W.Builder()
    b.add(op, [0] * nin, ip=ip, fp=fp)
    arr = b.build()
    arr[0]["inp"][:] = -1
    return arr


def test_mix_endpoints_and_factor_input():
    a, b = [0.1, 0.2, 0.3], [0.9, 0.5, 0.0]
    assert np.allclose(O.eval_node(_node(W.OP_MIX, fp=[0.0]), a, b), a, atol=0)
    assert np.allclose(O.eval_node(_node(W.OP_MIX, fp=[1.0]), a, b), b, atol=0)
    got = O.eval_node(_node(W.OP_MIX, fp=[0.9]), a, b, c=[0.25, 9, 9])
    assert np.allclose(got, [0.3, 0.275, 0.225], atol=1e-15)
    got = O.eval_node(_node(W.OP_MIX, fp=[0.0]), a, b, c=[7.0, 0, 0])  # factor clamped to 1
    assert np.allclose(got, b, atol=0)


def test_ramp_hits_stop_colours():
    fp = [0.0, 0.25, 0.75, 1.0, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 1.0, 0.0, 0.5]
    nd = _node(W.OP_RAMP, fp=fp, ip=[4])
    cols = np.array(fp[4:]).reshape(4, 3).astype(np.float32).astype(np.float64)
    for k, t in enumerate([0.0, 0.25, 0.75, 1.0]):
        assert np.allclose(O.eval_node(nd, [t, 0, 0]), cols[k], atol=1e-7)
    assert np.allclose(O.eval_node(nd, [-3.0, 0, 0]), cols[0], atol=0)
    assert np.allclose(O.eval_node(nd, [5.0, 0, 0]), cols[3], atol=0)
    assert np.allclose(O.eval_node(nd, [0.5, 0, 0]), (cols[1] + cols[2]) / 2, atol=1e-7)
    # two-stop ramp with stops inside (0,1): constant outside, linear inside
    nd2 = _node(W.OP_RAMP, fp=[0.2, 0.6, 0, 0, 0.0, 0.0, 0.0, 1.0, 0.5, 0.25], ip=[2])
    assert np.allclose(O.eval_node(nd2, [0.1, 0, 0]), [0, 0, 0], atol=0)
    assert np.allclose(O.eval_node(nd2, [0.3, 0, 0]), [0.25, 0.125, 0.0625], atol=1e-7)


def test_checker_parity():
    fp = [4.0, 0.1, 0.2, 0.3, 0.7, 0.8, 0.9]
    nd = _node(W.OP_CHECKER, fp=fp, nin=1)
    c1 = np.float32([0.1, 0.2, 0.3]).astype(np.float64)
    c2 = np.float32([0.7, 0.8, 0.9]).astype(np.float64)
    assert np.array_equal(O.eval_node(nd, [0.1, 0.1, 0]), c1)     # cells (0, 0)
    assert np.array_equal(O.eval_node(nd, [0.3, 0.1, 0]), c2)     # cells (1, 0)
    assert np.array_equal(O.eval_node(nd, [0.3, 0.3, 0]), c1)     # cells (1, 1)
    assert np.array_equal(O.eval_node(nd, [0.25, 0.0, 0]), c2)    # edge belongs to the upper cell
    assert np.array_equal(O.eval_node(nd, [-0.1, 0.1, 0]), c2)    # cells (-1, 0)


def test_affine_identity_and_rotation():
    ident = _node(W.OP_UV_AFFINE, fp=[1, 0, 0, 1, 0, 0], nin=1)
    assert np.array_equal(O.eval_node(ident, [0.3, 0.7, 0.0]), [0.3, 0.7, 0.0])
    rot = _node(W.OP_UV_AFFINE, fp=[0, -1, 1, 0, 2, 3], nin=1)
    assert np.allclose(O.eval_node(rot, [0.3, 0.7, 0.0]), [2 - 0.7, 3 + 0.3, 0.0], atol=1e-15)


def test_add_mul_pow_facing_clamp():
    a, b = [0.6, 0.2, -0.5], [0.7, 0.1, 0.2]
    assert np.allclose(O.eval_node(_node(W.OP_ADD, nin=2), a, b), [1.0, 0.3, 0.0], atol=1e-15)
    assert np.allclose(O.eval_node(_node(W.OP_MUL, nin=2), a, b), [0.42, 0.02, 0.0], atol=1e-15)
    assert np.allclose(O.eval_node(_node(W.OP_POW, fp=[1.0], nin=1), [0.3, 0.9, -2]), [0.3, 0.9, 0], atol=0)
    assert np.allclose(O.eval_node(_node(W.OP_POW, fp=[2.0], nin=1), [0.5, 1.5, 0]), [0.25, 1.0, 0], atol=0)
    d = [0.0, 0.6, 0.8]
    assert np.allclose(O.eval_node(_node(W.OP_FACING, fp=d, nin=1), [0.0, -1.0, 0.0]), [0.6] * 3, atol=1e-7)


def test_inputs_of_shading_point():
    sp = [0.1, 0.2, 1.0, 2.0, 3.0, 0.0, 0.0, 1.0]
    assert np.allclose(O.eval_node(_node(W.OP_UV)), [0, 0, 0])
    assert np.allclose(O.eval_node(_node(W.OP_UV), sp=sp), [0.1, 0.2, 0])
    assert np.allclose(O.eval_node(_node(W.OP_POSITION), sp=sp), [1, 2, 3])
    assert np.allclose(O.eval_node(_node(W.OP_NORMAL), sp=sp), [0, 0, 1])
    assert np.allclose(O.eval_node(_node(W.OP_CONST, fp=[0.5, 0.25, 2.0])), [0.5, 0.25, 2.0])


def test_tiny_material_by_hand():
    # Mix(ramp(noise), c1, 0.5) * c2 written out from the primitives above.
    m = W.material_tiny()
    u, v = 0.37, 0.81
    sp = [u, v, 0, 0, 0, 0, 0, 1]
    n = min(1.0, max(0.0, 0.5 + (O.perlin(u * 8, v * 8, 1) + 0.5 * O.perlin(u * 16, v * 16, 2)) / 1.5))
    pos = np.float32([0.0, 0.33, 0.66, 1.0]).astype(np.float64)
    cols = np.float32(m[2]["fp"][4:16]).astype(np.float64).reshape(4, 3)
    k = int(np.searchsorted(pos, n, side="right") - 1)
    w = (n - pos[k]) / (pos[k + 1] - pos[k])
    ramp = cols[k] + (cols[k + 1] - cols[k]) * w
    c1 = np.float32([0.8, 0.3, 0.2]).astype(np.float64)
    c2 = np.float32([0.9, 0.85, 0.7]).astype(np.float64)
    expected = (ramp + (c1 - ramp) * 0.5) * c2
    got = O.eval_point_nocache(m, sp)
    assert np.allclose(got, expected, atol=1e-14)
