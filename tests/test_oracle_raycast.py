"""Pins of the ray-caster oracle that generates shading points (UV, material, ray-cone
gradients; Sec. 3.1 takes them from the renderer and cites Akenine-Moller et al. 2021 for
the cone).  Expected values come from the published SplitMix64 stream and from closed
forms of a floor seen from above, a sphere seen head-on and the footprint of a cone."""
import math
import os

import numpy as np
import pytest

from oracle import raycast as R
from paper_2305_07238_gb300 import workload as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hash_vectors.txt")


def _golden_splitmix():
    out = []
    for line in open(GOLDEN):
        f = line.split()
        if f and f[0] == "splitmix64":
            out.append((int(f[1], 16), int(f[2], 16)))
    return out


def test_counter_stream_is_the_published_sequence():
    # seeded with 0, the k-th output is the output function of k * gamma
    gold = _golden_splitmix()
    assert len(gold) == 3
    for k, (state, output) in enumerate(gold, start=1):
        assert state == (k * R.GAMMA) & R.MASK64
        assert int(R.splitmix64_at(0, k)) == output


def test_jitter_by_hand():
    # pass 0, pixel 0 -> output 1 = 0xE220A8397B1DCDAF: bits 40..63 and 16..39
    jx, jy = R.jitter(0, 0, np.array([0]))
    assert jx[0] == 0xE220A8 / 2 ** 24 and jy[0] == 0x397B1D / 2 ** 24
    # pass 1 starts 2^32 outputs further on
    jx1, _ = R.jitter(0, 1, np.array([0]))
    r = int(R.splitmix64_at(0, (1 << 32) + 1))
    assert jx1[0] == (r >> 40) / 2 ** 24
    jx, jy = R.jitter(7, 3, np.arange(100000))
    assert jx.min() >= 0 and jx.max() < 1 and abs(jx.mean() - 0.5) < 0.01 and abs(jy.mean() - 0.5) < 0.01


def _floor_scene(s=0.25, h=2.0, W_=6, H_=4, th=0.4):
    objs = np.zeros(1, dtype=W.OBJECT_DTYPE)
    objs[0] = (W.KIND_PLANE, 5, 0 | (2 << 8), s, (0.0, 1.0, 0.0, 0.0))
    cam = {"eye": np.array([0.0, h, 0.0], np.float32), "fwd": np.array([0.0, -1.0, 0.0], np.float32),
           "right": np.array([1.0, 0.0, 0.0], np.float32), "up": np.array([0.0, 0.0, -1.0], np.float32),
           "tan_half_y": np.float32(th), "width": W_, "height": H_}
    return objs, cam


def test_floor_from_above_closed_form():
    s, h, W_, H_, th = 0.25, 2.0, 6, 4, np.float32(0.4)
    objs, cam = _floor_scene(s, h, W_, H_, th)
    r = R.cast(objs, cam, seed=3, pass_index=2)
    pix = np.arange(W_ * H_)
    jx, jy = R.jitter(3, 2, pix)
    sx = (2 * (pix % W_ + jx) / W_ - 1) * float(th) * W_ / H_
    sy = (1 - 2 * (pix // W_ + jy) / H_) * float(th)
    # the ray (sx, -1, -sy) from (0, h, 0) meets y = 0 at (h sx, 0, -h sy), at distance h |dir|
    norm = np.sqrt(sx * sx + 1 + sy * sy)
    assert np.allclose(r["px"], h * sx, atol=1e-12) and np.allclose(r["pz"], -h * sy, atol=1e-12)
    assert np.allclose(r["py"], 0.0, atol=1e-12) and np.allclose(r["t"], h * norm, rtol=1e-12)
    assert np.allclose(r["u"], np.mod(s * h * sx, 1.0), atol=1e-12)
    assert np.allclose(r["v"], np.mod(-s * h * sy, 1.0), atol=1e-12)
    assert np.all(r["mat"] == 5) and np.allclose(r["ny"], 1.0)
    # cone width w = t 2 tan / H; minor axis of length w, major of length w |dir| (1/|N.d|),
    # both in the floor, where the projection scales lengths by s
    w = h * norm * 2 * float(th) / H_
    g1 = np.hypot(r["g1u"], r["g1v"])
    g2 = np.hypot(r["g2u"], r["g2v"])
    assert np.allclose(g1, s * w, rtol=1e-12) and np.allclose(g2, s * w * norm, rtol=1e-12)
    assert np.allclose(r["g1u"] * r["g2u"] + r["g1v"] * r["g2v"], 0.0, atol=1e-15)


def test_sphere_head_on():
    objs = np.zeros(2, dtype=W.OBJECT_DTYPE)
    objs[0] = (W.KIND_PLANE, 1, 0 | (1 << 8), 1.0, (0.0, 0.0, 1.0, -50.0))    # back wall z = -50
    objs[1] = (W.KIND_SPHERE, 2, 0 | (2 << 8), 1.0, (0.0, 0.0, 0.0, 1.0))     # unit sphere
    cam = {"eye": np.array([0.0, 0.0, 10.0], np.float32), "fwd": np.array([0.0, 0.0, -1.0], np.float32),
           "right": np.array([1.0, 0.0, 0.0], np.float32), "up": np.array([0.0, 1.0, 0.0], np.float32),
           "tan_half_y": np.float32(1e-3), "width": 3, "height": 3}
    r = R.cast(objs, cam, seed=1, pass_index=0)
    assert np.all(r["obj"] == 1) and np.all(r["mat"] == 2)
    P = np.stack([r["px"], r["py"], r["pz"]], axis=1)
    N = np.stack([r["nx"], r["ny"], r["nz"]], axis=1)
    assert np.allclose(np.linalg.norm(P, axis=1), 1.0, atol=1e-12)
    assert np.allclose(N, P, atol=1e-12) and np.all(r["nz"] > 0.999)
    assert np.allclose(r["t"], 9.0, atol=1e-4)


def test_footprint_axes_closed_forms():
    # head-on: a circle of diameter w, axes orthogonal and tangent
    A1, A2, ndotd, L = R.footprint_axes([[0, 1, 0]], [[0, -1, 0]], np.array([2.0]))
    assert L[0] == 0 and ndotd[0] == -1
    assert math.isclose(np.linalg.norm(A1), 2.0) and math.isclose(np.linalg.norm(A2), 2.0)
    assert abs(A1[0] @ A2[0]) < 1e-15 and abs(A1[0][1]) < 1e-15 and abs(A2[0][1]) < 1e-15
    # oblique by theta: the major axis lies along the tangent part of d, stretched by 1/cos
    th = 1.1
    d = np.array([[math.sin(th), -math.cos(th), 0.0]])
    A1, A2, _, _ = R.footprint_axes([[0, 1, 0]], d, np.array([0.5]))
    assert np.allclose(np.abs(A1[0]), [0, 0, 0.5]) and np.allclose(A2[0], [0.5 / math.cos(th), 0, 0])
    # grazing: the stretch is capped at 1 / COS_MIN
    d = np.array([[math.cos(1e-6), -math.sin(1e-6), 0.0]])
    _, A2, _, _ = R.footprint_axes([[0, 1, 0]], d, np.array([1.0]))
    assert math.isclose(np.linalg.norm(A2), 1.0 / R.COS_MIN)


def test_room_scene_invariants():
    sc = W.Scene(W.SceneSpec(width=160, height=90))
    r = R.cast(sc.objects, sc.camera, seed=0, pass_index=0)
    assert np.all(np.isfinite(r["t"]))                                  # a closed room
    bx, by, bz = sc.spec.room
    assert np.all(np.abs(r["px"]) <= bx + 1e-9) and np.all((r["py"] >= -1e-9) & (r["py"] <= by + 1e-9))
    assert np.all(np.abs(r["pz"]) <= bz + 1e-9)
    P = np.stack([r["px"], r["py"], r["pz"]], axis=1)
    N = np.stack([r["nx"], r["ny"], r["nz"]], axis=1)
    assert np.allclose(np.linalg.norm(N, axis=1), 1.0)
    assert np.all((r["u"] >= 0) & (r["u"] < 1) & (r["v"] >= 0) & (r["v"] < 1))
    for k, ob in enumerate(sc.objects):
        sel = r["obj"] == k
        p = np.asarray(ob["p"], dtype=np.float64)
        assert np.all(r["mat"][sel] == ob["mat"])
        if ob["kind"] == W.KIND_PLANE:
            assert np.allclose(P[sel] @ p[:3], p[3], atol=1e-9)
            # the projection of an axis-aligned wall is isotropic: closed-form footprint
            d = (P[sel] - sc.camera["eye"].astype(np.float64)) / r["t"][sel, None]
            cosv = np.maximum(np.abs(d @ p[:3]), R.COS_MIN)
            w = r["t"][sel] * 2 * float(sc.camera["tan_half_y"]) / sc.camera["height"]
            s = float(ob["uv_scale"])
            assert np.allclose(np.hypot(r["g1u"][sel], r["g1v"][sel]), s * w, rtol=1e-9)
            assert np.allclose(np.hypot(r["g2u"][sel], r["g2v"][sel]), s * w / cosv, rtol=1e-9)
        else:
            assert np.allclose(np.linalg.norm(P[sel] - p[:3], axis=1), p[3], atol=1e-9)
    assert r["robust"].mean() > 0.99


def test_floor_levels_follow_eq1():
    # on the floor the smaller gradient is the minor axis, of length s w, so Eq. 1 gives
    # floor(-log2(s w)) there; the oracle's level function must agree on the FP32 values
    from oracle import oracle as O
    s, h, W_, H_, th = 0.25, 2.0, 6, 4, np.float32(0.02)
    objs, cam = _floor_scene(s, h, W_, H_, th)
    r = R.cast(objs, cam, seed=9, pass_index=1)
    w = r["t"] * 2 * float(th) / H_
    expect = np.clip(np.floor(-np.log2(s * w)), 0, 13).astype(int)
    got = [O.level(np.float32(a), np.float32(b), np.float32(c), np.float32(d))
           for a, b, c, d in zip(r["g1u"], r["g1v"], r["g2u"], r["g2v"])]
    # away from a power of two (where FP32 rounding may tip the floor) they agree exactly
    frac = -np.log2(s * w) - np.floor(-np.log2(s * w))
    ok = (frac > 1e-4) & (frac < 1 - 1e-4)
    assert ok.sum() > 0 and np.array_equal(np.asarray(got)[ok], expect[ok])
