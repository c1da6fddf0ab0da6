"""FP64 oracle of the ray caster that generates shading points (TEST INFRASTRUCTURE ONLY).

Only the test suite, the smoke check and the benchmark's CPU legs may use this module.
It shares no code with the CUDA library: every formula below is written again from its
source.

What it computes, per pixel of a pinhole camera, one sample per pass:
  * the sample position inside the pixel, from a counter-based SplitMix64 stream (Steele,
    Lea & Flood 2014): the k-th output of the generator seeded with `seed` is the output
    function of seed + k * 0x9E3779B97F4A7C15, with k = pass * 2^32 + pixel + 1; the top 24
    bits give the x offset, the next 24 bits (bits 16..39) the y offset, each times 2^-24;
  * the closest hit of the ray with the scene's planes and spheres (t > 1e-4);
  * the shading point the paper's renderer would hand to the material system (Sec. 3.1):
    position, normal, material, texture coordinates of a planar projection, and the
    texture-coordinate gradients along both axes of the ray cone's elliptic footprint
    (Sec. 3.1 cites Akenine-Moller et al. 2021 for them).  A primary ray from a pinhole
    has a cone of spread angle 2 tan(fov_y / 2) / height and zero initial width, so its
    width at distance t is that angle times t.  The footprint's minor axis, of that width,
    lies along N x d; its major axis along the tangent part of d, stretched by 1 / |N . d|
    (clamped to at most 1000).  The gradients are these axes mapped by the projection.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1
T_MIN = 1e-4
COS_MIN = 1e-3          # |N . d| below this is clamped (grazing hits)
CROSS_MIN = 1e-6        # |N x d| below this: head-on, the minor axis takes a fixed tangent


def splitmix64_output(z):
    """SplitMix64 output function of a state (numpy uint64 arrays wrap mod 2^64)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def splitmix64_at(seed: int, k):
    """The k-th output (k >= 1) of SplitMix64 seeded with `seed`."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & MASK64) + k * np.uint64(GAMMA)
    return splitmix64_output(state)


def jitter(seed: int, pass_index: int, pixel):
    """Sample offsets (x, y) in [0, 1) of the given pixels for one pass."""
    pixel = np.asarray(pixel, dtype=np.uint64)
    r = splitmix64_at(seed, (np.uint64(pass_index) << np.uint64(32)) + pixel + np.uint64(1))
    jx = (r >> np.uint64(40)).astype(np.float64) * 2.0 ** -24
    jy = ((r >> np.uint64(16)) & np.uint64(0xFFFFFF)).astype(np.float64) * 2.0 ** -24
    return jx, jy


def footprint_axes(N, d, width):
    """The two axes of a ray cone's footprint on a surface of normal N hit along the unit
    direction d, for a cone of the given width at the hit (rows of N, d; width per row):
    A1 of length `width` along N x d (a fixed tangent when the hit is head-on), A2 along the
    tangent part of d (N x A1 when head-on) of length width / max(|N . d|, COS_MIN)."""
    N = np.atleast_2d(np.asarray(N, dtype=np.float64))
    d = np.atleast_2d(np.asarray(d, dtype=np.float64))
    width = np.asarray(width, dtype=np.float64)
    ndotd = np.sum(N * d, axis=1)
    cosv = np.maximum(np.abs(ndotd), COS_MIN)
    m1 = np.cross(N, d)
    L = np.linalg.norm(m1, axis=1)
    head_on = L < CROSS_MIN
    helper = np.where(np.abs(N[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    m1 = np.where(head_on[:, None], np.cross(N, helper), m1)
    m1 /= np.linalg.norm(m1, axis=1, keepdims=True)
    m2 = np.where(head_on[:, None], np.cross(N, m1), d - ndotd[:, None] * N)
    m2 /= np.linalg.norm(m2, axis=1, keepdims=True)
    return width[..., None] * m1, (width / cosv)[..., None] * m2, ndotd, L


def cast(objects, camera, seed: int, pass_index: int, rows=None) -> dict:
    """Shading points of one pass (scanline order; rows = (y0, y1) restricts to a band).
    Returns float64 arrays u, v, px, py, pz, nx, ny, nz, g1u, g1v, g2u, g2v, uint32 mat,
    the hit object `obj`, and `robust`: hits whose object, and whose footprint branch,
    cannot change under a relative perturbation of about 1e-4 (used to compare with a
    lower-precision evaluation of the same formulas)."""
    W, H = int(camera["width"]), int(camera["height"])
    y0, y1 = rows if rows is not None else (0, H)
    pix = np.arange(y0 * W, y1 * W, dtype=np.int64)
    x = (pix % W).astype(np.float64)
    y = (pix // W).astype(np.float64)
    jx, jy = jitter(seed, pass_index, pix)
    th = float(camera["tan_half_y"])
    eye = np.asarray(camera["eye"], dtype=np.float64)
    fwd = np.asarray(camera["fwd"], dtype=np.float64)
    right = np.asarray(camera["right"], dtype=np.float64)
    up = np.asarray(camera["up"], dtype=np.float64)
    sx = (2.0 * (x + jx) / W - 1.0) * th * (W / H)
    sy = (1.0 - 2.0 * (y + jy) / H) * th
    d = fwd[None, :] + sx[:, None] * right[None, :] + sy[:, None] * up[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)

    n_pts, n_obj = len(pix), len(objects)
    tk = np.full((n_obj, n_pts), np.inf)          # closest valid distance per object
    disc_rel = np.full((n_obj, n_pts), np.inf)    # sphere discriminant / r^2
    for k, ob in enumerate(objects):
        p = np.asarray(ob["p"], dtype=np.float64)
        if int(ob["kind"]) == 0:
            nrm, dd = p[:3], p[3]
            den = d @ nrm
            with np.errstate(divide="ignore", invalid="ignore"):
                t = (dd - eye @ nrm) / den
            tk[k] = np.where(t > T_MIN, t, np.inf)
        else:
            # the discriminant as r^2 - |q|^2, q the offset of the centre from the ray's
            # closest approach (Haines et al. 2019): the same value as b^2 - (|oc|^2 - r^2)
            # without its cancellation
            c, r = p[:3], p[3]
            oc = eye - c
            b = d @ oc
            q = oc[None, :] - b[:, None] * d
            disc = r * r - np.sum(q * q, axis=1)
            s = np.sqrt(np.maximum(disc, 0.0))
            t0, t1 = -b - s, -b + s
            t = np.where(t0 > T_MIN, t0, np.where(t1 > T_MIN, t1, np.inf))
            tk[k] = np.where(disc >= 0.0, t, np.inf)
            disc_rel[k] = np.where(disc >= 0.0, disc / (r * r), np.inf)
    obj = np.argmin(tk, axis=0)
    srt = np.sort(tk, axis=0)
    t = srt[0]
    gap_ok = (srt[1] - srt[0]) > 1e-3 * srt[0] if n_obj > 1 else np.ones(n_pts, bool)
    P = eye[None, :] + t[:, None] * d
    N = np.zeros_like(P)
    mat = np.zeros(n_pts, dtype=np.uint32)
    scale = np.zeros(n_pts)
    a0 = np.zeros(n_pts, dtype=np.int64)
    a1 = np.zeros(n_pts, dtype=np.int64)
    tangent_ok = np.ones(n_pts, bool)
    for k, ob in enumerate(objects):
        sel = obj == k
        if not sel.any():
            continue
        p = np.asarray(ob["p"], dtype=np.float64)
        if int(ob["kind"]) == 0:
            N[sel] = p[:3]
        else:
            N[sel] = (P[sel] - p[:3]) / p[3]
            tangent_ok[sel] = disc_rel[k][sel] > 1e-4
        mat[sel] = int(ob["mat"])
        scale[sel] = float(ob["uv_scale"])
        a0[sel] = int(ob["axes"]) & 0xFF
        a1[sel] = int(ob["axes"]) >> 8
    idx = np.arange(n_pts)
    uu = scale * P[idx, a0]
    vv = scale * P[idx, a1]
    u = uu - np.floor(uu)
    v = vv - np.floor(vv)
    # ray cone footprint (Sec. 3.1)
    width = t * (2.0 * th / H)
    A1, A2, ndotd, L = footprint_axes(N, d, width)
    g1u, g1v = scale * A1[idx, a0], scale * A1[idx, a1]
    g2u, g2v = scale * A2[idx, a0], scale * A2[idx, a1]
    # an FP32 distance to a plane keeps a relative error of a few 1e-6 above |N . d| = 0.05
    robust = gap_ok & tangent_ok & (np.abs(ndotd) > 0.05) & ((L > 2.0 * CROSS_MIN) | (L < 0.5 * CROSS_MIN))
    return {"u": u, "v": v, "mat": mat, "px": P[:, 0], "py": P[:, 1], "pz": P[:, 2],
            "nx": N[:, 0], "ny": N[:, 1], "nz": N[:, 2], "g1u": g1u, "g1v": g1v, "g2u": g2u, "g2v": g2v,
            "obj": obj, "t": t, "robust": robust}
