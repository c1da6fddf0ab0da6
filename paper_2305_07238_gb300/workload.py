"""Seeded synthetic inputs: material networks in the IR format and shading-point streams.

This module only draws random numbers that shape inputs.  It holds none of the
method's arithmetic (no texel quantisation, hashing, node evaluation or caching),
so both the CUDA path and the CPU oracle can take their inputs from it.

The paper's scenes (Classroom, Junk Shop, ...; Sec. 4) are not available, so the
streams below stand in for them:

* ``tiny``     -- one 8-node material (2-octave gradient noise on UV -> 4-stop colour
  ramp -> mix with a constant colour -> multiply), 64x64 pixels x 4 spp, UV uniform
  on [0,1)^2, processed as 4 passes of 4096 points.
* ``frame``    -- randomly generated networks (node counts log-uniform), materials
  drawn per 8x8 pixel tile from a Zipf law, UV an affine function of the pixel
  position inside the tile plus per-sample jitter, position on a per-tile plane,
  one normal per tile, one sample per pixel per pass; optionally ray-cone gradients
  per sample, or whole path-traced passes (direct samples, then indirect points of
  later bounces that land anywhere in the scene, each with its visibility class).
* ``scene``    -- a closed room of planes with spheres on its floor, a material per
  object (Zipf) and a pinhole camera: the input of the ray caster that generates
  shading points.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# --------------------------------------------------------------------------------------
# IR format.  The operator numbering and the node layout are the library's input format;
# the C header of the library and the oracle each state them again.
# --------------------------------------------------------------------------------------
OP_UV = 0
OP_POSITION = 1
OP_NORMAL = 2
OP_CONST = 3
OP_UV_AFFINE = 4
OP_FBM = 5
OP_VORONOI = 6
OP_CHECKER = 7
OP_RAMP = 8
OP_MIX = 9
OP_ADD = 10
OP_MUL = 11
OP_POW = 12
OP_FACING = 13
NUM_OPS = 14

OP_NAMES = {
    OP_UV: "UV", OP_POSITION: "POSITION", OP_NORMAL: "NORMAL", OP_CONST: "CONST",
    OP_UV_AFFINE: "UV_AFFINE", OP_FBM: "FBM", OP_VORONOI: "VORONOI", OP_CHECKER: "CHECKER",
    OP_RAMP: "RAMP", OP_MIX: "MIX", OP_ADD: "ADD", OP_MUL: "MUL", OP_POW: "POW",
    OP_FACING: "FACING",
}

NODE_DTYPE = np.dtype(
    [("op", "<u4"), ("inp", "<i4", (4,)), ("ip", "<i4", (4,)), ("fp", "<f4", (16,))],
    align=False,
)
assert NODE_DTYPE.itemsize == 100

POINT_FIELDS = ("u", "v", "mat", "px", "py", "pz", "nx", "ny", "nz")
# optional per-point ray-cone texture-coordinate gradients (the two axes of the footprint)
CONE_FIELDS = ("g1u", "g1v", "g2u", "g2v")


class Builder:
    """Appends nodes in topological order; returns each node's index (its node ID)."""

    def __init__(self):
        self.rows = []

    def add(self, op, inputs=(), ip=(), fp=()):
        inp = [-1, -1, -1, -1]
        for k, x in enumerate(inputs):
            inp[k] = -1 if x is None else int(x)
        ipv = [0, 0, 0, 0]
        for k, x in enumerate(ip):
            ipv[k] = int(x)
        fpv = [0.0] * 16
        for k, x in enumerate(fp):
            fpv[k] = float(x)
        self.rows.append((op, inp, ipv, fpv))
        return len(self.rows) - 1

    def __len__(self):
        return len(self.rows)

    def build(self) -> np.ndarray:
        arr = np.zeros(len(self.rows), dtype=NODE_DTYPE)
        for i, (op, inp, ipv, fpv) in enumerate(self.rows):
            arr[i]["op"] = op
            arr[i]["inp"] = inp
            arr[i]["ip"] = ipv
            arr[i]["fp"] = fpv
        return arr


# --------------------------------------------------------------------------------------
# The tiny 8-node material
# --------------------------------------------------------------------------------------
def material_tiny() -> np.ndarray:
    """UV -> 2-octave noise (scale 8, lacunarity 2, gain 0.5) -> 4-stop ramp at
    0, .33, .66, 1 -> mix with a constant colour (factor 0.5) -> multiply by a
    constant colour.  Node 7 is the output."""
    b = Builder()
    uv = b.add(OP_UV)
    n = b.add(OP_FBM, [uv], ip=[2, 1], fp=[8.0, 2.0, 0.5])
    ramp = b.add(OP_RAMP, [n], ip=[4], fp=[0.0, 0.33, 0.66, 1.0,
                                          0.05, 0.10, 0.40,
                                          0.20, 0.55, 0.30,
                                          0.85, 0.75, 0.20,
                                          0.95, 0.95, 0.90])
    c1 = b.add(OP_CONST, fp=[0.8, 0.3, 0.2])
    fac = b.add(OP_CONST, fp=[0.5, 0.5, 0.5])
    mix = b.add(OP_MIX, [ramp, c1, fac])
    c2 = b.add(OP_CONST, fp=[0.9, 0.85, 0.7])
    b.add(OP_MUL, [mix, c2])
    return b.build()


def points_uniform(n: int, seed: int = 0, n_mats: int = 1) -> dict:
    """n shading points with UV uniform on [0,1)^2, random position and unit normal."""
    rng = np.random.Generator(np.random.PCG64(seed))
    uv = rng.random((2, n))
    p = rng.uniform(-4.0, 4.0, (3, n))
    nrm = rng.normal(size=(3, n))
    nrm /= np.linalg.norm(nrm, axis=0, keepdims=True)
    mat = rng.integers(0, n_mats, n) if n_mats > 1 else np.zeros(n)
    return _pack(uv[0], uv[1], mat, p, nrm)


def _pack(u, v, mat, p, nrm) -> dict:
    return {
        "u": np.ascontiguousarray(u, dtype=np.float32),
        "v": np.ascontiguousarray(v, dtype=np.float32),
        "mat": np.ascontiguousarray(mat, dtype=np.uint32),
        "px": np.ascontiguousarray(p[0], dtype=np.float32),
        "py": np.ascontiguousarray(p[1], dtype=np.float32),
        "pz": np.ascontiguousarray(p[2], dtype=np.float32),
        "nx": np.ascontiguousarray(nrm[0], dtype=np.float32),
        "ny": np.ascontiguousarray(nrm[1], dtype=np.float32),
        "nz": np.ascontiguousarray(nrm[2], dtype=np.float32),
    }


def _fields(pts: dict):
    return POINT_FIELDS + (CONE_FIELDS if all(k in pts for k in CONE_FIELDS) else ()) + \
        (("vis",) if "vis" in pts else ())


def slice_points(pts: dict, lo: int, hi: int) -> dict:
    return {k: np.ascontiguousarray(pts[k][lo:hi]) for k in _fields(pts)}


def concat_points(parts) -> dict:
    return {k: np.concatenate([p[k] for p in parts]) for k in _fields(parts[0])}


# --------------------------------------------------------------------------------------
# Random material networks
# --------------------------------------------------------------------------------------
def _loguniform(rng, lo, hi):
    return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


class _NetGen:
    """Grows one network: UV-only texture trees joined by shading-point dependent nodes."""

    def __init__(self, rng, smooth=False):
        self.rng = rng
        self.smooth = smooth   # low-frequency textures only (no checker), for surrogates
        self.b = Builder()
        self.uv = self.b.add(OP_UV)
        self.pos = None
        self.nor = None

    # -- helpers ------------------------------------------------------------------
    def _seed(self):
        return int(self.rng.integers(0, 2**31 - 1))

    def _color(self):
        return [float(x) for x in self.rng.uniform(0.0, 1.0, 3)]

    def _position(self):
        if self.pos is None:
            self.pos = self.b.add(OP_POSITION)
        return self.pos

    def _normal(self):
        if self.nor is None:
            self.nor = self.b.add(OP_NORMAL)
        return self.nor

    def _fbm_params(self, scale_lo, scale_hi, max_freq):
        rng = self.rng
        s = _loguniform(rng, scale_lo, scale_hi)
        lac = float(rng.uniform(1.8, 2.2))
        gain = float(rng.uniform(0.4, 0.6))
        oct_cap = 1 + int(math.floor(math.log(max_freq / s) / math.log(lac))) if s < max_freq else 1
        octaves = int(rng.integers(1, max(1, min(8, oct_cap)) + 1))
        return [octaves, self._seed()], [s, lac, gain]

    # -- UV-only trees ---------------------------------------------------------------
    def _coord(self, budget):
        """A texture coordinate: the UV node itself or an affine map of it."""
        if budget >= 1 and self.rng.random() < 0.5:
            th = float(self.rng.uniform(0.0, 2.0 * math.pi))
            sc = _loguniform(self.rng, 0.5, 1.5 if self.smooth else 2.0)
            c, s = sc * math.cos(th), sc * math.sin(th)
            off = [float(x) for x in self.rng.uniform(0.0, 4.0, 2)]
            return self.b.add(OP_UV_AFFINE, [self.uv], fp=[c, -s, s, c, off[0], off[1]]), 1
        return self.uv, 0

    def _texture(self, budget):
        """A texture leaf using about `budget` nodes (>= 1)."""
        rng = self.rng
        kind = rng.choice(["fbm", "fbm", "voronoi"] if self.smooth else ["fbm", "fbm", "voronoi", "checker"])
        if kind == "checker":
            s = float(2 ** int(rng.integers(1, 10)))
            return self.b.add(OP_CHECKER, [self.uv], fp=[s] + self._color() + self._color())
        coord, used = self._coord(budget - 1)
        if kind == "fbm":
            ip, fp = self._fbm_params(0.5, 2.0, 4.0) if self.smooth else self._fbm_params(2.0, 16.0, 256.0)
            return self.b.add(OP_FBM, [coord], ip=ip, fp=fp)
        s = _loguniform(rng, 0.5, 2.0) if self.smooth else _loguniform(rng, 2.0, 32.0)
        return self.b.add(OP_VORONOI, [coord], ip=[0, self._seed()], fp=[s])

    def _ramp(self, src):
        rng = self.rng
        ns = int(rng.integers(2, 5))
        pos = []
        for k in range(ns):
            base = k / (ns - 1)
            jit = 0.1 / (ns - 1)
            pos.append(float(min(1.0, max(0.0, base + rng.uniform(-jit, jit)))))
        pos[0], pos[-1] = min(pos[0], 0.1), max(pos[-1], 0.9)
        pos = sorted(pos)
        fp = pos + [0.0] * (4 - ns)
        for _ in range(ns):
            fp += self._color()
        return self.b.add(OP_RAMP, [src], ip=[ns], fp=fp)

    def tree(self, budget):
        """A UV-only tree of about `budget` nodes; returns its top node."""
        rng = self.rng
        if budget <= 2:
            return self._texture(budget)
        r = rng.random()
        if r < 0.25:
            src = self.tree(budget - 1)
            if rng.random() < 0.6:
                return self._ramp(src)
            return self.b.add(OP_POW, [src], fp=[float(rng.uniform(1.0, 2.0))])
        rest = budget - 1
        if r < 0.7:
            # mix of two sub-trees with a constant factor or a third sub-tree
            if rest >= 6 and rng.random() < 0.5:
                ka = max(2, int(rest * rng.uniform(0.3, 0.5)))
                kb = max(2, int((rest - ka) * rng.uniform(0.4, 0.6)))
                kc = max(1, rest - ka - kb)
                a, b_, c = self.tree(ka), self.tree(kb), self.tree(kc)
                return self.b.add(OP_MIX, [a, b_, c])
            ka = max(1, int(rest * rng.uniform(0.3, 0.7)))
            a, b_ = self.tree(ka), self.tree(max(1, rest - ka))
            return self.b.add(OP_MIX, [a, b_], fp=[float(rng.uniform(0.0, 1.0))])
        ka = max(1, int(rest * rng.uniform(0.3, 0.7)))
        a = self.tree(ka)
        if rng.random() < 0.3:
            b_ = self.b.add(OP_CONST, fp=self._color())
            if rest - ka > 1:
                b_ = self.b.add(OP_MIX, [b_, self.tree(rest - ka - 1)],
                                fp=[float(rng.uniform(0.2, 0.8))])
        else:
            b_ = self.tree(max(1, rest - ka))
        return self.b.add(OP_ADD if rng.random() < 0.4 else OP_MUL, [a, b_])

    # -- shading-point dependent factors -------------------------------------------------
    def sp_factor(self):
        rng = self.rng
        r = rng.random()
        if r < 0.4:
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            return self.b.add(OP_FACING, [self._normal()], fp=[float(x) for x in d])
        if r < 0.75:
            ip, fp = self._fbm_params(0.5, 4.0, 32.0)
            return self.b.add(OP_FBM, [self._position()], ip=ip, fp=fp)
        if r < 0.9:
            return self.b.add(OP_VORONOI, [self._position()], ip=[0, self._seed()],
                              fp=[_loguniform(rng, 0.5, 4.0)])
        s = float(2 ** int(rng.integers(-1, 3)))
        return self.b.add(OP_CHECKER, [self._position()], fp=[s] + self._color() + self._color())


def random_material(rng: np.random.Generator, n_nodes: int, sp_frac: float,
                    n_trees: int | None = None, smooth: bool = False) -> np.ndarray:
    """A network of about n_nodes nodes in which about sp_frac of the nodes depend on
    position or normal.  UV-only texture trees (noise, Worley, checker, ramps, mixes,
    add/multiply, power) are joined by MIX nodes whose factor depends on the shading
    point, so the top node of each tree is a cacheable node."""
    g = _NetGen(rng, smooth=smooth)
    n_sp = max(2, int(round(sp_frac * n_nodes)))
    if n_trees is None:
        n_trees = max(1, n_sp // 2)
    n_uv = max(2 * n_trees, n_nodes - n_sp - 1)
    w = rng.dirichlet(np.ones(n_trees)) if n_trees > 1 else np.ones(1)
    sizes = [max(2, int(round(x * n_uv))) for x in w]
    trees = [g.tree(s) for s in sizes]
    acc = trees[0]
    if len(trees) == 1:
        acc = g.b.add(OP_MIX, [acc, g.b.add(OP_CONST, fp=g._color()), g.sp_factor()])
    for t in trees[1:]:
        acc = g.b.add(OP_MIX, [acc, t, g.sp_factor()])
    # spend what is left of the SP budget on SP-class post-processing
    while len(g.b) < n_nodes:
        r = rng.random()
        if r < 0.4:
            acc = g.b.add(OP_MUL, [acc, g.sp_factor()])
        elif r < 0.7:
            acc = g.b.add(OP_POW, [acc], fp=[float(rng.uniform(1.0, 2.0))])
        else:
            acc = g.b.add(OP_MIX, [acc, g.b.add(OP_CONST, fp=g._color()), g.sp_factor()])
    return g.b.build()


def random_materials(n_mats: int, lo: int, hi: int, sp_frac: float, seed: int = 0) -> list:
    """n_mats networks with node counts log-uniform on [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mats = []
    for _ in range(n_mats):
        n = int(round(_loguniform(rng, lo, hi)))
        mats.append(random_material(rng, n, sp_frac))
    return mats


def surrogate_materials(n_mats: int, lo: int = 500, hi: int = 2000, seed: int = 0) -> list:
    """Networks whose one cacheable node sits on a deep UV-only tree of low-frequency
    textures (noise of 1-3 octaves at scales 0.5-2, Worley at 0.5-2, ramps, mixes,
    add/multiply, power), feeding a single shading-point dependent mix: the shape a
    learned surrogate stands in for.  Node counts log-uniform on [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64([seed, 4]))
    mats = []
    for _ in range(n_mats):
        n = int(round(_loguniform(rng, lo, hi)))
        mats.append(random_material(rng, n, 2.0 / n, n_trees=1, smooth=True))
    return mats


# --------------------------------------------------------------------------------------
# Frame-shaped shading-point streams
# --------------------------------------------------------------------------------------
@dataclass
class FrameSpec:
    width: int = 1920
    height: int = 1080
    tile: int = 8
    n_mats: int = 64
    zipf_s: float = 1.1
    delta_lo: float = 2.0 ** -12
    delta_hi: float = 2.0 ** -8
    seed: int = 0
    aniso_hi: float = 4.0       # ray-cone footprints: axis ratio log-uniform on [1, aniso_hi]
    spread: float = 0.5         # footprint width = delta * 2^U(-spread, spread) per sample


class Frame:
    """Per-tile material, UV mapping and surface plane; points() draws one pass."""

    def __init__(self, spec: FrameSpec):
        self.spec = spec
        rng = np.random.Generator(np.random.PCG64([spec.seed, 1]))
        tx = (spec.width + spec.tile - 1) // spec.tile
        ty = (spec.height + spec.tile - 1) // spec.tile
        nt = tx * ty
        ranks = np.arange(1, spec.n_mats + 1, dtype=np.float64)
        pz = ranks ** (-spec.zipf_s)
        pz /= pz.sum()
        rank_to_mat = rng.permutation(spec.n_mats)
        self.tile_mat = rank_to_mat[rng.choice(spec.n_mats, size=nt, p=pz)].astype(np.uint32)
        self.tile_o = rng.random((nt, 2))
        self.tile_delta = np.exp(rng.uniform(math.log(spec.delta_lo), math.log(spec.delta_hi), nt))
        nrm = rng.normal(size=(nt, 3))
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        self.tile_n = nrm
        helper = np.where(np.abs(nrm[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]),
                          np.array([[0.0, 1.0, 0.0]]))
        e1 = np.cross(nrm, helper)
        e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
        self.tile_e1 = e1
        self.tile_e2 = np.cross(nrm, e1)
        self.tile_c = rng.uniform(-8.0, 8.0, (nt, 3))
        # ray-cone footprint of a tile: orientation and axis ratio of the ellipse in UV
        crng = np.random.Generator(np.random.PCG64([spec.seed, 5]))
        self.tile_theta = crng.uniform(0.0, 2.0 * math.pi, nt)
        self.tile_aniso = np.exp(crng.uniform(0.0, math.log(spec.aniso_hi), nt))
        self.tiles_x = tx
        ys, xs = np.mgrid[0:spec.height, 0:spec.width]
        self.px_x = xs.ravel()
        self.px_y = ys.ravel()
        self.pix_tile = (self.px_y // spec.tile) * tx + (self.px_x // spec.tile)

    @property
    def n_pixels(self):
        return self.spec.width * self.spec.height

    def _pixel_layout(self):
        """Per-pixel copies of the per-tile quantities (built once, then reused)."""
        if getattr(self, "_pix", None) is None:
            t = self.pix_tile
            spec = self.spec
            self._pix = {
                "bx": (self.px_x % spec.tile).astype(np.float64),
                "by": (self.px_y % spec.tile).astype(np.float64),
                "fx": self.px_x.astype(np.float64), "fy": self.px_y.astype(np.float64),
                "ou": np.ascontiguousarray(self.tile_o[t, 0]), "ov": np.ascontiguousarray(self.tile_o[t, 1]),
                "d": self.tile_delta[t],
                "c": [np.ascontiguousarray(self.tile_c[t, k]) for k in range(3)],
                "e1": [np.ascontiguousarray(self.tile_e1[t, k]) for k in range(3)],
                "e2": [np.ascontiguousarray(self.tile_e2[t, k]) for k in range(3)],
                "mat": np.ascontiguousarray(self.tile_mat[t], dtype=np.uint32),
                "n": [np.ascontiguousarray(self.tile_n[t, k], dtype=np.float32) for k in range(3)],
                "cos": np.cos(self.tile_theta[t]), "sin": np.sin(self.tile_theta[t]),
                "aniso": self.tile_aniso[t],
            }
        return self._pix

    def points(self, pass_index: int, rows: tuple | None = None, cones: bool = False) -> dict:
        """One sample per pixel (scanline order) for pass `pass_index`; `rows` = (y0, y1)
        restricts to a band of pixel rows (same draws as the full pass).  cones: add the
        ray-cone gradients of every sample (CONE_FIELDS): an ellipse of the tile's
        orientation and axis ratio whose minor axis is delta * 2^U(-spread, spread)."""
        spec = self.spec
        rng = np.random.Generator(np.random.PCG64([spec.seed, 2, pass_index]))
        jit = rng.random((2, self.n_pixels))
        sel = slice(None)
        if rows is not None:
            sel = slice(rows[0] * spec.width, rows[1] * spec.width)
        L = self._pixel_layout()
        jx, jy = jit[0][sel], jit[1][sel]
        d = L["d"][sel]
        u = np.mod(L["ou"][sel] + d * (L["bx"][sel] + jx), 1.0)
        v = np.mod(L["ov"][sel] + d * (L["by"][sel] + jy), 1.0)
        w = 0.01
        wx = w * (L["fx"][sel] + jx)
        wy = w * (L["fy"][sel] + jy)
        p = [(L["c"][k][sel] + wx * L["e1"][k][sel] + wy * L["e2"][k][sel]) * 0.25 for k in range(3)]
        out = _pack(u, v, L["mat"][sel], p, [L["n"][k][sel] for k in range(3)])
        if cones:
            crng = np.random.Generator(np.random.PCG64([spec.seed, 6, pass_index]))
            f = d * np.exp2(crng.uniform(-spec.spread, spec.spread, self.n_pixels)[sel])
            c, s_, b = L["cos"][sel], L["sin"][sel], L["aniso"][sel]
            out.update(g1u=(f * c).astype(np.float32), g1v=(f * s_).astype(np.float32),
                       g2u=(-f * b * s_).astype(np.float32), g2v=(f * b * c).astype(np.float32))
        return out

    def points_paths(self, pass_index: int, bounce_frac=(0.5, 0.25), rows: tuple | None = None) -> dict:
        """One pass of a path tracer as one batch: the directly visible sample of every
        pixel (points() of the pass, visibility class 0), then for bounce k = 1, 2, ... the
        shading points of the paths still alive, a fraction bounce_frac[k-1] of the pixels,
        carrying class k in "vis".  An indirect ray lands anywhere in the scene, mostly off
        the parts the camera sees: each such point takes the material of a tile drawn
        uniformly from the frame (or from the band `rows`), a UV uniform on [0,1)^2 of that
        material and a position uniform in the scene's box, with that tile's normal."""
        spec = self.spec
        direct = self.points(pass_index, rows=rows)
        n0 = len(direct["u"])
        lo = rows[0] * spec.width if rows is not None else 0
        parts, vis = [direct], [np.zeros(n0, dtype=np.uint8)]
        L = self._pixel_layout()
        rng = np.random.Generator(np.random.PCG64([spec.seed, 7, pass_index]))
        for k, frac in enumerate(bounce_frac, start=1):
            m = int(round(frac * n0))
            pix = lo + rng.integers(0, n0, m)
            uv = rng.random((2, m))
            pos = rng.uniform(-4.0, 4.0, (3, m))
            parts.append(_pack(uv[0], uv[1], L["mat"][pix], pos, [L["n"][q][pix] for q in range(3)]))
            vis.append(np.full(m, k, dtype=np.uint8))
        out = {f: np.concatenate([p[f] for p in parts]) for f in POINT_FIELDS}
        out["vis"] = np.concatenate(vis)
        return out

    def points_torch(self, pass_index: int, device="cuda", rows: tuple | None = None) -> dict:
        """The same recipe drawn with torch's generator on `device` (for long sequences of
        passes whose host generation would dominate); the jitter comes from a different
        generator, so the values differ from points().  Returns torch tensors (mat as
        int32), SoA like points()."""
        import torch
        spec = self.spec
        key = ("_tpix", str(device))
        if getattr(self, "_tpix_key", None) != key:
            L = self._pixel_layout()
            T = lambda a: torch.as_tensor(a, device=device)
            self._tpix = {k: ([T(x) for x in v] if isinstance(v, list) else T(v)) for k, v in L.items()}
            self._tpix["mat"] = T(L["mat"].view(np.int32))
            self._tpix_key = key
        L = self._tpix
        g = torch.Generator(device=device)
        g.manual_seed(((spec.seed * 1_000_003) ^ (pass_index * 7919) ^ 0x5EED) & 0x7FFFFFFFFFFFFFFF)
        jit = torch.rand((2, self.n_pixels), generator=g, device=device, dtype=torch.float64)
        sel = slice(None)
        if rows is not None:
            sel = slice(rows[0] * spec.width, rows[1] * spec.width)
        jx, jy = jit[0][sel], jit[1][sel]
        d = L["d"][sel]
        u = torch.remainder(L["ou"][sel] + d * (L["bx"][sel] + jx), 1.0)
        v = torch.remainder(L["ov"][sel] + d * (L["by"][sel] + jy), 1.0)
        wx = 0.01 * (L["fx"][sel] + jx)
        wy = 0.01 * (L["fy"][sel] + jy)
        out = {"u": u.float().contiguous(), "v": v.float().contiguous(), "mat": L["mat"][sel].contiguous()}
        for k, name in enumerate(("px", "py", "pz")):
            out[name] = ((L["c"][k][sel] + wx * L["e1"][k][sel] + wy * L["e2"][k][sel]) * 0.25).float().contiguous()
        for k, name in enumerate(("nx", "ny", "nz")):
            out[name] = L["n"][k][sel].contiguous()
        return out


# --------------------------------------------------------------------------------------
# Procedural scene for the ray caster: a closed room and spheres resting on its floor
# --------------------------------------------------------------------------------------
# One record per object.  kind 0 = plane {n (unit), d}: the points x with n.x = d, the room
# on the side n.x >= d; kind 1 = sphere {centre, radius}.  Texture coordinates are a planar
# projection: (u, v) = fractional parts of uv_scale * (x[a0], x[a1]), a0 = axes & 0xFF,
# a1 = axes >> 8.  The layout is the library's input format; its C header states it again.
OBJECT_DTYPE = np.dtype([("kind", "<u4"), ("mat", "<u4"), ("axes", "<u4"), ("uv_scale", "<f4"),
                         ("p", "<f4", (4,))])
KIND_PLANE, KIND_SPHERE = 0, 1
CAMERA_FIELDS = ("eye", "fwd", "right", "up")


@dataclass
class SceneSpec:
    n_mats: int = 64
    n_spheres: int = 24
    room: tuple = (8.0, 6.0, 8.0)      # half width, height, half depth
    zipf_s: float = 1.1
    width: int = 1920
    height: int = 1080
    fov_y_deg: float = 60.0
    eye: tuple = (0.0, 3.0, 7.5)
    target: tuple = (0.0, 1.0, 0.0)
    seed: int = 0


class Scene:
    """Objects (OBJECT_DTYPE records) and a pinhole camera whose basis is given as FP32
    vectors: rays leave `eye` along fwd + sx right + sy up, with sx, sy the pixel's
    position on the image plane scaled by tan_half_y (and the aspect ratio for sx)."""

    def __init__(self, spec: SceneSpec):
        self.spec = spec
        rng = np.random.Generator(np.random.PCG64([spec.seed, 11]))
        bx, by, bz = spec.room
        planes = [((0, 1, 0), 0.0, (0, 2)), ((0, -1, 0), -by, (0, 2)),
                  ((1, 0, 0), -bx, (2, 1)), ((-1, 0, 0), -bx, (2, 1)),
                  ((0, 0, 1), -bz, (0, 1)), ((0, 0, -1), -bz, (0, 1))]
        n_obj = len(planes) + spec.n_spheres
        ranks = np.arange(1, spec.n_mats + 1, dtype=np.float64)
        pz = ranks ** (-spec.zipf_s)
        pz /= pz.sum()
        rank_to_mat = rng.permutation(spec.n_mats)
        mats = rank_to_mat[rng.choice(spec.n_mats, size=n_obj, p=pz)]
        scales = np.exp(rng.uniform(math.log(0.05), math.log(0.5), n_obj))
        objs = np.zeros(n_obj, dtype=OBJECT_DTYPE)
        for k, (nrm, d, axes) in enumerate(planes):
            objs[k] = (KIND_PLANE, mats[k], axes[0] | (axes[1] << 8), scales[k], (*nrm, d))
        for k in range(spec.n_spheres):
            r = float(np.exp(rng.uniform(math.log(0.3), math.log(1.5))))
            cx = float(rng.uniform(-bx + r, bx - r))
            cz = float(rng.uniform(-bz + r, bz - 2.0 - r))
            objs[len(planes) + k] = (KIND_SPHERE, mats[len(planes) + k], 0 | (2 << 8), scales[len(planes) + k],
                                     (cx, r, cz, r))
        self.objects = objs
        eye = np.array(spec.eye, dtype=np.float64)
        fwd = np.array(spec.target, dtype=np.float64) - eye
        fwd /= np.linalg.norm(fwd)
        right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
        right /= np.linalg.norm(right)
        up = np.cross(right, fwd)
        self.camera = {"eye": eye.astype(np.float32), "fwd": fwd.astype(np.float32),
                       "right": right.astype(np.float32), "up": up.astype(np.float32),
                       "tan_half_y": np.float32(math.tan(math.radians(spec.fov_y_deg) / 2.0)),
                       "width": spec.width, "height": spec.height}
