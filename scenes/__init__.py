"""Seeded synthetic scenes and per-frame motion for photon-path verification.

This module only produces input data: triangle soups, per-object albedo,
per-frame rigid transforms and light poses.  It contains none of the
path-verification arithmetic, so both the CUDA library and the FP64 CPU
oracle consume its output without sharing any method code.

Randomness comes from a counter-based SplitMix64 hash evaluated with numpy
uint64 arithmetic (wrapping), and trigonometry from Python's ``math`` module
on small tables, so a scene is reproducible bit for bit from its seed.

Workloads (all coordinates in metres, y up):

* ``tiny_box``  -- open 2x2x2 box (10 triangles) + unit cube moving +0.05 x per
  frame, one point light at (0, 1.8, 0), albedo 0.7, 10 000 paths, 3 bounces.
* ``city``      -- 100x100 m floor with 16 666 random boxes (~200k triangles),
  4 moving tori (2048 triangles each), a 1x1 m area light translating 0.1 m per
  frame; 1M paths, 7 bounces, tau = 1 %.
* ``villa``     -- 4x3 rooms of 5x5x3 m, exactly 2 000 000 static triangles
  (shell, furniture, 30 % small clutter), 10 moving tori (5000 triangles each),
  one point light, one static and one moving (and tilting) area light;
  3M paths, 7 bounces.

These stand in for the paper's Conference / Armadillo / Villa scenes (Sec. 5),
whose meshes are not available: the shapes, sizes, motion and light types
follow the paper's description, the geometry itself is procedural.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Tuple

import numpy as np

LIGHT_POINT = 0
LIGHT_RECT = 1

_U64 = np.uint64


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on a uint64 array."""
    with np.errstate(over="ignore"):
        z = x + _U64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> _U64(30))) * _U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> _U64(27))) * _U64(0x94D049BB133111EB)
        return z ^ (z >> _U64(31))


class Stream:
    """Counter-based uniform stream: value i = hash(seed, tag, i)."""

    def __init__(self, seed: int, tag: int):
        with np.errstate(over="ignore"):
            base = _splitmix64(np.array([seed * 0x100000001B3 + tag], dtype=np.uint64))[0]
        self._base = base
        self._off = 0

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        idx = np.arange(self._off, self._off + n, dtype=np.uint64)
        self._off += n
        with np.errstate(over="ignore"):
            h = _splitmix64(idx * _U64(0xD1B54A32D192ED03) + self._base)
        u = (h >> _U64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def integers(self, n: int, hi: int) -> np.ndarray:
        return np.minimum((self.uniform(n) * hi).astype(np.int64), hi - 1)

    def permutation(self, n: int) -> np.ndarray:
        return np.argsort(self.uniform(n), kind="stable")


@dataclass
class Light:
    """A light pose.  ``normal`` is the emitting side of a rectangle,
    ``tangent`` the direction of its ``size[0]`` edge; both ignored for
    point lights.  ``power`` is the RGB flux, split evenly over ``n_paths``."""
    type: int
    pos: Tuple[float, float, float]
    normal: Tuple[float, float, float] = (0.0, -1.0, 0.0)
    tangent: Tuple[float, float, float] = (1.0, 0.0, 0.0)
    size: Tuple[float, float] = (0.0, 0.0)
    power: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    n_paths: int = 0

    def as_f32(self) -> "Light":
        f = lambda v: tuple(float(np.float32(x)) for x in v)
        return Light(self.type, f(self.pos), f(self.normal), f(self.tangent),
                     f(self.size), f(self.power), int(self.n_paths))


@dataclass
class Scene:
    name: str
    verts: np.ndarray            # float32 [T,3,3]; dynamic objects in object-local space
    tri_object: np.ndarray       # uint32 [T]
    object_dynamic: np.ndarray   # uint8 [O]
    object_albedo: np.ndarray    # float32 [O,3]
    max_bounces: int
    diag: float                  # scene diagonal: unit of all geometric tolerances
    atlas_rect: Tuple[float, float, float, float]   # x0, z0, x1, z1 (top-down XZ)
    seed: int
    frames: int
    tau: float
    _xform_fn: Callable[[int], np.ndarray] = field(repr=False, default=None)
    _light_fn: Callable[[int], List[Light]] = field(repr=False, default=None)

    @property
    def n_tris(self) -> int:
        return int(self.verts.shape[0])

    @property
    def n_objects(self) -> int:
        return int(self.object_dynamic.shape[0])

    def xforms(self, frame: int) -> np.ndarray:
        """float32 [O,12] row-major 3x4 [R | t] per object at ``frame`` (1-based)."""
        return self._xform_fn(frame)

    def lights(self, frame: int) -> List[Light]:
        return [l.as_f32() for l in self._light_fn(frame)]

    @property
    def n_paths(self) -> int:
        return int(sum(l.n_paths for l in self._light_fn(1)))

    def world_verts(self, frame: int) -> np.ndarray:
        """World-space float64 vertices at ``frame`` (for plotting/tests only)."""
        x = self.xforms(frame).astype(np.float64).reshape(-1, 3, 4)
        m = x[self.tri_object]
        v = self.verts.astype(np.float64)
        return np.einsum("tij,tkj->tki", m[:, :, :3], v) + m[:, None, :, 3]


# ----------------------------------------------------------------------------
# geometry helpers (plain float64 numpy; output rounded to float32 once)
# ----------------------------------------------------------------------------

def _quad_grid(origin, eu, ev, nu: int, nv: int) -> np.ndarray:
    """Tessellate the parallelogram origin + s*eu + t*ev (s,t in [0,1]) into
    nu x nv cells, 2 triangles each: float64 [2*nu*nv,3,3]."""
    o = np.asarray(origin, np.float64)
    eu = np.asarray(eu, np.float64)
    ev = np.asarray(ev, np.float64)
    i = np.arange(nu, dtype=np.float64)
    j = np.arange(nv, dtype=np.float64)
    s0 = (i / nu)[:, None]
    s1 = ((i + 1) / nu)[:, None]
    t0 = (j / nv)[None, :]
    t1 = ((j + 1) / nv)[None, :]

    def P(s, t):
        return o + s[..., None] * eu + t[..., None] * ev

    p00 = P(np.broadcast_to(s0, (nu, nv)), np.broadcast_to(t0, (nu, nv))).reshape(-1, 3)
    p10 = P(np.broadcast_to(s1, (nu, nv)), np.broadcast_to(t0, (nu, nv))).reshape(-1, 3)
    p11 = P(np.broadcast_to(s1, (nu, nv)), np.broadcast_to(t1, (nu, nv))).reshape(-1, 3)
    p01 = P(np.broadcast_to(s0, (nu, nv)), np.broadcast_to(t1, (nu, nv))).reshape(-1, 3)
    a = np.stack([p00, p10, p11], axis=1)
    b = np.stack([p00, p11, p01], axis=1)
    return np.stack([a, b], axis=1).reshape(-1, 3, 3)


def _boxes(lo: np.ndarray, hi: np.ndarray, n: int = 1, bottom: bool = True) -> np.ndarray:
    """Axis-aligned boxes [B,3] lo/hi, each face an n x n grid:
    float64 [B, F*2*n*n, 3, 3] with F = 6 (or 5 without the bottom face)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    unit = []
    x0, x1 = 0.0, 1.0
    faces = [
        ((0, 0, 0), (0, 0, 1), (0, 1, 0)),   # x = 0
        ((1, 0, 0), (0, 1, 0), (0, 0, 1)),   # x = 1
        ((0, 1, 0), (0, 0, 1), (1, 0, 0)),   # y = 1 (top)
        ((0, 0, 0), (0, 1, 0), (1, 0, 0)),   # z = 0
        ((0, 0, 1), (1, 0, 0), (0, 1, 0)),   # z = 1
    ]
    if bottom:
        faces.append(((0, 0, 0), (1, 0, 0), (0, 0, 1)))  # y = 0
    for o, eu, ev in faces:
        unit.append(_quad_grid(o, eu, ev, n, n))
    unit = np.concatenate(unit, axis=0)                       # [K,3,3] in [0,1]^3
    ext = (hi - lo)[:, None, None, :]
    return lo[:, None, None, :] + unit[None] * ext


def _torus(nu: int, nv: int, R: float, r: float, vertical: bool) -> np.ndarray:
    """Torus of nu x nv quads (2*nu*nv triangles) centred at the origin.
    Horizontal: ring in the XZ plane; vertical: ring in the XY plane."""
    cu = np.array([math.cos(2.0 * math.pi * i / nu) for i in range(nu + 1)])
    su = np.array([math.sin(2.0 * math.pi * i / nu) for i in range(nu + 1)])
    cv = np.array([math.cos(2.0 * math.pi * j / nv) for j in range(nv + 1)])
    sv = np.array([math.sin(2.0 * math.pi * j / nv) for j in range(nv + 1)])
    rad = R + r * cv[None, :]                                # [nu+1, nv+1]
    a = rad * cu[:, None]
    b = rad * su[:, None]
    c = np.broadcast_to(r * sv[None, :], a.shape)
    if vertical:
        P = np.stack([a, b, c], axis=-1)
    else:
        P = np.stack([a, c, b], axis=-1)
    p00 = P[:-1, :-1].reshape(-1, 3)
    p10 = P[1:, :-1].reshape(-1, 3)
    p11 = P[1:, 1:].reshape(-1, 3)
    p01 = P[:-1, 1:].reshape(-1, 3)
    t1 = np.stack([p00, p10, p11], axis=1)
    t2 = np.stack([p00, p11, p01], axis=1)
    return np.stack([t1, t2], axis=1).reshape(-1, 3, 3)


def _identity_xforms(n: int) -> np.ndarray:
    x = np.zeros((n, 12), np.float32)
    x[:, 0] = x[:, 5] = x[:, 10] = 1.0
    return x


def _yaw(deg: float) -> np.ndarray:
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


class _Builder:
    def __init__(self):
        self.tris: List[np.ndarray] = []
        self.obj: List[np.ndarray] = []
        self.dyn: List[int] = []
        self.alb: List[np.ndarray] = []

    def add(self, tris: np.ndarray, albedo, dynamic: bool = False) -> int:
        oid = len(self.dyn)
        tris = np.asarray(tris, np.float64).reshape(-1, 3, 3)
        self.tris.append(tris)
        self.obj.append(np.full(tris.shape[0], oid, np.uint32))
        self.dyn.append(1 if dynamic else 0)
        self.alb.append(np.asarray(albedo, np.float64).reshape(3))
        return oid

    def add_many(self, tris: np.ndarray, albedo: np.ndarray) -> None:
        """tris [B,K,3,3], albedo [B,3]: one static object per box."""
        B, K = tris.shape[:2]
        base = len(self.dyn)
        self.tris.append(tris.reshape(-1, 3, 3))
        self.obj.append(np.repeat(np.arange(base, base + B, dtype=np.uint32), K))
        self.dyn.extend([0] * B)
        self.alb.extend(list(np.asarray(albedo, np.float64)))

    def arrays(self):
        verts = np.concatenate(self.tris, axis=0).astype(np.float32)
        obj = np.concatenate(self.obj).astype(np.uint32)
        dyn = np.asarray(self.dyn, np.uint8)
        alb = np.stack(self.alb).astype(np.float32)
        return verts, obj, dyn, alb


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def tiny_box(n_paths: int = 10_000, seed: int = 1) -> Scene:
    """Open 2x2x2 box + moving unit cube + point light (smallest workload)."""
    b = _Builder()
    shell = []
    shell.append(_quad_grid((-1, 0, -1), (2, 0, 0), (0, 0, 2), 1, 1))   # floor y=0
    shell.append(_quad_grid((-1, 2, -1), (0, 0, 2), (2, 0, 0), 1, 1))   # ceiling y=2
    shell.append(_quad_grid((-1, 0, -1), (0, 2, 0), (0, 0, 2), 1, 1))   # wall x=-1
    shell.append(_quad_grid((1, 0, -1), (0, 0, 2), (0, 2, 0), 1, 1))    # wall x=+1
    shell.append(_quad_grid((-1, 0, -1), (2, 0, 0), (0, 2, 0), 1, 1))   # wall z=-1
    b.add(np.concatenate(shell), (0.7, 0.7, 0.7))
    cube = _boxes(np.array([[-0.5, -0.5, -0.5]]), np.array([[0.5, 0.5, 0.5]]))[0]
    cube_id = b.add(cube, (0.7, 0.7, 0.7), dynamic=True)
    verts, obj, dyn, alb = b.arrays()
    n_obj = dyn.shape[0]

    def xf(frame: int) -> np.ndarray:
        x = _identity_xforms(n_obj)
        x[cube_id, 3] = -0.4 + 0.05 * (frame - 1)
        x[cube_id, 7] = 0.6
        x[cube_id, 11] = 0.0
        return x

    def lf(frame: int) -> List[Light]:
        return [Light(LIGHT_POINT, (0.0, 1.8, 0.0), power=(100.0, 100.0, 100.0), n_paths=n_paths)]

    return Scene("tiny_box", verts, obj, dyn, alb, max_bounces=3, diag=math.sqrt(12.0),
                 atlas_rect=(-1.0, -1.0, 1.0, 1.0), seed=seed, frames=2, tau=0.01,
                 _xform_fn=xf, _light_fn=lf)


def city(n_paths: int = 1_000_000, seed: int = 2, n_boxes: int = 16_666) -> Scene:
    """Procedural city grid: 100x100 m floor, ~200k triangles of random boxes,
    4 dynamic tori on sinusoidal paths (amplitude 2 m), one 1x1 m area light
    translating 0.1 m/frame along +x (its tangent)."""
    st = Stream(seed, 1)
    b = _Builder()
    b.add(_quad_grid((-50, 0, -50), (0, 0, 100), (100, 0, 0), 1, 1), st.uniform(3, 0.3, 0.8))

    centres = [(6.0, 2.5, 6.0), (-6.0, 2.5, 6.0), (-6.0, 2.5, -6.0), (6.0, 2.5, -6.0)]
    axes = [0, 2, 0, 2]
    R, r, amp = 1.0, 0.35, 2.0

    G = 130
    cell = 100.0 / G
    gi, gj = np.meshgrid(np.arange(G), np.arange(G), indexing="ij")
    cx = -50.0 + (gi.reshape(-1) + 0.5) * cell
    cz = -50.0 + (gj.reshape(-1) + 0.5) * cell
    keep = np.ones(cx.shape[0], bool)
    for (x0, _, z0), ax in zip(centres, axes):
        hx = (amp if ax == 0 else 0.0) + R + r + 0.6
        hz = (amp if ax == 2 else 0.0) + R + r + 0.6
        keep &= ~((np.abs(cx - x0) < hx) & (np.abs(cz - z0) < hz))
    # keep the region under the light's path clear of nothing: boxes stay
    idx = np.nonzero(keep)[0]
    idx = idx[Stream(seed, 2).permutation(idx.shape[0])][:n_boxes]
    idx = np.sort(idx)
    nb = idx.shape[0]
    sx = st.uniform(nb, 0.3, 0.7)
    sz = st.uniform(nb, 0.3, 0.7)
    h = st.uniform(nb, 0.5, 5.0)
    jx = (st.uniform(nb) - 0.5) * (cell - sx)
    jz = (st.uniform(nb) - 0.5) * (cell - sz)
    lo = np.stack([cx[idx] + jx - 0.5 * sx, np.zeros(nb), cz[idx] + jz - 0.5 * sz], axis=1)
    hi = np.stack([cx[idx] + jx + 0.5 * sx, h, cz[idx] + jz + 0.5 * sz], axis=1)
    b.add_many(_boxes(lo, hi), st.uniform(3 * nb, 0.3, 0.8).reshape(nb, 3))

    torus = _torus(32, 32, R, r, vertical=False)
    tids = [b.add(torus, st.uniform(3, 0.3, 0.8), dynamic=True) for _ in range(4)]
    verts, obj, dyn, alb = b.arrays()
    n_obj = dyn.shape[0]

    def xf(frame: int) -> np.ndarray:
        x = _identity_xforms(n_obj)
        for j, (oid, (x0, y0, z0), ax) in enumerate(zip(tids, centres, axes)):
            off = amp * math.sin(2.0 * math.pi * (frame - 1) / 30.0 + j * math.pi / 2.0)
            p = [x0, y0, z0]
            p[ax] += off
            x[oid, 3], x[oid, 7], x[oid, 11] = p
        return x

    def lf(frame: int) -> List[Light]:
        return [Light(LIGHT_RECT, (0.1 * (frame - 1), 12.0, 0.0), (0.0, -1.0, 0.0), (1.0, 0.0, 0.0),
                      (1.0, 1.0), (1000.0, 1000.0, 1000.0), n_paths)]

    diag = math.sqrt(100.0 ** 2 + 12.0 ** 2 + 100.0 ** 2)
    return Scene("city", verts, obj, dyn, alb, max_bounces=7, diag=diag,
                 atlas_rect=(-50.0, -50.0, 50.0, 50.0), seed=seed, frames=30, tau=0.01,
                 _xform_fn=xf, _light_fn=lf)


def villa(n_paths_per_light: int = 1_000_000, seed: int = 3, n_static: int = 2_000_000,
          moving_light: str = "torch") -> Scene:
    """Villa-shaped interior: 4x3 rooms of 5x5x3 m with 1x2.1 m doors, exactly
    ``n_static`` static triangles (tessellated shell, detailed furniture boxes,
    30 % small clutter), 10 dynamic tori (5000 triangles, translating with
    amplitude 1 m and yawing 2 deg/frame), a ceiling point light, a static
    0.5x0.5 m ceiling area light and a moving, tilting 0.3x0.3 m torch.

    ``moving_light = "point"``: the torch stays at its first pose and the
    ceiling point light moves instead, 0.05 m/frame along a 1 m radius loop
    under the ceiling of its room (the case whose origin update needs a
    visibility ray per path)."""
    if moving_light not in ("torch", "point"):
        raise ValueError("villa: moving_light is 'torch' or 'point'")
    st = Stream(seed, 1)
    b = _Builder()
    NX, NZ, RS, H = 4, 3, 5.0, 3.0
    W, D = NX * RS, NZ * RS
    cellsz = 0.0825

    def wall_rect(o, eu, ev, lu, lv, alb):
        nu = max(1, int(round(lu / cellsz)))
        nv = max(1, int(round(lv / cellsz)))
        eu = np.asarray(eu, np.float64) * lu
        ev = np.asarray(ev, np.float64) * lv
        b.add(_quad_grid(o, eu, ev, nu, nv), alb)

    floor_alb = (0.6, 0.5, 0.4)
    wall_alb = (0.75, 0.75, 0.7)
    for i in range(NX):
        for k in range(NZ):
            x0, z0 = i * RS, k * RS
            wall_rect((x0, 0, z0), (0, 0, 1), (1, 0, 0), RS, RS, floor_alb)
            wall_rect((x0, H, z0), (1, 0, 0), (0, 0, 1), RS, RS, (0.8, 0.8, 0.8))
    dw, dh = 1.0, 2.1

    def wall_with_door(o, along, length, door: bool):
        o = np.asarray(o, np.float64)
        a = np.asarray(along, np.float64)
        up = np.array([0.0, 1.0, 0.0])
        if not door:
            wall_rect(o, a, up, length, H, wall_alb)
            return
        d0 = 0.5 * (length - dw)
        wall_rect(o, a, up, d0, H, wall_alb)
        wall_rect(o + a * (d0 + dw), a, up, length - d0 - dw, H, wall_alb)
        wall_rect(o + a * d0 + up * dh, a, up, dw, H - dh, wall_alb)

    for k in range(NZ):          # walls along x at z = k*RS ... including outer
        pass
    for kz in range(NZ + 1):
        for i in range(NX):
            inner = 0 < kz < NZ
            wall_with_door((i * RS, 0.0, kz * RS), (1, 0, 0), RS, door=inner)
    for kx in range(NX + 1):
        for k in range(NZ):
            inner = 0 < kx < NX
            wall_with_door((kx * RS, 0.0, k * RS), (0, 0, 1), RS, door=inner)
    n_shell = sum(t.shape[0] for t in b.tris)

    # furniture: 20 boxes per room, each face an n x n grid
    n_furn = 20 * NX * NZ
    nf = 18
    rx = st.integers(n_furn, NX)
    rz = st.integers(n_furn, NZ)
    fw = st.uniform(n_furn, 0.3, 1.6)
    fd = st.uniform(n_furn, 0.3, 1.6)
    fh = st.uniform(n_furn, 0.3, 2.0)
    fx = rx * RS + 0.15 + st.uniform(n_furn) * (RS - 0.3 - fw)
    fz = rz * RS + 0.15 + st.uniform(n_furn) * (RS - 0.3 - fd)
    flo = np.stack([fx, np.zeros(n_furn), fz], axis=1)
    fhi = np.stack([fx + fw, fh, fz + fd], axis=1)
    b.add_many(_boxes(flo, fhi, n=nf), st.uniform(3 * n_furn, 0.3, 0.8).reshape(n_furn, 3))
    n_furn_tris = n_furn * 6 * 2 * nf * nf

    # clutter: small boxes on floors and on furniture tops, padded to n_static
    rest = n_static - n_shell - n_furn_tris
    if rest < 0:
        raise ValueError("villa: shell + furniture exceed the static triangle budget")
    n_clut = rest // 12
    n_single = rest - 12 * n_clut
    on_furn = st.uniform(n_clut) < 0.5
    fsel = st.integers(n_clut, n_furn)
    cs = st.uniform(3 * n_clut, 0.03, 0.2).reshape(n_clut, 3)
    # floor placement
    crx = st.integers(n_clut, NX)
    crz = st.integers(n_clut, NZ)
    cx = crx * RS + 0.05 + st.uniform(n_clut) * (RS - 0.1 - cs[:, 0])
    cz = crz * RS + 0.05 + st.uniform(n_clut) * (RS - 0.1 - cs[:, 2])
    cy = np.zeros(n_clut)
    # furniture-top placement
    tx = flo[fsel, 0] + st.uniform(n_clut) * np.maximum(fw[fsel] - cs[:, 0], 0.0)
    tz = flo[fsel, 2] + st.uniform(n_clut) * np.maximum(fd[fsel] - cs[:, 2], 0.0)
    cx = np.where(on_furn, tx, cx)
    cz = np.where(on_furn, tz, cz)
    cy = np.where(on_furn, fh[fsel], cy)
    clo = np.stack([cx, cy, cz], axis=1)
    chi = clo + cs
    b.add_many(_boxes(clo, chi), st.uniform(3 * n_clut, 0.3, 0.8).reshape(n_clut, 3))
    if n_single:
        px = st.uniform(n_single, 0.2, W - 0.2)
        pz = st.uniform(n_single, 0.2, D - 0.2)
        for s in range(n_single):
            t = np.array([[px[s], 0.01, pz[s]], [px[s] + 0.05, 0.01, pz[s]], [px[s], 0.01, pz[s] + 0.05]])
            b.add(t, (0.5, 0.5, 0.5))

    torus = _torus(50, 50, 0.3, 0.1, vertical=True)
    n_tori = 10
    tor_room = [(0, 0), (1, 0), (2, 0), (3, 0), (0, 1), (1, 1), (3, 1), (0, 2), (1, 2), (2, 2)]
    tor_c = []
    tor_ax = []
    for j, (i, k) in enumerate(tor_room):
        tor_c.append((i * RS + 2.5, 1.3 + 0.1 * (j % 3), k * RS + 2.5))
        tor_ax.append(0 if j % 2 == 0 else 2)
    tids = [b.add(torus, st.uniform(3, 0.3, 0.8), dynamic=True) for _ in range(n_tori)]
    verts, obj, dyn, alb = b.arrays()
    n_obj = dyn.shape[0]
    assert int((dyn[obj] == 0).sum()) == n_static

    def xf(frame: int) -> np.ndarray:
        x = _identity_xforms(n_obj)
        for j, oid in enumerate(tids):
            f = frame - 1
            off = 1.0 * math.sin(2.0 * math.pi * f / 60.0 + j * 0.7)
            p = list(tor_c[j])
            p[tor_ax[j]] += off
            Rm = _yaw(2.0 * f + 17.0 * j)
            x[oid, 0:3] = Rm[0]
            x[oid, 4:7] = Rm[1]
            x[oid, 8:11] = Rm[2]
            x[oid, 3], x[oid, 7], x[oid, 11] = p
        return x

    P = (300.0, 300.0, 300.0)

    def lf(frame: int) -> List[Light]:
        f = frame - 1
        fp = f if moving_light == "point" else 0
        ang_p = 0.05 * fp                # the ceiling light's loop: 0.05 m/frame, radius 1 m
        p_pos = (2.5 + math.cos(ang_p) - 1.0, 2.9, 2.5 + math.sin(ang_p))
        if moving_light == "point":
            f = 0
        ang = 0.05 * f / 1.0            # 0.05 m/frame along a 1 m radius loop
        cxk, czk = 3 * RS + 2.5, 2 * RS + 2.5
        pos = (cxk + math.cos(ang), 2.5, czk + math.sin(ang))    # above the furniture (<= 2.2 m)
        tilt = math.radians(10.0) * math.sin(2.0 * math.pi * f / 60.0)
        # torch points down, tilted about x by +-10 degrees
        nrm = (0.0, -math.cos(tilt), math.sin(tilt))
        tan = (1.0, 0.0, 0.0)
        return [
            Light(LIGHT_POINT, p_pos, power=P, n_paths=n_paths_per_light),
            Light(LIGHT_RECT, (2 * RS + 2.5, 2.98, RS + 2.5), (0.0, -1.0, 0.0), (1.0, 0.0, 0.0),
                  (0.5, 0.5), P, n_paths_per_light),
            Light(LIGHT_RECT, pos, nrm, tan, (0.3, 0.3), P, n_paths_per_light),
        ]

    diag = math.sqrt(W * W + H * H + D * D)
    return Scene("villa", verts, obj, dyn, alb, max_bounces=7, diag=diag,
                 atlas_rect=(0.0, 0.0, W, D), seed=seed, frames=60, tau=0.01,
                 _xform_fn=xf, _light_fn=lf)


def by_name(name: str, **kw) -> Scene:
    return {"tiny_box": tiny_box, "city": city, "villa": villa}[name](**kw)


def perturbed_theta(theta, n_lights: int, seed: int = 2111) -> np.ndarray:
    """Seeded target pose of the adjoint workload: every light's position
    moved by N(0, 5 cm) per axis, its normal by N(0, 0.02) per component,
    its intensity factor times 1.1, and every dynamic object's translation
    moved by N(0, 5 cm) per axis (theta layout: per light pos 3, normal 3,
    intensity 1; then per dynamic object translation 3)."""
    rng = np.random.default_rng(seed)
    th = np.array(theta, np.float64, copy=True)
    for l in range(n_lights):
        th[7 * l:7 * l + 3] += rng.normal(0.0, 0.05, 3)
        th[7 * l + 3:7 * l + 6] += rng.normal(0.0, 0.02, 3)
        th[7 * l + 6] *= 1.1
    th[7 * n_lights:] += rng.normal(0.0, 0.05, th.shape[0] - 7 * n_lights)
    return th


def district(n_tris: int, n_paths: int, n_lights: int = 1, max_bounces: int = 7, n_tori: int = 4,
             seed: int = 5) -> Scene:
    """City-like district of about ``n_tris`` triangles: a square floor with
    random boxes at the city's density (0.77 m grid cells, sides U[0.3, 0.7] m,
    heights U[0.5, 5] m), ``n_tori`` (1..4) tori of 2048 triangles on x or z
    sinusoids (amplitude 2 m, period 30 frames) and 1..3 lights sharing
    ``n_paths``: a 1x1 m area light at 12 m translating 0.1 m/frame, a static
    point light at 8 m, a static 0.5x0.5 m area light at 10 m."""
    st = Stream(seed, 1)
    b = _Builder()
    cell = 100.0 / 130.0
    n_boxes = max(1, (n_tris - 2 - 2048 * n_tori) // 12)
    G = int(math.ceil(math.sqrt(n_boxes / 0.9))) + 4
    L = G * cell
    h = 0.5 * L
    b.add(_quad_grid((-h, 0, -h), (0, 0, L), (L, 0, 0), 1, 1), st.uniform(3, 0.3, 0.8))
    q = max(L / 6.0, 6.0)
    centres = [(q, 2.5, q), (-q, 2.5, q), (-q, 2.5, -q), (q, 2.5, -q)][:n_tori]
    axes = [0, 2, 0, 2][:n_tori]
    R, r, amp = 1.0, 0.35, 2.0
    gi, gj = np.meshgrid(np.arange(G), np.arange(G), indexing="ij")
    cx = -h + (gi.reshape(-1) + 0.5) * cell
    cz = -h + (gj.reshape(-1) + 0.5) * cell
    keep = np.ones(cx.shape[0], bool)
    for (x0, _, z0), ax in zip(centres, axes):
        hx = (amp if ax == 0 else 0.0) + R + r + 0.6
        hz = (amp if ax == 2 else 0.0) + R + r + 0.6
        keep &= ~((np.abs(cx - x0) < hx) & (np.abs(cz - z0) < hz))
    idx = np.nonzero(keep)[0]
    idx = np.sort(idx[Stream(seed, 2).permutation(idx.shape[0])][:n_boxes])
    nb = idx.shape[0]
    sx = st.uniform(nb, 0.3, 0.7)
    sz = st.uniform(nb, 0.3, 0.7)
    hh = st.uniform(nb, 0.5, 5.0)
    jx = (st.uniform(nb) - 0.5) * (cell - sx)
    jz = (st.uniform(nb) - 0.5) * (cell - sz)
    lo = np.stack([cx[idx] + jx - 0.5 * sx, np.zeros(nb), cz[idx] + jz - 0.5 * sz], axis=1)
    hi = np.stack([cx[idx] + jx + 0.5 * sx, hh, cz[idx] + jz + 0.5 * sz], axis=1)
    b.add_many(_boxes(lo, hi), st.uniform(3 * nb, 0.3, 0.8).reshape(nb, 3))
    torus = _torus(32, 32, R, r, vertical=False)
    tids = [b.add(torus, st.uniform(3, 0.3, 0.8), dynamic=True) for _ in range(n_tori)]
    verts, obj, dyn, alb = b.arrays()
    n_obj = dyn.shape[0]
    n_lights = max(1, min(3, n_lights))
    per = [n_paths // n_lights + (1 if l < n_paths % n_lights else 0) for l in range(n_lights)]

    def xf(frame: int) -> np.ndarray:
        x = _identity_xforms(n_obj)
        for j, (oid, (x0, y0, z0), ax) in enumerate(zip(tids, centres, axes)):
            off = amp * math.sin(2.0 * math.pi * (frame - 1) / 30.0 + j * math.pi / 2.0)
            p = [x0, y0, z0]
            p[ax] += off
            x[oid, 3], x[oid, 7], x[oid, 11] = p
        return x

    def lf(frame: int) -> List[Light]:
        ls = [Light(LIGHT_RECT, (0.1 * (frame - 1), 12.0, 0.0), (0.0, -1.0, 0.0), (1.0, 0.0, 0.0), (1.0, 1.0),
                    (1000.0, 1000.0, 1000.0), per[0])]
        if n_lights >= 2:
            ls.append(Light(LIGHT_POINT, (0.25 * h, 8.0, -0.25 * h), power=(500.0, 500.0, 500.0), n_paths=per[1]))
        if n_lights >= 3:
            ls.append(Light(LIGHT_RECT, (-0.25 * h, 10.0, 0.25 * h), (0.0, -1.0, 0.0), (1.0, 0.0, 0.0), (0.5, 0.5),
                            (500.0, 500.0, 500.0), per[2]))
        return ls

    diag = math.sqrt(2.0 * L * L + 12.0 ** 2)
    return Scene(f"district{n_tris}", verts, obj, dyn, alb, max_bounces=max_bounces, diag=diag,
                 atlas_rect=(-h, -h, h, h), seed=seed, frames=60, tau=0.01, _xform_fn=xf, _light_fn=lf)


def batch16(seed: int = 4) -> List[Scene]:
    """Sixteen independent districts of uneven size: triangles log-spaced from
    10k to 2M, paths log-spaced from 50k to 3M (paired by a seeded
    permutation), 1 to 3 lights, bounce caps cycling 1..7, 1 to 4 tori."""
    tris = np.geomspace(10_000, 2_000_000, 16)
    paths = np.geomspace(50_000, 3_000_000, 16)
    perm = Stream(seed, 9).permutation(16)
    return [district(int(tris[i]), int(paths[perm[i]]), n_lights=1 + i % 3, max_bounces=1 + (3 * i) % 7,
                     n_tori=1 + i % 4, seed=100 * seed + i) for i in range(16)]
