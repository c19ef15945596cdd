"""ctypes wrapper of the FP64 brute-force CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is what the CUDA path is checked
against; only the test suite, the smoke check and the benchmark's CPU
baseline may import it.  It shares no code with the CUDA library: both only
consume the seeded arrays of the ``scenes`` package.

Path records on this side are AoS: ``photons[n, B, 8]`` float32 with
(x, y, z, prim-as-int32-bits, E_r, E_g, E_b, path-length) per photon (the
32-byte record of Sec. 4), ``info[n]`` uint32 (Sec. 4 bit fields) and
``origin[n, 3]`` float32.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")

MODE_NAIVE_AABB = 0
MODE_NAIVE_EXACT = 1
MODE_ERROR = 2
FLAG_TEST_OLD_TRIS = 1
FLAG_ERROR_EXACT = 2

AMB_TRACE = 1
AMB_VERIFY = 2
AMB_CONT = 4
AMB_ENERGY = 8
AMB_LIGHT = 16

INFO_REPLACE = 1 << 30
INFO_REUSE_LIGHT = 1 << 31


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no floating-point contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Light(C.Structure):
    _fields_ = [("type", C.c_int32), ("pos", C.c_float * 3), ("normal", C.c_float * 3),
                ("tangent", C.c_float * 3), ("size", C.c_float * 2), ("power", C.c_float * 3),
                ("n_paths", C.c_uint32)]


class Camera(C.Structure):
    """Pinhole camera: pos, target, up, vertical field of view (radians), pixels."""
    _fields_ = [("pos", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3), ("fov_y", C.c_float),
                ("width", C.c_uint32), ("height", C.c_uint32)]

    @classmethod
    def make(cls, pos, target, up, fov_y, width, height):
        c = cls()
        c.pos[:] = [float(v) for v in pos]
        c.target[:] = [float(v) for v in target]
        c.up[:] = [float(v) for v in up]
        c.fov_y = float(fov_y)
        c.width, c.height = int(width), int(height)
        return c


class _Stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "paths", "segments_tested", "segments_amb", "vis_rays", "cont_rays", "trace_rays",
        "energy_tests", "energy_amb", "n_reemit", "n_tail", "n_updated", "n_truncated", "n_pruned", "n_filled",
        "rays_amb")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class _Choice(C.Structure):
    _fields_ = [("script", C.c_void_p), ("n_script", C.c_int32), ("pos", C.c_int32), ("n_alt_next", C.c_int32),
                ("open", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        P = C.c_void_p
        L.or_scene_create.restype = P
        L.or_scene_create.argtypes = [P, C.c_uint32, P, C.c_uint32, P, P, C.c_double, C.c_uint32]
        L.or_scene_destroy.argtypes = [P]
        L.or_scene_set_poses.argtypes = [P, P, P, P, P, C.c_uint32]
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_trace.argtypes = [P, P, C.c_uint32, C.c_uint64, C.c_uint32, P, P, P, P, P]
        L.or_verify.argtypes = [P, P, C.c_uint32, C.c_int32, C.c_double, C.c_uint32, C.c_uint64, C.c_uint32, P, P,
                                P, P, P, P]
        L.or_scene_set_dm.restype = C.c_int32
        L.or_scene_set_dm.argtypes = [P, P, P]
        L.or_dm_reset.argtypes = [P]
        L.or_dm_cells.restype = C.c_uint32
        L.or_dm_cells.argtypes = [P, C.c_uint32]
        L.or_dm_target.restype = C.c_uint32
        L.or_dm_target.argtypes = [P, C.c_uint32, C.c_uint32]
        L.or_dm_counts.argtypes = [P, C.c_uint32, P]
        L.or_dm_set_counts.argtypes = [P, C.c_uint32, P]
        L.or_dm_cell_of.restype = C.c_int32
        L.or_dm_cell_of.argtypes = [P, C.c_uint32, P, P]
        L.or_splat.argtypes = [P, P, C.c_uint32, P, P, P, P, C.c_double, P, P]
        L.or_dm_turn.restype = C.c_float
        L.or_dm_turn.argtypes = [C.c_float, C.c_float]
        L.or_compact.restype = C.c_uint32
        L.or_compact.argtypes = [P, C.c_uint32, P]
        L.or_retrace.argtypes = [P, P, C.c_uint32, C.c_uint64, C.c_uint32, P, P, P, P, P]
        L.or_deposit.argtypes = [P, C.c_uint32, P, C.c_uint32, C.c_uint32, C.c_uint32,
                                 C.c_float, C.c_float, C.c_float, C.c_float, P]
        L.or_photon_texels.argtypes = [P, C.c_uint32, P, C.c_uint32, C.c_uint32, C.c_uint32,
                                       C.c_float, C.c_float, C.c_float, C.c_float, P]
        L.or_closest_hit.restype = C.c_int32
        L.or_closest_hit.argtypes = [P, P, P, C.c_double, C.c_int32, P, P]
        L.or_num_threads.restype = C.c_int32
        L.or_trace_path.argtypes = [P, C.c_uint32, C.c_uint64, C.c_uint32, P, P, P, P, P]
        L.or_verify_path.restype = C.c_int32
        L.or_verify_path.argtypes = [P, C.c_uint32, C.c_int32, C.c_double, C.c_uint32, P, P, P, P, P, P]
        L.or_retrace_path.argtypes = [P, C.c_uint32, C.c_uint64, C.c_uint32, P, P, P, P, P]
        L.or_theta_size.restype = C.c_uint32
        L.or_theta_size.argtypes = [P]
        L.or_theta_current.argtypes = [P, P]
        L.or_model_deposit.argtypes = [P, P, C.c_uint32, P, P, P, P, C.c_uint32, C.c_uint32, C.c_float, C.c_float,
                                       C.c_float, C.c_float, P]
        L.or_adjoint.argtypes = [P, P, C.c_uint32, P, P, P, P, C.c_uint32, C.c_uint32, C.c_float, C.c_float,
                                 C.c_float, C.c_float, P, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def num_threads() -> int:
    return int(lib().or_num_threads())


def _lights(ls):
    arr = (_Light * len(ls))()
    for i, l in enumerate(ls):
        arr[i].type = l.type
        arr[i].pos[:] = list(l.pos)
        arr[i].normal[:] = list(l.normal)
        arr[i].tangent[:] = list(l.tangent)
        arr[i].size[:] = list(l.size)
        arr[i].power[:] = list(l.power)
        arr[i].n_paths = l.n_paths
    return arr


@dataclass
class Paths:
    """Oracle-side path records for a subset of path ids.

    For the paths whose decisions may be ambiguous the records also carry
    what is needed to list their admissible outcomes: ``snap`` holds the
    records at the last point they were checked (or uploaded), ``pending``
    the steps applied since, and ``branches`` -- for paths that met an
    ambiguous decision earlier -- the oracle records, at ``snap`` time, that
    every check so far has accepted (see ``OracleScene.outcomes``)."""
    ids: np.ndarray                 # uint32 [n]
    info: np.ndarray                # uint32 [n]
    origin: np.ndarray              # float32 [n,3]
    photons: np.ndarray             # float32 [n,B,8]
    amb: np.ndarray                 # uint32 [n] ambiguity bits (accumulated)
    stats: dict = field(default_factory=dict)
    snap: tuple = None              # (info, origin, photons) at the last check; None: before the first trace
    pending: list = field(default_factory=list)     # steps since snap: (kind, frames, args)
    branches: dict = field(default_factory=dict)    # position -> [(info, origin, photons)] at snap time
    oracle: object = field(default=None, repr=False)
    opened: set = field(default_factory=set)         # positions whose admissible records could not be listed

    def record(self, i: int):
        return int(self.info[i]), self.origin[i].copy(), self.photons[i].copy()

    def subset(self, idx) -> "Paths":
        """The paths at positions ``idx``, with their snapshot, pending steps
        and accepted branches."""
        idx = np.asarray(idx, np.int64)
        pos = {int(j): k for k, j in enumerate(idx)}
        snap = None if self.snap is None else tuple(a[idx].copy() for a in self.snap)
        br = {pos[i]: list(v) for i, v in self.branches.items() if i in pos}
        return Paths(self.ids[idx].copy(), self.info[idx].copy(), self.origin[idx].copy(), self.photons[idx].copy(),
                     self.amb[idx].copy(), dict(self.stats), snap, list(self.pending), br, self.oracle,
                     {pos[i] for i in self.opened if i in pos})

    def adopt_branches(self) -> None:
        """Paths with an ambiguous decision take the first record the last
        check accepted (an oracle record: the outcome the device's result
        agreed with) in place of the oracle's default outcome; e.g. before
        comparing quantities computed from the records, such as a deposit."""
        for i, recs in self.branches.items():
            self.info[i], self.origin[i], self.photons[i] = recs[0][0], recs[0][1], recs[0][2]
            if self.snap is not None:
                self.snap[0][i], self.snap[1][i], self.snap[2][i] = recs[0][0], recs[0][1], recs[0][2]
            self.branches[i] = [recs[0]]

    def rebase(self) -> None:
        """The current records become the shared starting point (e.g. after
        uploading them to the device): no pending steps, no branches."""
        self.snap = (self.info.copy(), self.origin.copy(), self.photons.copy())
        self.pending = []
        self.branches = {}
        self.opened = set()

    @property
    def nseg(self) -> np.ndarray:
        return (self.info >> 22) & 15

    @property
    def start(self) -> np.ndarray:
        return (self.info >> 26) & 15

    @property
    def prim(self) -> np.ndarray:
        return self.photons[..., 3].view(np.int32)

    def copy(self) -> "Paths":
        snap = None if self.snap is None else tuple(a.copy() for a in self.snap)
        return Paths(self.ids.copy(), self.info.copy(), self.origin.copy(), self.photons.copy(),
                     self.amb.copy(), dict(self.stats), snap, list(self.pending),
                     {k: list(v) for k, v in self.branches.items()}, self.oracle, set(self.opened))


class OracleScene:
    """Oracle view of a ``scenes.Scene`` at a pair of (old, new) frames."""

    def __init__(self, scene):
        self.scene = scene
        self.B = int(scene.max_bounces)
        L = lib()
        self._keep = (np.ascontiguousarray(scene.verts, np.float32),
                      np.ascontiguousarray(scene.tri_object, np.uint32),
                      np.ascontiguousarray(scene.object_dynamic, np.uint8),
                      np.ascontiguousarray(scene.object_albedo, np.float32))
        v, to, dy, al = self._keep
        self._h = L.or_scene_create(_p(v), scene.n_tris, _p(to), scene.n_objects, _p(dy), _p(al),
                                    float(scene.diag), self.B)
        self.frames = None
        self._poses = None

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_scene_destroy(self._h)
            self._h = None

    def set_frames(self, frame_old: int, frame_new: int) -> None:
        self.set_poses(self.scene.xforms(frame_old), self.scene.xforms(frame_new),
                       self.scene.lights(frame_old), self.scene.lights(frame_new))
        self.frames = (frame_old, frame_new)

    def set_poses(self, xf_old, xf_new, lights_old, lights_new) -> None:
        xo = np.ascontiguousarray(xf_old, np.float32)
        xn = np.ascontiguousarray(xf_new, np.float32)
        lo, ln = _lights(lights_old), _lights(lights_new)
        lib().or_scene_set_poses(self._h, _p(xo), _p(xn), C.cast(lo, C.c_void_p),
                                 C.cast(ln, C.c_void_p), len(lights_new))
        self._poses = (xo, xn, list(lights_old), list(lights_new))
        self.frames = None

    def _restore_poses(self, poses, frames) -> None:
        if poses is not None:
            self.set_poses(*poses)
        self.frames = frames

    def trace(self, ids, seed: int, frame: int) -> Paths:
        ids = np.ascontiguousarray(ids, np.uint32)
        n = ids.shape[0]
        p = Paths(ids, np.zeros(n, np.uint32), np.zeros((n, 3), np.float32),
                  np.zeros((n, self.B, 8), np.float32), np.zeros(n, np.uint32))
        st = _Stats()
        lib().or_trace(self._h, _p(ids), n, seed, frame, _p(p.info), _p(p.origin), _p(p.photons),
                       _p(p.amb), C.byref(st))
        p.stats = st.as_dict()
        p.oracle = self
        p.pending = [("trace", self.frames, (int(seed), int(frame)))]
        return p

    def verify(self, paths: Paths, mode: int, tau: float, flags: int = 0, seed: int = 0, frame: int = 0):
        """In place; returns (segment mask [n], stats).  Ambiguity bits are
        OR-ed into ``paths.amb``.  seed and frame key the prune draws of the
        distribution maps."""
        n = paths.ids.shape[0]
        mask = np.zeros(n, np.uint32)
        amb = np.zeros(n, np.uint32)
        st = _Stats()
        lib().or_verify(self._h, _p(paths.ids), n, mode, float(tau), flags, int(seed), int(frame), _p(paths.info),
                        _p(paths.origin), _p(paths.photons), _p(mask), _p(amb), C.byref(st))
        paths.amb |= amb
        paths.pending.append(("verify", self.frames, (int(mode), float(tau), int(flags))))
        return mask, st.as_dict()

    def retrace(self, paths: Paths, seed: int, frame: int) -> dict:
        n = paths.ids.shape[0]
        amb = np.zeros(n, np.uint32)
        st = _Stats()
        lib().or_retrace(self._h, _p(paths.ids), n, seed, frame, _p(paths.info), _p(paths.origin),
                         _p(paths.photons), _p(amb), C.byref(st))
        paths.amb |= amb
        paths.pending.append(("retrace", self.frames, (int(seed), int(frame))))
        return st.as_dict()

    # ---- admissible outcomes of the paths whose decisions are ambiguous
    def run_path(self, steps, pid: int, rec, script=()):
        """``steps`` (kind, frames, args) applied to one path record under a
        decision script; returns ((info, origin, photons), n_alt_next, open),
        or None when a step cannot run per path (a distribution map, or poses
        not set through set_frames).  ``open``: a closest hit of the run met a
        triangle whose crossing distance the band leaves undetermined over a
        stretch of the ray (the ray runs within eps of its plane), so records
        with a hit anywhere on that stretch are admissible as well."""
        L = lib()
        info = np.array([rec[0]], np.uint32)
        org = np.ascontiguousarray(rec[1], np.float32).copy()
        ph = np.ascontiguousarray(rec[2], np.float32).copy()
        amb = np.zeros(1, np.uint32)
        mask = np.zeros(1, np.uint32)
        sc = np.ascontiguousarray(script, np.uint8)
        ch = _Choice(sc.ctypes.data if sc.size else None, int(sc.size), 0, 0, 0)
        for kind, frames, args in steps:
            if frames is None:
                return None
            if self.frames != frames:
                self.set_frames(*frames)
            if kind == "trace":
                L.or_trace_path(self._h, pid, args[0], args[1], _p(info), _p(org), _p(ph), _p(amb), C.byref(ch))
            elif kind == "verify":
                if L.or_verify_path(self._h, pid, args[0], args[1], args[2], _p(info), _p(org), _p(ph), _p(mask),
                                    _p(amb), C.byref(ch)) != 0:
                    return None
            else:
                L.or_retrace_path(self._h, pid, args[0], args[1], _p(info), _p(org), _p(ph), _p(amb), C.byref(ch))
        return (int(info[0]), org, ph), int(ch.n_alt_next), bool(ch.open)

    def outcomes(self, steps, pid: int, rec, max_runs: int = 96, max_depth: int = 12):
        """Every record path ``pid`` can end with when ``steps`` run from record
        ``rec`` and each ambiguous decision takes each of its admissible
        outcomes (depth-first over decision scripts).  Returns (records,
        complete, open); complete is False when the run or depth bound cut
        the search, open is True when some run met a hit whose distance the
        band leaves undetermined over a stretch (see run_path), and records
        is None when the steps cannot run per path.  The scene's poses are as
        before on return."""
        poses, frames = getattr(self, "_poses", None), self.frames
        try:
            return self._outcomes(steps, pid, rec, max_runs, max_depth)
        finally:
            if self.frames != frames:
                self._restore_poses(poses, frames)

    def _outcomes(self, steps, pid, rec, max_runs, max_depth):
        out, stack, runs, opened = [], [()], 0, False
        while stack:
            script = stack.pop()
            r = self.run_path(steps, pid, rec, script)
            if r is None:
                return None, False, False
            runs += 1
            rec_out, n_alt, op = r
            opened |= op
            if n_alt == 0 or len(script) >= max_depth:
                out.append(rec_out)
                if n_alt:
                    return out, False, opened
            else:
                stack.extend(script + (c,) for c in reversed(range(n_alt)))
            if runs >= max_runs and stack:
                return out, False, opened
        return out, True, opened

    # ---- screen-space splat (Fig. 2 splat/gather, radius kernel)
    def splat(self, paths: Paths, cam: "Camera", radius: float):
        """(image [h, w, 3] float64, ambiguous pixels [h, w] bool) at the current pose."""
        img = np.zeros((cam.height, cam.width, 3), np.float64)
        amb = np.zeros((cam.height, cam.width), np.uint8)
        lib().or_splat(self._h, _p(paths.ids), paths.ids.shape[0], _p(paths.info), _p(paths.origin),
                       _p(paths.photons), C.byref(cam), float(radius), _p(img), _p(amb))
        return img, amb.astype(bool)

    # ---- distribution maps (Sec. 3.1)
    def set_dm(self, rect=(0, 0, 0, 0), point=(0, 0)) -> None:
        """Give every rectangle light a rect[0..3] map over (x, y, sin^2 theta,
        phi/2pi) and every point light a point[0..1] map over ((1-z)/2,
        phi/2pi); call after set_frames.  Zeros: no map."""
        r = np.ascontiguousarray(rect, np.uint32)
        q = np.ascontiguousarray(point, np.uint32)
        if lib().or_scene_set_dm(self._h, _p(r), _p(q)) != 0:
            raise ValueError("distribution map larger than 2^20 cells")

    def dm_reset(self) -> None:
        lib().or_dm_reset(self._h)

    def dm_cells(self, light: int) -> int:
        return int(lib().or_dm_cells(self._h, light))

    def dm_counts(self, light: int) -> np.ndarray:
        out = np.zeros(self.dm_cells(light), np.uint32)
        lib().or_dm_counts(self._h, light, _p(out))
        return out

    def dm_set_counts(self, light: int, counts) -> None:
        c = np.ascontiguousarray(counts, np.uint32)
        assert c.shape[0] == self.dm_cells(light)
        lib().or_dm_set_counts(self._h, light, _p(c))

    def dm_targets(self, light: int) -> np.ndarray:
        return np.array([lib().or_dm_target(self._h, light, c) for c in range(self.dm_cells(light))], np.uint32)

    def dm_cell_of(self, light: int, x1, o) -> int:
        a = np.ascontiguousarray(x1, np.float32)
        b = np.ascontiguousarray(o, np.float32)
        return int(lib().or_dm_cell_of(self._h, light, _p(a), _p(b)))

    # ---- differentiable deposit model (frozen triangles and directions)
    def theta_current(self) -> np.ndarray:
        th = np.zeros(lib().or_theta_size(self._h), np.float64)
        lib().or_theta_current(self._h, _p(th))
        return th

    def model_deposit(self, paths: Paths, theta, width: int, height: int, rect) -> np.ndarray:
        th = np.ascontiguousarray(theta, np.float64)
        atlas = np.zeros((height, width, 3), np.float64)
        x0, z0, x1, z1 = (float(np.float32(v)) for v in rect)
        lib().or_model_deposit(self._h, _p(paths.ids), paths.ids.shape[0], _p(paths.info), _p(paths.origin),
                               _p(paths.photons), _p(th), width, height, x0, z0, x1, z1, _p(atlas))
        return atlas

    def adjoint(self, paths: Paths, theta, G, rect):
        """(dL/dtheta, per-path scores) for G = dL/datlas [h, w, 3]."""
        th = np.ascontiguousarray(theta, np.float64)
        G = np.ascontiguousarray(G, np.float64)
        height, width = G.shape[:2]
        dth = np.zeros_like(th)
        score = np.zeros(paths.ids.shape[0], np.float64)
        x0, z0, x1, z1 = (float(np.float32(v)) for v in rect)
        lib().or_adjoint(self._h, _p(paths.ids), paths.ids.shape[0], _p(paths.info), _p(paths.origin),
                         _p(paths.photons), _p(th), width, height, x0, z0, x1, z1, _p(G), _p(dth), _p(score))
        return dth, score

    def closest_hit(self, o, d, tlo: float, exclude: int = -1):
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        t = C.c_double()
        a = C.c_int32()
        prim = lib().or_closest_hit(self._h, _p(o), _p(d), tlo, exclude, C.byref(t), C.byref(a))
        return int(prim), float(t.value), bool(a.value)


def dm_turn(x: float, y: float) -> float:
    """Fraction of a turn of the angle of (x, y) as the map's parametrisation computes it."""
    return float(lib().or_dm_turn(float(x), float(y)))


def compact(info: np.ndarray) -> np.ndarray:
    """Ascending positions whose replace bit is set (the oracle's definition)."""
    info = np.ascontiguousarray(info, np.uint32)
    out = np.zeros(info.shape[0], np.uint32)
    c = lib().or_compact(_p(info), info.shape[0], _p(out))
    return out[:c]


def photon_texels(paths: Paths, width: int, height: int, rect) -> np.ndarray:
    """int32 [n, B, 2]: the texel (tx, tz) deposit() assigns to each stored
    photon, (-1, -1) past a path's photon count."""
    B = paths.photons.shape[1]
    out = np.zeros((paths.ids.shape[0], B, 2), np.int32)
    x0, z0, x1, z1 = (float(np.float32(v)) for v in rect)
    lib().or_photon_texels(_p(np.ascontiguousarray(paths.info)), paths.ids.shape[0],
                           _p(np.ascontiguousarray(paths.photons)), B, width, height, x0, z0, x1, z1, _p(out))
    return out


def deposit(paths: Paths, width: int, height: int, rect) -> np.ndarray:
    """float64 [height, width, 3] atlas of incident photon energy."""
    atlas = np.zeros((height, width, 3), np.float64)
    B = paths.photons.shape[1]
    x0, z0, x1, z1 = (float(np.float32(v)) for v in rect)
    lib().or_deposit(_p(np.ascontiguousarray(paths.info)), paths.ids.shape[0],
                     _p(np.ascontiguousarray(paths.photons)), B, width, height, x0, z0, x1, z1,
                     _p(atlas))
    return atlas
