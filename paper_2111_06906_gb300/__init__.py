"""Python binding of the GB300 path-verification library (``include/pv.h``).

Argument marshalling only: every step of the path runs in the CUDA kernels of
``_build/libpv.so``.  PyTorch supplies device memory (``data_ptr()``) and
streams; nothing here computes on the data.  Importing works without a GPU;
every call that reaches the library fails loudly if the library was not built.

Path buffers follow ``pv_paths`` (Sec. 4 of the paper, row k = photon k of
every path): ``info`` int32 [N] (uint32 bits), ``origin`` float32 [3, N],
``pa`` float32 [B, N, 4] (hit position, primitive id bits), ``pb`` float32
[B, N, 4] (incident RGB energy, path length).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpv.so")

PV_OK = 0
PV_LIGHT_POINT, PV_LIGHT_RECT = 0, 1
PV_MODE_NAIVE_AABB, PV_MODE_NAIVE_EXACT, PV_MODE_ERROR = 0, 1, 2
PV_FLAG_TEST_OLD_TRIS, PV_FLAG_ERROR_EXACT = 1, 2
PV_BUILD_DYN_REBUILD = 1
PV_BUILD_STATIC_LBVH = 2
PV_BUILD_REFIT_CLIMB = 4
PV_INFO_NSEG_SHIFT, PV_INFO_START_SHIFT = 22, 26
PV_INFO_REPLACE, PV_INFO_REUSE_LIGHT = 1 << 30, 1 << 31

EXPORTS = ["pv_build_scene", "pv_update_dynamic", "pv_verify_paths", "pv_retrace_invalid", "pv_verify_retrace",
           "pv_verify_retrace_deposit", "pv_verify_retrace_deposit_delta", "pv_stage_timing", "pv_stage_times", "pv_trace_all",
           "pv_trace_all_deposit",
           "pv_compact_replace", "pv_compact_replace_static", "pv_deposit", "pv_set_traversal_limit",
           "pv_read_device_status", "pv_destroy_scene", "pv_status_string", "pv_theta_size", "pv_theta_current",
           "pv_model_deposit", "pv_adjoint_deposit", "pv_budget_list", "pv_batch_create", "pv_batch_frame",
           "pv_batch_autotune", "pv_batch_tuning", "pv_batch_set_config", "pv_batch_get_config", "pv_batch_step_times",
           "pv_batch_destroy", "pv_distribution_map_cells", "pv_read_distribution_map", "pv_splat_workspace_bytes",
           "pv_splat", "pv_fma_probe"]
PV_BATCH_MAX_SCENES = 32
PV_STATIC_COMPACT_MAX_PATHS = 1 << 26


class PvError(RuntimeError):
    pass


class PvLight(C.Structure):
    _fields_ = [("type", C.c_int32), ("pos", C.c_float * 3), ("normal", C.c_float * 3), ("tangent", C.c_float * 3),
                ("size", C.c_float * 2), ("power", C.c_float * 3), ("n_paths", C.c_uint32)]


class PvSceneDesc(C.Structure):
    _fields_ = [("verts", C.c_void_p), ("n_tris", C.c_uint32), ("tri_object", C.c_void_p), ("n_objects", C.c_uint32),
                ("object_dynamic", C.c_void_p), ("object_albedo", C.c_void_p), ("object_xform", C.c_void_p),
                ("n_lights", C.c_uint32), ("lights", C.c_void_p), ("max_bounces", C.c_uint32),
                ("scene_diag", C.c_float), ("flags", C.c_uint32), ("dm_rect", C.c_uint32 * 4),
                ("dm_point", C.c_uint32 * 2)]


class PvPaths(C.Structure):
    _fields_ = [("n", C.c_uint32), ("max_bounces", C.c_uint32), ("info", C.c_void_p), ("origin", C.c_void_p),
                ("pa", C.c_void_p), ("pb", C.c_void_p)]


class PvVerifyParams(C.Structure):
    _fields_ = [("mode", C.c_int32), ("tau", C.c_float), ("flags", C.c_uint32), ("frame", C.c_uint32),
                ("seed", C.c_uint64)]


class PvAtlas(C.Structure):
    _fields_ = [("data", C.c_void_p), ("width", C.c_uint32), ("height", C.c_uint32), ("x0", C.c_float),
                ("z0", C.c_float), ("x1", C.c_float), ("z1", C.c_float), ("scale_log2", C.c_int32)]


class PvCamera(C.Structure):
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


class PvBatchScene(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("paths", PvPaths), ("d_list", C.c_void_p), ("d_count", C.c_void_p),
                ("d_stats", C.c_void_p), ("seed", C.c_uint64)]


class PvBatchConfig(C.Structure):
    _fields_ = [("verify_mapping", C.c_int32), ("verify_threads", C.c_int32), ("trace_steps", C.c_int32),
                ("trace_blocks", C.c_int32), ("stack", C.c_int32)]


STATS_FIELDS = ["n_paths", "n_listed", "n_reemit", "n_tail", "n_updated", "n_truncated", "n_cont", "vis_rays",
                "cont_rays", "trace_rays", "segments_tested", "photons_written", "n_pruned", "n_filled"]
STATS_FIELDS64 = ["node_visits", "tri_tests"]
STATS_WORDS = len(STATS_FIELDS) + 2 * len(STATS_FIELDS64)

_lib = None


def load():
    """Load ``libpv.so``; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise PvError(f"CUDA library missing at {LIB_PATH}: run paper_2111_06906_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.pv_build_scene.argtypes = [C.POINTER(PvSceneDesc), P, C.POINTER(C.c_void_p)]
        L.pv_update_dynamic.argtypes = [P, P, P, P]
        L.pv_verify_paths.argtypes = [P, C.POINTER(PvPaths), C.POINTER(PvVerifyParams), P, P, P, P]
        L.pv_retrace_invalid.argtypes = [P, C.POINTER(PvPaths), P, P, C.c_uint64, C.c_uint32, P, P]
        L.pv_verify_retrace.argtypes = [P, C.POINTER(PvPaths), C.POINTER(PvVerifyParams), P, P]
        L.pv_verify_retrace_deposit.argtypes = [P, C.POINTER(PvPaths), C.POINTER(PvVerifyParams), C.POINTER(PvAtlas),
                                                P, P]
        L.pv_verify_retrace_deposit_delta.argtypes = [P, C.POINTER(PvPaths), C.POINTER(PvVerifyParams),
                                                      C.POINTER(PvAtlas), P, P]
        L.pv_stage_timing.argtypes = [P, C.c_uint32]
        L.pv_stage_times.argtypes = [P, P, P]
        L.pv_trace_all.argtypes = [P, C.POINTER(PvPaths), C.c_uint64, C.c_uint32, P, P]
        L.pv_trace_all_deposit.argtypes = [P, C.POINTER(PvPaths), C.c_uint64, C.c_uint32, C.POINTER(PvAtlas), P, P]
        L.pv_compact_replace.argtypes = [P, C.POINTER(PvPaths), P, P, P]
        L.pv_compact_replace_static.argtypes = [P, C.c_uint32, P, P, P]
        L.pv_deposit.argtypes = [P, C.POINTER(PvPaths), C.POINTER(PvAtlas), P]
        L.pv_set_traversal_limit.argtypes = [P, C.c_uint32]
        L.pv_read_device_status.argtypes = [P]
        L.pv_destroy_scene.argtypes = [P]
        L.pv_destroy_scene.restype = None
        L.pv_theta_size.argtypes = [P]
        L.pv_theta_current.argtypes = [P, P]
        L.pv_model_deposit.argtypes = [P, C.POINTER(PvPaths), P, P, C.c_uint32, C.c_uint32, P, P]
        L.pv_adjoint_deposit.argtypes = [P, C.POINTER(PvPaths), P, P, C.c_uint32, C.c_uint32, P, P, P, P]
        L.pv_budget_list.argtypes = [P, P, P, P, C.c_uint32, P, P, P]
        L.pv_batch_create.argtypes = [C.POINTER(PvBatchScene), C.c_uint32, C.POINTER(PvVerifyParams), P,
                                      C.POINTER(C.c_void_p)]
        L.pv_batch_frame.argtypes = [P, P, P, C.c_uint32, P]
        L.pv_batch_autotune.argtypes = [P, C.c_uint32]
        L.pv_batch_tuning.argtypes = [P]
        L.pv_batch_set_config.argtypes = [P, C.POINTER(PvBatchConfig)]
        L.pv_batch_get_config.argtypes = [P, C.POINTER(PvBatchConfig)]
        L.pv_batch_step_times.argtypes = [P, P]
        L.pv_batch_destroy.argtypes = [P]
        L.pv_distribution_map_cells.argtypes = [P, C.c_uint32]
        L.pv_splat_workspace_bytes.argtypes = [P, C.c_uint32, C.c_uint32]
        L.pv_splat_workspace_bytes.restype = C.c_size_t
        L.pv_splat.argtypes = [P, C.POINTER(PvPaths), C.POINTER(PvCamera), C.c_float, P, P, C.c_size_t, P]
        L.pv_read_distribution_map.argtypes = [P, C.c_uint32, P]
        L.pv_fma_probe.argtypes = [C.c_uint32, C.c_uint32, P, P, P]
        L.pv_batch_destroy.restype = None
        L.pv_status_string.argtypes = [C.c_int]
        L.pv_status_string.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("pv_destroy_scene", "pv_status_string", "pv_batch_destroy", "pv_splat_workspace_bytes"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def pv_status_string(rc: int) -> str:
    return load().pv_status_string(int(rc)).decode()


def _check(name: str, rc: int) -> None:
    if rc != PV_OK:
        raise PvError(f"{name}: {pv_status_string(rc)} ({rc})")


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def make_lights(lights) -> C.Array:
    """Pack objects with type/pos/normal/tangent/size/power/n_paths into pv_light[]."""
    arr = (PvLight * len(lights))()
    for i, l in enumerate(lights):
        arr[i].type = int(l.type)
        arr[i].pos[:] = [float(v) for v in l.pos]
        arr[i].normal[:] = [float(v) for v in l.normal]
        arr[i].tangent[:] = [float(v) for v in l.tangent]
        arr[i].size[:] = [float(v) for v in l.size]
        arr[i].power[:] = [float(v) for v in l.power]
        arr[i].n_paths = int(l.n_paths)
    return arr


@dataclass
class Paths:
    """Caller-owned device path buffers (torch tensors)."""
    info: "object"
    origin: "object"
    pa: "object"
    pb: "object"

    @classmethod
    def allocate(cls, n: int, max_bounces: int, device="cuda"):
        import torch
        return cls(torch.zeros(n, dtype=torch.int32, device=device),
                   torch.zeros(3, n, dtype=torch.float32, device=device),
                   torch.zeros(max_bounces, n, 4, dtype=torch.float32, device=device),
                   torch.zeros(max_bounces, n, 4, dtype=torch.float32, device=device))

    @property
    def n(self) -> int:
        return int(self.info.shape[0])

    @property
    def max_bounces(self) -> int:
        return int(self.pa.shape[0])

    def struct(self) -> PvPaths:
        for t in (self.info, self.origin, self.pa, self.pb):
            if not t.is_contiguous():
                raise PvError("path buffers must be contiguous")
        return PvPaths(self.n, self.max_bounces, self.info.data_ptr(), self.origin.data_ptr(), self.pa.data_ptr(),
                       self.pb.data_ptr())


def pv_build_scene(verts, tri_object, object_dynamic, object_albedo, lights, max_bounces: int, scene_diag: float,
                   object_xform=None, flags: int = 0, stream=None, dm_rect=(0, 0, 0, 0),
                   dm_point=(0, 0)) -> C.c_void_p:
    """Build a scene from host arrays (copied); returns the opaque handle.
    dm_rect / dm_point: distribution-map resolutions of the rectangle and
    point lights (zeros: no map)."""
    L = load()
    keep = [np.ascontiguousarray(verts, np.float32), np.ascontiguousarray(tri_object, np.uint32),
            np.ascontiguousarray(object_dynamic, np.uint8), np.ascontiguousarray(object_albedo, np.float32)]
    xf = None if object_xform is None else np.ascontiguousarray(object_xform, np.float32)
    la = make_lights(lights)
    d = PvSceneDesc(keep[0].ctypes.data, keep[0].shape[0], keep[1].ctypes.data, keep[2].shape[0], keep[2].ctypes.data,
                    keep[3].ctypes.data, 0 if xf is None else xf.ctypes.data, len(lights), C.cast(la, C.c_void_p),
                    int(max_bounces), float(scene_diag), int(flags), (C.c_uint32 * 4)(*[int(v) for v in dm_rect]),
                    (C.c_uint32 * 2)(*[int(v) for v in dm_point]))
    h = C.c_void_p()
    _check("pv_build_scene", L.pv_build_scene(C.byref(d), _stream(stream), C.byref(h)))
    return h


def pv_update_dynamic(scene, xforms=None, lights=None, stream=None) -> None:
    """``lights``: a list of lights, or an array already packed by make_lights."""
    xf = None if xforms is None else np.ascontiguousarray(xforms, np.float32)
    la = None if lights is None else (lights if isinstance(lights, C.Array) else make_lights(lights))
    _check("pv_update_dynamic", load().pv_update_dynamic(
        scene, None if xf is None else xf.ctypes.data_as(C.c_void_p), None if la is None else C.cast(la, C.c_void_p),
        _stream(stream)))


def pv_verify_paths(scene, paths: Paths, mode: int, tau: float, flags: int, d_list, d_count, d_stats=None,
                    stream=None, seed: int = 0, frame: int = 0) -> None:
    """seed / frame key the distribution maps' prune draws."""
    ps = paths.struct()
    prm = PvVerifyParams(int(mode), float(tau), int(flags), int(frame), int(seed))
    _check("pv_verify_paths", load().pv_verify_paths(scene, C.byref(ps), C.byref(prm), _ptr(d_list), _ptr(d_count),
                                                      _ptr(d_stats), _stream(stream)))


def pv_retrace_invalid(scene, paths: Paths, d_list, d_count, seed: int, frame: int, d_stats=None, stream=None) -> None:
    ps = paths.struct()
    _check("pv_retrace_invalid", load().pv_retrace_invalid(scene, C.byref(ps), _ptr(d_list), _ptr(d_count),
                                                            int(seed), int(frame), _ptr(d_stats), _stream(stream)))


def pv_verify_retrace(scene, paths: Paths, mode: int, tau: float, flags: int, seed: int, frame: int, d_stats=None,
                      stream=None) -> None:
    """pv_verify_paths + pv_retrace_invalid in one call (same records and counters, no list)."""
    ps = paths.struct()
    prm = PvVerifyParams(int(mode), float(tau), int(flags), int(frame), int(seed))
    _check("pv_verify_retrace", load().pv_verify_retrace(scene, C.byref(ps), C.byref(prm), _ptr(d_stats),
                                                          _stream(stream)))


def pv_stage_timing(scene, n: int) -> None:
    _check("pv_stage_timing", load().pv_stage_timing(scene, int(n)))


STAGES = ["clears", "k_verify", "between", "retrace_kernel", "call"]


def pv_stage_times(scene, n: int) -> np.ndarray:
    """[calls, 5] milliseconds of the last recorded pv_verify_retrace calls, columns as ``STAGES``
    (see include/pv.h)."""
    E = len(STAGES)
    ms = np.zeros(E * max(int(n), 1), np.float32)
    cnt = C.c_uint32(0)
    _check("pv_stage_times", load().pv_stage_times(scene, ms.ctypes.data_as(C.c_void_p), C.byref(cnt)))
    return ms[:E * cnt.value].reshape(cnt.value, E)


def pv_fma_probe(blocks: int, iters: int, d_sink, stream=None) -> int:
    """Enqueue the FP32 fused multiply-add probe; returns how many FMAs it executes."""
    fmas = C.c_uint64(0)
    _check("pv_fma_probe", load().pv_fma_probe(int(blocks), int(iters), _ptr(d_sink), C.byref(fmas), _stream(stream)))
    return int(fmas.value)


def pv_trace_all(scene, paths: Paths, seed: int, frame: int, d_stats=None, stream=None) -> None:
    ps = paths.struct()
    _check("pv_trace_all", load().pv_trace_all(scene, C.byref(ps), int(seed), int(frame), _ptr(d_stats),
                                                _stream(stream)))


def pv_trace_all_deposit(scene, paths: Paths, seed: int, frame: int, atlas, rect, scale_log2: int, d_stats=None,
                         stream=None) -> None:
    """pv_trace_all + pv_deposit in one kernel (same records, counters and atlas)."""
    ps = paths.struct()
    a = _atlas(atlas, rect, scale_log2)
    _check("pv_trace_all_deposit", load().pv_trace_all_deposit(scene, C.byref(ps), int(seed), int(frame), C.byref(a),
                                                                _ptr(d_stats), _stream(stream)))


def pv_compact_replace(scene, paths: Paths, d_list, d_count, stream=None) -> None:
    ps = paths.struct()
    _check("pv_compact_replace", load().pv_compact_replace(scene, C.byref(ps), _ptr(d_list), _ptr(d_count),
                                                            _stream(stream)))


def pv_compact_replace_static(d_info, n: int, d_list, d_count, stream=None) -> None:
    """Allocation-free compaction for callers that must not allocate device
    memory while running (no scene needed; at most 2^26 paths)."""
    _check("pv_compact_replace_static", load().pv_compact_replace_static(_ptr(d_info), int(n), _ptr(d_list),
                                                                          _ptr(d_count), _stream(stream)))


def _atlas(atlas, rect, scale_log2: int) -> PvAtlas:
    H, W = int(atlas.shape[0]), int(atlas.shape[1])
    return PvAtlas(atlas.data_ptr(), W, H, float(rect[0]), float(rect[1]), float(rect[2]), float(rect[3]),
                   int(scale_log2))


def pv_deposit(scene, paths: Paths, atlas, rect, scale_log2: int, stream=None) -> None:
    """``atlas``: int64 tensor [H, W, 3] (uint64 fixed point, cleared here)."""
    ps = paths.struct()
    a = _atlas(atlas, rect, scale_log2)
    _check("pv_deposit", load().pv_deposit(scene, C.byref(ps), C.byref(a), _stream(stream)))


def pv_verify_retrace_deposit(scene, paths: Paths, mode: int, tau: float, flags: int, seed: int, frame: int, atlas,
                              rect, scale_log2: int, d_stats=None, stream=None) -> None:
    """pv_verify_retrace + pv_deposit in one call (same records, counters and atlas)."""
    ps = paths.struct()
    prm = PvVerifyParams(int(mode), float(tau), int(flags), int(frame), int(seed))
    a = _atlas(atlas, rect, scale_log2)
    _check("pv_verify_retrace_deposit", load().pv_verify_retrace_deposit(scene, C.byref(ps), C.byref(prm), C.byref(a),
                                                                          _ptr(d_stats), _stream(stream)))


def pv_verify_retrace_deposit_delta(scene, paths: Paths, mode: int, tau: float, flags: int, seed: int, frame: int,
                                    atlas, rect, scale_log2: int, d_stats=None, stream=None) -> None:
    """pv_verify_retrace_deposit on an atlas that holds the deposit of the entry records (not cleared: the
    touched paths' entry photons are taken out and their final photons added; same atlas bit for bit)."""
    ps = paths.struct()
    prm = PvVerifyParams(int(mode), float(tau), int(flags), int(frame), int(seed))
    a = _atlas(atlas, rect, scale_log2)
    _check("pv_verify_retrace_deposit_delta",
           load().pv_verify_retrace_deposit_delta(scene, C.byref(ps), C.byref(prm), C.byref(a), _ptr(d_stats),
                                                  _stream(stream)))


def _rect(rect):
    r = (C.c_float * 4)(*[float(v) for v in rect])
    return r, C.cast(r, C.c_void_p)


def pv_theta_size(scene) -> int:
    n = int(load().pv_theta_size(scene))
    if n < 0:
        _check("pv_theta_size", n)
    return n


def pv_theta_current(scene) -> np.ndarray:
    """Parameters of the differentiable deposit model at the current poses:
    per light [pos 3, normal 3, intensity factor 1], per dynamic object
    [translation 3] (float32, host)."""
    th = np.zeros(pv_theta_size(scene), np.float32)
    _check("pv_theta_current", load().pv_theta_current(scene, th.ctypes.data_as(C.c_void_p)))
    return th


def pv_model_deposit(scene, paths: Paths, theta, atlas, rect, stream=None) -> None:
    """Add the model's cubic B-spline splat under ``theta`` (float32 device tensor)
    to ``atlas`` (float32 device tensor [H, W, 3], not cleared)."""
    ps = paths.struct()
    keep, r = _rect(rect)
    H, W = int(atlas.shape[0]), int(atlas.shape[1])
    _check("pv_model_deposit", load().pv_model_deposit(scene, C.byref(ps), _ptr(theta), _ptr(atlas), W, H, r,
                                                        _stream(stream)))


def pv_adjoint_deposit(scene, paths: Paths, theta, grad_atlas, rect, dtheta, score=None, stream=None) -> None:
    """Add dL/dtheta for the atlas gradient ``grad_atlas`` ([H, W, 3]) into
    ``dtheta``; per-path scores into ``score`` (float32 [N]) when given."""
    ps = paths.struct()
    keep, r = _rect(rect)
    H, W = int(grad_atlas.shape[0]), int(grad_atlas.shape[1])
    _check("pv_adjoint_deposit", load().pv_adjoint_deposit(scene, C.byref(ps), _ptr(theta), _ptr(grad_atlas), W, H,
                                                            r, _ptr(dtheta), _ptr(score), _stream(stream)))


def pv_budget_list(scene, d_list, d_count, score, budget: int, d_out, d_out_count, stream=None) -> None:
    """The ``budget`` listed paths of largest score, in ascending id order."""
    _check("pv_budget_list", load().pv_budget_list(scene, _ptr(d_list), _ptr(d_count), _ptr(score), int(budget),
                                                    _ptr(d_out), _ptr(d_out_count), _stream(stream)))


_model_fn = None


def _model_function():
    """torch.autograd.Function over pv_model_deposit / pv_adjoint_deposit
    (built on first use so that importing needs no torch)."""
    global _model_fn
    if _model_fn is None:
        import torch

        class ModelDeposit(torch.autograd.Function):
            @staticmethod
            def forward(ctx, theta, scene, paths, height, width, rect):
                th = theta.detach().to(torch.float32).contiguous()
                atlas = torch.zeros(height, width, 3, dtype=torch.float32, device=th.device)
                pv_model_deposit(scene, paths, th, atlas, rect)
                ctx.save_for_backward(th)
                ctx.scene, ctx.paths, ctx.rect = scene, paths, rect
                return atlas

            @staticmethod
            def backward(ctx, grad):
                (th,) = ctx.saved_tensors
                d = torch.zeros_like(th)
                pv_adjoint_deposit(ctx.scene, ctx.paths, th, grad.to(torch.float32).contiguous(), ctx.rect, d)
                return d, None, None, None, None, None

        _model_fn = ModelDeposit
    return _model_fn


def model_deposit(scene, paths: Paths, theta, height: int, width: int, rect):
    """Differentiable atlas (float32 [height, width, 3]) of the stored paths
    under ``theta``; ``backward`` runs the CUDA adjoint."""
    return _model_function().apply(theta, scene, paths, int(height), int(width), tuple(float(v) for v in rect))


class Batch:
    """Handle of a pv_batch plus the host objects its calls must keep alive."""

    def __init__(self, handle, n):
        self.handle = handle
        self.n = n

    def __bool__(self):
        return bool(self.handle)


def pv_batch_create(items, mode: int, tau: float, flags: int = 0, stream=None) -> Batch:
    """items: sequence of (scene, Paths, d_list, d_count, d_stats or None, seed); d_list and d_count None
    for every scene: no lists, Alg. 1 fused with the re-trace."""
    arr = (PvBatchScene * len(items))()
    for i, (scene, paths, d_list, d_count, d_stats, seed) in enumerate(items):
        arr[i].scene = scene.value if isinstance(scene, C.c_void_p) else scene
        arr[i].paths = paths.struct()
        arr[i].d_list = d_list.data_ptr() if d_list is not None else None
        arr[i].d_count = d_count.data_ptr() if d_count is not None else None
        arr[i].d_stats = d_stats.data_ptr() if d_stats is not None else None
        arr[i].seed = int(seed)
    prm = PvVerifyParams(int(mode), float(tau), int(flags), 0, 0)
    h = C.c_void_p()
    _check("pv_batch_create", load().pv_batch_create(arr, len(items), C.byref(prm), _stream(stream), C.byref(h)))
    return Batch(h, len(items))


class BatchPoses:
    """The per-scene poses of one batched frame, marshalled once: xforms / lights are per scene a float32
    [n_objects, 12] array / list of lights, or None (whole argument or per entry).  Reusable."""

    def __init__(self, n: int, xforms, lights):
        self.keep = []
        self.xf = None
        if xforms is not None:
            self.xf = (C.c_void_p * n)()
            for i, x in enumerate(xforms):
                if x is not None:
                    a = np.ascontiguousarray(x, np.float32)
                    self.keep.append(a)
                    self.xf[i] = a.ctypes.data
        self.lt = None
        if lights is not None:
            self.lt = (C.c_void_p * n)()
            for i, l in enumerate(lights):
                if l is not None:
                    a = make_lights(l)
                    self.keep.append(a)
                    self.lt[i] = C.cast(a, C.c_void_p).value


def pv_batch_frame(batch: Batch, xforms, lights, frame: int, stream=None) -> None:
    """xforms / lights as BatchPoses takes them, or a BatchPoses as ``xforms`` (``lights`` ignored)."""
    poses = xforms if isinstance(xforms, BatchPoses) else BatchPoses(batch.n, xforms, lights)
    _check("pv_batch_frame", load().pv_batch_frame(batch.handle,
                                                    None if poses.xf is None else C.cast(poses.xf, C.c_void_p),
                                                    None if poses.lt is None else C.cast(poses.lt, C.c_void_p),
                                                    int(frame), _stream(stream)))


def pv_batch_autotune(batch: Batch, frames_per_candidate: int = 1) -> None:
    _check("pv_batch_autotune", load().pv_batch_autotune(batch.handle, int(frames_per_candidate)))


def pv_batch_tuning(batch: Batch) -> bool:
    rc = int(load().pv_batch_tuning(batch.handle))
    if rc < 0:
        _check("pv_batch_tuning", rc)
    return rc == 1


def pv_batch_set_config(batch: Batch, **cfg) -> None:
    c = PvBatchConfig()
    _check("pv_batch_get_config", load().pv_batch_get_config(batch.handle, C.byref(c)))
    for k, v in cfg.items():
        setattr(c, k, int(v))
    _check("pv_batch_set_config", load().pv_batch_set_config(batch.handle, C.byref(c)))


def pv_batch_get_config(batch: Batch) -> dict:
    c = PvBatchConfig()
    _check("pv_batch_get_config", load().pv_batch_get_config(batch.handle, C.byref(c)))
    return {k: int(getattr(c, k)) for k, _ in PvBatchConfig._fields_}


def pv_batch_step_times(batch: Batch):
    """[pose update, verify, continuation, compaction, re-trace] in ms."""
    a = (C.c_float * 5)()
    _check("pv_batch_step_times", load().pv_batch_step_times(batch.handle, C.cast(a, C.c_void_p)))
    return [float(x) for x in a]


def pv_batch_destroy(batch: Batch) -> None:
    if batch and batch.handle:
        load().pv_batch_destroy(batch.handle)
        batch.handle = None


def pv_splat_workspace_bytes(scene, width: int, height: int) -> int:
    return int(load().pv_splat_workspace_bytes(scene, int(width), int(height)))


def pv_splat(scene, paths: Paths, cam: PvCamera, radius: float, image, work, stream=None) -> None:
    """Splat the stored photons into ``image`` (float32 [h, w, 3] device
    tensor, written); ``work``: device tensor of pv_splat_workspace_bytes."""
    ps = paths.struct()
    _check("pv_splat", load().pv_splat(scene, C.byref(ps), C.byref(cam), float(radius), _ptr(image), _ptr(work),
                                        int(work.numel() * work.element_size()), _stream(stream)))


def pv_distribution_map_cells(scene, light: int) -> int:
    n = int(load().pv_distribution_map_cells(scene, int(light)))
    if n < 0:
        _check("pv_distribution_map_cells", n)
    return n


def pv_read_distribution_map(scene, light: int) -> np.ndarray:
    """Current counts DM_C of a light's distribution map (synchronises)."""
    out = np.zeros(pv_distribution_map_cells(scene, light), np.uint32)
    _check("pv_read_distribution_map", load().pv_read_distribution_map(scene, int(light),
                                                                        out.ctypes.data_as(C.c_void_p)))
    return out


def pv_set_traversal_limit(scene, max_visits: int) -> None:
    _check("pv_set_traversal_limit", load().pv_set_traversal_limit(scene, int(max_visits)))


def pv_read_device_status(scene) -> int:
    return int(load().pv_read_device_status(scene))


def pv_destroy_scene(scene) -> None:
    if scene:
        load().pv_destroy_scene(scene)


def stats_dict(d_stats) -> dict:
    """Decode a ``pv_frame_stats`` device buffer (int32 tensor)."""
    v = d_stats.cpu().numpy().view(np.uint32)
    out = {k: int(v[i]) for i, k in enumerate(STATS_FIELDS)}
    w = v[len(STATS_FIELDS):].copy().view(np.uint64)
    out.update({k: int(w[i]) for i, k in enumerate(STATS_FIELDS64)})
    return out


def new_stats(device="cuda"):
    """Zeroed ``pv_frame_stats`` (8-byte aligned int32 tensor)."""
    import torch
    return torch.zeros(STATS_WORDS, dtype=torch.int32, device=device)
