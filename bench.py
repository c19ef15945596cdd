#!/usr/bin/env python
"""Benchmark of the per-frame path-verification hot path on one GB300.

One step = one frame of the reuse pipeline on the seeded villa workload
(2M static triangles, 10 yawing tori of 5000 triangles, a ceiling point
light, a static area light and a moving, tilting torch; 3M photon paths of up
to 7 bounces; error-based mode with tau = 1 %):  pv_update_dynamic ->
pv_verify_retrace_deposit (origin update, dynamic occlusions, then Alg. 1, the
re-trace and the atlas deposit in one persistent kernel).  Beside it, on the
same frames: the same library's trace-all frame (pv_update_dynamic ->
pv_trace_all_deposit: every path re-traced, its photons deposited in the
same kernel as they are stored), the separate calls (pv_verify_paths ->
pv_retrace_invalid -> pv_deposit), tau in {0, 0.5, 1, 5} % over 60 frames,
the naive modes of Sec. 3.2 against the error-based one, the same villa with
its ceiling point light moving (visibility rays in the origin update), and
per-kernel durations set against the measured HBM bandwidth and the measured
FP32 fused multiply-add rate.  The city workload and the 16-scene batch are
measured after it as secondary fields of the same line.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "photon paths verified+reused+retraced/s and frame ms vs trace-all on 1 GB300"
MODES = {"naive_aabb": 0, "naive_exact": 1, "error": 2}
WORKLOADS = {
    "villa": "villa-shaped interior: 4x3 rooms, 2M static tris (30% clutter), 10 yawing tori of 5000 tris, "
             "point light + static area light + moving tilting torch; 3M paths, <=7 bounces",
    "city": "procedural city: 100x100 m floor, 16666 random boxes (200k static tris), 4 tori of 2048 tris on "
            "sinusoidal paths (2 m amplitude), 1x1 m area light translating 0.1 m/frame; 1M paths, <=7 bounces",
    "tiny_box": "open 2x2x2 box (10 tris) + moving unit cube (12 tris), point light; 10k paths, <=3 bounces",
    "batch16": "16 independent districts: 10k to 2M tris, 50k to 3M paths (12.4M in all), 1 to 3 lights, "
               "bounce caps 1 to 7, 1 to 4 moving tori; one batched graph-captured frame per step, tuned",
}
# Algorithmic FP32 work of a traversal: 20 operations per ray-box slab test (four per 4-wide node) and 35 per
# Moller-Trumbore ray-triangle test, times the node visits and triangle tests the library counts.
OPS_PER_SLAB, OPS_PER_TRI = 20, 35
OPS_PER_NODE = 4 * OPS_PER_SLAB
# DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum, median over the launches of one
# capture of this benchmark, summarised under profiles/) of the kernels in the per-kernel table.  They hold
# only for the kernel sources they were captured on: the digest of csrc/ and include/ at capture time.  Any other
# source digest reports no traffic.
NCU_TRAFFIC = {
    "digest": "eea445baffede396",
    "villa": {"k_refit_wide": 4974592, "k_verify_box": 367724288, "k_cont_trace<deposit>": 991691136,
              "k_compact": 12016384, "k_trace (re-trace)": 204486016, "k_deposit": 644327424,
              "k_trace<deposit> (trace-all)": 892445952},
    "city": {"k_refit_wide": 825088, "k_verify_box": 88076672, "k_cont_trace<deposit>": 218518272,
             "k_compact": 4012288, "k_trace (re-trace)": 57209856, "k_deposit": 160499712,
             "k_trace<deposit> (trace-all)": 164392320},
}
TAUS = (0.0, 0.005, 0.01, 0.05)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="villa", choices=list(WORKLOADS))
    ap.add_argument("--mode", default="error", choices=list(MODES))
    ap.add_argument("--tau", type=float, default=None)
    ap.add_argument("--atlas", type=int, default=1024)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--sweep-frames", type=int, default=60, help="frames per tau / mode / moving-point-light row")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-dm", action="store_true", help="skip the distribution-map frame measurement")
    ap.add_argument("--no-splat", action="store_true", help="skip the 1920x1080 screen-space splat measurement")
    ap.add_argument("--no-sweeps", action="store_true", help="skip the tau, mode and moving-point-light rows")
    ap.add_argument("--no-secondary", action="store_true", help="villa only: skip the city and batch16 fields")
    ap.add_argument("--tune-frames", type=int, default=16, help="batch16: frames per tuner candidate")
    ap.add_argument("--build-flags", type=int, default=0, help="pv_scene_desc flags (2: Morton-code static tree)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def source_digest() -> str:
    """Digest of the library's kernel sources and headers (csrc/, include/)."""
    h = hashlib.sha256()
    dirs = [os.path.join(ROOT, "paper_2111_06906_gb300", "csrc"), os.path.join(ROOT, "include")]
    for d in dirs:
        for f in sorted(os.listdir(d)):
            if f.endswith((".cu", ".cuh", ".h")):
                h.update(f.encode())
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(fh.read())
    return h.hexdigest()[:16]


class Clocks:
    """SM clock and clock-event reasons sampled during the timed region: every
    5 ms through NVML (the driver's libnvidia-ml, read-only queries), else
    nvidia-smi every 50 ms."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.samples = []             # (sm_mhz, max_mhz, reasons bitmask or names)
        self.stop = threading.Event()
        self.source = None

    def _nvml(self):
        import ctypes as C
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        dev = C.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(self.index), C.byref(dev)) != 0:
            return None
        fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        return lib, dev, fn

    def _poll_nvml(self, lib, dev, fn):
        import ctypes as C
        sm, mx, rs = C.c_uint(), C.c_uint(), C.c_ulonglong()
        while not self.stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(dev, 1, C.byref(sm)) == 0 and
                    lib.nvmlDeviceGetMaxClockInfo(dev, 1, C.byref(mx)) == 0 and fn(dev, C.byref(rs)) == 0):
                self.samples.append((float(sm.value), float(mx.value),
                                     {n for bit, n in self.REASONS.items() if rs.value & bit}))
            time.sleep(0.005)

    def __enter__(self):
        try:
            h = self._nvml()
        except (OSError, AttributeError):
            h = None
        if h:
            self.source = "nvml 5 ms"
            self.t = threading.Thread(target=self._poll_nvml, args=h, daemon=True)
            self.t.start()
            return self
        try:
            self.source = "nvidia-smi 50 ms"
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            f = [x.strip() for x in line.strip().split(",")]
            if len(f) < 7:
                continue
            try:
                self.samples.append((float(f[0]), float(f[1]),
                                     {n for n, v in zip(names, f[3:7]) if v.lower().startswith("active")}))
            except ValueError:
                continue

    def __exit__(self, *a):
        self.stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if getattr(self, "t", None):
            self.t.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [x[0] for x in self.samples]
        reasons = set().union(*[x[2] for x in self.samples])
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(x[1] for x in self.samples)),
                "reasons": sorted(reasons), "samples": len(sm), "source": self.source}


def scene_for(name, **kw):
    import scenes
    return scenes.by_name(name, **kw)


def fma_peak(pv, torch, dev, sms, stream, local):
    """The FP32 fused multiply-add rate of this GPU: the library's probe kernel
    over 8 blocks of 256 threads per SM, median of 10 timed launches after 40
    untimed ones, SM clock sampled meanwhile."""
    blocks = 8 * sms
    sink = torch.zeros(blocks, dtype=torch.float32, device=dev)
    ms, fmas = [], 0
    clocks = Clocks(local)
    with clocks:
        for i in range(50):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fmas = pv.pv_fma_probe(blocks, 512, sink)
            e1.record(stream)
            if i >= 40:
                ms.append((e0, e1))
        torch.cuda.synchronize()
    t = float(np.median([a.elapsed_time(b) for a, b in ms]))
    rate = fmas / (t * 1e-3)
    ck = clocks.summary()
    return {"kernel": "k_fma_probe", "top_s": rate / 1e12, "fmas_per_launch": fmas, "ms": t, "blocks": blocks,
            "threads_per_block": 256, "sm_count": sms, "sm_mhz": ck.get("sm_mhz"),
            "fma_per_sm_per_clock": rate / (sms * ck["sm_mhz"] * 1e6) if ck.get("sm_mhz") else None,
            "note": "FP32 fused multiply-adds per second (one FMA = one op), 8 independent chains per thread"}


# ----------------------------------------------------------------------------- one workload on one scene
class Workload:
    """One scene, its path buffers and atlas, and the frame loops timed on it."""

    def __init__(self, pv, torch, sc, args, dev, stream, rank, K, W, frames_needed):
        self.pv, self.torch, self.sc, self.args, self.dev, self.stream = pv, torch, sc, args, dev, stream
        self.K, self.W = K, W
        self.mode = MODES[args.mode]
        self.tau = sc.tau if args.tau is None else args.tau
        self.seed = sc.seed + 7919 * rank
        self.N, self.B = sc.n_paths, sc.max_bounces
        self.xfs = {f: np.ascontiguousarray(sc.xforms(f), np.float32) for f in range(1, frames_needed + 1)}
        self.lts = {f: pv.make_lights(sc.lights(f)) for f in range(1, frames_needed + 1)}
        t0 = time.time()
        self.h = pv.pv_build_scene(sc.verts, sc.tri_object, sc.object_dynamic, sc.object_albedo, sc.lights(1), self.B,
                                   sc.diag, object_xform=self.xfs[1], flags=args.build_flags)
        self.build_s = time.time() - t0
        self.P = pv.Paths.allocate(self.N, self.B, dev)
        A = args.atlas
        self.A = A
        self.atlas = torch.zeros(A, A, 3, dtype=torch.int64, device=dev)
        self.scale = 40 if sc.name != "tiny_box" else 31
        self.lst = torch.zeros(self.N, dtype=torch.int32, device=dev)
        self.cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        self.lst2 = torch.zeros(self.N, dtype=torch.int32, device=dev)
        self.cnt2 = torch.zeros(1, dtype=torch.int32, device=dev)
        self.stats = torch.zeros(2 * K + 2, pv.STATS_WORDS, dtype=torch.int32, device=dev)

    def ev(self):
        return self.torch.cuda.Event(enable_timing=True)

    def barrier(self, ws):
        self.torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        self.torch.cuda.synchronize()

    def restart(self, lts=None):
        """Back to the poses of frame 1 and a fresh trace-all, so every loop runs frames 2, 3, ..."""
        lts = lts or self.lts
        self.pv.pv_update_dynamic(self.h, self.xfs[1], lts[1])
        self.pv.pv_trace_all(self.h, self.P, self.seed, 1)
        return 1

    def reuse_frame(self, f, st, atlas=None, mode=None, tau=None, lts=None, flags=0):
        lts = lts or self.lts
        self.pv.pv_update_dynamic(self.h, self.xfs[f], lts[f])
        self.pv.pv_verify_retrace_deposit(self.h, self.P, self.mode if mode is None else mode,
                                          self.tau if tau is None else tau, flags, self.seed, f,
                                          self.atlas if atlas is None else atlas, self.sc.atlas_rect, self.scale, st)

    def mean_photons(self):
        info = self.P.info.cpu().numpy().view(np.uint32)
        return float(np.minimum((info >> 22) & 15, self.B).mean())

    # ---- the headline: K reuse frames, only the two events that bracket them
    def headline(self, ws, local):
        frame = self.restart()
        for _ in range(self.W):
            frame += 1
            self.reuse_frame(frame, self.stats[-1])
        self.barrier(ws)
        clocks = Clocks(local)
        with clocks:
            start, stop = self.ev(), self.ev()
            start.record(self.stream)
            for i in range(self.K):
                self.reuse_frame(frame + 1 + i, self.stats[i])
            stop.record(self.stream)
            self.barrier(ws)
        self.first_timed = frame + 1
        ms = start.elapsed_time(stop) / self.K
        rows = [self.pv.stats_dict(self.stats[i]) for i in range(self.K)]
        return ms, rows, clocks.summary(), self.mean_photons(), self.pv.pv_read_device_status(self.h)

    # ---- the same frames with per-frame events and the library's stage events
    def instrumented(self, ws, rows_head):
        pv, K = self.pv, self.K
        frame = self.restart()
        for _ in range(self.W):
            frame += 1
            self.reuse_frame(frame, self.stats[-1])
        pv.pv_stage_timing(self.h, K)
        self.barrier(ws)
        ev = []
        for i in range(K):
            f = frame + 1 + i
            e = [self.ev() for _ in range(3)]
            e[0].record(self.stream)
            pv.pv_update_dynamic(self.h, self.xfs[f], self.lts[f])
            e[1].record(self.stream)
            pv.pv_verify_retrace_deposit(self.h, self.P, self.mode, self.tau, 0, self.seed, f, self.atlas,
                                         self.sc.atlas_rect, self.scale, self.stats[K + i])
            e[2].record(self.stream)
            ev.append(e)
        self.barrier(ws)
        stages = pv.pv_stage_times(self.h, K)
        pv.pv_stage_timing(self.h, 0)
        per_frame = np.array([e[0].elapsed_time(e[2]) for e in ev])
        update = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
        same = all(pv.stats_dict(self.stats[K + i]) == rows_head[i] for i in range(K))
        return {"per_frame_ms": per_frame, "update_ms": update,
                "stages_ms": dict(zip(pv.STAGES, [float(x) for x in stages.mean(axis=0)])), "counters_match": same}

    # ---- atlas carried from frame to frame
    def delta(self, ws):
        pv, torch = self.pv, self.torch
        atlas_full = self.atlas.clone()
        atlas_delta = torch.zeros_like(self.atlas)
        frame = self.restart()
        pv.pv_deposit(self.h, self.P, atlas_delta, self.sc.atlas_rect, self.scale)

        def delta_frame(f):
            pv.pv_update_dynamic(self.h, self.xfs[f], self.lts[f])
            pv.pv_verify_retrace_deposit_delta(self.h, self.P, self.mode, self.tau, 0, self.seed, f, atlas_delta,
                                               self.sc.atlas_rect, self.scale, self.stats[-1])

        for _ in range(self.W):
            frame += 1
            delta_frame(frame)
        self.barrier(ws)
        s, e = self.ev(), self.ev()
        s.record(self.stream)
        for i in range(self.K):
            delta_frame(frame + 1 + i)
        e.record(self.stream)
        self.barrier(ws)
        ms = s.elapsed_time(e) / self.K
        equal = bool(torch.equal(atlas_delta, atlas_full))
        return {"call": "pv_verify_retrace_deposit_delta", "ms_per_frame": ms, "paths_per_s": self.N / (ms * 1e-3),
                "atlas_equal_to_full_deposit": equal}

    # ---- the separate calls, with events between them; then the compaction alone on each frame's marks
    def separate(self, ws):
        pv, K = self.pv, self.K
        frame = self.restart()
        self.stats[:2 * K].zero_()                  # counters accumulate
        for _ in range(self.W):
            frame += 1
            pv.pv_update_dynamic(self.h, self.xfs[frame], self.lts[frame])
            pv.pv_verify_paths(self.h, self.P, self.mode, self.tau, 0, self.lst, self.cnt, self.stats[-1])
            pv.pv_retrace_invalid(self.h, self.P, self.lst, self.cnt, self.seed, frame, self.stats[-1])
            pv.pv_deposit(self.h, self.P, self.atlas, self.sc.atlas_rect, self.scale)
        self.barrier(ws)
        s, e = self.ev(), self.ev()
        ev = []
        s.record(self.stream)
        for i in range(K):
            f = frame + 1 + i
            x = [self.ev() for _ in range(5)]
            x[0].record(self.stream)
            pv.pv_update_dynamic(self.h, self.xfs[f], self.lts[f])
            x[1].record(self.stream)
            pv.pv_verify_paths(self.h, self.P, self.mode, self.tau, 0, self.lst, self.cnt, self.stats[i])
            x[2].record(self.stream)
            pv.pv_retrace_invalid(self.h, self.P, self.lst, self.cnt, self.seed, f, self.stats[K + i])
            x[3].record(self.stream)
            pv.pv_deposit(self.h, self.P, self.atlas, self.sc.atlas_rect, self.scale)
            x[4].record(self.stream)
            ev.append(x)
        e.record(self.stream)
        self.barrier(ws)
        ms = s.elapsed_time(e) / K
        parts = np.array([[x[j].elapsed_time(x[j + 1]) for j in range(4)] for x in ev]).mean(axis=0)
        rows_v = [pv.stats_dict(self.stats[i]) for i in range(K)]
        rows_r = [pv.stats_dict(self.stats[K + i]) for i in range(K)]
        # the compaction alone (pv_compact_replace, the k_compact kernel) on the marks of each verified frame
        frame = self.restart()
        cms = []
        for i in range(self.W + K):
            frame += 1
            pv.pv_update_dynamic(self.h, self.xfs[frame], self.lts[frame])
            pv.pv_verify_paths(self.h, self.P, self.mode, self.tau, 0, self.lst, self.cnt, self.stats[-1])
            a, b = self.ev(), self.ev()
            a.record(self.stream)
            pv.pv_compact_replace(self.h, self.P, self.lst2, self.cnt2)
            b.record(self.stream)
            pv.pv_retrace_invalid(self.h, self.P, self.lst, self.cnt, self.seed, frame, self.stats[-1])
            if i >= self.W:
                cms.append((a, b))
        self.barrier(ws)
        compact_ms = float(np.mean([a.elapsed_time(b) for a, b in cms]))
        return {"ms_per_frame": ms, "parts": dict(zip(["update", "verify", "retrace", "deposit"],
                                                      [float(v) for v in parts])),
                "compact_ms": compact_ms}, rows_v, rows_r

    # ---- trace-all on the same frames
    def trace_all(self, ws):
        pv, K = self.pv, self.K
        frame = self.restart()
        for _ in range(self.W):
            frame += 1
            pv.pv_update_dynamic(self.h, self.xfs[frame], self.lts[frame])
            pv.pv_trace_all_deposit(self.h, self.P, self.seed, frame, self.atlas, self.sc.atlas_rect, self.scale,
                                    self.stats[-1])
        self.stats[:K].zero_()
        self.barrier(ws)
        s, e = self.ev(), self.ev()
        ev = []
        s.record(self.stream)
        for i in range(K):
            f = frame + 1 + i
            x = [self.ev() for _ in range(3)]
            x[0].record(self.stream)
            pv.pv_update_dynamic(self.h, self.xfs[f], self.lts[f])
            x[1].record(self.stream)
            pv.pv_trace_all_deposit(self.h, self.P, self.seed, f, self.atlas, self.sc.atlas_rect, self.scale,
                                    self.stats[i])
            x[2].record(self.stream)
            ev.append(x)
        e.record(self.stream)
        self.barrier(ws)
        ms = s.elapsed_time(e) / K
        parts = np.array([[x[j].elapsed_time(x[j + 1]) for j in range(2)] for x in ev]).mean(axis=0)
        per_frame = np.array([x[0].elapsed_time(x[2]) for x in ev])
        rows = [pv.stats_dict(self.stats[i]) for i in range(K)]
        return ms, dict(zip(["update", "trace_all_deposit"], [float(v) for v in parts])), per_frame, rows, \
            self.mean_photons()

    # ---- end to end through the public API: host poses in, atlas and stats out (pinned), every frame
    def end_to_end(self, ws):
        """Two atlases alternate: frame i's result is copied to the host on a
        copy stream while frame i + 1 computes, and the host waits for frame
        i's copy before it launches frame i + 2."""
        torch, K = self.torch, self.K
        A = self.A
        atl = [self.atlas, torch.zeros_like(self.atlas)]
        host_atlas = [torch.empty(A, A, 3, dtype=torch.int64, pin_memory=True) for _ in range(2)]
        host_stats = [torch.empty(self.pv.STATS_WORDS, dtype=torch.int32, pin_memory=True) for _ in range(2)]
        copy_stream = torch.cuda.Stream(device=self.dev)
        done = [torch.cuda.Event(), torch.cuda.Event()]
        copied = [None, None]

        def e2e_frame(i, f):
            b = i % 2
            if copied[b] is not None:
                copied[b].synchronize()           # the host has frame i - 2's result; its buffers are free
                self.stream.wait_event(copied[b])
            self.reuse_frame(f, self.stats[-1 - b], atl[b])
            done[b].record(self.stream)
            copy_stream.wait_event(done[b])
            with torch.cuda.stream(copy_stream):
                host_atlas[b].copy_(atl[b], non_blocking=True)
                host_stats[b].copy_(self.stats[-1 - b], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy_stream)
            copied[b] = ev

        frame = self.restart()
        for i in range(self.W):
            frame += 1
            e2e_frame(i, frame)
        for ev in copied:
            ev.synchronize()
        self.barrier(ws)
        t = time.perf_counter()
        for i in range(K):
            frame += 1
            e2e_frame(i, frame)
        for ev in copied:
            ev.synchronize()
        e2e_s = (time.perf_counter() - t) / K
        h2d = 12 * 4 * int(self.sc.object_dynamic.sum()) + 64 * len(self.sc.lights(1))
        return {"value": None, "unit": "paths/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": int(host_atlas[0].numel() * 8 + host_stats[0].numel() * 4), "_s": e2e_s}

    # ---- F frames from a fresh trace-all with one setting: mean frame time and per-frame counters
    def run_frames(self, F, mode=None, tau=None, lts=None, stage=False, flags=0):
        """Frames 2..F+1 from a fresh trace-all, timed together; with ``stage``
        the same frames again with the library's stage events."""
        pv = self.pv
        lts = lts or self.lts
        self.restart(lts)
        self.stats[-2].zero_()
        self.torch.cuda.synchronize()
        s, e = self.ev(), self.ev()
        s.record(self.stream)
        for f in range(2, F + 2):
            self.reuse_frame(f, self.stats[-2], mode=mode, tau=tau, lts=lts, flags=flags)
        e.record(self.stream)
        self.torch.cuda.synchronize()
        ms = s.elapsed_time(e) / F
        st = pv.stats_dict(self.stats[-2])
        per = {k: v / F for k, v in st.items()}
        out = {"frames": F, "ms_per_frame": ms, "paths_per_s": self.N / (ms * 1e-3),
               "rays_per_frame": per["vis_rays"] + per["cont_rays"] + per["trace_rays"],
               "vis_rays_per_frame": per["vis_rays"], "cont_rays_per_frame": per["cont_rays"],
               "retrace_rays_per_frame": per["trace_rays"], "listed_per_frame": per["n_listed"],
               "cont_paths_per_frame": per["n_cont"], "reemit_per_frame": per["n_reemit"],
               "tails_per_frame": per["n_tail"], "updated_per_frame": per["n_updated"]}
        if stage:
            self.restart(lts)
            pv.pv_stage_timing(self.h, F)
            for f in range(2, F + 2):
                self.reuse_frame(f, self.stats[-1], mode=mode, tau=tau, lts=lts, flags=flags)
            t = pv.pv_stage_times(self.h, F).mean(axis=0)
            pv.pv_stage_timing(self.h, 0)
            out["stages_ms"] = dict(zip(pv.STAGES, [float(x) for x in t]))
        out["device_status"] = pv.pv_read_device_status(self.h)
        return out

    def destroy(self):
        self.pv.pv_destroy_scene(self.h)


def kernel_table(w, head_rows, inst, sep, rows_v, rows_r, ta, rows_ta, L_reuse, L_ta, hbm_peak, fma):
    """Per-kernel durations (CUDA events) against the algorithmic bytes each
    kernel must move (and, for traversals, the algorithmic FP32 work)."""
    agg = lambda key, rows: float(np.mean([r[key] for r in rows]))
    N = w.N
    n_dyn_tris = int((w.sc.object_dynamic[w.sc.tri_object] != 0).sum())
    photons = N * L_reuse                                   # stored photons after a reuse frame
    listed, tails, cont = agg("n_listed", head_rows), agg("n_tail", head_rows), agg("n_cont", head_rows)
    new_photons = agg("photons_written", head_rows)
    traffic = NCU_TRAFFIC.get(w.sc.name, {}) if NCU_TRAFFIC.get("digest") == source_digest() else {}

    def row(kernel, where, ms, nbytes, unit_note, ops=None):
        r = {"kernel": kernel, "timed": where, "duration_ms": ms, "algorithmic_bytes": nbytes,
             "bytes_per_unit": unit_note, "achieved_gbs": nbytes / (ms * 1e-3) / 1e9,
             "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / hbm_peak, "traffic": traffic.get(kernel),
             "traffic_over_algorithmic": traffic[kernel] / nbytes if kernel in traffic and nbytes else None}
        if ops is not None:
            r["algorithmic_ops"] = ops
            r["achieved_top_s"] = ops / (ms * 1e-3) / 1e12
            r["alu_frac"] = ops / (ms * 1e-3) / 1e12 / fma["top_s"]
        return r

    ops = lambda rows: OPS_PER_NODE * agg("node_visits", rows) + OPS_PER_TRI * agg("tri_tests", rows)
    st = inst["stages_ms"]
    t = [
        row("k_refit_wide", "pose update of the instrumented reuse frames", inst["update_ms"],
            n_dyn_tris * (36 + 48 + 128 / 3.0),
            "per dynamic triangle: 36 B object-local corners read, 48 B world triangle written, a third of a "
            "128 B wide node written"),
        row("k_verify_box", "stage events of pv_verify_retrace_deposit", st["k_verify"],
            N * (16 + 1) + 16.0 * photons + 8.0 * (listed - tails) + 4.0 * cont,
            "per path 4 B info + 12 B origin read, 1 B touched mark written; 16 B per stored photon (position row) "
            "read; 4 B info + 4 B list entry per listed path; 4 B per Alg. 1 list entry"),
        row("k_cont_trace<deposit>", "stage events of pv_verify_retrace_deposit", st["retrace_kernel"],
            N * 4 + 32.0 * photons + 8.0 * (listed + cont) + 32.0 * new_photons + 32.0 * L_reuse * cont,
            "deposit: 4 B info + 32 B per stored photon read; re-trace: 4 B list entry + 4 B info per listed or "
            "Alg. 1 path, 32 B per new photon written; Alg. 1: 32 B per stored photon of each path it checks",
            ops(head_rows)),
        row("k_compact", "pv_compact_replace on each verified frame's marks", sep["compact_ms"],
            N * 4 + 4.0 * agg("n_listed", rows_v), "4 B info read per path, 4 B per listed id written"),
        row("k_trace (re-trace)", "pv_retrace_invalid of the separate calls", sep["parts"]["retrace"],
            8.0 * agg("n_listed", rows_v) + 32.0 * agg("photons_written", rows_r) + 32.0 * agg("n_tail", rows_v),
            "4 B list entry + 4 B info per listed path, 32 B start photon read per tail, 32 B per new photon "
            "written", ops(rows_r)),
        row("k_deposit", "pv_deposit of the separate calls", sep["parts"]["deposit"], N * 4 + 32.0 * photons,
            "4 B info per path + 32 B per stored photon read (the atlas stays in L2)"),
        row("k_trace<deposit> (trace-all)", "pv_trace_all_deposit of the trace-all frames", ta["trace_all_deposit"],
            N * 16 + 32.0 * agg("photons_written", rows_ta),
            "12 B origin + 4 B info written per path, 32 B per photon written (deposited from registers, the "
            "atlas stays in L2)", ops(rows_ta)),
    ]
    return t


def measure(pv, torch, sc, args, dev, stream, ws, rank, local, fma, full: bool):
    """Every loop on one workload; ``full`` adds the tau, mode and moving-point-light rows."""
    K, W = args.steps, args.warmup
    F = args.sweep_frames
    frames_needed = max(W + K + 2, F + 2)
    w = Workload(pv, torch, sc, args, dev, stream, rank, K, W, frames_needed)
    pk, pk_kind = peaks()
    reuse_ms, head_rows, clocks, L_reuse, status = w.headline(ws, local)
    inst = w.instrumented(ws, head_rows)
    delta = w.delta(ws)
    sep, rows_v, rows_r = w.separate(ws)
    trace_ms, ta_parts, ta_per_frame, rows_ta, L_ta = w.trace_all(ws)
    e2e = None if args.no_e2e else w.end_to_end(ws)
    agg = lambda key, rows: float(np.mean([r[key] for r in rows]))
    kt = kernel_table(w, head_rows, inst, sep, rows_v, rows_r, ta_parts, rows_ta, L_reuse, L_ta, pk["hbm_gbs"], fma)
    rays_reuse = agg("vis_rays", head_rows) + agg("cont_rays", head_rows) + agg("trace_rays", head_rows)
    res = {"workload": f"{sc.name}: {WORKLOADS[sc.name]}", "paths": w.N, "max_bounces": w.B, "mode": args.mode,
           "tau": w.tau, "frames_timed": K, "first_timed_frame": w.first_timed,
           "l2": "inputs larger than L2 (path buffers %.0f MB)" % (w.N * (4 + 12 + 32 * w.B) / 1e6),
           "reuse_ms_per_frame": reuse_ms, "trace_all_ms_per_frame": trace_ms,
           "speedup_vs_trace_all": trace_ms / reuse_ms,
           "reuse_ms_parts": {"update": inst["update_ms"],
                              "verify_retrace_deposit": float(np.mean(inst["per_frame_ms"])) - inst["update_ms"]},
           "instrumented_ms_per_frame": float(np.mean(inst["per_frame_ms"])),
           "instrumented_counters_match": inst["counters_match"],
           "per_frame_ms_p50_p90": {"reuse": [float(np.percentile(inst["per_frame_ms"], q)) for q in (50, 90)],
                                    "trace_all": [float(np.percentile(ta_per_frame, q)) for q in (50, 90)],
                                    "note": "from the per-frame events of the instrumented loops"},
           "verify_retrace_deposit_stages_ms": inst["stages_ms"],
           "delta_deposit": delta, "separate_calls": sep, "trace_all_ms_parts": ta_parts,
           "rays_per_frame_reuse": rays_reuse, "rays_per_frame_trace_all": agg("trace_rays", rows_ta),
           "listed_per_frame": agg("n_listed", head_rows), "cont_paths_per_frame": agg("n_cont", head_rows),
           "tails_per_frame": agg("n_tail", head_rows), "vis_rays_per_frame": agg("vis_rays", head_rows),
           "mean_photons_per_path": L_reuse,
           "retrace_node_visits_per_ray": agg("node_visits", rows_r) / max(agg("trace_rays", rows_r), 1),
           "retrace_tri_tests_per_ray": agg("tri_tests", rows_r) / max(agg("trace_rays", rows_r), 1),
           "scene_build_s": w.build_s, "build_flags": args.build_flags, "kernels": kt}
    if full and not args.no_sweeps:
        res["tau_sweep"] = {f"{tau:g}": w.run_frames(F, tau=tau) for tau in TAUS}
        for row in res["tau_sweep"].values():
            row["speedup_vs_trace_all"] = trace_ms / row["ms_per_frame"]
        res["modes_tau_1pct"] = {m: w.run_frames(F, mode=MODES[m], tau=0.01) for m in MODES}
        # error mode with the moved objects' triangles in place of their boxes (PV_FLAG_ERROR_EXACT)
        res["modes_tau_1pct"]["error_triangle_tests"] = w.run_frames(F, mode=MODES["error"], tau=0.01, flags=2)
        res["modes_tau_1pct"]["trace_all_rays_per_frame"] = agg("trace_rays", rows_ta)
        if sc.name == "villa":
            import scenes
            vp = scenes.villa(moving_light="point")
            lts = {f: pv.make_lights(vp.lights(f)) for f in range(1, F + 2)}
            row = w.run_frames(F, lts=lts, stage=True)
            row["light"] = "ceiling point light moving 0.05 m/frame on a 1 m loop, torch static"
            row["speedup_vs_trace_all"] = trace_ms / row["ms_per_frame"]
            res["moving_point_light"] = row
    out = {"res": res, "value": w.N / (reuse_ms * 1e-3), "reuse_ms": reuse_ms, "trace_ms": trace_ms, "e2e": e2e,
           "clocks": clocks, "kernels": kt, "N": w.N}
    if not args.no_splat and sc.name != "tiny_box":
        res["splat"] = time_splat(pv, w.h, w.P, sc, K, W, stream, dev)
    if not args.no_adjoint and sc.name == "city":
        res["adjoint"] = time_adjoint(pv, w.h, w.P, sc, w.N, w.A, K, W, stream, dev)
    res["device_status"] = [status, pv.pv_read_device_status(w.h)]
    w.destroy()
    del w
    torch.cuda.empty_cache()
    if not args.no_dm and sc.name == "city":
        xfs = {f: sc.xforms(f) for f in range(1, W + K + 3)}
        lts = {f: sc.lights(f) for f in range(1, W + K + 3)}
        res["distribution_maps"] = time_dm(pv, sc, MODES[args.mode], res["tau"], sc.seed + 7919 * rank, K, W, xfs,
                                           lts, stream, dev)
        torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------- ours
def run_ours(args, ws, rank, local):
    import torch

    import paper_2111_06906_gb300 as pv
    from paper_2111_06906_gb300 import build as pvbuild
    pvbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fma = fma_peak(pv, torch, dev, sms, stream, local)
    head = measure(pv, torch, scene_for(args.workload), args, dev, stream, ws, rank, local, fma, full=True)
    secondary = {}
    if args.workload == "villa" and not args.no_secondary:
        city = measure(pv, torch, scene_for("city"), args, dev, stream, ws, rank, local, fma, full=False)
        secondary["city"] = dict(city["res"], value_paths_per_s=city["value"])
        b16 = run_batch(args, ws, rank, local, print_line=False)
        if b16 is not None:
            secondary["batch16"] = b16

    # ---- max over ranks
    e2e = head["e2e"]
    vals = torch.tensor([head["reuse_ms"], head["trace_ms"], e2e["_s"] if e2e else 0.0], dtype=torch.float64,
                        device=dev)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(vals, op=dist.ReduceOp.MAX)
    reuse_ms, trace_ms, e2e_s = vals.tolist()
    if rank != 0:
        return
    pk, pk_kind = peaks()
    cfg = head["res"]
    cfg["reuse_ms_per_frame"], cfg["trace_all_ms_per_frame"] = reuse_ms, trace_ms
    cfg["speedup_vs_trace_all"] = trace_ms / reuse_ms
    cfg.update(secondary)
    dom = next(k for k in head["kernels"] if k["kernel"] == "k_cont_trace<deposit>")
    roof = {"kernel": "k_cont_trace<deposit> (pv_verify_retrace_deposit: Alg. 1, re-trace, deposit)",
            "bound": "alu", "achieved": dom["achieved_top_s"], "peak": fma["top_s"], "unit": "Top/s",
            "frac": dom["achieved_top_s"] / fma["top_s"], "traffic": dom["traffic"],
            "traffic_note": "ncu DRAM bytes per launch, null unless captured on these kernel sources",
            "duration_ms": dom["duration_ms"],
            "peak_kind": "measured: k_fma_probe, FP32 fused multiply-adds per second on this GPU",
            "algorithmic_ops": dom["algorithmic_ops"],
            "ops_rule": f"{OPS_PER_NODE} per 4-wide node visit ({OPS_PER_SLAB} per slab test), {OPS_PER_TRI} per "
                        "triangle test, times the counted visits and tests",
            "hbm": {"achieved": dom["achieved_gbs"], "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": dom["hbm_frac"],
                    "algorithmic_bytes": dom["algorithmic_bytes"], "peak_kind": pk_kind},
            "fma_probe": fma, "hbm_peak": {"value": pk["hbm_gbs"], "unit": "GB/s", "kind": pk_kind},
            "kernels": head["kernels"], "source_digest": source_digest()}
    # kernels per reuse frame: the pose update with the top level (k_refit_wide), k_verify_box, and k_cont_trace
    # (Alg. 1, re-trace and deposit); the call's two memsets are not kernels of the library
    launches_per_frame = 3
    out = {"metric": METRIC, "value": ws * head["N"] / (reuse_ms * 1e-3), "unit": "paths/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": reuse_ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
           "roofline": roof, "gpu_launches": launches_per_frame * args.steps, "clocks": head["clocks"]}
    if e2e:
        e2e["value"] = ws * head["N"] / e2e_s
        e2e.pop("_s")
        out["e2e"] = e2e
    if not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(args.workload, MODES[args.mode], cfg["tau"], args.cpu_seconds)
    print(json.dumps(out), flush=True)


SPLAT_CAMERAS = {"city": ((0.0, 45.0, 35.0), (0.0, 0.0, 0.0), 0.3), "villa": ((10.0, 2.5, 2.0), (14.0, 0.5, 6.0), 0.08)}


def time_splat(pv, h, P, sc, K, W, stream, dev):
    """Screen-space splat (primary-ray G-buffer + radius kernel) of the current
    records at 1920 x 1080, 60 degree vertical field of view, timed per call."""
    import torch
    pos, target, radius = SPLAT_CAMERAS.get(sc.name, ((0.0, 1.5, 0.9), (0.0, 0.0, 0.0), 0.1))
    Wd, Hd = 1920, 1080
    cam = pv.PvCamera.make(pos, target, (0.0, 1.0, 0.0), math.radians(60.0), Wd, Hd)
    img = torch.zeros(Hd, Wd, 3, dtype=torch.float32, device=dev)
    work = torch.empty(pv.pv_splat_workspace_bytes(h, Wd, Hd), dtype=torch.uint8, device=dev)
    ms = []
    for i in range(W + K):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        pv.pv_splat(h, P, cam, radius, img, work)
        e[1].record(stream)
        if i >= W:
            ms.append(e)
    torch.cuda.synchronize()
    t = float(np.mean([a.elapsed_time(b) for a, b in ms]))
    lit = float((img.sum(-1) > 0).float().mean())
    return {"resolution": [Wd, Hd], "camera": {"pos": pos, "target": target, "fov_y_deg": 60.0},
            "radius": radius, "ms": t, "lit_fraction": lit, "photons": int(((P.info.view(torch.int32) >> 22) & 15)
                                                                            .clamp(max=sc.max_bounces).sum())}


def time_dm(pv, sc, mode, tau, seed, K, W, xfs, lts, stream, dev):
    """Reuse frames (update, verify with compute DM_C / prune / fill, re-trace)
    of a second copy of the scene whose lights carry distribution maps:
    8 x 8 x 64 x 64 for rectangles, 64 x 64 for point lights."""
    import torch
    rect, point = (8, 8, 64, 64), (64, 64)
    h = pv.pv_build_scene(sc.verts, sc.tri_object, sc.object_dynamic, sc.object_albedo, lts[1], sc.max_bounces,
                          sc.diag, object_xform=xfs[1], dm_rect=rect, dm_point=point)
    N = sc.n_paths
    P = pv.Paths.allocate(N, sc.max_bounces, dev)
    lst = torch.zeros(N, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    stats = torch.zeros(K, pv.STATS_WORDS, dtype=torch.int32, device=dev)
    scratch = pv.new_stats(dev)
    pv.pv_trace_all(h, P, seed, 1)
    ev = []
    for i in range(W + K):
        f = 2 + i
        st = scratch if i < W else stats[i - W]
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        pv.pv_update_dynamic(h, xfs[f], lts[f])
        pv.pv_verify_paths(h, P, mode, tau, 0, lst, cnt, st, seed=seed, frame=f)
        e[1].record(stream)
        pv.pv_retrace_invalid(h, P, lst, cnt, seed, f, st)
        e[2].record(stream)
        if i >= W:
            ev.append(e)
    torch.cuda.synchronize()
    rows = [pv.stats_dict(stats[i]) for i in range(K)]
    status = pv.pv_read_device_status(h)
    cells = [pv.pv_distribution_map_cells(h, l) for l in range(len(lts[1]))]
    pv.pv_destroy_scene(h)
    verify_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    retrace_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    mean = lambda k: float(np.mean([r[k] for r in rows]))
    return {"maps": {"rect": list(rect), "point": list(point)}, "cells_per_light": cells,
            "frame_ms": verify_ms + retrace_ms, "update_verify_dm_ms": verify_ms, "retrace_ms": retrace_ms,
            "pruned_per_frame": mean("n_pruned"), "filled_per_frame": mean("n_filled"),
            "listed_per_frame": mean("n_listed"), "device_status": status}


def time_adjoint(pv, h, P, sc, N, A, K, W, stream, dev):
    """Forward model splat and adjoint on the current path records, L2 loss
    against the atlas at the seeded perturbed pose (G = 2 (A - T) formed once,
    outside the timed calls); each call timed alone with CUDA events, L2
    flushed before each by writing a 256 MB buffer."""
    import torch

    import scenes
    rect = sc.atlas_rect
    th0 = torch.as_tensor(pv.pv_theta_current(h), device=dev)
    ths = torch.as_tensor(scenes.perturbed_theta(th0.cpu().numpy(), len(sc.lights(1))), dtype=torch.float32,
                          device=dev)
    T = torch.zeros(A, A, 3, dtype=torch.float32, device=dev)
    pv.pv_model_deposit(h, P, ths, T, rect)
    At = torch.zeros_like(T)
    pv.pv_model_deposit(h, P, th0, At, rect)
    G = 2 * (At - T)
    dth = torch.zeros_like(th0)
    score = torch.zeros(N, dtype=torch.float32, device=dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    fwd = []
    for i in range(W + K):
        flush.zero_()
        At.zero_()
        dth.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        pv.pv_model_deposit(h, P, th0, At, rect)
        e[1].record(stream)
        flush.zero_()
        e[2].record(stream)
        pv.pv_adjoint_deposit(h, P, th0, G, rect, dth, score)
        e[3].record(stream)
        if i >= W:
            fwd.append(e)
    torch.cuda.synchronize()
    f_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in fwd]))
    b_ms = float(np.mean([e[2].elapsed_time(e[3]) for e in fwd]))
    info = P.info.cpu().numpy().view(np.uint32)
    photons = float(np.minimum((info >> 22) & 15, sc.max_bounces).sum())
    # algorithmic bytes: per path info + origin + score, per photon PA + PB rows;
    # the atlas (read-modify-write forward, G read backward) once
    b_fwd = 16.0 * N + 32.0 * photons + 2 * 12.0 * A * A
    b_bwd = 20.0 * N + 32.0 * photons + 12.0 * A * A
    pk, pk_kind = peaks()
    return {"atlas": f"{A}x{A} RGB f32, uniform cubic B-spline splat", "loss": "L2 against the seeded perturbed pose",
            "forward_ms": f_ms, "adjoint_ms": b_ms, "paths_per_s_fwd_bwd": N / ((f_ms + b_ms) * 1e-3),
            "photons": photons, "theta": int(th0.numel()),
            "roofline_adjoint": {"kernel": "k_adjoint", "bound": "hbm", "achieved": b_bwd / (b_ms * 1e-3) / 1e9,
                                 "peak": pk["hbm_gbs"], "unit": "GB/s",
                                 "frac": b_bwd / (b_ms * 1e-3) / 1e9 / pk["hbm_gbs"], "peak_kind": pk_kind},
            "roofline_forward": {"kernel": "k_model_deposit", "bound": "hbm",
                                 "achieved": b_fwd / (f_ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                 "frac": b_fwd / (f_ms * 1e-3) / 1e9 / pk["hbm_gbs"], "peak_kind": pk_kind}}


# ----------------------------------------------------------------------------- batch of 16 scenes
def run_batch(args, ws, rank, local, print_line=True):
    """Sixteen uneven scenes per frame: the batched, tuned, graph-replayed
    frame (Alg. 1 fused with the re-trace) against the same scenes driven
    one after another through the single-scene calls (pv_update_dynamic,
    pv_verify_retrace: same frames, bit-identical results) and against
    trace-all of every scene."""
    import torch

    import paper_2111_06906_gb300 as pv
    import scenes
    from paper_2111_06906_gb300 import build as pvbuild
    pvbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scs = scenes.batch16()
    mode = MODES[args.mode]
    tau = 0.01 if args.tau is None else args.tau
    K, W = args.steps, args.warmup
    stream = torch.cuda.Stream(device=dev)
    n_total = sum(sc.n_paths for sc in scs)

    def make():
        out = []
        for i, sc in enumerate(scs):
            h = pv.pv_build_scene(sc.verts, sc.tri_object, sc.object_dynamic, sc.object_albedo, sc.lights(1),
                                  sc.max_bounces, sc.diag, object_xform=sc.xforms(1), stream=stream)
            P = pv.Paths.allocate(sc.n_paths, sc.max_bounces, dev)
            st = pv.new_stats(dev)
            seed = sc.seed + 7919 * rank
            pv.pv_trace_all(h, P, seed, 1, None, stream)
            out.append((h, P, st, seed))
        return out

    t0 = time.time()
    with torch.cuda.stream(stream):
        B = make()
    build_s = time.time() - t0
    # no lists asked for: Alg. 1 runs inside the batched re-trace kernel
    batch = pv.pv_batch_create([(h, P, None, None, st, seed) for (h, P, st, seed) in B], mode, tau, 0, stream)
    frame = 1

    # every frame's poses marshalled before the run, so the timed loop holds only the library call
    poses = {}

    def batch_frame(f):
        if f not in poses:
            poses[f] = pv.BatchPoses(len(scs), [sc.xforms(f) for sc in scs], [sc.lights(f) for sc in scs])
        pv.pv_batch_frame(batch, poses[f], None, f, stream)

    pv.pv_batch_autotune(batch, max(1, args.tune_frames))
    tune_frames = 0
    while pv.pv_batch_tuning(batch):
        frame += 1
        tune_frames += 1
        batch_frame(frame)
    for _ in range(W):
        frame += 1
        batch_frame(frame)
    for f in range(frame + 1, frame + K + 1):
        poses[f] = pv.BatchPoses(len(scs), [sc.xforms(f) for sc in scs], [sc.lights(f) for sc in scs])
    with torch.cuda.stream(stream):
        for x in B:
            x[2].zero_()                      # counters of the timed frames only
    stream.synchronize()
    first = frame + 1
    clocks = Clocks(local)
    with clocks:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t = time.perf_counter()
        e0.record(stream)
        for _ in range(K):
            frame += 1
            batch_frame(frame)
        e1.record(stream)
        stream.synchronize()
        wall = (time.perf_counter() - t) / K
    batch_ms = e0.elapsed_time(e1) / K
    cfg = pv.pv_batch_get_config(batch)
    step_ms = pv.pv_batch_step_times(batch)
    stats_b = [pv.stats_dict(x[2]) for x in B]
    pv.pv_batch_destroy(batch)
    status_b = [pv.pv_read_device_status(x[0]) for x in B]
    for x in B:
        pv.pv_destroy_scene(x[0])
    del B
    torch.cuda.empty_cache()

    # the same frames, scene after scene through the single-scene calls
    with torch.cuda.stream(stream):
        A = make()
    for f in range(2, first):
        for sc, (h, P, st, seed) in zip(scs, A):
            pv.pv_update_dynamic(h, sc.xforms(f), sc.lights(f), stream)
            pv.pv_verify_retrace(h, P, mode, tau, 0, seed, f, None, stream)
    stream.synchronize()
    pre = {f: [(np.ascontiguousarray(sc.xforms(f), np.float32), pv.make_lights(sc.lights(f))) for sc in scs]
           for f in range(first, first + K)}
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for f in range(first, first + K):
        for (xf, lt), (h, P, st, seed) in zip(pre[f], A):
            pv.pv_update_dynamic(h, xf, lt, stream)
            pv.pv_verify_retrace(h, P, mode, tau, 0, seed, f, st, stream)
    e3.record(stream)
    stream.synchronize()
    seq_ms = e2.elapsed_time(e3) / K
    # trace-all of every scene, same frames
    pre = {f: [(np.ascontiguousarray(sc.xforms(f), np.float32), pv.make_lights(sc.lights(f))) for sc in scs]
           for f in range(first + K, first + 2 * K)}
    e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e4.record(stream)
    for f in range(first + K, first + 2 * K):
        for (xf, lt), (h, P, st, seed) in zip(pre[f], A):
            pv.pv_update_dynamic(h, xf, lt, stream)
            pv.pv_trace_all(h, P, seed, f, None, stream)
    e5.record(stream)
    stream.synchronize()
    trace_ms = e4.elapsed_time(e5) / K
    status_a = [pv.pv_read_device_status(x[0]) for x in A]
    for x in A:
        pv.pv_destroy_scene(x[0])
    del A
    torch.cuda.empty_cache()
    if rank != 0:
        return None
    agg = lambda key, rows: float(sum(r[key] for r in rows)) / K
    summary = {"workload": f"batch16: {WORKLOADS['batch16']}", "paths": n_total, "mode": args.mode, "tau": tau,
               "frames_timed": K, "l2": "inputs larger than L2", "batch_frame_ms": batch_ms,
               "value_paths_per_s": ws * n_total / (batch_ms * 1e-3),
               "batch_frame_wall_ms": wall * 1e3, "sequential_single_scene_ms": seq_ms,
               "speedup_vs_sequential": seq_ms / batch_ms, "trace_all_ms": trace_ms,
               "speedup_vs_trace_all": trace_ms / batch_ms, "tuned_config": cfg, "tune_frames": tune_frames,
               "tuned_step_ms": dict(zip(["update", "verify", "continue", "compact", "retrace"], step_ms)),
               "listed_per_frame": agg("n_listed", stats_b), "rays_per_frame": agg("trace_rays", stats_b)
               + agg("cont_rays", stats_b) + agg("vis_rays", stats_b),
               "scene_build_s": build_s, "device_status": status_b + status_a, "clocks": clocks.summary()}
    if not print_line:
        return summary
    out = {"metric": METRIC, "value": ws * n_total / (batch_ms * 1e-3), "unit": "paths/s", "n_gpus": ws, "steps": K,
           "warmup": W, "ms_per_step": batch_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic", "config": summary,
           # graph kernel nodes per frame: prologue, transform + wide refit with the top levels, verify, Alg. 1 +
           # re-trace
           "gpu_launches": 4 * K, "clocks": clocks.summary()}
    print(json.dumps(out), flush=True)
    return summary


# ----------------------------------------------------------------------------- oracle
def _oracle_sample(workload, n_sample, seed_off=0):
    import oracle
    sc = scene_for(workload)
    ids = np.sort(np.random.default_rng(1234 + seed_off).choice(sc.n_paths, n_sample, replace=False)).astype(np.uint32)
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    p = o.trace(ids, sc.seed, 1)
    return sc, o, p


def _oracle_frame(o, sc, p, mode, tau, f):
    """One frame of the oracle on the sample; returns its verify and
    re-trace counters."""
    import oracle
    o.set_frames(f - 1, f)
    _, sv = o.verify(p, mode, tau)
    sr = o.retrace(p, sc.seed, f)
    oracle.deposit(p, 1024, 1024, sc.atlas_rect)
    return sv, sr


def _ambiguity(stats):
    """Queries the oracle flags ambiguous (a decision that a perturbation of
    1e-6 x the scene diagonal could flip), over all its queries: segment tests
    against moved objects, trace, Alg. 1 and visibility rays."""
    amb = sum(s.get("segments_amb", 0) + s.get("rays_amb", 0) for s in stats)
    seg = sum(s.get("segments_tested", 0) for s in stats)
    rays = sum(s.get("trace_rays", 0) + s.get("cont_rays", 0) + s.get("vis_rays", 0) for s in stats)
    return {"ambiguous_queries": int(amb), "segment_tests": int(seg), "rays": int(rays),
            "share": amb / max(seg + rays, 1),
            "segments_ambiguous_share": sum(s.get("segments_amb", 0) for s in stats) / max(seg, 1)}


CPU_SAMPLE = {"villa": 200, "city": 4000, "tiny_box": 10000}


def cpu_baseline(workload, mode, tau, seconds):
    """The oracle as it stands, on this host's cores, on a bounded sample:
    the sample's paths traced at frame 1 (untimed), then frames 2..30 run in
    order with frames 2, 15 and 30 timed (fewer when the time bound ends the
    run first); the full frame's time is extrapolated from the sample."""
    import oracle
    n_sample = CPU_SAMPLE[workload]
    sc, o, p = _oracle_sample(workload, n_sample)
    timed = {2, 15, 30}
    ts, stats = {}, []
    t_all = time.perf_counter()
    for f in range(2, 31):
        t = time.perf_counter()
        stats += _oracle_frame(o, sc, p, mode, tau, f)
        if f in timed:
            ts[f] = time.perf_counter() - t
        if time.perf_counter() - t_all > seconds and ts:
            break
    dt = float(np.mean(list(ts.values())))
    return {"value": n_sample / dt, "unit": "paths/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n_sample} seeded paths of the {workload} workload (verify + retrace + deposit, FP64 brute "
                      f"force over all {sc.n_tris} triangles), frames {sorted(ts)} timed of the run from frame 2",
            "frame_s": {str(k): v for k, v in sorted(ts.items())},
            "full_frame_s_extrapolated": sc.n_paths * dt / n_sample,
            "ambiguity": _ambiguity(stats)}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    sc0 = scene_for(args.workload)
    mode = MODES[args.mode]
    tau = sc0.tau if args.tau is None else args.tau
    n_sample = {"city": 2000, "villa": 300, "tiny_box": 10000}[args.workload]
    sc, o, p = _oracle_sample(args.workload, n_sample)
    f = 1
    for _ in range(args.warmup):
        f += 1
        _oracle_frame(o, sc, p, mode, tau, f)
    t = time.perf_counter()
    for _ in range(args.steps):
        f += 1
        _oracle_frame(o, sc, p, mode, tau, f)
    dt = (time.perf_counter() - t) / args.steps
    val = n_sample / dt
    sample = (f"{n_sample} seeded paths of the {args.workload} workload per step "
              f"(verify + retrace + deposit, FP64 brute force)")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "paths/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "mode": args.mode, "tau": tau,
                      "sample_paths": n_sample},
           "cpu_baseline": {"value": val, "unit": "paths/s", "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, ws, rank)
        elif args.workload == "batch16":
            run_batch(args, ws, rank, local)
        else:
            run_ours(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
