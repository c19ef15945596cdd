#!/usr/bin/env python
"""Benchmark of the per-frame path-verification hot path on one GB300.

One step = one frame of the reuse pipeline on the seeded city workload
(200k static triangles, 4 moving tori, a 1x1 m area light translating
0.1 m/frame, 1M photon paths of up to 7 bounces, error-based mode with
tau = 1 %):  pv_update_dynamic -> pv_verify_retrace_deposit (origin
update, dynamic occlusions, compaction, then Alg. 1, the re-trace and the
atlas deposit in one persistent kernel).  The same frames through the
separate calls (pv_verify_paths -> pv_retrace_invalid -> pv_deposit) and the
same library's trace-all frame (pv_update_dynamic -> pv_trace_all ->
pv_deposit) are timed beside it.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
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
    "city": "procedural city: 100x100 m floor, 16666 random boxes (200k static tris), 4 tori of 2048 tris on "
            "sinusoidal paths (2 m amplitude), 1x1 m area light translating 0.1 m/frame; 1M paths, <=7 bounces",
    "villa": "villa-shaped interior: 4x3 rooms, 2M static tris (30% clutter), 10 yawing tori of 5000 tris, "
             "point light + static area light + moving tilting torch; 3M paths, <=7 bounces",
    "tiny_box": "open 2x2x2 box (10 tris) + moving unit cube (12 tris), point light; 10k paths, <=3 bounces",
    "batch16": "16 independent districts: 10k to 2M tris, 50k to 3M paths (12.4M in all), 1 to 3 lights, "
               "bounce caps 1 to 7, 1 to 4 moving tori; one batched graph-captured frame per step, tuned",
}
# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) of one k_cont_trace<deposit> launch of a
# timed reuse frame, measured on the same kernel code
TRACE_TRAFFIC = {"city": 204794112 + 21009664, "villa": 940165632 + 104417536}
# warp instructions issued by one launch of the same kernel (ncu smsp__inst_executed.sum, same capture), and the
# average active lanes per issued instruction (smsp__thread_inst_executed_per_inst_executed.ratio)
TRACE_WARP_INST = {"city": (173336291, 9.57), "villa": (592380139, 12.04)}
SCHEDULERS_PER_SM = 4
OPS_PER_NODE = 107    # FP32-pipe ops per wide-node visit (four slab tests + ordering network), from the source
OPS_PER_TRI = 40      # FP32-pipe ops per Moller-Trumbore test, counted from the source
SM_COUNT, FP32_LANES = 152, 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="city", choices=list(WORKLOADS))
    ap.add_argument("--mode", default="error", choices=list(MODES))
    ap.add_argument("--tau", type=float, default=None)
    ap.add_argument("--atlas", type=int, default=1024)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-dm", action="store_true", help="skip the distribution-map frame measurement")
    ap.add_argument("--no-splat", action="store_true", help="skip the 1920x1080 screen-space splat measurement")
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


def scene_for(name, rank=0):
    import scenes
    return scenes.by_name(name)


# ----------------------------------------------------------------------------- ours
def run_ours(args, ws, rank, local):
    import torch

    import paper_2111_06906_gb300 as pv
    from paper_2111_06906_gb300 import build as pvbuild
    pvbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc = scene_for(args.workload)
    mode = MODES[args.mode]
    tau = sc.tau if args.tau is None else args.tau
    seed = sc.seed + 7919 * rank
    N, B = sc.n_paths, sc.max_bounces
    frames_needed = args.warmup + args.steps + 2      # every loop restarts at frame 1: the same frames timed
    xfs = {f: sc.xforms(f) for f in range(1, frames_needed + 1)}
    lts = {f: sc.lights(f) for f in range(1, frames_needed + 1)}

    t0 = time.time()
    h = pv.pv_build_scene(sc.verts, sc.tri_object, sc.object_dynamic, sc.object_albedo, lts[1], B, sc.diag,
                          object_xform=xfs[1], flags=args.build_flags)
    build_s = time.time() - t0
    P = pv.Paths.allocate(N, B, dev)
    A = args.atlas
    atlas = torch.zeros(A, A, 3, dtype=torch.int64, device=dev)
    scale = 40 if args.workload != "tiny_box" else 31
    lst = torch.zeros(N, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    K, W = args.steps, args.warmup
    stats = torch.zeros(4 * K + 2, pv.STATS_WORDS, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def restart():
        # back to the pose of frame 1 and a fresh bootstrap, so that every loop below runs frames 2, 3, ...
        pv.pv_update_dynamic(h, xfs[1], lts[1])
        pv.pv_trace_all(h, P, seed, 1)
        return 1

    frame = restart()

    def reuse_frame(f, st, at=None):
        pv.pv_update_dynamic(h, xfs[f], lts[f])
        pv.pv_verify_retrace_deposit(h, P, mode, tau, 0, seed, f, atlas if at is None else at, sc.atlas_rect, scale,
                                     st)

    def timed_loop(fn, first_frame, rows_a, rows_b):
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(K)]
        for i in range(K):
            f = first_frame + i
            e = ev[i]
            e[0].record(stream)
            pv.pv_update_dynamic(h, xfs[f], lts[f])
            e[1].record(stream)
            fn(f, rows_a[i], rows_b[i], e)
            e[4].record(stream)
        return ev

    def fused_body(f, st_v, st_r, e):
        pv.pv_verify_retrace_deposit(h, P, mode, tau, 0, seed, f, atlas, sc.atlas_rect, scale, st_v)
        e[2].record(stream)
        e[3].record(stream)

    def separate_body(f, st_v, st_r, e):
        pv.pv_verify_paths(h, P, mode, tau, 0, lst, cnt, st_v)
        e[2].record(stream)
        pv.pv_retrace_invalid(h, P, lst, cnt, seed, f, st_r)
        e[3].record(stream)
        pv.pv_deposit(h, P, atlas, sc.atlas_rect, scale)

    def trace_body(f, st_v, st_r, e):
        e[2].record(stream)
        pv.pv_trace_all(h, P, seed, f, st_r)
        e[3].record(stream)
        pv.pv_deposit(h, P, atlas, sc.atlas_rect, scale)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- reuse pipeline, one call from verification to re-trace (headline): only the two events that bracket
    # the K frames, nothing recorded between the library's launches
    for i in range(W):
        frame += 1
        reuse_frame(frame, stats[-1])
    barrier()
    clocks = Clocks(local)
    with clocks:
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for i in range(K):
            reuse_frame(frame + 1 + i, stats[i])
        stop.record(stream)
        barrier()
    frame += K
    reuse_ms = start.elapsed_time(stop) / K
    st_reuse = [pv.stats_dict(stats[i]) for i in range(K)]
    info_np = P.info.cpu().numpy().view(np.uint32)
    mean_L = float(((info_np >> 22) & 15).mean())
    status = pv.pv_read_device_status(h)

    # ---- the same frames again with events between the calls and the library's own stage events
    frame = restart()
    for i in range(W):
        frame += 1
        reuse_frame(frame, stats[-1])
    pv.pv_stage_timing(h, K)                   # the library records its stages' events in the timed frames
    barrier()
    ev = timed_loop(fused_body, frame + 1, stats[K:2 * K], stats[K:2 * K])
    barrier()
    frame += K
    reuse_parts = np.array([[e[j].elapsed_time(e[j + 1]) for j in range(4)] for e in ev]).mean(axis=0)
    stage_ms = pv.pv_stage_times(h, K).mean(axis=0)     # k_verify, compaction, fused kernel, whole call
    pv.pv_stage_timing(h, 0)
    per_frame = np.array([e[0].elapsed_time(e[4]) for e in ev])
    instrumented_ms = float(per_frame.mean())
    reuse_pct = [float(np.percentile(per_frame, q)) for q in (50, 90)]
    same = all(pv.stats_dict(stats[K + i]) == st_reuse[i] for i in range(K))

    # ---- the same frames with the atlas carried from frame to frame (pv_verify_retrace_deposit_delta): only the
    # paths a frame changes leave and re-enter it; the final atlas must equal the full deposit's
    atlas_full = atlas.clone()
    atlas_delta = torch.zeros_like(atlas)
    frame = restart()
    pv.pv_deposit(h, P, atlas_delta, sc.atlas_rect, scale)

    def delta_frame(f, st):
        pv.pv_update_dynamic(h, xfs[f], lts[f])
        pv.pv_verify_retrace_deposit_delta(h, P, mode, tau, 0, seed, f, atlas_delta, sc.atlas_rect, scale, st)

    for i in range(W):
        frame += 1
        delta_frame(frame, stats[-1])
    barrier()
    start4 = torch.cuda.Event(enable_timing=True)
    stop4 = torch.cuda.Event(enable_timing=True)
    start4.record(stream)
    for i in range(K):
        delta_frame(frame + 1 + i, stats[-1])
    stop4.record(stream)
    barrier()
    frame += K
    delta_ms = start4.elapsed_time(stop4) / K
    delta_equal = bool(torch.equal(atlas_delta, atlas_full))
    del atlas_full, atlas_delta

    # ---- the same frames through the separate calls (pv_verify_paths, then pv_retrace_invalid)
    frame = restart()
    stats[:2 * K].zero_()                      # counters accumulate
    for i in range(W):
        frame += 1
        pv.pv_update_dynamic(h, xfs[frame], lts[frame])
        pv.pv_verify_paths(h, P, mode, tau, 0, lst, cnt, stats[-1])
        pv.pv_retrace_invalid(h, P, lst, cnt, seed, frame, stats[-1])
        pv.pv_deposit(h, P, atlas, sc.atlas_rect, scale)
    barrier()
    start3 = torch.cuda.Event(enable_timing=True)
    stop3 = torch.cuda.Event(enable_timing=True)
    start3.record(stream)
    ev3 = timed_loop(separate_body, frame + 1, stats[:K], stats[K:2 * K])
    stop3.record(stream)
    barrier()
    frame += K
    sep_ms = start3.elapsed_time(stop3) / K
    sep_parts = np.array([[e[j].elapsed_time(e[j + 1]) for j in range(4)] for e in ev3]).mean(axis=0)
    st_retrace = [pv.stats_dict(stats[K + i]) for i in range(K)]

    # ---- trace-all baseline (same library, same GPU), on the same frames
    frame = restart()
    for i in range(W):
        frame += 1
        pv.pv_update_dynamic(h, xfs[frame], lts[frame])
        pv.pv_trace_all(h, P, seed, frame, stats[-1])
        pv.pv_deposit(h, P, atlas, sc.atlas_rect, scale)
    barrier()
    start2 = torch.cuda.Event(enable_timing=True)
    stop2 = torch.cuda.Event(enable_timing=True)
    start2.record(stream)
    ev2 = timed_loop(trace_body, frame + 1, stats[2 * K:3 * K], stats[3 * K:4 * K])
    stop2.record(stream)
    barrier()
    frame += K
    trace_ms = start2.elapsed_time(stop2) / K
    parts2 = np.array([[e[j].elapsed_time(e[j + 1]) for j in range(4)] for e in ev2]).mean(axis=0)
    per_frame2 = np.array([e[0].elapsed_time(e[4]) for e in ev2])
    trace_pct = [float(np.percentile(per_frame2, q)) for q in (50, 90)]
    st_trace = [pv.stats_dict(stats[3 * K + i]) for i in range(K)]

    # ---- end to end through the API: host poses in, atlas and stats out (pinned), every frame.  Two atlases
    # alternate: frame i's result is copied to the host on a copy stream while frame i + 1 computes, and the
    # host waits for frame i's copy before it launches frame i + 2
    e2e = None
    if not args.no_e2e:
        atl = [atlas, torch.zeros_like(atlas)]
        host_atlas = [torch.empty(A, A, 3, dtype=torch.int64, pin_memory=True) for _ in range(2)]
        host_stats = [torch.empty(pv.STATS_WORDS, dtype=torch.int32, pin_memory=True) for _ in range(2)]
        copy_stream = torch.cuda.Stream(device=dev)
        done = [torch.cuda.Event(), torch.cuda.Event()]
        copied = [None, None]

        def e2e_frame(i, f):
            b = i % 2
            if copied[b] is not None:
                copied[b].synchronize()           # the host has frame i - 2's result; its buffers are free
                stream.wait_event(copied[b])
            reuse_frame(f, stats[-1 - b], atl[b])
            done[b].record(stream)
            copy_stream.wait_event(done[b])
            with torch.cuda.stream(copy_stream):
                host_atlas[b].copy_(atl[b], non_blocking=True)
                host_stats[b].copy_(stats[-1 - b], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy_stream)
            copied[b] = ev

        # the same frames as the device-timed loop, from a fresh bootstrap
        frame = restart()
        for i in range(W):
            frame += 1
            e2e_frame(i, frame)
        for ev in copied:
            ev.synchronize()
        barrier()
        t = time.perf_counter()
        for i in range(K):
            frame += 1
            e2e_frame(i, frame)
        for ev in copied:
            ev.synchronize()
        e2e_s = (time.perf_counter() - t) / K
        h2d = 12 * 4 * int(sc.object_dynamic.sum()) + 64 * len(lts[1])
        e2e = {"value": None, "unit": "paths/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": int(host_atlas[0].numel() * 8 + host_stats[0].numel() * 4), "_s": e2e_s}
    # ---- differentiable model: forward splat and adjoint of an L2 atlas loss
    adjoint = None if args.no_adjoint else time_adjoint(pv, h, P, sc, N, A, K, W, stream, dev)
    # ---- screen-space splat of the current records at 1920 x 1080
    splat = None if args.no_splat or args.workload == "tiny_box" else time_splat(pv, h, P, sc, K, W, stream, dev)
    # ---- the same reuse frames with distribution maps on the lights (Sec. 3.1)
    dm = None if args.no_dm or args.workload == "tiny_box" else time_dm(pv, sc, mode, tau, seed, K, W, xfs, lts,
                                                                          stream, dev)
    status2 = pv.pv_read_device_status(h)
    pv.pv_destroy_scene(h)

    # ---- max over ranks
    vals = torch.tensor([reuse_ms, trace_ms, e2e["_s"] if e2e else 0.0], dtype=torch.float64, device=dev)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(vals, op=dist.ReduceOp.MAX)
    reuse_ms, trace_ms, e2e_s = vals.tolist()
    if rank != 0:
        return

    pk, pk_kind = peaks()
    names = ["update", "verify_retrace", "-", "deposit"]
    agg = lambda key, rows: float(np.mean([r[key] for r in rows]))
    # dominant kernel: the persistent kernel of pv_verify_retrace_deposit (Alg. 1, the re-trace and the atlas
    # deposit), timed by the library's own events; its traversal work comes from the counted node visits and
    # triangle tests of the call (k_verify traverses only for moving point lights: vis_rays = 0 here)
    ops = OPS_PER_NODE * agg("node_visits", st_reuse) + OPS_PER_TRI * agg("tri_tests", st_reuse)
    ops_peak = SM_COUNT * FP32_LANES * pk.get("sm_max_mhz", 2070.0) * 1e6
    achieved = ops / (float(stage_ms[2]) * 1e-3)
    roof = {"kernel": "k_cont_trace<deposit> (pv_verify_retrace_deposit)", "bound": "alu",
            "achieved": achieved / 1e12, "peak": ops_peak / 1e12, "unit": "Top/s", "frac": achieved / ops_peak,
            "duration_ms": float(stage_ms[2]),
            "traffic": TRACE_TRAFFIC.get(args.workload), "traffic_unit": "bytes per launch (ncu)",
            "peak_kind": f"derived: {SM_COUNT} SMs x {FP32_LANES} FP32 lanes x max SM clock"}
    if args.workload in TRACE_WARP_INST:
        # the same kernel against the issue rate: warp instructions per launch (ncu) over the live duration,
        # against one instruction per scheduler per clock; lanes per instruction give the SIMT efficiency
        inst, lanes = TRACE_WARP_INST[args.workload]
        issue_peak = SM_COUNT * SCHEDULERS_PER_SM * pk.get("sm_max_mhz", 2070.0) * 1e6
        issue = inst / (float(stage_ms[2]) * 1e-3)
        roof["issue"] = {"achieved": issue / 1e9, "peak": issue_peak / 1e9, "unit": "G warp-inst/s",
                         "frac": issue / issue_peak, "active_lanes_per_inst": lanes, "simt_efficiency": lanes / 32.0,
                         "source": "warp instructions per launch from ncu, duration live"}
    rays_reuse = agg("vis_rays", st_reuse) + agg("cont_rays", st_reuse) + agg("trace_rays", st_reuse)
    rays_trace = agg("trace_rays", st_trace)
    value = ws * N / (reuse_ms * 1e-3)
    cfg = {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "paths": N, "max_bounces": B,
           "mode": args.mode, "tau": tau, "frames_timed": K,
           "l2": "inputs larger than L2 (path buffers %.0f MB)" % (N * (4 + 12 + 32 * B) / 1e6),
           "reuse_ms_per_frame": reuse_ms, "trace_all_ms_per_frame": trace_ms,
           "speedup_vs_trace_all": trace_ms / reuse_ms,
           "reuse_ms_parts": {"update": float(reuse_parts[0]), "verify_retrace_deposit": float(reuse_parts[1])},
           "instrumented_ms_per_frame": instrumented_ms, "instrumented_counters_match": same,
           "per_frame_ms_p50_p90": {"reuse": reuse_pct, "trace_all": trace_pct,
                                    "note": "from the per-frame events of the instrumented loops"},
           "delta_deposit": {"call": "pv_verify_retrace_deposit_delta", "ms_per_frame": delta_ms,
                             "paths_per_s": ws * N / (delta_ms * 1e-3), "atlas_equal_to_full_deposit": delta_equal},
           "verify_retrace_deposit_stages_ms": {"k_verify": float(stage_ms[0]), "compaction": float(stage_ms[1]),
                                                "k_cont_trace+deposit": float(stage_ms[2]),
                                                "call": float(stage_ms[3])},
           "separate_calls": {"ms_per_frame": sep_ms,
                              "parts": dict(zip(["update", "verify", "retrace", "deposit"],
                                                [float(x) for x in sep_parts]))},
           "trace_all_ms_parts": dict(zip(["update", "-", "trace_all", "deposit"], [float(x) for x in parts2])),
           "rays_per_frame_reuse": rays_reuse, "rays_per_frame_trace_all": rays_trace,
           "listed_per_frame": agg("n_listed", st_reuse), "cont_paths_per_frame": agg("n_cont", st_reuse),
           "tails_per_frame": agg("n_tail", st_reuse), "vis_rays_per_frame": agg("vis_rays", st_reuse),
           "mean_photons_per_path": mean_L,
           "retrace_node_visits_per_ray": agg("node_visits", st_retrace) / max(agg("trace_rays", st_retrace), 1),
           "retrace_tri_tests_per_ray": agg("tri_tests", st_retrace) / max(agg("trace_rays", st_retrace), 1),
           "scene_build_s": build_s, "build_flags": args.build_flags, "device_status": [status, status2]}
    # kernels per reuse frame: the pose update with the top level (k_refit_wide), k_verify_box, and k_cont_trace
    # (Alg. 1, re-trace and deposit); the two memsets of the call are not kernels of the library
    launches_per_frame = 3
    out = {"metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": ws, "steps": K, "warmup": W,
           "ms_per_step": reuse_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic", "config": cfg, "roofline": roof,
           "gpu_launches": launches_per_frame * K, "clocks": clocks.summary()}
    if adjoint:
        cfg["adjoint"] = adjoint
    if dm:
        cfg["distribution_maps"] = dm
    if splat:
        cfg["splat"] = splat
    if e2e:
        e2e["value"] = ws * N / e2e_s
        e2e.pop("_s")
        out["e2e"] = e2e
    if not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(args.workload, mode, tau, args.cpu_seconds)
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
    fwd, bwd = [], []
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
def run_batch(args, ws, rank, local):
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

    def make(copy):
        out = []
        for i, sc in enumerate(scs):
            h = pv.pv_build_scene(sc.verts, sc.tri_object, sc.object_dynamic, sc.object_albedo, sc.lights(1),
                                  sc.max_bounces, sc.diag, object_xform=sc.xforms(1), stream=stream)
            P = pv.Paths.allocate(sc.n_paths, sc.max_bounces, dev)
            lst = torch.zeros(sc.n_paths, dtype=torch.int32, device=dev)
            cnt = torch.zeros(1, dtype=torch.int32, device=dev)
            st = pv.new_stats(dev)
            seed = sc.seed + 7919 * rank
            pv.pv_trace_all(h, P, seed, 1, None, stream)
            out.append((h, P, lst, cnt, st, seed))
        return out

    t0 = time.time()
    with torch.cuda.stream(stream):
        B = make(1)
    build_s = time.time() - t0
    # no lists asked for: Alg. 1 runs inside the batched re-trace kernel
    batch = pv.pv_batch_create([(h, P, None, None, st, seed) for (h, P, lst, cnt, st, seed) in B], mode, tau, 0,
                               stream)
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
            x[4].zero_()                      # counters of the timed frames only
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
    stats_b = [pv.stats_dict(x[4]) for x in B]
    pv.pv_batch_destroy(batch)
    status_b = [pv.pv_read_device_status(x[0]) for x in B]
    for x in B:
        pv.pv_destroy_scene(x[0])
    del B
    torch.cuda.empty_cache()

    # the same frames, scene after scene through the single-scene calls
    with torch.cuda.stream(stream):
        A = make(0)
    for f in range(2, first):
        for sc, (h, P, lst, cnt, st, seed) in zip(scs, A):
            pv.pv_update_dynamic(h, sc.xforms(f), sc.lights(f), stream)
            pv.pv_verify_retrace(h, P, mode, tau, 0, seed, f, None, stream)
    stream.synchronize()
    pre = {f: [(np.ascontiguousarray(sc.xforms(f), np.float32), pv.make_lights(sc.lights(f))) for sc in scs]
           for f in range(first, first + K)}
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for f in range(first, first + K):
        for (xf, lt), (h, P, lst, cnt, st, seed) in zip(pre[f], A):
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
        for (xf, lt), (h, P, lst, cnt, st, seed) in zip(pre[f], A):
            pv.pv_update_dynamic(h, xf, lt, stream)
            pv.pv_trace_all(h, P, seed, f, None, stream)
    e5.record(stream)
    stream.synchronize()
    trace_ms = e4.elapsed_time(e5) / K
    status_a = [pv.pv_read_device_status(x[0]) for x in A]
    for x in A:
        pv.pv_destroy_scene(x[0])
    if rank != 0:
        return
    agg = lambda key, rows: float(sum(r[key] for r in rows)) / K
    pk, pk_kind = peaks()
    ops = OPS_PER_NODE * agg("node_visits", stats_b) + OPS_PER_TRI * agg("tri_tests", stats_b)
    ops_peak = SM_COUNT * FP32_LANES * pk.get("sm_max_mhz", 2070.0) * 1e6
    achieved = ops / (batch_ms * 1e-3)
    out = {"metric": METRIC, "value": ws * n_total / (batch_ms * 1e-3), "unit": "paths/s", "n_gpus": ws, "steps": K,
           "warmup": W, "ms_per_step": batch_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"batch16: {WORKLOADS['batch16']}", "paths": n_total, "mode": args.mode, "tau": tau,
                      "frames_timed": K, "l2": "inputs larger than L2", "batch_frame_ms": batch_ms,
                      "batch_frame_wall_ms": wall * 1e3, "sequential_single_scene_ms": seq_ms,
                      "speedup_vs_sequential": seq_ms / batch_ms, "trace_all_ms": trace_ms,
                      "speedup_vs_trace_all": trace_ms / batch_ms, "tuned_config": cfg, "tune_frames": tune_frames,
                      "tuned_step_ms": dict(zip(["update", "verify", "continue", "compact", "retrace"], step_ms)),
                      "listed_per_frame": agg("n_listed", stats_b), "rays_per_frame": agg("trace_rays", stats_b)
                      + agg("cont_rays", stats_b) + agg("vis_rays", stats_b),
                      "scene_build_s": build_s, "device_status": status_b + status_a},
           "roofline": {"kernel": "whole batched frame (traversal-bound)", "bound": "alu",
                        "achieved": achieved / 1e12, "peak": ops_peak / 1e12, "unit": "Top/s",
                        "frac": achieved / ops_peak, "traffic": None,
                        "peak_kind": f"derived: {SM_COUNT} SMs x {FP32_LANES} FP32 lanes x max SM clock"},
           # graph kernel nodes per frame: prologue, transform + wide refit, poses + top level, verify,
           # compaction, Alg. 1 + re-trace
           "gpu_launches": 6 * K, "clocks": clocks.summary()}
    print(json.dumps(out), flush=True)


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
    import oracle
    o.set_frames(f - 1, f)
    o.verify(p, mode, tau)
    o.retrace(p, sc.seed, f)
    oracle.deposit(p, 1024, 1024, sc.atlas_rect)


def cpu_baseline(workload, mode, tau, seconds):
    """The oracle as it stands, on this host's cores, on a bounded sample."""
    import oracle
    n_sample = {"city": 4000, "villa": 600, "tiny_box": 10000}[workload]
    sc, o, p = _oracle_sample(workload, n_sample)
    t = time.perf_counter()
    frames = 0
    f = 1
    while time.perf_counter() - t < seconds and frames < 60:
        f += 1
        _oracle_frame(o, sc, p, mode, tau, f)
        frames += 1
    dt = time.perf_counter() - t
    return {"value": n_sample * frames / dt, "unit": "paths/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n_sample} seeded paths of the {workload} workload, frames 2..{f} "
                      f"(verify + retrace + deposit, FP64 brute force over all {sc.n_tris} triangles)"}


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
