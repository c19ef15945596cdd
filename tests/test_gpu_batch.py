"""GPU tests of the batched frame (include/pv_batch.h).

Every scene of a batch must end each frame with exactly the records, lists
and counters that the single-scene calls (pv_update_dynamic,
pv_verify_paths, pv_retrace_invalid with the same seed and frame) produce:
the same device code runs, only the mapping of work to threads differs, so
the comparison is bit-exact (the traversal counters of the warp-per-path
verify mapping are the one documented exception).  A second check runs the
batch against the FP64 oracle.
"""
import math

import numpy as np
import pytest

import oracle
import scenes
import paper_2111_06906_gb300 as pv
from scenes import LIGHT_POINT, Light
from tests import gpu_util as gu
from tests import scene_kit as kit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2111_06906_gb300 import build
    build.build()
    pv.load()


def _torch():
    import torch
    return torch


def _moving_point_light(n_paths=3000):
    """Tiny box shell with a torus and a point light that moves every frame."""
    sc = kit.box_with_torus(n_paths, B=3, seed=5)
    sc._light_fn = lambda f: [Light(LIGHT_POINT, (0.05 * (f - 1), 1.8, 0.02 * (f - 1)), power=(100.0,) * 3,
                                    n_paths=n_paths)]
    return sc


def _mix():
    """Uneven scenes: point and area lights, 1 to 7 bounces, 2k to 40k paths."""
    return [scenes.tiny_box(n_paths=5000),
            kit.box_with_torus(4000, B=4),
            kit.rect_light_over_floor(2000, shift=lambda f: (0.03 * (f - 1), 0.0, 0.0), B=1, R=3.0),
            _moving_point_light(),
            scenes.city(n_paths=40000, n_boxes=1500)]


class Lane:
    """One scene driven twice: through the single-scene calls and in a batch
    (with distribution maps of the given resolutions on its lights)."""

    def __init__(self, sc, seed, dm_rect=(0, 0, 0, 0), dm_point=(0, 0)):
        torch = _torch()
        self.sc, self.seed = sc, seed
        self.dm = any(dm_rect) or any(dm_point)
        self.h1 = gu.lib_scene(sc, dm_rect=dm_rect, dm_point=dm_point)
        self.h2 = gu.lib_scene(sc, dm_rect=dm_rect, dm_point=dm_point)
        n, B = sc.n_paths, sc.max_bounces
        self.P1 = pv.Paths.allocate(n, B)
        self.P2 = pv.Paths.allocate(n, B)
        pv.pv_trace_all(self.h1, self.P1, seed, 1)
        pv.pv_trace_all(self.h2, self.P2, seed, 1)
        self.l1 = torch.zeros(n, dtype=torch.int32, device="cuda")
        self.c1 = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.l2 = torch.zeros(n, dtype=torch.int32, device="cuda")
        self.c2 = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.s1 = pv.new_stats()
        self.s2 = pv.new_stats()

    def item(self, lists=True):
        return (self.h2, self.P2, self.l2 if lists else None, self.c2 if lists else None, self.s2, self.seed)

    def single_frame(self, f, mode, tau, flags):
        pv.pv_update_dynamic(self.h1, self.sc.xforms(f), self.sc.lights(f))
        pv.pv_verify_paths(self.h1, self.P1, mode, tau, flags, self.l1, self.c1, self.s1, seed=self.seed, frame=f)
        pv.pv_retrace_invalid(self.h1, self.P1, self.l1, self.c1, self.seed, f, self.s1)

    def compare(self, traversal_counters=True, lists=True):
        torch = _torch()
        for a, b in ((self.P1.info, self.P2.info), (self.P1.origin, self.P2.origin), (self.P1.pa, self.P2.pa),
                     (self.P1.pb, self.P2.pb)):
            assert torch.equal(a.view(torch.int32), b.view(torch.int32))
        if lists:
            n1, n2 = int(self.c1.item()), int(self.c2.item())
            assert n1 == n2
            assert torch.equal(self.l1[:n1], self.l2[:n2])
        if self.dm:
            for l in range(len(self.sc.lights(1))):
                assert np.array_equal(pv.pv_read_distribution_map(self.h1, l), pv.pv_read_distribution_map(self.h2, l))
        d1, d2 = pv.stats_dict(self.s1), pv.stats_dict(self.s2)
        if not traversal_counters:
            for k in ("node_visits", "tri_tests"):
                d1.pop(k)
                d2.pop(k)
        assert d1 == d2, (d1, d2)

    def close(self):
        for h in (self.h1, self.h2):
            assert pv.pv_read_device_status(h) == 0
            pv.pv_destroy_scene(h)


def _run(lanes, batch, frames, mode, tau, flags, traversal_counters=True, lists=True):
    for f in frames:
        for ln in lanes:
            ln.single_frame(f, mode, tau, flags)
        pv.pv_batch_frame(batch, [ln.sc.xforms(f) for ln in lanes], [ln.sc.lights(f) for ln in lanes], f)
        for ln in lanes:
            ln.compare(traversal_counters, lists)


CONFIGS = [
    {},
    {"verify_mapping": 1},
    {"verify_mapping": 2, "verify_threads": 64},
    {"verify_threads": 64, "trace_steps": 16},
    {"verify_threads": 128, "trace_steps": 32, "trace_blocks": 2},
    {"stack": 64},
]


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: ",".join(f"{k}={v}" for k, v in c.items()) or "default")
def test_batch_matches_single_scene_calls(cfg):
    lanes = [Lane(sc, 11 + 7 * i) for i, sc in enumerate(_mix())]
    b = pv.pv_batch_create([ln.item() for ln in lanes], pv.PV_MODE_ERROR, 0.01)
    if cfg:
        pv.pv_batch_set_config(b, **cfg)
    _run(lanes, b, range(2, 7), pv.PV_MODE_ERROR, 0.01, 0, traversal_counters=cfg.get("verify_mapping", 0) != 1)
    pv.pv_batch_destroy(b)
    for ln in lanes:
        ln.close()


@pytest.mark.parametrize("mode,flags", [(pv.PV_MODE_NAIVE_AABB, 0), (pv.PV_MODE_NAIVE_EXACT, 0),
                                        (pv.PV_MODE_ERROR, pv.PV_FLAG_ERROR_EXACT)])
@pytest.mark.parametrize("mapping", [0, 1])
def test_batch_modes_match_single_scene_calls(mode, flags, mapping):
    lanes = [Lane(sc, 3 + i) for i, sc in enumerate(_mix()[:4])]
    b = pv.pv_batch_create([ln.item() for ln in lanes], mode, 0.01, flags)
    pv.pv_batch_set_config(b, verify_mapping=mapping)
    _run(lanes, b, range(2, 5), mode, 0.01, flags, traversal_counters=mapping != 1)
    pv.pv_batch_destroy(b)
    for ln in lanes:
        ln.close()


@pytest.mark.parametrize("mapping", [0, 1, 2])
def test_batch_verify_few_blocks_matches_single_scene_calls(monkeypatch, mapping):
    """Two verify blocks for the whole batch: each block loops over 64-path
    tiles of every scene in turn and restages the scene's shared state at each
    change; records, lists and counters stay those of the single-scene calls."""
    monkeypatch.setenv("PV_VERIFY_MAX_BLOCKS", "2")
    lanes = [Lane(sc, 9 + i) for i, sc in enumerate(_mix())]
    b = pv.pv_batch_create([ln.item() for ln in lanes], pv.PV_MODE_ERROR, 0.01)
    pv.pv_batch_set_config(b, verify_mapping=mapping, verify_threads=64)
    _run(lanes, b, range(2, 5), pv.PV_MODE_ERROR, 0.01, 0, traversal_counters=mapping != 1)
    pv.pv_batch_destroy(b)
    for ln in lanes:
        ln.close()


def test_batch_flat_mapping_error_exact_matches_single_scene_calls():
    lanes = [Lane(sc, 5 + i) for i, sc in enumerate(_mix()[:4])]
    b = pv.pv_batch_create([ln.item() for ln in lanes], pv.PV_MODE_ERROR, 0.01, pv.PV_FLAG_ERROR_EXACT)
    pv.pv_batch_set_config(b, verify_mapping=2)
    _run(lanes, b, range(2, 5), pv.PV_MODE_ERROR, 0.01, pv.PV_FLAG_ERROR_EXACT)
    pv.pv_batch_destroy(b)
    for ln in lanes:
        ln.close()


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: ",".join(f"{k}={v}" for k, v in c.items()) or "default")
def test_fused_batch_matches_single_scene_calls(cfg):
    """Batches without lists run Alg. 1 inside the re-trace kernel; records and counters stay those of
    the separate single-scene calls."""
    lanes = [Lane(sc, 13 + 5 * i) for i, sc in enumerate(_mix())]
    b = pv.pv_batch_create([ln.item(lists=False) for ln in lanes], pv.PV_MODE_ERROR, 0.01)
    if cfg:
        pv.pv_batch_set_config(b, **cfg)
    _run(lanes, b, range(2, 7), pv.PV_MODE_ERROR, 0.01, 0, traversal_counters=cfg.get("verify_mapping", 0) != 1,
         lists=False)
    pv.pv_batch_destroy(b)
    for ln in lanes:
        ln.close()


@pytest.mark.parametrize("mode,flags", [(pv.PV_MODE_NAIVE_AABB, 0), (pv.PV_MODE_ERROR, pv.PV_FLAG_ERROR_EXACT)])
def test_fused_batch_modes_and_tuner(mode, flags):
    lanes = [Lane(sc, 7 + i) for i, sc in enumerate(_mix()[:4])]
    b = pv.pv_batch_create([ln.item(lists=False) for ln in lanes], mode, 0.01, flags)
    pv.pv_batch_autotune(b, 1)
    f = 2
    while pv.pv_batch_tuning(b):
        _run(lanes, b, [f], mode, 0.01, flags, traversal_counters=False, lists=False)
        f += 1
        assert f < 60
    times = pv.pv_batch_step_times(b)
    assert times[2] < 0.02 and times[4] > 0.0          # no separate continuation kernel: only event spacing
    cfg = pv.pv_batch_get_config(b)
    _run(lanes, b, range(f, f + 3), mode, 0.01, flags, traversal_counters=cfg["verify_mapping"] != 1, lists=False)
    pv.pv_batch_destroy(b)
    for ln in lanes:
        ln.close()


def _dm_lanes(seed0):
    """Mapped scenes (a translating area light with a 4^4 map, a point light
    with an 8 x 8 map) beside unmapped ones."""
    point = kit.floor_and_light(3200, B=2, R=20.0)
    point._light_fn = lambda f: [Light(LIGHT_POINT, (0.31 * (f - 1), 1.0, -0.17 * (f - 1)), power=(1.0,) * 3,
                                       n_paths=3200)]
    rect = kit.rect_light_over_floor(2560, shift=lambda f: (0.11 * (f - 1), 0.0, 0.07 * (f - 1)), B=2, R=3.0)
    return [Lane(rect, seed0, dm_rect=(4, 4, 4, 4)), Lane(scenes.tiny_box(n_paths=3000), seed0 + 1),
            Lane(point, seed0 + 2, dm_point=(8, 8)), Lane(kit.box_with_torus(3000, B=3), seed0 + 3)]


@pytest.mark.parametrize("mode", [pv.PV_MODE_NAIVE_AABB, pv.PV_MODE_ERROR])
def test_batch_with_distribution_maps_matches_single_scene_calls(mode):
    """Compute DM_C (fused with the origin update), prune (Eq. 1, two passes)
    and fill inside the batched frame, eagerly and replayed from the
    captured graph: records, lists, counters (pruned and filled included) and
    every DM_C count equal the single-scene calls'."""
    lanes = _dm_lanes(31)
    b = pv.pv_batch_create([ln.item() for ln in lanes], mode, 0.01)
    pv.pv_batch_autotune(b, 1)
    f = 2
    while pv.pv_batch_tuning(b):                       # eager frames, every tuner candidate
        _run(lanes, b, [f], mode, 0.01, 0, traversal_counters=False)
        f += 1
        assert f < 60
    _run(lanes, b, range(f, f + 4), mode, 0.01, 0,       # graph replays
         traversal_counters=pv.pv_batch_get_config(b)["verify_mapping"] != 1)
    tot = pv.stats_dict(lanes[0].s2)
    assert tot["n_filled"] > 0 and tot["n_pruned"] > 0
    pv.pv_batch_destroy(b)
    for ln in lanes:
        ln.close()


def test_batch_with_distribution_maps_needs_lists():
    lanes = _dm_lanes(41)
    with pytest.raises(pv.PvError):
        pv.pv_batch_create([ln.item(lists=False) for ln in lanes], pv.PV_MODE_ERROR, 0.01)
    for ln in lanes:
        ln.close()


def test_batch_lists_for_some_scenes_only_is_refused():
    lanes = [Lane(sc, 3 + i) for i, sc in enumerate(_mix()[:2])]
    with pytest.raises(pv.PvError):
        pv.pv_batch_create([lanes[0].item(lists=True), lanes[1].item(lists=False)], pv.PV_MODE_ERROR, 0.01)
    for ln in lanes:
        ln.close()


def test_batch_autotune_then_graph():
    lanes = [Lane(sc, 5 + i) for i, sc in enumerate(_mix())]
    b = pv.pv_batch_create([ln.item() for ln in lanes], pv.PV_MODE_ERROR, 0.01)
    pv.pv_batch_autotune(b, 1)
    f = 2
    while pv.pv_batch_tuning(b):
        for ln in lanes:
            ln.single_frame(f, pv.PV_MODE_ERROR, 0.01, 0)
        pv.pv_batch_frame(b, [ln.sc.xforms(f) for ln in lanes], [ln.sc.lights(f) for ln in lanes], f)
        cfg = pv.pv_batch_get_config(b)
        for ln in lanes:
            ln.compare(traversal_counters=False)
        f += 1
        assert f < 60
    cfg = pv.pv_batch_get_config(b)
    assert cfg["verify_mapping"] in (0, 1, 2) and cfg["trace_steps"] in (16, 32, 64) and cfg["stack"] in (32, 64)
    times = pv.pv_batch_step_times(b)
    assert len(times) == 5 and all(t >= 0 for t in times)
    _run(lanes, b, range(f, f + 3), pv.PV_MODE_ERROR, 0.01, 0, traversal_counters=cfg["verify_mapping"] != 1)
    pv.pv_batch_destroy(b)
    for ln in lanes:
        ln.close()


def test_batch_against_oracle():
    """Two frames of a batch of the tiny box and the moving torus against the FP64 oracle."""
    torch = _torch()
    mix = [scenes.tiny_box(n_paths=4000), kit.box_with_torus(3000, B=4), _moving_point_light(2000)]
    items, ctx = [], []
    for i, sc in enumerate(mix):
        seed = 21 + i
        o = oracle.OracleScene(sc)
        o.set_frames(1, 1)
        op = o.trace(np.arange(sc.n_paths, dtype=np.uint32), seed, 1)
        h = gu.lib_scene(sc, frame=1)
        P = pv.Paths.allocate(sc.n_paths, sc.max_bounces)
        gu.upload(P, op)
        lst = torch.zeros(sc.n_paths, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        items.append((h, P, lst, cnt, None, seed))
        ctx.append((sc, o, op, h, P, lst, cnt, seed))
    b = pv.pv_batch_create(items, pv.PV_MODE_ERROR, 0.01)
    for f in (2, 3):
        pv.pv_batch_frame(b, [c[0].xforms(f) for c in ctx], [c[0].lights(f) for c in ctx], f)
        for k, (sc, o, op, h, P, lst, cnt, seed) in enumerate(ctx):
            o.set_frames(f - 1, f)
            o.verify(op, pv.PV_MODE_ERROR, 0.01)
            o.retrace(op, seed, f)
            r = gu.compare(gu.download(P), op, sc.diag)
            print(sc.name, f, {k: r[k] for k in ("n", "ambiguous", "ambiguous_matched", "ambiguous_open")})
            gu.assert_parity(r)
            assert r["ambiguous"] <= 3, r                # measured: 0 to 1 flagged path per frame
            gu.upload(P, op)                          # continue both sides from the oracle's records
    pv.pv_batch_destroy(b)
    for c in ctx:
        assert pv.pv_read_device_status(c[3]) == 0
        pv.pv_destroy_scene(c[3])


def test_batch_argument_errors():
    torch = _torch()
    sc = scenes.tiny_box(n_paths=1000)
    h = gu.lib_scene(sc)
    P = pv.Paths.allocate(sc.n_paths, sc.max_bounces)
    lst = torch.zeros(sc.n_paths, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(pv.PvError):                   # the same scene twice
        pv.pv_batch_create([(h, P, lst, cnt, None, 1), (h, P, lst, cnt, None, 1)], pv.PV_MODE_ERROR, 0.01)
    hr = gu.lib_scene(sc, flags=pv.PV_BUILD_DYN_REBUILD)
    with pytest.raises(pv.PvError):                   # rebuild mode cannot be replayed
        pv.pv_batch_create([(hr, P, lst, cnt, None, 1)], pv.PV_MODE_ERROR, 0.01)
    bn = pv.pv_batch_create([(h, P, lst, cnt, None, 1)], pv.PV_MODE_NAIVE_AABB, 0.01)
    with pytest.raises(pv.PvError):                   # the flat mapping serves error mode only
        pv.pv_batch_set_config(bn, verify_mapping=2)
    pv.pv_batch_destroy(bn)
    b = pv.pv_batch_create([(h, P, lst, cnt, None, 1)], pv.PV_MODE_ERROR, 0.01)
    pv.pv_batch_set_config(b, verify_mapping=2)
    with pytest.raises(pv.PvError):
        pv.pv_batch_set_config(b, trace_steps=5)
    with pytest.raises(pv.PvError):
        pv.pv_batch_step_times(b)
    pv.pv_batch_destroy(b)
    for x in (h, hr):
        pv.pv_destroy_scene(x)
