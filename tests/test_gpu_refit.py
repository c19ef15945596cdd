"""The refit without dependent levels (each dynamic wide node's box from the
run of triangles under it) against the level-by-level climb
(PV_BUILD_REFIT_CLIMB): both must give the same boxes, so two scenes that
differ only in that flag must give the same records, lists and traversal
counters, frame after frame (Sec. 3: the dynamic objects' BVHs are refitted
to the new poses)."""
from __future__ import annotations

import math

import numpy as np
import pytest

import scenes
import paper_2111_06906_gb300 as pv
from scenes import LIGHT_POINT, Light
from tests import gpu_util as gu
from tests import scene_kit as kit

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2111_06906_gb300 import build
    build.build()
    pv.load()


def _mixed_objects(n_paths=20000):
    """The tiny box's shell with six dynamic objects of 1, 3, 12, 576, 4096 and
    2 triangles: roots that are leaves, roots with only leaf children, and runs
    that span many warps.  Objects move on different frames (some frames move
    only some of them), the large torus also yaws."""
    s0 = scenes.tiny_box(n_paths=n_paths)
    shell = s0.verts[s0.tri_object == 0].astype(np.float64)
    one = np.array([[[-0.1, 0.0, 0.0], [0.1, 0.0, 0.0], [0.0, 0.15, 0.0]]])
    three = kit.quad((-0.1, 0.0, -0.1), (0.2, 0.0, 0.0), (0.0, 0.0, 0.2))[:1]
    three = np.concatenate([three, one + 0.05, one - 0.05])
    cube = scenes._boxes(np.array([[-0.1, -0.1, -0.1]]), np.array([[0.1, 0.1, 0.1]]))[0]
    small = scenes._torus(24, 12, 0.25, 0.06, vertical=True)
    big = scenes._torus(64, 32, 0.45, 0.1, vertical=False)
    two = kit.quad((-0.05, 0.0, -0.05), (0.1, 0.0, 0.0), (0.0, 0.1, 0.0))
    parts = [(shell, (0.7, 0.6, 0.5), False), (one, (0.5, 0.5, 0.5), True), (three, (0.6, 0.4, 0.4), True),
             (cube, (0.7, 0.7, 0.7), True), (small, (0.4, 0.8, 0.6), True), (big, (0.8, 0.7, 0.3), True),
             (two, (0.3, 0.3, 0.9), True)]
    n_obj = len(parts)
    home = {1: (-0.6, 1.2, 0.5), 2: (0.6, 0.3, -0.5), 3: (0.0, 0.4, 0.6), 4: (-0.4, 0.9, -0.2),
            5: (0.1, 1.0, 0.0), 6: (0.7, 1.5, 0.7)}

    def xf(f):
        x = scenes._identity_xforms(n_obj)
        for o, (hx, hy, hz) in home.items():
            t = f if (o + f) % 3 else f - 1           # each object sits still on some frames
            x[o, 3], x[o, 7], x[o, 11] = hx + 0.03 * t, hy + 0.01 * math.sin(t), hz - 0.02 * t
        R = scenes._yaw(7.0 * f)
        x[5, [0, 1, 2, 4, 5, 6, 8, 9, 10]] = R.reshape(-1)
        return x

    lights = lambda f: [Light(LIGHT_POINT, (0.0, 1.8, 0.0), power=(100.0, 100.0, 100.0), n_paths=n_paths)]
    return kit.build(parts, lights, xf, B=4, diag=math.sqrt(12.0), name="mixed_objects", seed=13)


def _paths_equal(P1, P2):
    torch = _torch()
    for a, b in ((P1.info, P2.info), (P1.origin, P2.origin), (P1.pa, P2.pa), (P1.pb, P2.pb)):
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))


def _chain(sc, frames, mode=2, tau=0.01):
    torch = _torch()
    n = sc.n_paths
    hs = [gu.lib_scene(sc), gu.lib_scene(sc, flags=pv.PV_BUILD_REFIT_CLIMB)]
    Ps = [pv.Paths.allocate(n, sc.max_bounces) for _ in hs]
    for h, P in zip(hs, Ps):
        pv.pv_trace_all(h, P, sc.seed, 1)
    _paths_equal(*Ps)
    for f in frames:
        got = []
        for h, P in zip(hs, Ps):
            lst = torch.zeros(n, dtype=torch.int32, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
            st = pv.new_stats()
            gu.advance(h, sc, f)
            pv.pv_verify_paths(h, P, mode, tau, 0, lst, cnt, st, seed=sc.seed, frame=f)
            pv.pv_retrace_invalid(h, P, lst, cnt, sc.seed, f, st)
            c = int(cnt.item())
            got.append((lst[:c].clone(), pv.stats_dict(st)))
        _paths_equal(*Ps)
        assert torch.equal(got[0][0], got[1][0])
        assert got[0][1] == got[1][1], (f, got[0][1], got[1][1])
    for h in hs:
        assert pv.pv_read_device_status(h) == 0
        pv.pv_destroy_scene(h)
    return got[0][1]


def test_refit_runs_match_climb_mixed_objects():
    st = _chain(_mixed_objects(), range(2, 9))
    assert st["node_visits"] > 0


def test_refit_runs_match_climb_box_torus():
    _chain(kit.box_with_torus(8000, B=4), range(2, 7), mode=0)


def test_refit_runs_match_climb_city_fused():
    """Four 2048-triangle tori through the fused call, atlas included."""
    torch = _torch()
    sc = scenes.city(n_paths=100_000)
    n = sc.n_paths
    hs = [gu.lib_scene(sc), gu.lib_scene(sc, flags=pv.PV_BUILD_REFIT_CLIMB)]
    Ps = [pv.Paths.allocate(n, sc.max_bounces) for _ in hs]
    atl = [torch.zeros(256, 256, 3, dtype=torch.int64, device="cuda") for _ in hs]
    for h, P in zip(hs, Ps):
        pv.pv_trace_all(h, P, sc.seed, 1)
    for f in range(2, 6):
        sts = []
        for h, P, a in zip(hs, Ps, atl):
            st = pv.new_stats()
            gu.advance(h, sc, f)
            pv.pv_verify_retrace_deposit(h, P, 2, sc.tau, 0, sc.seed, f, a, sc.atlas_rect, 30, st)
            sts.append(pv.stats_dict(st))
        _paths_equal(*Ps)
        assert torch.equal(atl[0], atl[1])
        assert sts[0] == sts[1], (f, sts[0], sts[1])
    for h in hs:
        assert pv.pv_read_device_status(h) == 0
        pv.pv_destroy_scene(h)
