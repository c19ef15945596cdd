"""GPU tests of pv_verify_retrace, the one-call frame that runs Alg. 1 inside
the persistent re-trace kernel.

The fused call must leave exactly the records and counters that
pv_verify_paths followed by pv_retrace_invalid (same seed and frame) leave:
every path goes through the same device functions, only the order in which
paths are taken differs, so the comparison is bit-exact, traversal counters
included.  Scenes cover every verify variant (moving point light with
visibility rays, moving area light, moving objects, box and exact segment
tests), error-mode thresholds from 0 to 5 %, and a light with a
distribution map (where the call runs the separate kernels).  A last test
runs the fused call against the FP64 oracle.

pv_verify_retrace_deposit also deposits the atlas inside the same kernel;
its records, counters and integer atlas must equal those of
pv_verify_retrace followed by pv_deposit, bit for bit.
"""
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
    sc = kit.box_with_torus(n_paths, B=3, seed=5)
    sc._light_fn = lambda f: [Light(LIGHT_POINT, (0.05 * (f - 1), 1.8, 0.02 * (f - 1)), power=(100.0,) * 3,
                                    n_paths=n_paths)]
    return sc


SCENES = {
    "tiny_box": lambda: scenes.tiny_box(n_paths=5000),
    "box_torus": lambda: kit.box_with_torus(4000, B=4),
    "rect_light_moving": lambda: kit.rect_light_over_floor(2000, shift=lambda f: (0.03 * (f - 1), 0.0, 0.0), B=1,
                                                           R=3.0),
    "point_light_moving": _moving_point_light,
    "city_small": lambda: scenes.city(n_paths=40000, n_boxes=1500),
}


class Pair:
    """One scene driven through the separate calls (1) and the fused call (2)."""

    def __init__(self, sc, seed, dm_rect=(0, 0, 0, 0)):
        torch = _torch()
        self.sc, self.seed = sc, seed
        self.h1 = gu.lib_scene(sc, dm_rect=dm_rect)
        self.h2 = gu.lib_scene(sc, dm_rect=dm_rect)
        n, B = sc.n_paths, sc.max_bounces
        self.P1 = pv.Paths.allocate(n, B)
        self.P2 = pv.Paths.allocate(n, B)
        pv.pv_trace_all(self.h1, self.P1, seed, 1)
        pv.pv_trace_all(self.h2, self.P2, seed, 1)
        self.lst = torch.zeros(n, dtype=torch.int32, device="cuda")
        self.cnt = torch.zeros(1, dtype=torch.int32, device="cuda")

    def frame(self, f, mode, tau, flags):
        s1, s2 = pv.new_stats(), pv.new_stats()
        for h in (self.h1, self.h2):
            gu.advance(h, self.sc, f)
        pv.pv_verify_paths(self.h1, self.P1, mode, tau, flags, self.lst, self.cnt, s1, seed=self.seed, frame=f)
        pv.pv_retrace_invalid(self.h1, self.P1, self.lst, self.cnt, self.seed, f, s1)
        pv.pv_verify_retrace(self.h2, self.P2, mode, tau, flags, self.seed, f, s2)
        return pv.stats_dict(s1), pv.stats_dict(s2)

    def compare(self, d1, d2):
        torch = _torch()
        for name in ("info", "origin", "pa", "pb"):
            a, b = getattr(self.P1, name), getattr(self.P2, name)
            same = a.view(torch.int32) == b.view(torch.int32)
            assert bool(same.all()), (name, int((~same).sum()))
        assert d1 == d2, (d1, d2)

    def close(self):
        for h in (self.h1, self.h2):
            assert pv.pv_read_device_status(h) == 0
            pv.pv_destroy_scene(h)


MODES = [(pv.PV_MODE_ERROR, 0.01, 0), (pv.PV_MODE_ERROR, 0.0, 0), (pv.PV_MODE_ERROR, 0.05, 0),
         (pv.PV_MODE_ERROR, 0.01, pv.PV_FLAG_ERROR_EXACT), (pv.PV_MODE_NAIVE_AABB, 0.01, 0),
         (pv.PV_MODE_NAIVE_EXACT, 0.01, 0)]


@pytest.mark.parametrize("mode,tau,flags", MODES, ids=lambda v: str(v))
@pytest.mark.parametrize("name", list(SCENES))
def test_fused_frame_matches_separate_calls(name, mode, tau, flags):
    p = Pair(SCENES[name](), 17)
    tails = 0
    for f in range(2, 6):
        d1, d2 = p.frame(f, mode, tau, flags)
        p.compare(d1, d2)
        tails += d2["n_tail"]
        assert d2["n_listed"] >= d2["n_tail"]
    if mode == pv.PV_MODE_ERROR and tau == 0.01 and name in ("box_torus", "city_small", "point_light_moving"):
        assert tails > 0                           # Alg. 1 did hand paths straight to the re-trace
    p.close()


def _atlas(sc, res=256):
    torch = _torch()
    return torch.zeros(res, res, 3, dtype=torch.int64, device="cuda"), sc.atlas_rect, 40


@pytest.mark.parametrize("mode,tau,flags", [MODES[0], MODES[3], MODES[4]], ids=lambda v: str(v))
@pytest.mark.parametrize("name", list(SCENES))
def test_fused_deposit_matches_separate_calls(name, mode, tau, flags):
    """pv_verify_retrace_deposit against pv_verify_retrace + pv_deposit: records, counters and atlas."""
    torch = _torch()
    sc = SCENES[name]()
    p = Pair(sc, 19)
    a1, rect, scale = _atlas(sc)
    a2 = torch.full_like(a1, 12345)                # cleared by the call
    for f in range(2, 5):
        s1, s2 = pv.new_stats(), pv.new_stats()
        for h in (p.h1, p.h2):
            gu.advance(h, sc, f)
        pv.pv_verify_retrace(p.h1, p.P1, mode, tau, flags, p.seed, f, s1)
        pv.pv_deposit(p.h1, p.P1, a1, rect, scale)
        pv.pv_verify_retrace_deposit(p.h2, p.P2, mode, tau, flags, p.seed, f, a2, rect, scale, s2)
        p.compare(pv.stats_dict(s1), pv.stats_dict(s2))
        assert torch.equal(a1, a2), int((a1 != a2).sum())
        assert int(a1.sum()) > 0
    p.close()


def test_fused_deposit_without_motion_and_with_distribution_map():
    torch = _torch()
    for sc, dm, moving in ((kit.box_with_torus(3000, B=4), (0, 0, 0, 0), False),
                           (kit.rect_light_over_floor(2560, shift=lambda f: (0.11 * (f - 1), 0.0, 0.07 * (f - 1)), B=2,
                                                      R=3.0), (4, 4, 4, 4), True)):
        p = Pair(sc, 29, dm_rect=dm)
        a1, rect, scale = _atlas(sc, 128)
        a2 = torch.zeros_like(a1)
        for f in range(2, 4):
            s1, s2 = pv.new_stats(), pv.new_stats()
            ff = f if moving else 1
            for h in (p.h1, p.h2):
                gu.advance(h, sc, ff)
            pv.pv_verify_retrace(p.h1, p.P1, pv.PV_MODE_ERROR, 0.01, 0, p.seed, f, s1)
            pv.pv_deposit(p.h1, p.P1, a1, rect, scale)
            pv.pv_verify_retrace_deposit(p.h2, p.P2, pv.PV_MODE_ERROR, 0.01, 0, p.seed, f, a2, rect, scale, s2)
            p.compare(pv.stats_dict(s1), pv.stats_dict(s2))
            assert torch.equal(a1, a2)
        p.close()


@pytest.mark.parametrize("B", [1, 15])
def test_fused_deposit_bounce_caps(B):
    """The shortest and the longest stored paths (1 and 15 bounces) through the fused deposit call."""
    torch = _torch()
    sc = kit.box_with_torus(3000, B=B)
    p = Pair(sc, 43)
    a1, rect, scale = _atlas(sc, 64)
    a2 = torch.zeros_like(a1)
    for f in range(2, 5):
        s1, s2 = pv.new_stats(), pv.new_stats()
        for h in (p.h1, p.h2):
            gu.advance(h, sc, f)
        pv.pv_verify_paths(p.h1, p.P1, pv.PV_MODE_ERROR, 0.01, 0, p.lst, p.cnt, s1, seed=p.seed, frame=f)
        pv.pv_retrace_invalid(p.h1, p.P1, p.lst, p.cnt, p.seed, f, s1)
        pv.pv_deposit(p.h1, p.P1, a1, rect, scale)
        pv.pv_verify_retrace_deposit(p.h2, p.P2, pv.PV_MODE_ERROR, 0.01, 0, p.seed, f, a2, rect, scale, s2)
        p.compare(pv.stats_dict(s1), pv.stats_dict(s2))
        assert torch.equal(a1, a2)
    L = (p.P2.info.cpu().numpy().view(np.uint32) >> 22) & 15
    assert L.max() <= B and (B == 1 or L.max() > 4)
    p.close()


def test_fused_frame_with_distribution_map_matches_separate_calls():
    sc = kit.rect_light_over_floor(2560, shift=lambda f: (0.11 * (f - 1), 0.0, 0.07 * (f - 1)), B=2, R=3.0)
    p = Pair(sc, 23, dm_rect=(4, 4, 4, 4))
    for f in range(2, 5):
        d1, d2 = p.frame(f, pv.PV_MODE_ERROR, 0.01, 0)
        p.compare(d1, d2)
        assert np.array_equal(pv.pv_read_distribution_map(p.h1, 0), pv.pv_read_distribution_map(p.h2, 0))
    p.close()


def test_fused_frame_without_motion_keeps_every_path():
    sc = kit.box_with_torus(3000, B=4)
    p = Pair(sc, 5)
    before = [getattr(p.P2, k).clone() for k in ("info", "origin", "pa", "pb")]
    st = pv.new_stats()
    pv.pv_update_dynamic(p.h2, sc.xforms(1), sc.lights(1))       # the same pose again: nothing moved
    pv.pv_verify_retrace(p.h2, p.P2, pv.PV_MODE_ERROR, 0.01, 0, 5, 2, st)
    d = pv.stats_dict(st)
    assert d["n_listed"] == 0 and d["trace_rays"] == 0 and d["cont_rays"] == 0, d
    torch = _torch()
    for a, k in zip(before, ("info", "origin", "pa", "pb")):
        assert torch.equal(a, getattr(p.P2, k)), k
    p.close()


def test_fused_frame_against_oracle():
    """Three frames of the moving torus and the moving point light against the FP64 oracle."""
    for sc, seed in ((kit.box_with_torus(3000, B=4), 31), (_moving_point_light(2000), 37)):
        o = oracle.OracleScene(sc)
        o.set_frames(1, 1)
        op = o.trace(np.arange(sc.n_paths, dtype=np.uint32), seed, 1)
        h = gu.lib_scene(sc, frame=1)
        P = pv.Paths.allocate(sc.n_paths, sc.max_bounces)
        gu.upload(P, op)
        for f in (2, 3, 4):
            gu.advance(h, sc, f)
            pv.pv_verify_retrace(h, P, pv.PV_MODE_ERROR, 0.01, 0, seed, f)
            o.set_frames(f - 1, f)
            o.verify(op, pv.PV_MODE_ERROR, 0.01)
            o.retrace(op, seed, f)
            r = gu.compare(gu.download(P), op, sc.diag)
            print(sc.name, f, {k: r[k] for k in ("n", "ambiguous", "ambiguous_matched", "ambiguous_open")})
            gu.assert_parity(r)
            assert r["ambiguous"] <= 3, r                # measured: 0 to 1 flagged path per frame
            gu.upload(P, op)                          # continue both sides from the oracle's records
        assert pv.pv_read_device_status(h) == 0
        pv.pv_destroy_scene(h)


DELTA_MODES = [MODES[0], MODES[2], MODES[3], MODES[4], MODES[5]]


@pytest.mark.parametrize("mode,tau,flags", DELTA_MODES, ids=lambda v: str(v))
@pytest.mark.parametrize("name", list(SCENES))
def test_delta_deposit_matches_full_deposit(name, mode, tau, flags):
    """pv_verify_retrace_deposit_delta on an atlas carried from frame to frame against
    pv_verify_retrace_deposit on a cleared one: records, counters and atlas equal bit for bit every frame,
    re-emitted paths (moving lights), Alg. 1 paths, tails and naive re-traces included."""
    torch = _torch()
    sc = SCENES[name]()
    p = Pair(sc, 47)
    a1, rect, scale = _atlas(sc)
    a2 = torch.zeros_like(a1)
    pv.pv_deposit(p.h2, p.P2, a2, rect, scale)        # the entry records' deposit
    changed = 0
    for f in range(2, 6):
        s1, s2 = pv.new_stats(), pv.new_stats()
        for h in (p.h1, p.h2):
            gu.advance(h, sc, f)
        pv.pv_verify_retrace_deposit(p.h1, p.P1, mode, tau, flags, p.seed, f, a1, rect, scale, s1)
        pv.pv_verify_retrace_deposit_delta(p.h2, p.P2, mode, tau, flags, p.seed, f, a2, rect, scale, s2)
        d1, d2 = pv.stats_dict(s1), pv.stats_dict(s2)
        p.compare(d1, d2)
        assert torch.equal(a1, a2), int((a1 != a2).sum())
        changed += d2["n_listed"] + d2["n_cont"]
    assert changed > 0
    p.close()


def test_delta_deposit_without_motion_and_with_distribution_map():
    """Nothing moved: the carried atlas stays as it was.  Distribution maps: the delta call clears and
    deposits every path, so a wrong entry atlas does not survive."""
    torch = _torch()
    sc = kit.box_with_torus(3000, B=4)
    p = Pair(sc, 53)
    a, rect, scale = _atlas(sc, 128)
    pv.pv_deposit(p.h2, p.P2, a, rect, scale)
    before = a.clone()
    pv.pv_update_dynamic(p.h2, sc.xforms(1), sc.lights(1))
    st = pv.new_stats()
    pv.pv_verify_retrace_deposit_delta(p.h2, p.P2, pv.PV_MODE_ERROR, 0.01, 0, p.seed, 2, a, rect, scale, st)
    assert pv.stats_dict(st)["n_listed"] == 0
    assert torch.equal(a, before)
    p.close()

    sc = kit.rect_light_over_floor(2560, shift=lambda f: (0.11 * (f - 1), 0.0, 0.07 * (f - 1)), B=2, R=3.0)
    p = Pair(sc, 59, dm_rect=(4, 4, 4, 4))
    a1, rect, scale = _atlas(sc, 128)
    a2 = torch.full_like(a1, 777)                         # not the entry deposit: the call must not rely on it
    for f in range(2, 4):
        s1, s2 = pv.new_stats(), pv.new_stats()
        for h in (p.h1, p.h2):
            gu.advance(h, sc, f)
        pv.pv_verify_retrace_deposit(p.h1, p.P1, pv.PV_MODE_ERROR, 0.01, 0, p.seed, f, a1, rect, scale, s1)
        pv.pv_verify_retrace_deposit_delta(p.h2, p.P2, pv.PV_MODE_ERROR, 0.01, 0, p.seed, f, a2, rect, scale, s2)
        p.compare(pv.stats_dict(s1), pv.stats_dict(s2))
        assert torch.equal(a1, a2)
    p.close()


@pytest.mark.parametrize("B", [1, 15])
def test_delta_deposit_bounce_caps(B):
    torch = _torch()
    sc = kit.box_with_torus(3000, B=B)
    p = Pair(sc, 61)
    a1, rect, scale = _atlas(sc, 64)
    a2 = torch.zeros_like(a1)
    pv.pv_deposit(p.h2, p.P2, a2, rect, scale)
    for f in range(2, 5):
        s1, s2 = pv.new_stats(), pv.new_stats()
        for h in (p.h1, p.h2):
            gu.advance(h, sc, f)
        pv.pv_verify_retrace_deposit(p.h1, p.P1, pv.PV_MODE_ERROR, 0.01, 0, p.seed, f, a1, rect, scale, s1)
        pv.pv_verify_retrace_deposit_delta(p.h2, p.P2, pv.PV_MODE_ERROR, 0.01, 0, p.seed, f, a2, rect, scale, s2)
        p.compare(pv.stats_dict(s1), pv.stats_dict(s2))
        assert torch.equal(a1, a2)
    p.close()


@pytest.mark.parametrize("name", ["tiny_box", "box_torus", "point_light_moving", "city_small"])
def test_trace_all_deposit_matches_separate_calls(name):
    """pv_trace_all_deposit against pv_trace_all + pv_deposit: records, counters and atlas bit for bit, over
    three frames of moving geometry and lights, into an atlas that holds stale values before each call."""
    torch = _torch()
    sc = SCENES[name]()
    p = Pair(sc, 23)
    a1, rect, scale = _atlas(sc)
    a2 = torch.full_like(a1, 777)                  # cleared by the call
    for f in range(2, 5):
        s1, s2 = pv.new_stats(), pv.new_stats()
        for h in (p.h1, p.h2):
            gu.advance(h, sc, f)
        pv.pv_trace_all(p.h1, p.P1, p.seed, f, s1)
        pv.pv_deposit(p.h1, p.P1, a1, rect, scale)
        pv.pv_trace_all_deposit(p.h2, p.P2, p.seed, f, a2, rect, scale, s2)
        p.compare(pv.stats_dict(s1), pv.stats_dict(s2))
        assert torch.equal(a1, a2), int((a1 != a2).sum())
        assert int(a1.sum()) > 0
        a2.fill_(777)
    p.close()


def test_trace_all_deposit_with_distribution_map():
    """A stratified full trace with a map: the same records, counters and DM_C as pv_trace_all."""
    torch = _torch()
    sc = kit.rect_light_over_floor(2560, shift=lambda f: (0.11 * (f - 1), 0.0, 0.07 * (f - 1)), B=2, R=3.0)
    p = Pair(sc, 31, dm_rect=(4, 4, 4, 4))
    a1, rect, scale = _atlas(sc, 128)
    a2 = torch.zeros_like(a1)
    gu.advance(p.h1, sc, 2)
    gu.advance(p.h2, sc, 2)
    s1, s2 = pv.new_stats(), pv.new_stats()
    pv.pv_trace_all(p.h1, p.P1, p.seed, 2, s1)
    pv.pv_deposit(p.h1, p.P1, a1, rect, scale)
    pv.pv_trace_all_deposit(p.h2, p.P2, p.seed, 2, a2, rect, scale, s2)
    p.compare(pv.stats_dict(s1), pv.stats_dict(s2))
    assert torch.equal(a1, a2)
    assert np.array_equal(pv.pv_read_distribution_map(p.h1, 0), pv.pv_read_distribution_map(p.h2, 0))
    p.close()
