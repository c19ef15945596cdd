"""GPU parity of the distribution maps (Sec. 3.1: compute DM_C, prune with
Eq. 1 in two passes, fill DM_C) against the FP64 oracle, through the C ABI.

Every map decision is an integer one made from bit-identical inputs (the
float32 parametrisation of stored records and poses, counts, the 24-bit
Philox draw, prefix sums over ascending free lists), so info words (with
their cells), the DM_C counts, the pruned and filled counts and the re-trace
lists are compared bit-exact; re-traced records within the usual position
(1e-5 diag) and energy (1e-5) tolerances.  A decision the oracle flags as
ambiguous could shift counts for a whole light, so these scenes are chosen
without ambiguity and the tests assert that.
"""
import numpy as np
import pytest

import oracle
import scenes
import paper_2111_06906_gb300 as pv
from scenes import LIGHT_POINT, LIGHT_RECT, Light
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


def _point_over_floor(n, B=2):
    sc = kit.floor_and_light(n, B=B, R=20.0)
    sc._light_fn = lambda f: [Light(LIGHT_POINT, (0.31 * (f - 1), 1.0, -0.17 * (f - 1)), power=(1.0,) * 3,
                                    n_paths=n)]
    return sc


def _tilting_rect(n, B=2):
    sc = kit.rect_light_over_floor(n, shift=lambda f: (0.05 * (f - 1), 0.0, 0.0), B=B, R=3.0)
    nrm = lambda f: (0.08 * (f - 1), -1.0, 0.0)
    sc._light_fn = lambda f: [Light(LIGHT_RECT, (0.05 * (f - 1), 3.0, 0.0), nrm(f), (1.0, 0.0, 0.0), (1.0, 1.0),
                                    (100.0, 100.0, 100.0), n)]
    return sc


def _box_point(n):
    sc = kit.box_with_torus(n, B=3, seed=5)
    sc._light_fn = lambda f: [Light(LIGHT_POINT, (0.07 * (f - 1), 1.8, 0.03 * (f - 1)), power=(100.0,) * 3,
                                    n_paths=n)]
    return sc


CASES = {
    "rect_translating": (lambda: kit.rect_light_over_floor(2560, shift=lambda f: (0.11 * (f - 1), 0.0, 0.07 * (f - 1)),
                                                             B=2, R=3.0), (4, 4, 4, 4), (0, 0), 2),
    "rect_tilting": (lambda: _tilting_rect(2560), (4, 4, 4, 4), (0, 0), 2),
    "point_over_floor": (lambda: _point_over_floor(3200), (0, 0, 0, 0), (8, 8), 2),
    "box_point_torus": (lambda: _box_point(4096), (0, 0, 0, 0), (8, 8), 2),
}


def _compare_maps(h, o, sc):
    for l in range(len(sc.lights(1))):
        g = pv.pv_read_distribution_map(h, l)
        assert np.array_equal(g, o.dm_counts(l)), l


@pytest.mark.parametrize("name", list(CASES))
def test_dm_frames_match_oracle(name):
    torch = _torch()
    make, rect, point, mode = CASES[name]
    sc = make()
    seed = 41
    n = sc.n_paths
    ids = np.arange(n, dtype=np.uint32)
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    o.set_dm(rect, point)
    op = o.trace(ids, seed, 1)
    o.dm_reset()
    h = gu.lib_scene(sc, dm_rect=rect, dm_point=point)
    P = pv.Paths.allocate(n, sc.max_bounces)
    pv.pv_trace_all(h, P, seed, 1)
    r = gu.compare(gu.download(P), op, sc.diag)
    gu.assert_parity(r)
    assert r["ambiguous"] == 0, r
    _compare_maps(h, o, sc)
    gu.upload(P, op)
    lst = torch.zeros(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    pruned = filled = 0
    for f in (2, 3, 4):
        gu.advance(h, sc, f)
        st = pv.new_stats()
        pv.pv_verify_paths(h, P, mode, 0.01, 0, lst, cnt, st, seed=seed, frame=f)
        o.set_frames(f - 1, f)
        _, ost = o.verify(op, mode, 0.01, seed=seed, frame=f)
        assert int((op.amb != 0).sum()) == 0
        gv = gu.download(P)
        assert np.array_equal(gv.info, op.info), int((gv.info != op.info).sum())
        _compare_maps(h, o, sc)
        s = pv.stats_dict(st)
        assert (s["n_pruned"], s["n_filled"]) == (ost["n_pruned"], ost["n_filled"])
        pruned += s["n_pruned"]
        filled += s["n_filled"]
        k = int(cnt.item())
        assert np.array_equal(lst[:k].cpu().numpy().view(np.uint32), oracle.compact(op.info))
        pv.pv_retrace_invalid(h, P, lst, cnt, seed, f)
        o.retrace(op, seed, f)
        r = gu.compare(gu.download(P), op, sc.diag)
        gu.assert_parity(r)
        assert r["ambiguous"] == 0, r
        gu.upload(P, op)                               # continue both sides from identical records
    assert filled > 0
    assert pv.pv_read_device_status(h) == 0
    pv.pv_destroy_scene(h)


def test_dm_translation_by_whole_cells_refills_exactly():
    torch = _torch()
    sc = kit.rect_light_over_floor(800, shift=lambda f: (0.25 * (f - 1), 0.0, 0.0), B=1, R=1000.0)
    h = gu.lib_scene(sc, dm_rect=(8, 1, 1, 1))
    P = pv.Paths.allocate(sc.n_paths, 1)
    pv.pv_trace_all(h, P, 3, 1)
    assert np.array_equal(pv.pv_read_distribution_map(h, 0), np.full(8, 100, np.uint32))
    gu.advance(h, sc, 2)
    lst = torch.zeros(sc.n_paths, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = pv.new_stats()
    pv.pv_verify_paths(h, P, pv.PV_MODE_ERROR, 0.01, 0, lst, cnt, st, seed=3, frame=2)
    s = pv.stats_dict(st)
    assert s["n_pruned"] == 0 and s["n_filled"] == 200 and int(cnt.item()) == 200
    assert np.array_equal(pv.pv_read_distribution_map(h, 0), np.full(8, 100, np.uint32))
    info = gu.download(P).info
    assert set(np.unique(info[(info >> 30) & 1 == 1] & 0xFFFFF)) == {6, 7}
    pv.pv_destroy_scene(h)


def test_dm_full_size_city_invariants():
    """The city's moving area light with an 8 x 8 x 64 x 64 map (1M paths): every
    path is in exactly one cell after each frame, the counts add up, and no
    cell is short while free paths were spread beyond the deficits."""
    torch = _torch()
    sc = scenes.city()
    h = gu.lib_scene(sc, dm_rect=(8, 8, 64, 64))
    n = sc.n_paths
    assert pv.pv_distribution_map_cells(h, 0) == 8 * 8 * 64 * 64
    P = pv.Paths.allocate(n, sc.max_bounces)
    pv.pv_trace_all(h, P, 5, 1)
    t = pv.pv_read_distribution_map(h, 0)
    assert t.sum() == n and t.max() - t.min() <= 1
    lst = torch.zeros(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    for f in (2, 3, 4, 5):
        gu.advance(h, sc, f)
        st = pv.new_stats()
        pv.pv_verify_paths(h, P, pv.PV_MODE_ERROR, 0.01, 0, lst, cnt, st, seed=5, frame=f)
        dm = pv.pv_read_distribution_map(h, 0)
        info = P.info.cpu().numpy().view(np.uint32)
        assert dm.sum() == n
        assert np.array_equal(np.bincount(info & 0xFFFFF, minlength=dm.shape[0]), dm)
        s = pv.stats_dict(st)
        assert s["n_filled"] > 0
        pv.pv_retrace_invalid(h, P, lst, cnt, 5, f)
    assert pv.pv_read_device_status(h) == 0
    pv.pv_destroy_scene(h)
