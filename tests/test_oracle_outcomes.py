"""The oracle's list of admissible outcomes for paths with an ambiguous
decision (CPU).  A decision is ambiguous when a perturbation of 1e-6 x the
scene diagonal could flip it (an edge, a plane, a box face, an Eq. 2 or
AreClose threshold); the oracle then runs the path once per decision script,
each ambiguous decision taking each of its possible outcomes.  Pinned here:
a path with no ambiguous decision admits exactly the oracle's record; a
flagged path admits the oracle's record first and only records that are
valid traces; and the comparison used by the GPU tests accepts an admitted
alternative and rejects a record with a planted mistake."""
import numpy as np
import pytest

import oracle
import scenes
from tests import gpu_util as gu
from tests import scene_kit as kit


def _same(a, b):
    return a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def _records(p):
    return [p.record(i) for i in range(len(p.ids))]


@pytest.fixture(scope="module")
def city_trace():
    sc = scenes.city()
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    ids = np.sort(np.random.default_rng(3).choice(sc.n_paths, 3000, replace=False)).astype(np.uint32)
    return sc, o, o.trace(ids, sc.seed, 1)


def test_unflagged_paths_admit_only_the_oracle_record(city_trace):
    sc, o, p = city_trace
    B = sc.max_bounces
    blank = (0, np.zeros(3, np.float32), np.zeros((B, 8), np.float32))
    for i in np.nonzero(p.amb == 0)[0][:40]:
        recs, complete, _ = o.outcomes(p.pending, int(p.ids[i]), blank)
        assert complete and len(recs) == 1
        assert _same(recs[0], p.record(i))


def test_flagged_paths_admit_the_oracle_record_first_and_valid_alternatives(city_trace):
    sc, o, p = city_trace
    B = sc.max_bounces
    flagged = np.nonzero(p.amb != 0)[0]
    assert 0 < len(flagged) < 0.02 * len(p.ids)
    blank = (0, np.zeros(3, np.float32), np.zeros((B, 8), np.float32))
    world = sc.world_verts(1)
    several = 0
    for i in flagged:
        recs, complete, _ = o.outcomes(p.pending, int(p.ids[i]), blank)
        assert complete
        assert _same(recs[0], p.record(i))
        several += len(recs) > 1
        for info, org, ph in recs:
            assert np.array_equal(org, p.origin[i])            # the emission has no ambiguous decision
            L = (info >> 22) & 15
            for k in range(L):                                   # every photon lies on its primitive's plane
                prim = int(ph[k, 3:4].view(np.int32)[0])
                v = world[prim]
                n = np.cross(v[1] - v[0], v[2] - v[0])
                n /= np.linalg.norm(n)
                assert abs(np.dot(ph[k, :3].astype(np.float64) - v[0], n)) < 1e-5 * sc.diag
    assert several > 0


def test_compare_accepts_an_admitted_alternative_and_rejects_a_planted_mistake(city_trace):
    sc, o, p = city_trace
    B = sc.max_bounces
    blank = (0, np.zeros(3, np.float32), np.zeros((B, 8), np.float32))
    alt = None
    for i in np.nonzero(p.amb != 0)[0]:
        recs, _, _ = o.outcomes(p.pending, int(p.ids[i]), blank)
        for r in recs[1:]:
            if not _same(r, p.record(i)):
                alt = (i, r)
                break
        if alt:
            break
    assert alt is not None
    i, r = alt
    fake = p.copy()
    fake.info[i], fake.origin[i], fake.photons[i] = r
    res = gu.compare(fake, p.copy(), sc.diag)
    gu.assert_parity(res)
    assert res["ambiguous_matched"] == res["ambiguous"] > 0
    # the same path with a wrong primitive on its first photon matches no admitted record
    bad = fake.copy()
    wrong = np.array([int(r[2][0, 3:4].view(np.int32)[0]) + 1], np.int32).view(np.float32)[0]
    bad.photons[i, 0, 3] = wrong
    res = gu.compare(bad, p.copy(), sc.diag)
    assert res["bad_ambiguous"] == 1
    # and an unflagged path with a moved photon is a plain mismatch
    j = int(np.nonzero(p.amb == 0)[0][0])
    bad2 = p.copy()
    bad2.photons[j, 0, 0] += np.float32(1e-3 * sc.diag)
    res = gu.compare(bad2, p.copy(), sc.diag)
    assert res["bad_pos"] == 1 and res["bad_ambiguous"] == 0


def test_verify_outcomes_follow_the_accepted_branch():
    """Through a verify and a re-trace step, the alternatives are listed from
    the record accepted at the previous check, and a path that met no
    ambiguous decision stays on the oracle's own record."""
    sc = kit.box_with_torus(6000, B=4)
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    p = o.trace(np.arange(sc.n_paths, dtype=np.uint32), 1, 1)
    p.rebase()                                  # as after an upload: both sides start here
    o.set_frames(1, 2)
    q = p.copy()
    o.verify(q, oracle.MODE_ERROR, 0.01)
    flagged = np.nonzero(q.amb != 0)[0]
    # the trace's flags carry over: paths flagged only there admit just the oracle's verified record
    for i in flagged[:30]:
        recs, complete, _ = o.outcomes(q.pending, int(q.ids[i]), p.record(i))
        assert complete and _same(recs[0], q.record(i))
    r = gu.compare(q.copy(), q, sc.diag)        # the oracle's own records pass, and become the branches
    gu.assert_parity(r)
    assert r["ambiguous_matched"] == r["ambiguous"] == len(flagged)
    o.retrace(q, 1, 2)
    r2 = gu.compare(q.copy(), q, sc.diag)
    gu.assert_parity(r2)
    assert o.frames == (1, 2)                   # the enumeration left the scene's poses as they were


def test_segments_in_a_surface_plane_are_open():
    """When Alg. 1 moves a vertex onto a wall, the next segment can end on
    the same wall plane (two coplanar triangles).  Its query along it
    runs inside the plane, where the hit distance is undetermined over the
    triangle: the oracle reports the search as open (any point of that
    stretch is an admissible hit) instead of listing outcomes."""
    sc = kit.box_with_torus(8000, B=4)
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    p = o.trace(np.arange(sc.n_paths, dtype=np.uint32), 1, 1)
    p.rebase()
    o.set_frames(1, 2)
    q = p.copy()
    o.verify(q, oracle.MODE_ERROR, float("inf"))
    walls = [(0, -1.0), (0, 1.0), (1, 0.0), (1, 2.0), (2, -1.0)]     # the box's planes (axis, coordinate)
    in_plane, opened = set(), set()
    for i in np.nonzero(q.amb != 0)[0]:
        L = int(q.nseg[i])
        x = q.photons[i, :L, :3]                 # after Alg. 1 moved a vertex onto a wall
        if any(x[k, a] == c and x[k + 1, a] == c for k in range(L - 1) for a, c in walls):
            in_plane.add(int(i))
        _, _, op = o.outcomes(q.pending, int(q.ids[i]), p.record(i))
        if op:
            opened.add(int(i))
    assert len(in_plane) >= 2
    assert in_plane <= opened
