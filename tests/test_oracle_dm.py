"""Pins of the oracle's distribution maps (Sec. 3.1: compute DM_C, prune with
Eq. 1 in two passes, fill DM_C), CPU only.

The map's cells are boxes of the emission's sample space, so they are pinned
against the emission itself (equal probability, round trip), against exact
counting cases (stratified full trace, a light translated by whole cells),
against the expectation Eq. 1 fixes for the number of pruned paths, and its
angle routine against numpy's arctan2."""
import math

import numpy as np
import pytest

import oracle
import scenes
from scenes import LIGHT_POINT, Light
from tests import scene_kit as kit

MODE_ERROR = 2


def _traced(sc, rect=(0, 0, 0, 0), point=(0, 0), seed=3, frame=1, dm_after=False):
    o = oracle.OracleScene(sc)
    o.set_frames(frame, frame)
    if not dm_after:
        o.set_dm(rect, point)
    p = o.trace(np.arange(sc.n_paths, dtype=np.uint32), seed, frame)
    if dm_after:
        o.set_dm(rect, point)
    else:
        o.dm_reset()
    return o, p


def _cells(p):
    return p.info & 0xFFFFF


def test_turn_matches_arctan2():
    rng = np.random.default_rng(1)
    xy = rng.normal(size=(20000, 2)).astype(np.float32)
    got = np.array([oracle.dm_turn(x, y) for x, y in xy], np.float64)
    ref = np.mod(np.arctan2(xy[:, 1].astype(np.float64), xy[:, 0].astype(np.float64)), 2 * np.pi) / (2 * np.pi)
    d = np.abs(got - ref)
    d = np.minimum(d, 1.0 - d)                      # circular distance (0 and 1 are the same turn)
    assert d.max() < 3e-7, d.max()
    assert oracle.dm_turn(1.0, 0.0) == 0.0
    assert oracle.dm_turn(0.0, 1.0) == 0.25
    assert oracle.dm_turn(-1.0, 0.0) == 0.5
    assert oracle.dm_turn(0.0, -1.0) == 0.75
    assert oracle.dm_turn(0.0, 0.0) == 0.0
    assert abs(oracle.dm_turn(1.0, 1.0) - 0.125) < 1e-7
    assert all(0.0 <= oracle.dm_turn(x, -1e-30) < 1.0 for x in (1.0, -1.0))


@pytest.mark.parametrize("kind", ["rect", "point"])
def test_full_trace_is_stratified(kind):
    if kind == "rect":
        sc, rect, point, n_cells = kit.rect_light_over_floor(2560, B=1, R=3.0), (4, 4, 4, 4), (0, 0), 256
    else:
        sc, rect, point, n_cells = kit.floor_and_light(640, B=1), (0, 0, 0, 0), (8, 8), 64
    o, p = _traced(sc, rect, point)
    assert o.dm_cells(0) == n_cells
    t = o.dm_targets(0)
    assert t.sum() == sc.n_paths and (t == sc.n_paths // n_cells).all()
    assert np.array_equal(np.bincount(_cells(p), minlength=n_cells), t)
    assert np.array_equal(o.dm_counts(0), t)


@pytest.mark.parametrize("kind", ["rect", "point"])
def test_restricted_emission_maps_back_to_its_cell(kind):
    """Every path emitted inside its cell is mapped back to that cell by the
    parametrisation (up to paths within rounding of a cell boundary)."""
    if kind == "rect":
        sc, rect, point = kit.rect_light_over_floor(4096, B=1, R=6.0), (4, 4, 4, 4), (0, 0)
    else:
        sc, rect, point = kit.floor_and_light(4096, B=1), (0, 0, 0, 0), (16, 16)
    o, p = _traced(sc, rect, point)
    hit = np.nonzero(p.nseg > 0)[0]
    assert hit.size > 1000
    back = np.array([o.dm_cell_of(0, p.photons[i, 0, :3], p.origin[i]) for i in hit])
    assert (back == _cells(p)[hit]).sum() >= hit.size - 2


@pytest.mark.parametrize("kind", ["rect", "point"])
def test_cells_are_equiprobable_under_emission(kind):
    """Unrestricted emissions spread evenly over the cells (chi-square, 6 sigma):
    the parametrisation inverts the emission's sampling (sin^2 theta and
    phi / 2 pi for the cosine-weighted rectangle, (1 - z) / 2 for the sphere)."""
    if kind == "rect":
        sc, rect, point, n_cells = kit.rect_light_over_floor(51200, B=1, R=1000.0), (4, 4, 4, 4), (0, 0), 256
    else:
        sc, rect, point, n_cells = kit.two_planes(51200, B=1, R=1000.0), (0, 0, 0, 0), (16, 16), 256
    o, p = _traced(sc, rect, point, dm_after=True)   # traced without a map: unrestricted
    hit = np.nonzero(p.nseg > 0)[0]
    assert hit.size > 0.9 * sc.n_paths
    cells = np.array([o.dm_cell_of(0, p.photons[i, 0, :3], p.origin[i]) for i in hit])
    assert (cells >= 0).all()
    h = np.bincount(cells, minlength=n_cells).astype(np.float64)
    e = hit.size / n_cells
    chi2 = ((h - e) ** 2 / e).sum()
    dof = n_cells - 1
    assert abs(chi2 - dof) < 6 * math.sqrt(2 * dof), chi2


def test_translation_by_whole_cells_refills_exactly():
    """A rectangle light moved along its tangent by two of its eight x-cells:
    the paths of the first two cells leave the light, the last two cells empty,
    and the fill gives exactly those paths to exactly those cells."""
    shift = lambda f: (0.25 * (f - 1), 0.0, 0.0)
    sc = kit.rect_light_over_floor(800, shift=shift, B=1, R=1000.0)    # every path hits the floor
    o, p = _traced(sc, (8, 1, 1, 1), (0, 0))
    assert (p.nseg > 0).all()
    x0 = (p.info & 0xFFFFF) // 1
    o.set_frames(1, 2)
    _, st = o.verify(p, MODE_ERROR, 0.01, seed=3, frame=2)
    assert st["n_pruned"] == 0
    assert st["n_filled"] == 200
    assert np.array_equal(o.dm_counts(0), o.dm_targets(0))
    filled = (p.info & (1 << 30)) != 0
    assert set(np.unique(x0[filled])) == {0, 1}            # the paths that fell off the light
    assert set(np.unique(p.info[filled] & 0xFFFFF)) == {6, 7}
    o.retrace(p, 3, 2)
    hit = np.nonzero(filled & (p.nseg > 0))[0]
    back = np.array([o.dm_cell_of(0, p.photons[i, 0, :3], p.origin[i]) for i in hit])
    assert (back == (p.info[hit] & 0xFFFFF)).sum() >= hit.size - 1


def test_prune_count_matches_eq1_expectation():
    """Point light moved: cells with DM_C > DM_T lose each of their paths with
    probability (DM_C - DM_T) / DM_C, so the pruned total has expectation
    sum (DM_C - DM_T) (5 sigma over 200 independent draws); cells at or below
    their target lose none."""
    mv = lambda f: [Light(LIGHT_POINT, (0.6 * (f - 1), 1.0, 0.0), power=(1.0,) * 3, n_paths=3200)]
    sc = kit.floor_and_light(3200, B=1, R=20.0)
    sc._light_fn = mv
    o, p0 = _traced(sc, (0, 0, 0, 0), (8, 8))
    o.set_frames(1, 2)
    # counts before pruning, from the parametrisation at the new pose
    kept = np.nonzero(p0.nseg > 0)[0]
    pre = np.zeros(64, np.int64)
    cells = {}
    for i in kept:
        c = o.dm_cell_of(0, p0.photons[i, 0, :3], p0.origin[i])
        cells[i] = c
        pre[c] += 1
    t = o.dm_targets(0).astype(np.int64)
    over = pre > t
    assert over.any()
    expect_per = (pre - t)[over].sum()
    var_per = (pre[over] * ((pre - t)[over] / pre[over]) * (t[over] / pre[over])).sum()
    R, total = 200, 0
    for r in range(R):
        p = p0.copy()
        _, st = o.verify(p, MODE_ERROR, 0.01, seed=3, frame=1000 + r)
        total += st["n_pruned"]
    assert abs(total - R * expect_per) <= 5 * math.sqrt(R * var_per) + 1, (total, R * expect_per)
    # no path of a cell at or below its target is ever pruned (last draw)
    free = ((p.info >> 30) & 1).astype(bool) & (((p.info >> 26) & 15) == 0) & ((p.info >> 31) == 0)
    for i in kept:
        if not over[cells[i]]:
            assert not free[i], i


def test_fill_accounts_for_every_path():
    """Point light moved with many escaped paths: every free path is given a
    cell, the counts add up to the light's paths, and no cell stays below its
    target while free paths remain."""
    mv = lambda f: [Light(LIGHT_POINT, (0.3 * (f - 1), 1.0, 0.2 * (f - 1)), power=(1.0,) * 3, n_paths=6400)]
    sc = kit.floor_and_light(6400, B=1, R=20.0)
    sc._light_fn = mv
    o, p = _traced(sc, (0, 0, 0, 0), (8, 8))
    escaped = int((p.nseg == 0).sum())
    assert escaped > 1000
    for f in (2, 3, 4):
        o.set_frames(f - 1, f)
        _, st = o.verify(p, MODE_ERROR, 0.01, seed=3, frame=f)
        dm = o.dm_counts(0).astype(np.int64)
        t = o.dm_targets(0).astype(np.int64)
        assert dm.sum() == sc.n_paths
        assert np.array_equal(np.bincount(p.info & 0xFFFFF, minlength=64), dm)
        free = ((p.info >> 30) & 1).astype(bool) & (((p.info >> 26) & 15) == 0) & ((p.info >> 31) == 0)
        F = int(free.sum())
        assert st["n_filled"] == F and F >= escaped // 2
        filled = np.bincount(p.info[free] & 0xFFFFF, minlength=64)
        pre = dm - filled
        deficit = np.maximum(t - pre, 0)
        if F >= deficit.sum():
            assert (filled >= deficit).all() and (dm >= t).all()
        else:
            assert (filled == np.minimum(deficit, np.maximum(filled, 0))).all()
        o.retrace(p, 3, f)


def test_static_light_leaves_the_map_alone():
    sc = kit.rect_light_over_floor(1024, B=1, R=3.0)
    o, p = _traced(sc, (4, 4, 2, 2), (0, 0))
    before = o.dm_counts(0).copy()
    info = p.info.copy()
    o.set_frames(1, 2)                                  # nothing moves
    _, st = o.verify(p, MODE_ERROR, 0.01, seed=3, frame=2)
    assert st["n_pruned"] == 0 and st["n_filled"] == 0
    assert np.array_equal(o.dm_counts(0), before)
    assert np.array_equal(p.info, info)
