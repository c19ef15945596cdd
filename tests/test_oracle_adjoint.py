"""Pins of the oracle's differentiable deposit model and its adjoint (CPU).

The model freezes every stored path's triangles and sampled directions and
re-finds each photon on its (translated) triangle plane; the adjoint is
checked against central differences of the model itself, closed forms and an
independent cubic B-spline splat of the stored photons (written from the
distance form of the kernel, not the per-fraction polynomials the oracle
uses)."""
import numpy as np
import pytest

import oracle
import scenes
from tests import scene_kit as kit

W = H = 32


def _setup(sc, frame=1, n=None, seed=3):
    o = oracle.OracleScene(sc)
    o.set_frames(frame, frame)
    n = sc.n_paths if n is None else n
    p = o.trace(np.arange(n, dtype=np.uint32), seed, frame)
    return o, p


def _bspline(t):
    """Cardinal cubic B-spline as a function of the distance |t| in texels."""
    a = abs(t)
    if a < 1.0:
        return 2.0 / 3.0 - a * a + a ** 3 / 2.0
    if a < 2.0:
        return (2.0 - a) ** 3 / 6.0
    return 0.0


def _bspline_numpy(p, rect):
    """Independent splat of the stored photons: texel (i, j) with centre
    coordinate (i, j) gets B(u - i) B(v - j)."""
    x0, z0, x1, z1 = rect
    A = np.zeros((H, W, 3))
    for i in range(p.ids.shape[0]):
        for k in range(int(p.nseg[i])):
            x, z = float(p.photons[i, k, 0]), float(p.photons[i, k, 2])
            u = (x - x0) * W / (x1 - x0) - 0.5
            v = (z - z0) * H / (z1 - z0) - 0.5
            for ti in range(int(np.floor(u)) - 2, int(np.floor(u)) + 4):
                for tj in range(int(np.floor(v)) - 2, int(np.floor(v)) + 4):
                    if 0 <= ti < W and 0 <= tj < H:
                        w = _bspline(u - ti) * _bspline(v - tj)
                        A[tj, ti] += w * p.photons[i, k, 4:7].astype(np.float64)
    return A


def test_model_reproduces_stored_photons():
    sc = kit.box_with_torus(1500, B=4)
    o, p = _setup(sc)
    A = o.model_deposit(p, o.theta_current(), W, H, sc.atlas_rect)
    B = _bspline_numpy(p, sc.atlas_rect)
    assert np.allclose(A, B, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("which", ["point", "rect"])
def test_adjoint_matches_central_differences(which):
    if which == "point":
        sc = kit.box_with_torus(800, B=4)
        rect = sc.atlas_rect
    else:
        sc = kit.rect_light_over_floor(800, B=2, R=3.0)
        rect = (-3.0, -3.0, 3.0, 3.0)
    o, p = _setup(sc)
    th0 = o.theta_current()
    G = np.random.default_rng(1).normal(size=(H, W, 3))
    dth, _ = o.adjoint(p, th0, G, rect)
    h = 1e-6
    for j in range(th0.shape[0]):
        e = np.zeros_like(th0)
        e[j] = h
        Lp = (G * o.model_deposit(p, th0 + e, W, H, rect)).sum()
        Lm = (G * o.model_deposit(p, th0 - e, W, H, rect)).sum()
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - dth[j]) <= 1e-5 * max(abs(fd), 1.0), (j, fd, dth[j])
    # the moving parameters really matter in these scenes
    assert np.abs(dth).max() > 1e-3


def test_intensity_gradient_closed_form():
    """With G = 1 everywhere, dL/d(scale) = total energy the light deposits."""
    sc = kit.box_with_torus(1000, B=4)
    o, p = _setup(sc)
    th = o.theta_current()
    A = o.model_deposit(p, th, W, H, sc.atlas_rect)
    dth, score = o.adjoint(p, th, np.ones((H, W, 3)), sc.atlas_rect)
    assert dth[6] == pytest.approx(A.sum(), rel=1e-12)
    # scores: |dL/d(path scale)| = each path's deposited energy when G = 1
    assert score.sum() == pytest.approx(A.sum(), rel=1e-9)


def test_translation_within_a_plane_moves_nothing():
    """A dynamic floor moved within its own plane keeps every re-found hit."""
    R = 2.0
    floor = kit.quad((-R, 0, -R), (0, 0, 2 * R), (2 * R, 0, 0))
    lights = lambda f: [scenes.Light(scenes.LIGHT_POINT, (0.1, 1.0, -0.2), power=(1.0,) * 3, n_paths=2000)]
    sc = kit.build([(floor, (0.5,) * 3, True)], lights, B=1, diag=6.0, rect=(-2.0, -2.0, 2.0, 2.0))
    o, p = _setup(sc)
    th0 = o.theta_current()
    G = np.random.default_rng(2).normal(size=(H, W, 3))
    dth, _ = o.adjoint(p, th0, G, sc.atlas_rect)
    t = 7                                   # translation of the floor
    assert dth[t] == 0.0 and dth[t + 2] == 0.0
    assert abs(dth[t + 1]) > 1e-6           # moving it up or down does move the hits
    moved = th0.copy()
    moved[t] += 0.3
    moved[t + 2] -= 0.2
    assert np.allclose(o.model_deposit(p, moved, W, H, sc.atlas_rect), o.model_deposit(p, th0, W, H, sc.atlas_rect),
                       rtol=1e-12, atol=1e-15)
