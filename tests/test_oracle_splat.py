"""Pins of the oracle's screen-space splat (radius kernel), CPU only: the
kernel integrates to rho/pi E over a surface seen head-on, photons arriving
from behind the visible surface add nothing, and the splatted image of a
point light over a floor reproduces the closed-form irradiance
Phi h / (4 pi (h^2 + rho^2)^(3/2)) times rho/pi."""
import math

import numpy as np

import oracle
from tests import scene_kit as kit


def _one_photon(sc, x, origin, E):
    B = sc.max_bounces
    ph = np.zeros((1, B, 8), np.float32)
    ph[0, 0, :3] = x
    ph[0, 0, 3] = np.array([0], np.int32).view(np.float32)[0]
    ph[0, 0, 4:7] = E
    return oracle.Paths(np.zeros(1, np.uint32), np.array([1 << 22], np.uint32), np.array([origin], np.float32), ph,
                        np.zeros(1, np.uint32))


def _down_camera(height, half_extent, n):
    return oracle.Camera.make((0.0, height, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 1.0),
                              2.0 * math.atan(half_extent / height), n, n)


def test_kernel_integrates_to_albedo_over_pi():
    sc = kit.floor_and_light(10, B=1, R=20.0)            # floor y = 0, albedo 0.5
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    E = np.array([2.0, 3.0, 5.0], np.float32)
    p = _one_photon(sc, (0.013, 0.0, -0.021), (0.3, 2.0, 0.1), E)
    cam = _down_camera(10.0, 0.5, 200)
    img, _ = o.splat(p, cam, 0.1)       # flagged pixels lie on the floor's diagonal edge: same plane either way
    side = 2 * 0.5 / 200                                 # every pixel covers the same floor area
    total = img.sum(axis=(0, 1)) * side * side
    np.testing.assert_allclose(total, 0.5 / math.pi * E, rtol=0.01)
    # the pixel nearest the photon sees the kernel's peak 2 / (pi r^2)
    j, i = np.unravel_index(np.argmax(img[..., 0]), img.shape[:2])
    assert abs(img[j, i, 0] / (0.5 / math.pi * 2.0 * 2.0 / (math.pi * 0.01)) - 1.0) < 0.02


def test_photon_from_behind_adds_nothing():
    sc = kit.floor_and_light(10, B=1, R=20.0)
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    p = _one_photon(sc, (0.0, 0.0, 0.0), (0.0, -2.0, 0.0), np.ones(3, np.float32))
    img, _ = o.splat(p, _down_camera(10.0, 0.5, 64), 0.1)
    assert img.max() == 0.0


def test_point_light_irradiance_through_the_splat():
    """Direct photons of a point light at height 1 (flux 4 pi): the floor's
    irradiance is h / (h^2 + rho^2)^(3/2); the splat returns rho_albedo/pi
    times it (mean over the view 2 %, every pixel 6 sigma)."""
    n = 400_000
    sc = kit.floor_and_light(n, h=1.0, R=20.0, power=4.0 * math.pi, B=1)
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    p = o.trace(np.arange(n, dtype=np.uint32), 7, 1)
    cam = _down_camera(10.0, 1.0, 48)
    r = 0.15
    img, _ = o.splat(p, cam, r)
    side = 2.0 / 48
    c = (np.arange(48) + 0.5) * side - 1.0
    X, Z = np.meshgrid(-c, c[::-1], indexing="xy")        # right = -x, up = +z for this camera
    rho2 = X ** 2 + Z ** 2
    want = 0.5 / math.pi * 1.0 / (1.0 + rho2) ** 1.5
    got = img[..., 0]
    assert abs(got.mean() / want.mean() - 1.0) < 0.02
    # per pixel: about n E / (4 pi) pi r^2 photons under the kernel; the kernel-weighted
    # estimate has relative variance 4/3 / (expected count)
    expected = n * want / (0.5 / math.pi) / (4.0 * math.pi) * math.pi * r * r
    sigma = want * np.sqrt(4.0 / 3.0 / expected)
    assert (np.abs(got - want) < 6 * sigma + 0.02 * want).all()
