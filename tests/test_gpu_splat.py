"""GPU parity of the screen-space splat (radius kernel) against the FP64
oracle through the C ABI: the same stored records (the oracle's, uploaded)
and camera on both sides; pixels whose visible point, side test or
near-plane decision the oracle flags are excluded.  Tolerance: float32
G-buffer points and float atomics in any order, |gpu - oracle| <= 1e-4 of
the image maximum + 1e-4 relative."""
import math

import numpy as np
import pytest

import oracle
import scenes
import paper_2111_06906_gb300 as pv
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


CASES = {
    "tiny_box": (lambda: scenes.tiny_box(n_paths=6000), ((0.0, 1.5, 0.95), (0.0, 0.2, -0.4), (0.0, 1.0, 0.0)), 0.12),
    "box_torus": (lambda: kit.box_with_torus(5000, B=4), ((0.3, 1.2, 0.9), (-0.3, 0.5, -0.5), (0.0, 1.0, 0.0)), 0.1),
    "rect_floor": (lambda: kit.rect_light_over_floor(5000, B=2, R=3.0), ((0.0, 6.0, 4.0), (0.0, 0.0, 0.0),
                                                                          (0.0, 1.0, 0.0)), 0.25),
    "city_small": (lambda: scenes.city(n_paths=12000, n_boxes=1500), ((0.0, 45.0, 35.0), (0.0, 0.0, 0.0),
                                                                       (0.0, 1.0, 0.0)), 1.5),
}


@pytest.mark.parametrize("name", list(CASES))
def test_splat_matches_oracle(name):
    torch = _torch()
    make, (pos, target, up), radius = CASES[name]
    sc = make()
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    op = o.trace(np.arange(sc.n_paths, dtype=np.uint32), 9, 1)
    W, H = 160, 90
    cam_o = oracle.Camera.make(pos, target, up, math.radians(60.0), W, H)
    want, amb = o.splat(op, cam_o, radius)
    h = gu.lib_scene(sc)
    P = pv.Paths.allocate(sc.n_paths, sc.max_bounces)
    gu.upload(P, op)
    cam = pv.PvCamera.make(pos, target, up, math.radians(60.0), W, H)
    img = torch.zeros(H, W, 3, dtype=torch.float32, device="cuda")
    work = torch.empty(pv.pv_splat_workspace_bytes(h, W, H), dtype=torch.uint8, device="cuda")
    pv.pv_splat(h, P, cam, radius, img, work)
    got = img.cpu().numpy().astype(np.float64)
    ok = ~amb
    assert ok.mean() > 0.95 and want.max() > 0
    err = np.abs(got - want)[ok]
    tol = 1e-4 * want.max() + 1e-4 * np.abs(want)[ok]
    assert (err <= tol).all(), (float(err.max()), float(want.max()))
    assert pv.pv_read_device_status(h) == 0
    pv.pv_destroy_scene(h)


def test_splat_argument_errors():
    torch = _torch()
    sc = scenes.tiny_box(n_paths=1000)
    h = gu.lib_scene(sc)
    P = pv.Paths.allocate(sc.n_paths, sc.max_bounces)
    img = torch.zeros(10, 10, 3, device="cuda")
    work = torch.empty(pv.pv_splat_workspace_bytes(h, 10, 10), dtype=torch.uint8, device="cuda")
    good = ((0.0, 1.0, 0.9), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0))
    for cam, r, wk in [(pv.PvCamera.make(*good, 1.0, 10, 10), 0.0, work),
                       (pv.PvCamera.make(*good, 0.0, 10, 10), 0.1, work),
                       (pv.PvCamera.make((0, 1, 0), (0, 0, 0), (0, 1, 0), 1.0, 10, 10), 0.1, work),
                       (pv.PvCamera.make(*good, 1.0, 10, 10), 0.1, work[:100])]:
        with pytest.raises(pv.PvError):
            pv.pv_splat(h, P, cam, r, img, wk)
    pv.pv_destroy_scene(h)


def test_splat_full_hd_city():
    """1920 x 1080 splat of the city's 1M traced paths: finite, non-negative,
    lit, and repeatable up to the order of each pixel's sum."""
    torch = _torch()
    sc = scenes.city()
    h = gu.lib_scene(sc)
    P = pv.Paths.allocate(sc.n_paths, sc.max_bounces)
    pv.pv_trace_all(h, P, 5, 1)
    W, H = 1920, 1080
    cam = pv.PvCamera.make((0.0, 45.0, 35.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), math.radians(60.0), W, H)
    work = torch.empty(pv.pv_splat_workspace_bytes(h, W, H), dtype=torch.uint8, device="cuda")
    a = torch.zeros(H, W, 3, device="cuda")
    b = torch.zeros(H, W, 3, device="cuda")
    pv.pv_splat(h, P, cam, 0.3, a, work)
    pv.pv_splat(h, P, cam, 0.3, b, work)
    assert bool(torch.isfinite(a).all()) and float(a.min()) >= 0.0
    assert float((a.sum(-1) > 0).float().mean()) > 0.5
    assert float((a - b).abs().max()) <= 1e-5 * float(a.max())
    assert pv.pv_read_device_status(h) == 0
    pv.pv_destroy_scene(h)
