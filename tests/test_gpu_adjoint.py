"""GPU parity of the differentiable deposit model, its adjoint and the
ray-budget list, through the C ABI, against the FP64 oracle.

Tolerances (FP32 kernels, float atomics in any order):
  - model atlas: |gpu - oracle| <= 1e-4 max|atlas| per texel;
  - dL/dtheta: |gpu - oracle| <= 2e-3 max_j |dL/dtheta_j| + 1e-3 |dL/dtheta_j|.
    The cubic B-spline splat is twice continuously differentiable, so FP32
    and FP64 choosing different base texels for a photon on a texel-centre
    line changes neither the atlas nor the gradient beyond rounding;
  - per-path scores: |gpu - oracle| <= 1e-4 max score + 1e-4 |score|;
  - budget lists: bit-exact against a numpy ranking of the GPU's own scores.
"""
import numpy as np
import pytest

import oracle
import scenes
import paper_2111_06906_gb300 as pv
from tests import gpu_util as gu
from tests import scene_kit as kit

pytestmark = pytest.mark.gpu

W, H = 48, 40


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2111_06906_gb300 import build
    build.build()
    pv.load()


def _torch():
    import torch
    return torch


def _scene(name):
    if name == "box_torus":
        return kit.box_with_torus(4000, B=4)
    if name == "rect_floor":
        return kit.rect_light_over_floor(3000, B=2, R=3.0)
    if name == "city_small":
        return scenes.city(n_paths=12000, n_boxes=1500)
    if name == "villa_small":
        return scenes.villa(n_paths_per_light=3000)
    raise KeyError(name)


_cache = {}


def _traced(name):
    """(scene, oracle scene at frame 1, oracle paths traced with seed 5), built
    once per module: the read-only tests share them."""
    if name not in _cache:
        sc = _scene(name)
        o = oracle.OracleScene(sc)
        o.set_frames(1, 1)
        _cache[name] = (sc, o, o.trace(np.arange(sc.n_paths, dtype=np.uint32), 5, 1))
    return _cache[name]


def _setup(sc, frame=1, seed=5):
    """Oracle-traced paths uploaded into the library's buffers."""
    o = oracle.OracleScene(sc)
    o.set_frames(frame, frame)
    op = o.trace(np.arange(sc.n_paths, dtype=np.uint32), seed, frame)
    h = gu.lib_scene(sc, frame=frame)
    P = pv.Paths.allocate(sc.n_paths, sc.max_bounces)
    gu.upload(P, op)
    return o, op, h, P


def _setup_cached(name):
    sc, o, op = _traced(name)
    h = gu.lib_scene(sc, frame=1)
    P = pv.Paths.allocate(sc.n_paths, sc.max_bounces)
    gu.upload(P, op)
    return sc, o, op, h, P


def _linear_G(seed, noise=1e-3):
    rng = np.random.default_rng(seed)
    i = np.arange(W)[None, :, None]
    j = np.arange(H)[:, None, None]
    a, b, c = rng.normal(size=(3, 1, 1, 3))
    return a + b * i / W + c * j / H + noise * rng.normal(size=(H, W, 3))


def _perturbed(th0, n_lights, seed, amount=1.0):
    rng = np.random.default_rng(seed)
    th = th0.copy()
    for l in range(n_lights):
        th[7 * l:7 * l + 3] += amount * 0.01 * rng.normal(size=3)
        th[7 * l + 3:7 * l + 6] += amount * 0.01 * rng.normal(size=3)
        th[7 * l + 6] *= 1.0 + amount * 0.2 * rng.random()
    th[7 * n_lights:] += amount * 0.01 * rng.normal(size=th.shape[0] - 7 * n_lights)
    return th


def _gpu_model(h, P, th, rect):
    torch = _torch()
    A = torch.zeros(H, W, 3, dtype=torch.float32, device="cuda")
    pv.pv_model_deposit(h, P, torch.as_tensor(th, dtype=torch.float32, device="cuda"), A, rect)
    return A.cpu().numpy().astype(np.float64)


def _gpu_adjoint(h, P, th, G, rect, n):
    torch = _torch()
    d = torch.zeros(th.shape[0], dtype=torch.float32, device="cuda")
    s = torch.zeros(n, dtype=torch.float32, device="cuda")
    pv.pv_adjoint_deposit(h, P, torch.as_tensor(th, dtype=torch.float32, device="cuda"),
                          torch.as_tensor(G, dtype=torch.float32, device="cuda"), rect, d, s)
    return d.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64)


def _assert_dtheta(dg, do):
    tol = 2e-3 * np.abs(do).max() + 1e-3 * np.abs(do)
    bad = np.nonzero(np.abs(dg - do) > tol)[0]
    assert bad.size == 0, [(int(j), dg[j], do[j]) for j in bad[:8]]


@pytest.mark.parametrize("name", ["box_torus", "rect_floor", "city_small", "villa_small"])
def test_theta_current_matches_oracle(name):
    sc, o, _ = _traced(name)
    h = gu.lib_scene(sc, frame=1)
    assert pv.pv_theta_size(h) == o.theta_current().shape[0]
    np.testing.assert_allclose(pv.pv_theta_current(h), o.theta_current(), rtol=0, atol=1e-6)
    pv.pv_destroy_scene(h)


@pytest.mark.parametrize("name", ["box_torus", "rect_floor", "city_small", "villa_small"])
@pytest.mark.parametrize("perturb", [0.0, 1.0])
def test_model_deposit_parity(name, perturb):
    sc, o, op, h, P = _setup_cached(name)
    th = _perturbed(o.theta_current(), len(sc.lights(1)), seed=3, amount=perturb)
    Ag = _gpu_model(h, P, th, sc.atlas_rect)
    Ao = o.model_deposit(op, th, W, H, sc.atlas_rect)
    assert Ao.max() > 0
    err = np.abs(Ag - Ao).max() / Ao.max()
    assert err <= 1e-4, err
    assert pv.pv_read_device_status(h) == 0
    pv.pv_destroy_scene(h)


@pytest.mark.parametrize("name", ["box_torus", "rect_floor", "city_small", "villa_small"])
@pytest.mark.parametrize("perturb", [0.0, 1.0])
def test_adjoint_parity(name, perturb):
    sc, o, op, h, P = _setup_cached(name)
    th = _perturbed(o.theta_current(), len(sc.lights(1)), seed=4, amount=perturb)
    G = _linear_G(7)
    dg, _ = _gpu_adjoint(h, P, th, G, sc.atlas_rect, sc.n_paths)
    do, _ = o.adjoint(op, th, G, sc.atlas_rect)
    assert np.abs(do).max() > 0
    _assert_dtheta(dg, do)
    pv.pv_destroy_scene(h)


@pytest.mark.parametrize("name", ["box_torus", "city_small"])
def test_scores_parity_random_gradient(name):
    sc, o, op, h, P = _setup_cached(name)
    th = o.theta_current()
    G = np.random.default_rng(9).normal(size=(H, W, 3))
    _, sg = _gpu_adjoint(h, P, th, G, sc.atlas_rect, sc.n_paths)
    _, so = o.adjoint(op, th, G, sc.atlas_rect)
    tol = 1e-4 * so.max() + 1e-4 * so
    bad = np.nonzero(np.abs(sg - so) > tol)[0]
    assert bad.size == 0, [(int(i), sg[i], so[i]) for i in bad[:8]]
    pv.pv_destroy_scene(h)


def test_adjoint_against_fp32_central_differences():
    """The CUDA adjoint against central differences of the CUDA model itself.
    h = 1e-4: photons hit at grazing angles make the model strongly curved in
    the light's position (the truncation error at h = 1e-3 reaches 6 %), and
    the FP32 atlas noise, about 1e-7 of the loss, stays below 1 % of the
    derivative.  The loss is summed in FP64 from the FP32 atlases."""
    sc, o, op, h, P = _setup_cached("box_torus")
    th = o.theta_current()
    G = _linear_G(11, noise=0.0)
    dg, _ = _gpu_adjoint(h, P, th, G, sc.atlas_rect, sc.n_paths)
    step = 1e-4
    fd = np.zeros_like(th)
    for j in range(th.shape[0]):
        e = np.zeros_like(th)
        e[j] = step
        fd[j] = ((G * _gpu_model(h, P, th + e, sc.atlas_rect)).sum()
                 - (G * _gpu_model(h, P, th - e, sc.atlas_rect)).sum()) / (2 * step)
    tol = 1e-2 * np.abs(fd).max() + 1e-2 * np.abs(fd)
    assert (np.abs(dg - fd) <= tol).all(), np.c_[dg, fd]
    pv.pv_destroy_scene(h)


def test_intensity_gradient_is_total_deposit():
    """G = 1: dL/d(intensity) equals the model atlas's total; scores sum to it."""
    sc, o, op, h, P = _setup_cached("city_small")
    th = o.theta_current()
    A = _gpu_model(h, P, th, sc.atlas_rect)
    dg, sg = _gpu_adjoint(h, P, th, np.ones((H, W, 3)), sc.atlas_rect, sc.n_paths)
    assert dg[6] == pytest.approx(A.sum(), rel=1e-4)
    assert sg.sum() == pytest.approx(A.sum(), rel=1e-4)
    pv.pv_destroy_scene(h)


def test_autograd_function_matches_oracle():
    torch = _torch()
    sc, o, op, h, P = _setup_cached("box_torus")
    th0 = _perturbed(o.theta_current(), 1, seed=5)
    theta = torch.tensor(th0, dtype=torch.float32, device="cuda", requires_grad=True)
    G = _linear_G(13)
    A = pv.model_deposit(h, P, theta, H, W, sc.atlas_rect)
    loss = (A.double() * torch.as_tensor(G, device="cuda")).sum()
    loss.backward()
    do, _ = o.adjoint(op, th0, G, sc.atlas_rect)
    _assert_dtheta(theta.grad.cpu().numpy().astype(np.float64), do)
    Ao = o.model_deposit(op, th0, W, H, sc.atlas_rect)
    assert float(loss.detach()) == pytest.approx(float((G * Ao).sum()), rel=1e-4, abs=1e-4 * np.abs(G * Ao).sum())
    pv.pv_destroy_scene(h)


def test_empty_paths_and_argument_errors():
    torch = _torch()
    sc = _scene("box_torus")
    o, op, h, P = _setup(sc)
    th = torch.as_tensor(o.theta_current(), dtype=torch.float32, device="cuda")
    A = torch.zeros(H, W, 3, dtype=torch.float32, device="cuda")
    P.info.zero_()                                   # every path empty
    pv.pv_model_deposit(h, P, th, A, sc.atlas_rect)
    d = torch.zeros_like(th)
    s = torch.full((sc.n_paths,), 7.0, device="cuda")
    pv.pv_adjoint_deposit(h, P, th, A, sc.atlas_rect, d, s)
    assert float(A.abs().sum()) == 0.0 and float(d.abs().sum()) == 0.0 and float(s.abs().sum()) == 0.0
    for rect in [(0.0, 0.0, 0.0, 1.0), (1.0, 0.0, 0.0, 1.0)]:
        with pytest.raises(pv.PvError):
            pv.pv_model_deposit(h, P, th, A, rect)
    with pytest.raises(pv.PvError):
        pv.pv_adjoint_deposit(h, P, None, A, sc.atlas_rect, d)
    assert pv.pv_read_device_status(h) == 0
    pv.pv_destroy_scene(h)


def _budget_ref(lst, score, budget):
    s = score[lst].astype(np.float32)
    key = np.where(s > 0, s, np.float32(0)).view(np.uint32)
    order = np.lexsort((lst, ~key))                  # score descending, then id ascending
    return np.sort(lst[order[:budget]])


@pytest.mark.parametrize("count_frac,budget_frac,tie", [(0.3, 0.5, False), (0.3, 0.5, True), (1.0, 0.1, True),
                                                        (0.0, 0.5, False), (0.5, 0.0, False), (0.5, 2.0, False),
                                                        (0.05, 1.0, True)])
def test_budget_list_exact(count_frac, budget_frac, tie):
    torch = _torch()
    sc = _scene("rect_floor")                        # 3000 paths
    h = gu.lib_scene(sc)
    n = sc.n_paths
    rng = np.random.default_rng(int(1000 * count_frac + 10 * budget_frac) + tie)
    lst = np.sort(rng.choice(n, size=int(count_frac * n), replace=False)).astype(np.uint32)
    score = rng.random(n).astype(np.float32)
    if tie:                                          # many equal scores, zeros and negatives
        score = np.round(score * 4).astype(np.float32) / 4
        score[rng.random(n) < 0.1] = -1.0
    budget = int(budget_frac * len(lst))
    d_list = torch.zeros(n, dtype=torch.int32, device="cuda")
    d_list[: len(lst)] = torch.as_tensor(lst.view(np.int32), device="cuda")
    d_cnt = torch.tensor([len(lst)], dtype=torch.int32, device="cuda")
    out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    out_cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    pv.pv_budget_list(h, d_list, d_cnt, torch.as_tensor(score, device="cuda"), budget, out, out_cnt)
    got = out[: int(out_cnt.item())].cpu().numpy().view(np.uint32)
    want = _budget_ref(lst, score, min(budget, len(lst)))
    np.testing.assert_array_equal(got, want)
    assert pv.pv_read_device_status(h) == 0
    pv.pv_destroy_scene(h)


def test_budget_list_large_spans_radix_tiles():
    """300k listed of 1M paths (many sort tiles); scores from the adjoint."""
    torch = _torch()
    sc = scenes.city(n_paths=1_000_000, n_boxes=1500)
    h = gu.lib_scene(sc)
    P = pv.Paths.allocate(sc.n_paths, sc.max_bounces)
    pv.pv_trace_all(h, P, 3, 1)
    n = sc.n_paths
    th = torch.as_tensor(pv.pv_theta_current(h), device="cuda")
    G = torch.as_tensor(_linear_G(17, noise=0.5), dtype=torch.float32, device="cuda")
    d = torch.zeros_like(th)
    s = torch.zeros(n, dtype=torch.float32, device="cuda")
    pv.pv_adjoint_deposit(h, P, th, G, sc.atlas_rect, d, s)
    rng = np.random.default_rng(19)
    lst = np.sort(rng.choice(n, size=300_000, replace=False)).astype(np.uint32)
    d_list = torch.zeros(n, dtype=torch.int32, device="cuda")
    d_list[: len(lst)] = torch.as_tensor(lst.view(np.int32), device="cuda")
    d_cnt = torch.tensor([len(lst)], dtype=torch.int32, device="cuda")
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    out_cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    pv.pv_budget_list(h, d_list, d_cnt, s, 77_777, out, out_cnt)
    got = out[: int(out_cnt.item())].cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got, _budget_ref(lst, s.cpu().numpy(), 77_777))
    assert pv.pv_read_device_status(h) == 0
    pv.pv_destroy_scene(h)


def test_budgeted_retrace_flow_matches_oracle():
    """Verify (Alg. 1) -> adjoint scores -> budget list -> re-trace of the
    budget only: the re-traced paths match the oracle re-tracing the same ids,
    every other path keeps its record."""
    torch = _torch()
    sc = _scene("box_torus")
    o, op, h, P = _setup(sc)
    gu.advance(h, sc, 2)
    n = sc.n_paths
    lst = torch.zeros(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    pv.pv_verify_paths(h, P, pv.PV_MODE_ERROR, sc.tau, 0, lst, cnt)
    o.set_frames(1, 2)
    q = op.copy()
    o.verify(q, pv.PV_MODE_ERROR, sc.tau)
    listed = lst[: int(cnt.item())].cpu().numpy().view(np.uint32)
    assert listed.size > 20
    th = torch.as_tensor(pv.pv_theta_current(h), device="cuda")
    s = torch.zeros(n, dtype=torch.float32, device="cuda")
    pv.pv_adjoint_deposit(h, P, th, torch.ones(H, W, 3, device="cuda"), sc.atlas_rect, torch.zeros_like(th), s)
    budget = listed.size // 3
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    out_cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    pv.pv_budget_list(h, lst, cnt, s, budget, out, out_cnt)
    chosen = out[: int(out_cnt.item())].cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(chosen, _budget_ref(listed, s.cpu().numpy(), budget))
    before = gu.download(P)
    pv.pv_retrace_invalid(h, P, out, out_cnt, 9, 2)
    after = gu.download(P)
    rest = np.setdiff1d(np.arange(n, dtype=np.uint32), chosen)
    assert np.array_equal(after.info[rest], before.info[rest])
    assert np.array_equal(after.photons[rest], before.photons[rest])
    sub = q.subset(chosen)
    o.retrace(sub, 9, 2)
    got = gu.download(P, chosen)
    r = gu.compare(got, sub, sc.diag)
    print(r)
    gu.assert_parity(r)
    assert pv.pv_read_device_status(h) == 0
    pv.pv_destroy_scene(h)


def _l2_fd(model, T, th, step):
    """Central differences of sum((model(theta) - T)^2), summed in FP64."""
    fd = np.zeros_like(th)
    for j in range(th.shape[0]):
        e = np.zeros_like(th)
        e[j] = step
        fd[j] = (((model(th + e) - T) ** 2).sum() - ((model(th - e) - T) ** 2).sum()) / (2 * step)
    return fd


def test_adjoint_workload_city_l2_subset():
    """The adjoint workload: the city scene launched at full size (1M path
    slots), loss = L2 of the 1024 x 1024 atlas against the atlas at a seeded
    perturbed pose, on a seeded 20k-path subset (the other slots emptied;
    the records of both sides checked equal first).  Each side
    computes its own atlases, loss gradient G and dL/dtheta.  Checks: the
    gradient against the FP64 oracle's; the CUDA model's central differences
    (h = 1e-3) against the oracle's at the same h; and the CUDA adjoint
    against its own central differences, within the truncation error the
    FP64 oracle shows at that h (photons re-found at grazing incidence make
    the loss strongly curved on the scale of 1e-3) plus 1 %."""
    torch = _torch()
    sc = scenes.city()
    n, Wc, Hc, rect = sc.n_paths, 1024, 1024, sc.atlas_rect
    ids = np.sort(np.random.default_rng(20).choice(n, 20000, replace=False)).astype(np.uint32)
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    sub = o.trace(ids, 3, 1)
    h = gu.lib_scene(sc)
    P = pv.Paths.allocate(n, sc.max_bounces)
    pv.pv_trace_all(h, P, 3, 1)
    # every sampled path matches the oracle (an ambiguous one one of the outcomes it admits, which the oracle
    # then takes as its own record): both sides model the same stored paths
    r = gu.compare(gu.download(P, ids), sub, sc.diag)
    print(r)
    gu.assert_parity(r)
    on = torch.zeros(n, dtype=torch.bool, device="cuda")
    on[torch.as_tensor(sub.ids.astype(np.int64), device="cuda")] = True
    P.info[~on] = 0
    th0 = o.theta_current()
    ths = scenes.perturbed_theta(th0, 1)

    def model_o(th):
        return o.model_deposit(sub, th, Wc, Hc, rect)

    def model_g(th):
        A = torch.zeros(Hc, Wc, 3, dtype=torch.float32, device="cuda")
        pv.pv_model_deposit(h, P, torch.as_tensor(th, dtype=torch.float32, device="cuda"), A, rect)
        return A.double().cpu().numpy()

    T_o, T_g = model_o(ths), model_g(ths)
    G_o, G_g = 2 * (model_o(th0) - T_o), 2 * (model_g(th0) - T_g)
    d_o, _ = o.adjoint(sub, th0, G_o, rect)
    d_g, _ = _gpu_adjoint(h, P, th0, G_g, rect, n)
    _assert_dtheta(d_g, d_o)
    step = 1e-3
    fd_o, fd_g = _l2_fd(model_o, T_o, th0, step), _l2_fd(model_g, T_g, th0, step)
    assert np.all(np.abs(fd_g - fd_o) <= 1e-2 * np.abs(fd_o).max() + 1e-2 * np.abs(fd_o)), np.c_[fd_g, fd_o]
    trunc = np.abs(d_o - fd_o)
    tol = trunc + 1e-2 * np.abs(d_o).max() + 1e-2 * np.abs(d_o)
    assert np.all(np.abs(d_g - fd_g) <= tol), np.c_[d_g, fd_g, trunc]
    assert pv.pv_read_device_status(h) == 0
    pv.pv_destroy_scene(h)


def test_adjoint_workload_city_full_size_autograd():
    """Full adjoint workload through the autograd function (1M paths, 1024 x
    1024 atlas, L2 loss against the seeded perturbed pose): dL/d(intensity)
    equals its closed form 2 sum((A - T) A) / s, every parameter receives a
    finite gradient, and the per-path scores sum to the intensity gradient
    (up to sign) when G is the all-ones atlas."""
    torch = _torch()
    sc = scenes.city()
    n, Wc, Hc, rect = sc.n_paths, 1024, 1024, sc.atlas_rect
    h = gu.lib_scene(sc)
    P = pv.Paths.allocate(n, sc.max_bounces)
    pv.pv_trace_all(h, P, 3, 1)
    th0 = pv.pv_theta_current(h).astype(np.float64)
    ths = scenes.perturbed_theta(th0, 1)
    T = pv.model_deposit(h, P, torch.as_tensor(ths, dtype=torch.float32, device="cuda"), Hc, Wc, rect).detach()
    theta = torch.tensor(th0, dtype=torch.float32, device="cuda", requires_grad=True)
    A = pv.model_deposit(h, P, theta, Hc, Wc, rect)
    loss = ((A.double() - T.double()) ** 2).sum()
    loss.backward()
    g = theta.grad.double().cpu().numpy()
    assert np.all(np.isfinite(g)) and np.abs(g[7:]).max() > 0
    closed = float((2 * (A.double() - T.double()) * A.double()).sum().detach())
    assert g[6] == pytest.approx(closed, rel=1e-3, abs=1e-4 * abs(closed))
    d = torch.zeros(th0.shape[0], dtype=torch.float32, device="cuda")
    s = torch.zeros(n, dtype=torch.float32, device="cuda")
    pv.pv_adjoint_deposit(h, P, theta.detach(), torch.ones(Hc, Wc, 3, device="cuda"), rect, d, s)
    total = float(A.double().sum().detach())
    assert float(d[6]) == pytest.approx(total, rel=1e-3)
    assert float(s.double().sum()) == pytest.approx(total, rel=1e-3)
    assert pv.pv_read_device_status(h) == 0
    pv.pv_destroy_scene(h)
