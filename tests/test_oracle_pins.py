"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test checks the oracle against something the paper or mathematics fixes:
published generator vectors, the paper's Table 1, closed forms, invariants the
paper states (Sec. 3.2, 3.3), hand-derived cases and an independent brute force.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import scenes
from scenes import LIGHT_POINT, Light
from tests import scene_kit as kit

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers():
    for r in _kat():
        out = oracle.philox4x32_10(r[0:4], r[4:6])
        assert [int(x) for x in out] == r[6:10]


def test_table1_layout():
    """Record sizes reproduce the memory table (Sec. 5.2, Table 1)."""
    g = {}
    with open(os.path.join(GOLDEN, "table1_memory.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                g[k] = float(v)
    MiB = 1024.0 * 1024.0
    N, B = 5_000_000, 7
    info = N * np.dtype(np.uint32).itemsize / MiB
    origin = N * 3 * np.dtype(np.float32).itemsize / MiB
    photon_bytes = np.zeros((1, 1, 8), np.float32).nbytes        # oracle photon record
    photons = N * B * photon_bytes / MiB
    dm = 2 * 32 ** 4 * 4 / MiB
    pruned = N * 4 / MiB
    assert photon_bytes == 32
    assert round(info, 2) == g["path_information"]
    assert round(origin, 2) == g["path_origin"]
    assert round(dm, 3) == g["distribution_maps"]
    assert round(pruned, 2) == g["pruned_paths"]
    # the paper's sub-totals add its rounded rows
    assert round(round(info, 2) + round(origin, 2) + dm + round(pruned, 2), 2) == g["subtotal_lights"]
    assert round(round(info, 2) + round(origin, 2), 2) == g["subtotal_objects"]
    assert round(photons) == g["photon_map"]
    assert round(photons + info + origin + dm + pruned) == g["total_lights"]
    assert round(photons + info + origin) == g["total_objects"]
    # info word: 22 + 4 + 4 + 1 + 1 bits (Sec. 4): <= 15 segments, 2^22 cells
    assert 22 + 4 + 4 + 1 + 1 == 32
    assert oracle.INFO_REPLACE == 1 << 30 and oracle.INFO_REUSE_LIGHT == 1 << 31


def test_single_triangle_hand_values():
    tri = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0]]], np.float64)
    sc = kit.build([(tri, (0.5, 0.5, 0.5), False)],
                   lambda f: [Light(LIGHT_POINT, (0, 0, 5), n_paths=1)], diag=1.0)
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    down = [0.0, 0.0, -1.0]
    prim, t, amb = o.closest_hit([0.25, 0.25, 1.0], down, 1e-5)
    assert (prim, amb) == (0, False) and t == pytest.approx(1.0, abs=1e-15)
    prim, t, amb = o.closest_hit([0.5 + 1e-9, 0.5, 1.0], down, 1e-5)     # 7e-10 from an edge
    assert amb
    prim, t, amb = o.closest_hit([0.5 + 1e-3, 0.5, 1.0], down, 1e-5)     # outside by 7e-4
    assert (prim, amb) == (-1, False)
    prim, t, amb = o.closest_hit([0.5 - 1e-3, 0.5, 1.0], down, 1e-5)
    assert (prim, amb) == (0, False)
    prim, t, amb = o.closest_hit([0.25, 0.25, -1.0], down, 1e-5)         # behind the ray
    assert (prim, amb) == (-1, False)
    prim, t, amb = o.closest_hit([0.25, 0.25, 1e-5 + 1e-8], down, 1e-5)  # plane at t_min
    assert amb


def _moller_trumbore(V, o, d):
    """Independent closest hit: Moller & Trumbore (1997) in float64."""
    e1 = V[:, 1] - V[:, 0]
    e2 = V[:, 2] - V[:, 0]
    p = np.cross(d[None, :], e2)
    det = np.einsum("ij,ij->i", e1, p)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / det
        s = o[None, :] - V[:, 0]
        u = np.einsum("ij,ij->i", s, p) * inv
        q = np.cross(s, e1)
        v = (q @ d) * inv
        t = np.einsum("ij,ij->i", e2, q) * inv
    ok = (np.abs(det) > 1e-14) & (u >= 0) & (v >= 0) & (u + v <= 1)
    return t, ok, np.minimum(np.minimum(u, v), 1 - u - v)


def test_closest_hit_matches_independent_brute_force():
    sc = scenes.tiny_box()
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    V = sc.world_verts(1)
    rng = np.random.default_rng(5)
    tmin = 1e-5 * sc.diag
    checked = 0
    for _ in range(3000):
        org = rng.uniform([-0.95, 0.05, -0.95], [0.95, 1.95, 0.95])
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        prim, t, amb = o.closest_hit(org, d, tmin)
        if amb:
            continue
        tt, ok, margin = _moller_trumbore(V, org, d)
        ok &= tt > tmin
        if ok.any():
            k = int(np.argmin(np.where(ok, tt, np.inf)))
            if margin[k] < 1e-9:
                continue
            assert prim == k and t == pytest.approx(tt[k], rel=1e-12)
        else:
            assert prim == -1
        checked += 1
    assert checked > 2900


def test_single_bounce_irradiance_closed_form():
    """First-bounce deposit of an isotropic point light over a plane equals
    Phi * h / (4 pi (h^2 + r^2)^{3/2}) integrated over each texel (5 sigma)."""
    N, h = 400_000, 1.0
    sc = kit.floor_and_light(N, h=h, power=1.0, B=1)
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    p = o.trace(np.arange(N, dtype=np.uint32), seed=3, frame=1)
    W = 16
    atlas = oracle.deposit(p, W, W, (-2.0, -2.0, 2.0, 2.0))[..., 0]
    # exact texel integral of the irradiance by a 32x32 midpoint rule per texel
    edges = np.linspace(-2.0, 2.0, W + 1)
    sub = 32
    exp = np.zeros((W, W))
    for j in range(W):
        zs = edges[j] + (np.arange(sub) + 0.5) * (edges[j + 1] - edges[j]) / sub
        for i in range(W):
            xs = edges[i] + (np.arange(sub) + 0.5) * (edges[i + 1] - edges[i]) / sub
            X, Z = np.meshgrid(xs, zs)
            E = h / (4 * np.pi * (h * h + X * X + Z * Z) ** 1.5)
            exp[j, i] = E.mean() * (edges[1] - edges[0]) ** 2
    w = 1.0 / N                        # energy of one photon
    prob = exp / w / N                 # probability a path lands in the texel
    sigma = w * np.sqrt(N * prob * (1 - prob))
    z = (atlas - exp) / sigma
    inner = (slice(1, W - 1), slice(1, W - 1))      # the border texels also collect clamped photons
    assert np.abs(z[inner]).max() < 5.0
    e_in = exp[inner].sum()
    assert abs(atlas[inner].sum() / e_in - 1) < 5 * math.sqrt((1 - e_in) / (N * e_in))


def test_russian_roulette_energy_and_cosine_sampling():
    N = 100_000
    alb = (0.3, 0.5, 0.8)
    sc = kit.two_planes(N, albedo=alb, B=7)
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    p = o.trace(np.arange(N, dtype=np.uint32), seed=9, frame=1)
    L = p.nseg.astype(np.int64)
    q = 0.8
    # survival: P(L >= k+1 | L >= k) = q for k = 1..6 (binomial, 5 sigma)
    for k in range(1, 7):
        n_k = int((L >= k).sum())
        n_k1 = int((L >= k + 1).sum())
        assert abs(n_k1 - q * n_k) < 5 * math.sqrt(n_k * q * (1 - q)) + 1
    # energies: E1 = P/N exactly (as float32), E_{k+1} = E_k * rho / q
    E = p.photons[..., 4:7].astype(np.float64)
    sel = L >= 1
    assert np.all(p.photons[sel, 0, 4:7] == np.float32(1.0 / N))
    ratio = np.array(alb, np.float64) / q
    for k in range(1, 7):
        s = L >= k + 1
        want = E[s, k - 1] * ratio
        assert np.allclose(E[s, k], want, rtol=2e-7, atol=0)
    # cosine-weighted bounce directions: E[cos] = 2/3, E[cos^2] = 1/2
    P = p.photons[..., :3].astype(np.float64)
    s = L >= 2
    dv = P[s, 1] - P[s, 0]
    c = np.abs(dv[:, 1]) / np.linalg.norm(dv, axis=1)
    n = c.shape[0]
    assert abs(c.mean() - 2 / 3) < 5 * math.sqrt(1 / 18 / n)
    assert abs((c * c).mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)


def _traced(scene, n=None, seed=1, frame=1):
    o = oracle.OracleScene(scene)
    o.set_frames(frame, frame)
    n = scene.n_paths if n is None else n
    return o, o.trace(np.arange(n, dtype=np.uint32), seed=seed, frame=frame)


@pytest.mark.parametrize("mode,flags", [(0, 0), (1, 0), (2, 0), (2, oracle.FLAG_ERROR_EXACT)])
def test_static_scene_full_reuse(mode, flags):
    """No motion: every path is reused unchanged (Sec. 3)."""
    sc = kit.box_with_torus(3000)
    o, p = _traced(sc)
    q = p.copy()
    o.set_frames(1, 1)
    mask, st = o.verify(q, mode, 0.0, flags)
    assert (mask == 0).all() and len(oracle.compact(q.info)) == 0
    assert np.array_equal(q.info, p.info) and np.array_equal(q.photons, p.photons)
    assert np.array_equal(q.origin, p.origin)
    assert st["cont_rays"] == 0


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_object_moved_outside_paths_invalidates_nothing(mode):
    sc0 = scenes.tiny_box(n_paths=3000)
    cube = sc0.verts[sc0.tri_object == 1].astype(np.float64)
    shell = sc0.verts[sc0.tri_object == 0].astype(np.float64)
    xf = kit.translate(2, {1: lambda f: (3.0 + 0.05 * (f - 1), 1.0, 0.0)})
    sc = kit.build([(shell, (0.7,) * 3, False), (cube, (0.7,) * 3, True)], sc0._light_fn, xf, B=3,
                   diag=sc0.diag)
    o, p = _traced(sc)
    o.set_frames(1, 2)
    q = p.copy()
    mask, st = o.verify(q, mode, 0.01)
    assert st["segments_tested"] > 1000
    assert (mask == 0).all() and np.array_equal(q.photons, p.photons) and np.array_equal(q.info, p.info)


def test_inclusions_aabb_exact_error():
    """Boxes are conservative (Sec. 3.2): naive-AABB retraces a superset of
    naive-exact, from no later a vertex; error mode (Sec. 3.3) retraces a
    subset of naive-exact."""
    sc = kit.box_with_torus(6000)
    o, p = _traced(sc)
    o.set_frames(1, 2)
    res = {}
    for mode in (0, 1, 2):
        q = p.copy()
        o.verify(q, mode, 0.01)
        res[mode] = q
    amb = (res[0].amb | res[1].amb | res[2].amb) != 0
    lists = {m: set(np.nonzero(((res[m].info & oracle.INFO_REPLACE) != 0) & ~amb)[0]) for m in res}
    assert len(lists[1]) > 50
    assert lists[1] <= lists[0]
    assert len(lists[0]) > len(lists[1])
    assert lists[2] <= lists[1]
    both = sorted(lists[1])
    assert (res[0].start[both] <= res[1].start[both]).all()


def test_ordered_suffix_untouched():
    """Vertices before the first intersected segment are never modified
    (Sec. 3.2): true for every mode, before and after re-tracing."""
    sc = kit.box_with_torus(4000)
    o, p = _traced(sc)
    o.set_frames(1, 2)
    for mode in (0, 1, 2):
        q = p.copy()
        mask, _ = o.verify(q, mode, 0.01)
        first = np.array([(int(m) & -int(m)).bit_length() - 1 if m else 99 for m in mask])
        o.retrace(q, seed=1, frame=2)
        for i in np.nonzero(mask)[0]:
            keep = first[i] - 1            # photons 1..first-1 precede the segment
            assert np.array_equal(q.photons[i, :keep], p.photons[i, :keep])


def test_error_mode_monotone_in_tau():
    """E_N is always compared with the original E_O (Sec. 3.3), so a larger
    threshold never re-traces a path a smaller one keeps, nor from earlier."""
    sc = kit.box_with_torus(6000)
    o, p = _traced(sc)
    o.set_frames(1, 2)
    taus = [0.0, 0.005, 0.01, 0.05, 0.2, math.inf]
    out = []
    for tau in taus:
        q = p.copy()
        _, st = o.verify(q, 2, tau)
        out.append((q, st))
    amb = np.zeros(p.ids.shape[0], bool)
    for q, _ in out:
        amb |= q.amb != 0
    prev = None
    for (q, st), tau in zip(out, taus):
        rep = ((q.info & oracle.INFO_REPLACE) != 0) & ~amb
        if prev is not None:
            prq, prep = prev
            assert not (rep & ~prep).any()
            both = rep & prep
            assert (q.start[both] >= prq.start[both]).all()
        prev = (q, rep)
    assert out[-1][1]["n_tail"] == 0
    assert out[0][1]["n_tail"] > out[-2][1]["n_tail"]


def test_error_mode_rays_bounded_by_full_invalidation():
    """Alg. 1 traces at most one ray per segment from the first intersected
    one to the end of the path (Sec. 3.3: never more rays than re-tracing)."""
    sc = kit.box_with_torus(1500)
    o, p = _traced(sc)
    o.set_frames(1, 2)
    q = p.copy()
    mask, _ = o.verify(q, 0, 0.01)      # box test: same mask as error mode
    for i in np.nonzero(mask)[0][:300]:
        first = (int(mask[i]) & -int(mask[i])).bit_length() - 1
        one = oracle.Paths(p.ids[i:i + 1].copy(), p.info[i:i + 1].copy(), p.origin[i:i + 1].copy(),
                           p.photons[i:i + 1].copy(), p.amb[i:i + 1].copy())
        _, st = o.verify(one, 2, 0.01)
        assert st["cont_rays"] <= int(p.nseg[i]) - first + 1


def test_area_light_in_plane_translation_closed_form():
    """A light translated within its plane keeps every stored direction, so
    origins stay put and a path fails only if its origin leaves the light:
    fraction = shift / width (Sec. 3.1)."""
    N = 100_000
    sc = kit.rect_light_over_floor(N, shift=lambda f: (0.1 * (f - 1), 0.0, 0.0), R=1000.0)
    o, p = _traced(sc)
    o.set_frames(1, 2)
    q = p.copy()
    _, st = o.verify(q, 2, 0.01)
    frac = st["n_reemit"] / N
    assert abs(frac - 0.1) < 5 * math.sqrt(0.09 / N)
    ok = (q.info & oracle.INFO_REPLACE) == 0
    assert np.abs(q.origin[ok] - p.origin[ok]).max() <= 1e-6
    # no motion: origins unchanged bit for bit
    o.set_frames(1, 1)
    r = p.copy()
    o.verify(r, 2, 0.01)
    assert np.array_equal(r.origin, p.origin)


def test_area_light_failed_update_keeps_origin():
    """Sec. 3.1: DM_C counts only the paths "successfully updated"; the others
    are invalidated during the origin update.  A path whose update fails keeps
    the origin it had (its info word carries the decision; the re-trace emits
    it afresh), and a path whose update succeeds gets the point where its
    stored direction meets the new light plane, inside the rectangle."""
    N = 20_000
    a = math.radians(6.0)
    # lifted by 0.4 m, moved 0.3 m in x and tilted: some paths leave the rectangle, some fail Eq. 2 at tau = 2 %
    sc = kit.rect_light_over_floor(N, shift=lambda f: (0.3 * (f - 1), 0.4 * (f - 1), 0.0),
                                   normal=lambda f: (0.0, -1.0, 0.0) if f == 1 else (0.0, -math.cos(a), math.sin(a)))
    o, p = _traced(sc)
    o.set_frames(1, 2)
    for tau in (math.inf, 0.02):
        q = p.copy()
        _, st = o.verify(q, 2, tau)
        failed = ((q.info & oracle.INFO_REPLACE) != 0) & (q.start == 0)
        kept = ~failed & (p.nseg > 0)
        assert 0.05 * N < failed.sum() < 0.95 * N
        assert np.array_equal(q.origin[failed], p.origin[failed])
        L2 = sc.lights(2)[0]
        c = np.array(L2.pos, np.float64)
        n = np.array(L2.normal, np.float64)
        t = np.array(L2.tangent, np.float64)
        b = np.cross(n, t)
        org = q.origin[kept].astype(np.float64)
        assert np.abs((org - c) @ n).max() < 1e-5            # on the new plane
        assert (np.abs((org - c) @ t) <= 0.5 + 1e-5).all() and (np.abs((org - c) @ b) <= 0.5 + 1e-5).all()
        x1 = p.photons[kept, 0, :3].astype(np.float64)
        d_old = x1 - p.origin[kept]
        d_new = x1 - org
        cosang = (d_old * d_new).sum(1) / np.linalg.norm(d_old, axis=1) / np.linalg.norm(d_new, axis=1)
        assert (cosang > 1.0 - 1e-9).all()                     # the stored direction is kept
        if tau == math.inf:
            inf_failed = failed.sum()
        else:
            assert st["energy_tests"] > 0 and failed.sum() > inf_failed


def test_area_light_flip_and_tilt():
    N = 20_000
    flip = kit.rect_light_over_floor(N, normal=lambda f: (0.0, -1.0, 0.0) if f == 1 else (0.0, 1.0, 0.0))
    o, p = _traced(flip)
    o.set_frames(1, 2)
    q = p.copy()
    _, st = o.verify(q, 2, math.inf)
    assert st["n_reemit"] == N
    a = math.radians(5.0)
    tilt = kit.rect_light_over_floor(N, normal=lambda f: (0.0, -1.0, 0.0) if f == 1 else (0.0, -math.cos(a), math.sin(a)))
    o, p = _traced(tilt)
    o.set_frames(1, 2)
    q = p.copy()
    _, st_inf = o.verify(q, 2, math.inf)
    q = p.copy()
    _, st_0 = o.verify(q, 2, 0.0)
    assert st_0["n_reemit"] > st_inf["n_reemit"]
    assert st_inf["energy_tests"] > 0.8 * N


def _alg1_scene(kind):
    R = 2.0
    floor = kit.quad((-R, 0, -R), (0, 0, 2 * R), (2 * R, 0, 0))
    ceil = kit.quad((-R, 2, -R), (2 * R, 0, 0), (0, 0, 2 * R))
    if kind == "square":
        occ = kit.quad((-0.1, 0, -0.1), (0, 0, 0.2), (0.2, 0, 0))
        pose = {1: (5.0, 1.0, 0.5), 2: (0.03, 1.0, 0.5)}
    else:
        occ = np.array([[[-0.2, 0, -0.2], [0.2, 0, -0.2], [0.2, 0, 0.1]]], np.float64)
        pose = {1: (5.0, 1.0, 0.5), 2: (0.0, 1.0, 0.5)}
    parts = [(floor, (0.5,) * 3, False), (ceil, (0.5,) * 3, False), (occ, (0.5,) * 3, True)]
    lights = lambda f: [Light(LIGHT_POINT, (0.0, 1.9, 0.5), power=(0.01,) * 3, n_paths=1)]
    sc = kit.build(parts, lights, kit.translate(3, {2: lambda f: pose[f]}), B=3, diag=6.0)
    o = oracle.OracleScene(sc)
    o.set_frames(1, 2)
    ph = np.zeros((1, 3, 8), np.float32)
    ph[0, 0, :3] = (0.0, 0.0, 0.5)
    ph[0, 1, :3] = (0.5, 2.0, 0.0)
    ph[0, :2, 4:7] = 0.01
    prim = ph[..., 3].view(np.int32)
    prim[0, 0], prim[0, 1] = 0, 2
    p = oracle.Paths(np.zeros(1, np.uint32), np.array([2 << 22], np.uint32),
                     np.array([[0.0, 1.9, 0.5]], np.float32), ph, np.zeros(1, np.uint32))
    return o, p


def test_alg1_hand_built_occluder():
    g = json.load(open(os.path.join(GOLDEN, "alg1_cases.json")))["occluder_square"]
    o, p = _alg1_scene("square")
    for tau, exp in ((g["tau_fail"], g["expect_fail"]), (g["tau_pass"], g["expect_pass"])):
        q = p.copy()
        _, st = o.verify(q, 2, tau)
        assert q.amb[0] == 0
        assert int(q.nseg[0]) == exp["nseg"] and bool(q.info[0] & oracle.INFO_REPLACE) == exp["replace"]
        assert st["cont_rays"] == exp["cont_rays"]
        assert np.allclose(q.photons[0, 0, :3], exp["x1"], atol=1e-6) and int(q.prim[0, 0]) == exp["prim1"]
        if exp["replace"]:
            assert int(q.start[0]) == exp["start"]
        else:
            assert np.allclose(q.photons[0, 1, :3], exp["x2"], atol=1e-6) and int(q.prim[0, 1]) == exp["prim2"]
        assert np.array_equal(q.photons[0, :, 4:7], p.photons[0, :, 4:7])   # energy never rewritten
    # the ratio itself: between the two thresholds
    assert g["tau_fail"] < 1 - g["ratio"] < g["tau_pass"]
    for mode in (0, 1):
        q = p.copy()
        o.verify(q, mode, 0.01)
        e = g["expect_naive"]
        assert int(q.nseg[0]) == e["nseg"] and int(q.start[0]) == e["start"]
        assert bool(q.info[0] & oracle.INFO_REUSE_LIGHT) == e["reuse_light"]


def test_alg1_hand_built_skip_branch():
    g = json.load(open(os.path.join(GOLDEN, "alg1_cases.json")))["aabb_only_triangle"]
    o, p = _alg1_scene("triangle")
    q = p.copy()
    mask, st = o.verify(q, 2, 0.0)
    e = g["expect_error"]
    assert int(mask[0]) == 0b10 and q.amb[0] == 0
    assert st["cont_rays"] == e["cont_rays"] and not (q.info[0] & oracle.INFO_REPLACE)
    assert np.array_equal(q.photons, p.photons) and np.array_equal(q.info, p.info)
    q = p.copy()
    o.verify(q, 0, 0.0)
    e = g["expect_naive_aabb"]
    assert int(q.nseg[0]) == e["nseg"] and bool(q.info[0] & oracle.INFO_REUSE_LIGHT)
    q = p.copy()
    mask, _ = o.verify(q, 1, 0.0)
    assert int(mask[0]) == 0 and np.array_equal(q.photons, p.photons)


def test_point_light_visibility_when_light_moves():
    """A point light moved behind a wall can no longer see x1 (Sec. 3.1)."""
    R = 2.0
    floor = kit.quad((-R, 0, -R), (0, 0, 2 * R), (2 * R, 0, 0))
    wall = kit.quad((0.5, 0, -R), (0, 0, 2 * R), (0, 1.0, 0))           # x = 0.5, height 1
    lights = lambda f: [Light(LIGHT_POINT, (0.0 if f == 1 else 1.0, 0.5, 0.3), power=(1.0,) * 3, n_paths=4000)]
    sc = kit.build([(floor, (0.5,) * 3, False), (wall, (0.5,) * 3, False)], lights, B=1, diag=6.0)
    o, p = _traced(sc)
    o.set_frames(1, 2)
    q = p.copy()
    _, st = o.verify(q, 0, 0.01)
    x = p.photons[:, 0, 0]
    on_floor_left = (p.nseg >= 1) & (p.prim[:, 0] < 2) & (x < 0.5 - 1e-3)
    rep = (q.info & oracle.INFO_REPLACE) != 0
    assert st["vis_rays"] == int((p.nseg >= 1).sum())
    # light now at x=1 behind the wall: every floor photon left of the wall is blocked
    assert rep[on_floor_left].all()
    assert (q.origin[p.nseg >= 1] == np.float32([1.0, 0.5, 0.3])).all()


def test_deposit_sum_and_texel_edges():
    sc = kit.box_with_torus(2000)
    o, p = _traced(sc)
    atlas = oracle.deposit(p, 64, 32, sc.atlas_rect)
    L = p.nseg
    tot = sum(p.photons[i, :L[i], 4:7].astype(np.float64).sum(axis=0) for i in range(len(L)))
    assert np.allclose(atlas.sum(axis=(0, 1)), tot, rtol=1e-12)
    # texel decisions at the borders of the window (clamped)
    ph = np.zeros((5, 1, 8), np.float32)
    ph[:, 0, 0] = [-1.0, 1.0, -5.0, 0.0, np.nan]
    ph[:, 0, 2] = [-1.0, 1.0, 5.0, -1.0 + 2.0 / 32 * 0.5, 0.0]
    ph[:, 0, 4:7] = 1.0
    q = oracle.Paths(np.arange(5, dtype=np.uint32), np.full(5, 1 << 22, np.uint32), np.zeros((5, 3), np.float32),
                     ph, np.zeros(5, np.uint32))
    a = oracle.deposit(q, 64, 32, (-1.0, -1.0, 1.0, 1.0))[..., 0]
    assert a[0, 0] == 1 + 0      # (-1,-1) -> texel (0,0)
    assert a[31, 63] == 1        # (1,1) clamped to the last texel
    assert a[31, 0] == 1         # x below -> 0, z above -> last row
    assert a[0, 32] == 1         # x = 0 -> column 32, z in the first row
    assert a[16, 0] == 1         # NaN x -> column 0, z = 0 -> row 16
