"""The texel-edge rule of the sampled deposit check (CPU): a photon moved
across a texel edge by less than the band is accepted in either texel, a
moved one's energy must still be somewhere, and a photon moved by more than
the band, or a lost photon, fails."""
import numpy as np
import pytest

import oracle
import scenes
from tests import gpu_util as gu


@pytest.fixture(scope="module")
def traced():
    sc = scenes.tiny_box(4000)
    o = oracle.OracleScene(sc)
    o.set_frames(1, 1)
    return sc, o.trace(np.arange(sc.n_paths, dtype=np.uint32), sc.seed, 1)


def _edge_photon(q, W, rect):
    """A stored photon, and the x shift that moves it just across its texel's
    upper edge."""
    t = oracle.photon_texels(q, W, W, rect)
    i, k = map(int, np.argwhere(t[..., 0] >= 0)[0])
    x0, x1 = rect[0], rect[2]
    edge = x0 + (t[i, k, 0] + 1) * (x1 - x0) / W
    return i, k, np.float32(edge - q.photons[i, k, 0])


def test_moves_within_the_band_pass_and_beyond_it_fail(traced):
    sc, q = traced
    W, S = 64, 40
    rect = sc.atlas_rect
    base = oracle.deposit(q, W, W, rect)
    assert gu.check_deposit(base, q, W, W, rect, S, 0.0) == 0
    i, k, dx = _edge_photon(q, W, rect)
    moved = q.copy()
    moved.photons[i, k, 0] += dx * np.float32(1.001)          # now one texel over
    got = oracle.deposit(moved, W, W, rect)
    assert not np.array_equal(got, base)
    with pytest.raises(AssertionError):
        gu.check_deposit(got, q, W, W, rect, S, 0.0)
    assert gu.check_deposit(got, q, W, W, rect, S, float(dx) * 1.01) >= 1
    lost = q.copy()                                          # a photon's energy missing altogether
    lost.photons[i, k, 4:7] = 0.0
    with pytest.raises(AssertionError):
        gu.check_deposit(oracle.deposit(lost, W, W, rect), q, W, W, rect, S, float(dx) * 1.01)
