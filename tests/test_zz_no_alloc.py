"""The allocation-free compaction entry point (pv_compact_replace_static).

It serves callers that must not allocate device memory once running -- a
renderer that reserves its memory budget up front or whose device memory
belongs to another allocator, and frame loops that cannot take the
synchronisation an allocation may cause.  Its list and count must equal those
of the scene-based pv_compact_replace, on two calls in a row (the library's
fixed scratch array keeps the previous call's contents and must be cleared).
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import scenes
import paper_2111_06906_gb300 as pv
from tests import gpu_util as gu
from tests import scene_kit as kit


def test_rejects_sizes_beyond_the_limit():
    from paper_2111_06906_gb300 import build
    build.build()
    lib = pv.load()
    dummy = C.c_void_p(16)
    assert lib.pv_compact_replace_static(dummy, pv.PV_STATIC_COMPACT_MAX_PATHS + 1, dummy, dummy, None) == -6
    assert lib.pv_compact_replace_static(None, 10, None, dummy, None) == -1
    assert lib.pv_compact_replace_static(dummy, 10, dummy, None, None) == -1


@pytest.mark.gpu
@pytest.mark.parametrize("n", [3 * 4096 + 77, 100_003, pv.PV_STATIC_COMPACT_MAX_PATHS - 1,
                               pv.PV_STATIC_COMPACT_MAX_PATHS])
def test_matches_scene_compaction_on_two_calls_in_a_row(n):
    import torch
    from paper_2111_06906_gb300 import build
    build.build()
    lib = pv.load()
    lights = lambda f: [scenes.Light(scenes.LIGHT_POINT, (0.0, 1.0, 0.0), n_paths=n)]
    sc = kit.build([(kit.quad((-1, 0, -1), (0, 0, 2), (2, 0, 0)), (0.5,) * 3, False)], lights, B=1, diag=3.0)
    h = gu.lib_scene(sc)
    P = pv.Paths.allocate(n, 1)
    rng = np.random.default_rng(n)
    stream = torch.cuda.current_stream().cuda_stream
    for call, density in enumerate((0.3, 0.01)):        # dense then sparse: stale tile states would show
        bits = rng.random(n) < density
        info = np.where(bits, pv.PV_INFO_REPLACE, 0).astype(np.uint32) | (1 << 22)
        P.info.copy_(torch.as_tensor(info.view(np.int32), device="cuda"))
        ref_list = torch.zeros(n, dtype=torch.int32, device="cuda")
        ref_cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        pv.pv_compact_replace(h, P, ref_list, ref_cnt)
        got_list = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        got_cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rc = lib.pv_compact_replace_static(C.c_void_p(P.info.data_ptr()), n, C.c_void_p(got_list.data_ptr()),
                                           C.c_void_p(got_cnt.data_ptr()), C.c_void_p(stream))
        assert rc == 0, pv.pv_status_string(rc)
        torch.cuda.synchronize()
        c = int(ref_cnt.item())
        assert int(got_cnt.item()) == c == int(bits.sum())
        assert torch.equal(got_list[:c], ref_list[:c]), f"call {call}"
        if n >= pv.PV_STATIC_COMPACT_MAX_PATHS - 1:    # the array's last tile and its ticket word are in use
            assert np.array_equal(got_list[:c].cpu().numpy(), np.flatnonzero(bits).astype(np.int32))
    assert pv.pv_read_device_status(h) == 0
    pv.pv_destroy_scene(h)
    del P
    torch.cuda.empty_cache()
