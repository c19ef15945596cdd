"""The C-ABI library builds, loads and exports what include/*.h declare;
the Python structs match the C layout; host-side argument errors are
reported without touching a GPU (CPU only)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

import paper_2111_06906_gb300 as pv
from paper_2111_06906_gb300 import build as pvbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    pvbuild.build()
    return pv.load()


def _declared():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(pv_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert set(names) == set(pv.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", pv.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pv_\w+)", out))
    assert set(names) <= exported


def test_struct_layout_matches_header():
    probe = r"""
#include <stdio.h>
#include <stddef.h>
#include "pv.h"
#include "pv_batch.h"
#define S(t) printf(#t " %zu\n", sizeof(t));
#define O(t, f) printf(#t "." #f " %zu\n", offsetof(t, f));
int main(void) {
  S(pv_light) S(pv_scene_desc) S(pv_paths) S(pv_verify_params) S(pv_atlas) S(pv_frame_stats)
  O(pv_scene_desc, scene_diag) O(pv_scene_desc, flags) O(pv_paths, pb) O(pv_atlas, scale_log2)
  O(pv_light, n_paths) O(pv_frame_stats, photons_written)
  S(pv_batch_scene) S(pv_batch_config) O(pv_batch_scene, paths) O(pv_batch_scene, seed) O(pv_batch_config, stack)
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        open(c, "w").write(probe)
        exe = os.path.join(d, "probe")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = dict(l.rsplit(" ", 1) for l in subprocess.check_output([exe], text=True).splitlines())
    got = {k: int(v) for k, v in out.items()}
    assert got["pv_light"] == C.sizeof(pv.PvLight) == 64
    assert got["pv_scene_desc"] == C.sizeof(pv.PvSceneDesc)
    assert got["pv_paths"] == C.sizeof(pv.PvPaths)
    assert got["pv_verify_params"] == C.sizeof(pv.PvVerifyParams)
    assert got["pv_atlas"] == C.sizeof(pv.PvAtlas)
    assert got["pv_frame_stats"] == 4 * pv.STATS_WORDS
    assert got["pv_scene_desc.scene_diag"] == pv.PvSceneDesc.scene_diag.offset
    assert got["pv_scene_desc.flags"] == pv.PvSceneDesc.flags.offset
    assert got["pv_paths.pb"] == pv.PvPaths.pb.offset
    assert got["pv_atlas.scale_log2"] == pv.PvAtlas.scale_log2.offset
    assert got["pv_light.n_paths"] == pv.PvLight.n_paths.offset
    assert got["pv_frame_stats.photons_written"] == 4 * pv.STATS_FIELDS.index("photons_written")
    assert got["pv_batch_scene"] == C.sizeof(pv.PvBatchScene)
    assert got["pv_batch_config"] == C.sizeof(pv.PvBatchConfig)
    assert got["pv_batch_scene.paths"] == pv.PvBatchScene.paths.offset
    assert got["pv_batch_scene.seed"] == pv.PvBatchScene.seed.offset
    assert got["pv_batch_config.stack"] == pv.PvBatchConfig.stack.offset


def test_status_strings(lib):
    for code, text in [(0, "ok"), (-1, "invalid argument"), (-4, "BVH traversal stack overflow"),
                       (-5, "iteration cap reached"), (-6, "format limit exceeded"), (99, "unknown status")]:
        assert pv.pv_status_string(code) == text


def test_host_argument_errors_need_no_gpu(lib):
    h = C.c_void_p()
    assert lib.pv_build_scene(None, None, C.byref(h)) == -1
    assert lib.pv_build_scene(None, None, None) == -1
    # five lights: a format limit, found before any CUDA call
    import numpy as np
    v = np.zeros((1, 3, 3), np.float32)
    v[0, 1, 0] = v[0, 2, 2] = 1.0
    obj = np.zeros(1, np.uint32)
    dyn = np.zeros(1, np.uint8)
    alb = np.full((1, 3), 0.5, np.float32)

    class L:
        type, pos, normal, tangent, size, power, n_paths = 0, (0, 1, 0), (0, -1, 0), (1, 0, 0), (0, 0), (1, 1, 1), 10

    la = pv.make_lights([L] * 5)
    d = pv.PvSceneDesc(v.ctypes.data, 1, obj.ctypes.data, 1, dyn.ctypes.data, alb.ctypes.data, 0, 5,
                       C.cast(la, C.c_void_p), 3, 1.0, 0)
    assert lib.pv_build_scene(C.byref(d), None, C.byref(h)) == -6
    d.n_lights = 1
    d.max_bounces = 16
    assert lib.pv_build_scene(C.byref(d), None, C.byref(h)) == -6
    d.max_bounces = 3
    d.scene_diag = 0.0
    assert lib.pv_build_scene(C.byref(d), None, C.byref(h)) == -1
    bad = np.array([7], np.uint32)
    d.scene_diag = 1.0
    d.tri_object = bad.ctypes.data
    assert lib.pv_build_scene(C.byref(d), None, C.byref(h)) == -1
    assert lib.pv_update_dynamic(None, None, None, None) == -1
    assert lib.pv_verify_paths(None, None, None, None, None, None, None) == -1
    assert lib.pv_retrace_invalid(None, None, None, None, 0, 0, None, None) == -1
    assert lib.pv_trace_all(None, None, 0, 0, None, None) == -1
    assert lib.pv_compact_replace(None, None, None, None, None) == -1
    assert lib.pv_deposit(None, None, None, None) == -1
    assert lib.pv_read_device_status(None) == -1
    assert lib.pv_set_traversal_limit(None, 1) == -1
    assert lib.pv_stage_timing(None, 1) == -1
    assert lib.pv_trace_all_deposit(None, None, 1, 1, None, None, None) == -1
    fm = C.c_uint64(0)
    sink = C.c_void_p(16)
    assert lib.pv_fma_probe(0, 1, sink, C.byref(fm), None) == -1
    assert lib.pv_fma_probe(1, 0, sink, C.byref(fm), None) == -1
    assert lib.pv_fma_probe(1, 1, None, C.byref(fm), None) == -1
    lib.pv_destroy_scene(None)
    b = C.c_void_p()
    prm = pv.PvVerifyParams(2, 0.01, 0)
    assert lib.pv_batch_create(None, 1, C.byref(prm), None, C.byref(b)) == -1
    items = (pv.PvBatchScene * 40)()
    assert lib.pv_batch_create(items, 40, C.byref(prm), None, C.byref(b)) == -6
    assert lib.pv_batch_create(items, 0, C.byref(prm), None, C.byref(b)) == -1
    assert lib.pv_batch_frame(None, None, None, 0, None) == -1
    assert lib.pv_batch_autotune(None, 1) == -1
    assert lib.pv_batch_tuning(None) == -1
    assert lib.pv_batch_set_config(None, None) == -1
    assert lib.pv_batch_get_config(None, None) == -1
    lib.pv_batch_destroy(None)


def test_product_path_has_no_oracle_dependency():
    """The library and its binding never load the oracle (CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_2111_06906_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.replace("oracle-free", ""), f
