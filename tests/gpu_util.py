"""Helpers for the GPU parity tests: build a library scene from a seeded
scene, move path records between the oracle's AoS form and the library's
SoA buffers, and compare them field by field."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2111_06906_gb300 as pv


def lib_scene(sc, flags: int = 0, frame: int = 1, dm_rect=(0, 0, 0, 0), dm_point=(0, 0)):
    return pv.pv_build_scene(sc.verts, sc.tri_object, sc.object_dynamic, sc.object_albedo, sc.lights(frame),
                             sc.max_bounces, sc.diag, object_xform=sc.xforms(frame), flags=flags, dm_rect=dm_rect,
                             dm_point=dm_point)


def advance(h, sc, frame: int) -> None:
    pv.pv_update_dynamic(h, sc.xforms(frame), sc.lights(frame))


def upload(paths: pv.Paths, op: oracle.Paths) -> None:
    """Write oracle records (positions op.ids) into the device buffers."""
    import torch
    ids = torch.as_tensor(op.ids.astype(np.int64), device=paths.info.device)
    paths.info[ids] = torch.as_tensor(op.info.view(np.int32), device=paths.info.device)
    paths.origin[:, ids] = torch.as_tensor(op.origin.T.copy(), device=paths.info.device)
    ph = np.ascontiguousarray(np.transpose(op.photons, (1, 0, 2)))      # [B, n, 8]
    paths.pa[:, ids] = torch.as_tensor(ph[..., 0:4].copy(), device=paths.info.device)
    paths.pb[:, ids] = torch.as_tensor(ph[..., 4:8].copy(), device=paths.info.device)


def download(paths: pv.Paths, ids=None) -> oracle.Paths:
    """Device buffers -> oracle-layout records (at ``ids``, default all)."""
    import torch
    if ids is None:
        ids = np.arange(paths.n, dtype=np.uint32)
    t = torch.as_tensor(np.asarray(ids).astype(np.int64), device=paths.info.device)
    info = paths.info[t].cpu().numpy().view(np.uint32).copy()
    origin = paths.origin[:, t].cpu().numpy().T.copy()
    pa = paths.pa[:, t].cpu().numpy()
    pb = paths.pb[:, t].cpu().numpy()
    ph = np.concatenate([np.transpose(pa, (1, 0, 2)), np.transpose(pb, (1, 0, 2))], axis=2).copy()
    return oracle.Paths(np.asarray(ids, np.uint32), info, origin, ph, np.zeros(len(ids), np.uint32))


def compare(gpu: oracle.Paths, orc: oracle.Paths, diag: float, skip=None, pos_tol=1e-5, e_rtol=1e-5,
            check_info_bits=True):
    """Field-by-field comparison of two record sets (same ids), skipping the
    paths the oracle marks ambiguous.  Returns a dict of counts; every
    ``bad_*`` entry must be zero for parity."""
    amb = orc.amb != 0
    if skip is not None:
        amb = amb | skip
    ok = ~amb
    r = {"n": int(len(gpu.ids)), "ambiguous": int(amb.sum())}
    gi, oi = gpu.info[ok], orc.info[ok]
    if check_info_bits:
        r["bad_info"] = int((gi != oi).sum())
    else:
        r["bad_info"] = int((((gi >> 22) & 15) != ((oi >> 22) & 15)).sum())
    L = np.minimum((gi >> 22) & 15, (oi >> 22) & 15)
    B = gpu.photons.shape[1]
    kk = np.arange(B)[None, :] < L[:, None]
    gp, op = gpu.photons[ok], orc.photons[ok]
    r["bad_prim"] = int(((gp[..., 3].view(np.int32) != op[..., 3].view(np.int32)) & kk).sum())
    dpos = np.abs(gp[..., :3].astype(np.float64) - op[..., :3]).max(axis=-1)
    r["bad_pos"] = int(((dpos > pos_tol * diag) & kk).sum())
    r["max_dpos_over_diag"] = float((dpos * kk).max() / diag) if kk.any() else 0.0
    eo = op[..., 4:7].astype(np.float64)
    de = np.abs(gp[..., 4:7] - eo) / np.maximum(np.abs(eo), 1e-30)
    r["bad_energy"] = int(((de > e_rtol).any(axis=-1) & kk).sum())
    r["max_rel_denergy"] = float((de.max(axis=-1) * kk).max()) if kk.any() else 0.0
    drad = np.abs(gp[..., 7].astype(np.float64) - op[..., 7])
    r["bad_radius"] = int(((drad > e_rtol * np.abs(op[..., 7]) + pos_tol * diag) & kk).sum())
    do = np.abs(gpu.origin[ok].astype(np.float64) - orc.origin[ok]).max(axis=-1)
    r["bad_origin"] = int((do > pos_tol * diag).sum())
    return r


def assert_parity(r: dict) -> None:
    bad = {k: v for k, v in r.items() if k.startswith("bad_") and v}
    assert not bad, r
