"""Small hand-built scenes for the oracle pins and the GPU parity tests."""
from __future__ import annotations

import math

import numpy as np

import scenes
from scenes import LIGHT_POINT, LIGHT_RECT, Light, Scene


def quad(o, eu, ev, n=1):
    return scenes._quad_grid(o, eu, ev, n, n)


def build(parts, lights_fn, xform_fn=None, B=3, diag=1.0, rect=(-1.0, -1.0, 1.0, 1.0),
          name="kit", seed=7):
    """parts: list of (tris [K,3,3], albedo rgb, dynamic) -> Scene."""
    b = scenes._Builder()
    for tris, alb, dyn in parts:
        b.add(np.asarray(tris, np.float64), alb, dynamic=dyn)
    verts, obj, dyn, alb = b.arrays()
    n_obj = dyn.shape[0]
    if xform_fn is None:
        xform_fn = lambda f: scenes._identity_xforms(n_obj)
    return Scene(name, verts, obj, dyn, alb, max_bounces=B, diag=diag, atlas_rect=rect,
                 seed=seed, frames=2, tau=0.01, _xform_fn=xform_fn, _light_fn=lights_fn)


def translate(n_obj, moves):
    """xform function: moves = {object: callable(frame) -> (x, y, z)}."""
    def f(frame):
        x = scenes._identity_xforms(n_obj)
        for o, fn in moves.items():
            x[o, 3], x[o, 7], x[o, 11] = fn(frame)
        return x
    return f


def floor_and_light(n_paths, h=1.0, R=20.0, power=4.0 * math.pi, B=1):
    """Large floor quad at y = 0 and an isotropic point light at height h."""
    parts = [(quad((-R, 0, -R), (0, 0, 2 * R), (2 * R, 0, 0)), (0.5, 0.5, 0.5), False)]
    lights = lambda f: [Light(LIGHT_POINT, (0.0, h, 0.0), power=(power,) * 3, n_paths=n_paths)]
    return build(parts, lights, B=B, diag=2 * R * math.sqrt(2), rect=(-2.0, -2.0, 2.0, 2.0))


def two_planes(n_paths, albedo=(0.3, 0.5, 0.8), B=7, R=1000.0):
    """Floor y = 0 and ceiling y = 1 (both huge) with a point light between."""
    parts = [(quad((-R, 0, -R), (0, 0, 2 * R), (2 * R, 0, 0)), albedo, False),
             (quad((-R, 1, -R), (2 * R, 0, 0), (0, 0, 2 * R)), albedo, False)]
    lights = lambda f: [Light(LIGHT_POINT, (0.0, 0.5, 0.0), power=(1.0, 1.0, 1.0), n_paths=n_paths)]
    return build(parts, lights, B=B, diag=10.0, rect=(-5.0, -5.0, 5.0, 5.0))


def rect_light_over_floor(n_paths, shift=lambda f: (0.0, 0.0, 0.0), normal=lambda f: (0.0, -1.0, 0.0),
                          B=1, R=10.0):
    """Floor [-10,10]^2 and a 1x1 m area light at height 3 facing down; the
    light's pose per frame is pos = (0,3,0) + shift(f), normal(f)."""
    parts = [(quad((-R, 0, -R), (0, 0, 2 * R), (2 * R, 0, 0)), (0.5, 0.5, 0.5), False)]

    def lights(f):
        s = shift(f)
        return [Light(LIGHT_RECT, (s[0], 3.0 + s[1], s[2]), normal(f), (1.0, 0.0, 0.0), (1.0, 1.0),
                      (100.0, 100.0, 100.0), n_paths)]
    return build(parts, lights, B=B, diag=2 * R * math.sqrt(2), rect=(-R, -R, R, R))


def box_with_torus(n_paths, B=4, seed=11):
    """The tiny box's shell plus a vertical torus moving through it."""
    s0 = scenes.tiny_box(n_paths=n_paths)
    shell = s0.verts[s0.tri_object == 0].astype(np.float64)
    torus = scenes._torus(24, 12, 0.3, 0.1, vertical=True)
    parts = [(shell, (0.7, 0.6, 0.5), False), (torus, (0.4, 0.8, 0.6), True)]
    lights = lambda f: [Light(LIGHT_POINT, (0.0, 1.8, 0.0), power=(100.0, 100.0, 100.0), n_paths=n_paths)]
    xf = translate(2, {1: lambda f: (-0.3 + 0.08 * (f - 1), 0.9, 0.1 * (f - 1))})
    return build(parts, lights, xf, B=B, diag=math.sqrt(12.0), name="box_torus", seed=seed)
