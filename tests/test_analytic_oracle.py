"""Pins of the oracle's analytic scene (the paper's SDF primitives, Sec. 3.1), CPU only.

Each primitive's distance against its closed form; the union's minimum, owner and tie
rule; agreement with the FP64 bake (a separate implementation) at voxel centres; the
white furnace through a full update of an analytic closed room; and per-ray materials
against ray-sphere intersection in closed form.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def ascene(s: W.Scene, dims, h, origin=(0.0, 0.0, 0.0)):
    t, p = s.arrays()
    return O.OracleScene.analytic(t, p, s.albedo, s.emission, origin, dims, h)


def _one(t, params):
    s = W.Scene()
    s.add(t, params, (0.5, 0.5, 0.5))
    return ascene(s, (8, 8, 8), 1.0)


@pytest.mark.parametrize("t,params,point,want", [
    (W.SPHERE, [1, 2, 3, 0.5], [1, 2, 4], 0.5),
    (W.SPHERE, [1, 2, 3, 0.5], [1, 2, 3], -0.5),
    (W.BOX, [0, 0, 0, 1, 2, 3], [2, 0, 0], 1.0),
    (W.BOX, [0, 0, 0, 1, 2, 3], [2, 3, 0], 2 ** 0.5),
    (W.BOX, [0, 0, 0, 1, 2, 3], [0.5, 0, 0], -0.5),
    (W.BOX, [0, 0, 0, 1, 2, 3], [0, 0, -2.75], -0.25),
    (W.CAPSULE, [0, 0, 0, 0, 2, 0, 0.25], [1, 1, 0], 0.75),
    (W.CAPSULE, [0, 0, 0, 0, 2, 0, 0.25], [0, 3, 0], 0.75),
    (W.CAPSULE, [0, 0, 0, 0, 2, 0, 0.25], [0, -1, 0], 0.75),
    (W.PLANE_Y, [1.0], [5, 3, 2], 2.0),
    (W.INV_SPHERE, [0, 0, 0, 2], [1, 0, 0], 1.0),
    (W.INV_SPHERE, [0, 0, 0, 2], [3, 0, 0], -1.0),
])
def test_primitive_distances(t, params, point, want):
    d, own, _ = O.analytic_sdf(_one(t, params), np.array(point, dtype=float))
    assert abs(d - want) < 1e-15 and own == 0


def test_union_minimum_owner_and_ties():
    s = W.Scene()
    s.add(W.SPHERE, [0, 0, 0, 1], (0.1, 0.1, 0.1))
    s.add(W.SPHERE, [0, 0, 0, 1], (0.2, 0.2, 0.2))      # identical: ties go to the lower index
    s.add(W.BOX, [3, 0, 0, 0.5, 0.5, 0.5], (0.3, 0.3, 0.3))
    sc = ascene(s, (8, 8, 8), 1.0)
    d, own, sec = O.analytic_sdf(sc, np.array([0.0, 2.0, 0.0]))
    assert d == 1.0 and own == 0 and sec == 1.0
    d, own, sec = O.analytic_sdf(sc, np.array([2.25, 0.0, 0.0]))
    assert d == 0.25 and own == 2 and sec == 1.25


@pytest.mark.parametrize("kind", ["room", "open"])
def test_agrees_with_the_fp64_bake_at_voxel_centres(kind):
    if kind == "room":
        s, dims, h = W.room_scene(3), (16, 16, 16), 0.5
    else:
        s, dims, h = W.open_scene(5, size=16.0, n_prims=30), (16, 16, 16), 1.0
    b = W.bake(s, dims, h, keep64=True)
    sc = ascene(s, dims, h)
    nz, ny, nx = b.sdf64.shape
    rng = np.random.default_rng(0)
    for _ in range(600):
        x, y, z = (int(rng.integers(0, n)) for n in (nx, ny, nz))
        p = (np.array([x, y, z]) + 0.5) * h
        d, _, _ = O.analytic_sdf(sc, p)
        assert abs(d - b.sdf64[z, y, x]) < 1e-5          # float32-rounded primitive parameters


def test_white_furnace_analytic():
    Le = (0.5, 1.0, 2.0)
    s = W.room_scene(0, size=8.0, n_spheres=0, n_boxes=0, aperture=0.0, uniform_albedo=(0.0, 0.0, 0.0),
                     emission=Le, sun=False)
    s.add(W.SPHERE, [3.0, 3.0, 3.0, 1.2], (0.0, 0.0, 0.0), Le)
    sc = ascene(s, (32, 32, 32), 0.25)
    dims, org, sp = (4, 4, 4), (1.0, 1.0, 1.0), (2.0, 2.0, 2.0)
    st = W.probe_states(s, dims, org, sp, 0.25)
    g = O.make_grid(dims, org, sp, 32, 256, 0.01, 56.0, 0.97, k_bounce=1.0)
    out = O.update(sc, g, [], W.frame_rotation(3, 0), st)
    act = (st["flags"] & 1).astype(bool)
    assert np.allclose(out["irr"][act][:, 1:-1, 1:-1, :3], Le, rtol=1e-12)


def test_hit_materials_follow_the_nearest_primitive():
    """A closed room (emission 1) with a sphere of emission 5: a ray's radiance is 5 exactly
    when the ray meets the sphere (closed-form ray-sphere test) before the walls."""
    s = W.room_scene(0, size=8.0, n_spheres=0, n_boxes=0, aperture=0.0, uniform_albedo=(0.0, 0.0, 0.0),
                     emission=(1.0, 1.0, 1.0), sun=False)
    c, r = np.array([4.0, 4.0, 4.0]), 1.5
    s.add(W.SPHERE, list(c) + [r], (0.0, 0.0, 0.0), (5.0, 5.0, 5.0))
    sc = ascene(s, (32, 32, 32), 0.25)
    dims, org, sp = (2, 2, 2), (1.5, 1.5, 1.5), (5.0, 5.0, 5.0)
    st = W.probe_states(s, dims, org, sp, 0.25)
    g = O.make_grid(dims, org, sp, 64, 256, 0.01, 56.0, 0.0, k_bounce=0.0)
    rot = W.frame_rotation(2, 0)
    out = O.update(sc, g, [], rot, st)
    rays = out["rays"]
    for p in range(8):
        o = st["pos"][p].astype(np.float64)
        for i in range(64):
            d = rot.astype(np.float64) @ O.sf_dir(i, 64)
            oc = o - c
            b = np.dot(oc, d)
            disc = b * b - (np.dot(oc, oc) - r * r)
            hits_sphere = disc > 0 and -b - np.sqrt(disc) > 0
            want = 5.0 if hits_sphere else 1.0
            assert rays[p, i]["L"][0] == want, (p, i)
            assert rays[p, i]["owner"] == (s.types.__len__() if hits_sphere else rays[p, i]["owner"])
