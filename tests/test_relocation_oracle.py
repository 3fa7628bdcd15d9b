"""Pins of the oracle's probe relocation (Sec. 3.2, UpdateProbePos), CPU only.

The SDF of a plane bakes to an exactly linear field, so one Gauss-Newton step lands on
the clearance level to rounding. Near a sphere the probe moves radially to within the
bake bound of the level. The per-axis limit holds even when the surface is out of
reach, and such a probe ends inactive. Free probes stay put. History is rejected exactly
when the move from last frame's position exceeds threshold2.
"""
import numpy as np

import oracle as O
import workloads as W


def _scene(kind, **kw):
    s = W.Scene()
    if kind == "plane":
        s.add(W.PLANE_Y, [kw.get("y", 1.0)], (0.5, 0.5, 0.5))
    else:
        s.add(W.SPHERE, list(kw["c"]) + [kw["r"]], (0.5, 0.5, 0.5))
    return s


def _grid(dims, origin, spacing):
    return O.make_grid(dims, origin, spacing, 8, 64, 0.01, 300.0, 0.97)


def test_plane_one_step_to_the_clearance_level():
    h = 0.25
    baked = W.bake(_scene("plane", y=1.0), (32, 32, 32), h)
    osc = O.OracleScene(baked.sdf, h, (0, 0, 0), None)
    y0 = 1.0 + 0.25 * h  # a quarter voxel above the plane: inside the 2-voxel clearance
    g = _grid((2, 1, 2), (2.3, y0, 3.1), (2.0, 2.0, 2.0))
    r = O.relocate(osc, g, clearance_vox=2.0, reject_dist=0.0, max_offset=0.45)
    assert np.all(r["iters"] >= 1)
    assert np.allclose(r["pos"][:, 1], 1.0 + 2.0 * h, rtol=0, atol=1e-6)
    assert np.array_equal(r["pos"][:, 0], np.array([2.3, 4.3, 2.3, 4.3]))
    assert np.array_equal(r["pos"][:, 2], np.array([3.1, 3.1, 5.1, 5.1]))
    assert np.all(r["flags"] == 1)


def test_displacement_limit_and_a_probe_left_inside():
    h = 0.25
    baked = W.bake(_scene("plane", y=1.0), (32, 32, 32), h)
    osc = O.OracleScene(baked.sdf, h, (0, 0, 0), None)
    # 0.4 m under the surface: the level is 0.9 m away; a limit of 0.45 * 1 m stops it short
    g = _grid((1, 1, 1), (4.0, 0.6, 4.0), (1.0, 1.0, 1.0))
    r = O.relocate(osc, g, clearance_vox=2.0, reject_dist=0.0, max_offset=0.45, max_iters=16)
    assert abs(r["pos"][0, 1] - (0.6 + 0.45)) < 1e-12
    assert r["iters"][0] == 16
    assert r["flags"][0] == 0                       # 0.05 m = 0.2 voxel of clearance: not active
    # with a 2 m spacing the same probe reaches the level
    g = _grid((1, 1, 1), (4.0, 0.6, 4.0), (2.0, 2.0, 2.0))
    r = O.relocate(osc, g, clearance_vox=2.0, reject_dist=0.0, max_offset=0.45)
    assert abs(r["pos"][0, 1] - 1.5) < 1e-6 and r["flags"][0] == 1


def test_sphere_moves_radially_to_the_level():
    h, rad, c = 0.125, 1.5, np.array([4.0, 4.0, 4.0])
    baked = W.bake(_scene("sphere", c=c, r=rad), (64, 64, 64), h)
    osc = O.OracleScene(baked.sdf, h, (0, 0, 0), None)
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    home = c + (rad + 0.1) * u                      # 0.8 voxel outside the surface
    g = _grid((1, 1, 1), home, (2.0, 2.0, 2.0))
    r = O.relocate(osc, g, clearance_vox=3.0, reject_dist=0.0)
    p = r["pos"][0]
    bake_bound = 3 * h * h / (8 * rad) + 1e-3      # Taylor bound of the baked sphere + trilinear slack
    assert abs(np.linalg.norm(p - c) - (rad + 3.0 * h)) <= bake_bound
    assert np.linalg.norm(np.cross((p - c) / np.linalg.norm(p - c), u)) < 2e-3
    assert r["flags"][0] == 1


def test_free_probes_stay_and_history_rejection_rule():
    h = 0.25
    baked = W.bake(_scene("plane", y=1.0), (32, 32, 32), h)
    osc = O.OracleScene(baked.sdf, h, (0, 0, 0), None)
    g = _grid((2, 2, 1), (2.0, 4.0, 4.0), (1.0, 1.0, 1.0))   # 3 m and more above the plane
    home = W.probe_grid_positions((2, 2, 1), (2.0, 4.0, 4.0), (1.0, 1.0, 1.0))
    r = O.relocate(osc, g, clearance_vox=2.0, reject_dist=0.2)
    assert np.array_equal(r["pos"], home) and np.all(r["iters"] == 0) and np.all(r["flags"] == 1)
    last = home + np.array([[0.0, 0.3, 0.0], [0.0, 0.1, 0.0], [0.2, 0.0, 0.05], [0.0, 0.0, 0.0]])
    r = O.relocate(osc, g, clearance_vox=2.0, reject_dist=0.2, last_pos=last)
    dist = np.linalg.norm(home - last.astype(np.float32).astype(np.float64), axis=1)
    assert np.array_equal(r["flags"], np.where(dist > 0.2, 3, 1).astype(np.uint32))
    assert np.allclose(r["margin"][:, 1], dist - 0.2)
    r = O.relocate(osc, g, clearance_vox=2.0, reject_dist=0.0, last_pos=last)
    assert np.all(r["flags"] == 1)                   # threshold2 <= 0: no rejection
    r = O.relocate(osc, g, clearance_vox=0.0, reject_dist=0.0)
    assert np.array_equal(r["pos"], home)             # threshold1 <= 0: no probe moves
