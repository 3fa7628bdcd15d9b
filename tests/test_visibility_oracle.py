"""Pins of the oracle's interpolation with SDF probe visibility (Sec. 3.4), CPU only.

In open space every probe is visible, so the rule reduces to the plain interpolation,
bit for bit. A wall between probe columns hides the far column: a point in front of it
takes exactly the near column's irradiance, while the plain rule leaks the far one in.
Visibility grows with the softness parameter toward the hard binary test, stays in
[0, 1], and a point that sees no probe gets 0.
"""
import numpy as np

import oracle as O
import workloads as W


def _grid(dims, origin, spacing, bias_vox=1.0):
    return O.make_grid(dims, origin, spacing, 8, 128, 0.01, 300.0, 0.97, bias_vox=bias_vox)


def _maps(P, rng):
    irr = np.zeros((P, 8, 8, 4))
    irr[..., :3] = rng.uniform(0.1, 1.0, (P, 8, 8, 3))
    for p in range(P):
        irr[p] = O.border(irr[p])
    return irr


def test_open_space_equals_plain_interpolation():
    rng = np.random.default_rng(1)
    s = W.Scene()
    s.add(W.PLANE_Y, [0.1], (0.5, 0.5, 0.5))
    baked = W.bake(s, (64, 64, 64), 0.125)
    sc = O.OracleScene(baked.sdf, 0.125, (0, 0, 0), None)
    g = _grid((3, 3, 3), (3.0, 4.0, 3.0), (1.0, 1.0, 1.0))
    irr = _maps(27, rng)
    valid = np.ones(27, np.uint8)
    valid[5] = 0
    for _ in range(20):
        x = rng.uniform([3.0, 4.0, 3.0], [5.0, 6.0, 5.0])
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        vis_out, vis, _ = O.sample_irradiance_visible(sc, g, irr, valid, x, n, 8.0)
        plain = O.sample_irradiance(g, irr, valid, x, n)
        assert np.all((vis == 1.0) | (vis == -1.0))
        assert np.array_equal(vis_out, plain)


def _wall_setup():
    h = 0.125
    s = W.Scene()
    s.add(W.BOX, [4.0, 4.0, 4.0, h, 10.0, 10.0], (0.5, 0.5, 0.5))   # 2 voxels thick, x in [3.875, 4.125]
    baked = W.bake(s, (64, 64, 64), h)
    sc = O.OracleScene(baked.sdf, h, (0, 0, 0), None)
    g = _grid((2, 2, 2), (3.5, 3.5, 3.5), (1.0, 1.0, 1.0))
    A, B = np.array([0.2, 0.4, 0.6]), np.array([1.0, 0.8, 0.6])
    irr = np.zeros((8, 8, 8, 4))
    for p in range(8):
        irr[p, ..., :3] = A if p % 2 == 0 else B                 # x index 0: near column, 1: far column
    return sc, g, irr, A, B


def test_wall_hides_the_far_probes():
    sc, g, irr, A, B = _wall_setup()
    valid = np.ones(8, np.uint8)
    for x in ([3.8, 3.7, 3.9], [3.6, 4.2, 4.4], [3.75, 3.55, 3.8]):
        n = np.array([-1.0, 0.0, 0.0])
        out, vis, marg = O.sample_irradiance_visible(sc, g, irr, valid, np.array(x), n, 8.0)
        assert np.all(vis[1::2] == 0.0) and np.all(vis[0::2] == 1.0), vis
        assert np.allclose(out, A, rtol=0, atol=1e-12)
        plain = O.sample_irradiance(g, irr, valid, np.array(x), n)
        f = x[0] - 3.5
        assert np.allclose(plain, (1 - f) * A + f * B)            # the leak the visibility test removes
    # from the far side, the mirror image
    out, vis, _ = O.sample_irradiance_visible(sc, g, irr, valid, np.array([4.3, 3.9, 3.6]),
                                              np.array([1.0, 0.0, 0.0]), 8.0)
    assert np.allclose(out, B, rtol=0, atol=1e-12)


def test_softness_monotone_and_bounded_and_no_probe_visible():
    h, c, r = 0.125, np.array([4.0, 4.0, 4.0]), 0.6
    s = W.Scene()
    s.add(W.SPHERE, list(c) + [r], (0.5, 0.5, 0.5))
    baked = W.bake(s, (64, 64, 64), h)
    sc = O.OracleScene(baked.sdf, h, (0, 0, 0), None)
    g = _grid((2, 2, 2), (3.0, 3.0, 3.0), (2.0, 2.0, 2.0))
    irr = _maps(8, np.random.default_rng(3))
    valid = np.ones(8, np.uint8)
    x, n = np.array([3.3, 4.0 + r + 0.05, 3.2]), np.array([0.0, 1.0, 0.0])   # just above the sphere
    prev = None
    for k in (0.5, 2.0, 8.0, 64.0, 1e6):
        _, vis, _ = O.sample_irradiance_visible(sc, g, irr, valid, x, n, k)
        assert np.all((vis >= 0.0) & (vis <= 1.0))
        if prev is not None:
            assert np.all(vis >= prev - 1e-15)
        prev = vis
    _, soft, _ = O.sample_irradiance_visible(sc, g, irr, valid, x, n, 0.5)
    assert np.any((soft > 0.0) & (soft < 1.0))                    # a penumbra at low softness
    # a point inside the sphere's shell sees nothing: every trace starts in a hit
    out, vis, _ = O.sample_irradiance_visible(sc, g, irr, valid, c + np.array([0.0, 0.1, 0.0]),
                                              np.array([0.0, 1.0, 0.0]), 8.0)
    assert np.all(vis == 0.0) and np.array_equal(out, np.zeros(3))
