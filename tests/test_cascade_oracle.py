"""Pins of the oracle's mean value coordinates and cascade blending (Sec. 3.5), CPU only.

Mean value coordinates reproduce linear functions (sum lambda_j p_j = x) and sum to 1,
on a box and on the shell between two nested boxes. They interpolate at vertices and
faces. On a convex box they equal the defining spherical integral, lambda_j = the
integral of phi_j(p(w)) / r(w) over the integral of 1 / r(w), where r is the distance
along direction w to the surface and phi_j the barycentric weight of vertex j at the hit.
That integral is evaluated here by brute-force quadrature over a Fibonacci sphere, a
computation that shares nothing with the closed form. On the cascade's shell the same
integral, taken face by face over the surface by adaptive quadrature, pins the weight to
1e-10, also beside the faces' planes where the closed form cancels. The cascade weight is
1 inside the inner box and 0 on the outer box (1 everywhere without an inner box of
positive volume), and the blended irradiance reduces to one volume's plain interpolation
wherever the weight is 0 or 1.
"""
import numpy as np

import oracle as O

FACES = [(0, 4, 6, 2), (1, 3, 7, 5), (0, 1, 5, 4), (2, 6, 7, 3), (0, 2, 3, 1), (4, 5, 7, 6)]


def box(lo, hi, reversed_=False, base=0):
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    v = np.array([[hi[0] if c & 1 else lo[0], hi[1] if c & 2 else lo[1], hi[2] if c & 4 else lo[2]]
                  for c in range(8)])
    t = []
    for q in FACES:
        for tri in ((q[0], q[1], q[2]), (q[0], q[2], q[3])):
            t.append(tri[::-1] if reversed_ else tri)
    return v, np.array(t) + base


def test_linear_precision_and_unity_on_a_box():
    v, t = box([0, 0, 0], [2, 1, 3])
    rng = np.random.default_rng(0)
    for _ in range(50):
        x = rng.uniform([0.01, 0.01, 0.01], [1.99, 0.99, 2.99])
        lam, on = O.mvc(v, t, x)
        assert not on
        assert abs(lam.sum() - 1) < 1e-12
        assert np.abs(lam @ v - x).max() < 1e-12
        assert np.all(lam > 0)                       # convex domain: positive coordinates


def test_linear_precision_on_a_shell():
    vo, to = box([0, 0, 0], [4, 4, 4])
    vi, ti = box([1, 1, 1], [3, 3, 3], reversed_=True, base=8)
    v, t = np.concatenate([vo, vi]), np.concatenate([to, ti])
    rng = np.random.default_rng(1)
    n = 0
    while n < 50:
        x = rng.uniform(0.01, 3.99, 3)
        if np.all((x > 1) & (x < 3)):
            continue
        lam, _ = O.mvc(v, t, x)
        assert abs(lam.sum() - 1) < 1e-12 and np.abs(lam @ v - x).max() < 1e-11
        n += 1


def test_interpolation_at_vertices_and_faces():
    v, t = box([0, 0, 0], [1, 1, 1])
    lam, on = O.mvc(v, t, v[5])
    assert on and np.array_equal(lam, np.eye(8)[5])
    x = np.array([0.25, 0.0, 0.5])                   # on the face y = 0
    lam, on = O.mvc(v, t, x)
    assert on and abs(lam.sum() - 1) < 1e-12 and np.abs(lam @ v - x).max() < 1e-12
    assert np.all(lam[[2, 3, 6, 7]] == 0)            # only vertices of that face


def _spherical_integral(v, t, x, n=400_000):
    """lambda_j by quadrature of the mean-value integral over n Fibonacci-sphere directions."""
    i = np.arange(n) + 0.5
    z = 1 - 2 * i / n
    phi = np.pi * (1 + 5 ** 0.5) * i
    r = np.sqrt(1 - z * z)
    dirs = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    num, den = np.zeros(len(v)), 0.0
    best = np.full(n, np.inf)
    bary = np.zeros((n, 3))
    owner = np.zeros(n, int)
    for k, tri in enumerate(t):                      # ray-triangle (Moller-Trumbore) for every direction
        a, b, c = v[tri[0]], v[tri[1]], v[tri[2]]
        e1, e2 = b - a, c - a
        pvec = np.cross(dirs, e2)
        det = pvec @ e1
        ok = np.abs(det) > 1e-14
        inv = np.where(ok, 1 / np.where(ok, det, 1), 0)
        s = x - a
        uu = (pvec @ s) * inv
        q = np.cross(s, e1)
        vv = (dirs @ q) * inv
        tt = (q @ e2) * inv
        hit = ok & (uu >= 0) & (vv >= 0) & (uu + vv <= 1) & (tt > 0) & (tt < best)
        best[hit] = tt[hit]
        bary[hit] = np.stack([1 - uu[hit] - vv[hit], uu[hit], vv[hit]], axis=1)
        owner[hit] = k
    assert np.all(np.isfinite(best))
    w = 1 / best
    for k in range(3):
        np.add.at(num, t[owner, k], bary[:, k] * w)
    den = w.sum()
    return num / den


def test_closed_form_equals_the_spherical_integral_on_a_box():
    v, t = box([0, 0, 0], [2, 1, 1.5])
    for x in (np.array([0.7, 0.4, 0.6]), np.array([1.8, 0.15, 1.2])):
        lam, _ = O.mvc(v, t, x)
        ref = _spherical_integral(v, t, x)
        assert np.abs(lam - ref).max() < 2e-3, (lam, ref)


def _grid(dims, origin, spacing):
    return O.make_grid(dims, origin, spacing, 8, 64, 0.01, 100.0, 0.97)


def test_cascade_weight_limits():
    g = _grid((5, 4, 6), (1.0, 2.0, 0.0), (1.0, 1.0, 1.0))     # box [1,5]x[2,5]x[0,5], inner shrunk by 1
    assert O.cascade_weight(g, np.array([3.0, 3.5, 2.5])) == 1.0
    for x in ([1.0, 3.5, 2.5], [5.0, 3.0, 1.0], [2.0, 2.0, 4.0], [4.5, 5.0, 0.0]):
        assert O.cascade_weight(g, np.array(x)) < 1e-7        # rounding of the near-degenerate faces
    for x in ([2.0, 3.5, 2.5], [3.0, 3.0, 1.0]):                  # on the inner box
        assert O.cascade_weight(g, np.array(x)) > 1 - 1e-7
    ws = [O.cascade_weight(g, np.array([2.0 - s, 3.5, 2.5])) for s in np.linspace(0, 1, 11)]
    assert all(a >= b - 1e-12 for a, b in zip(ws, ws[1:]))        # falls toward the outer box
    g2 = _grid((2, 4, 6), (1.0, 2.0, 0.0), (1.0, 1.0, 1.0))     # too thin for an inner box
    assert O.cascade_weight(g2, np.array([1.5, 3.0, 2.0])) == 1.0


def test_cascade_sample_reduces_to_one_volume():
    rng = np.random.default_rng(2)
    fine = _grid((5, 5, 5), (2.0, 2.0, 2.0), (0.5, 0.5, 0.5))    # box [2,4]^3
    coarse = _grid((5, 5, 5), (0.0, 0.0, 0.0), (1.5, 1.5, 1.5))  # box [0,6]^3
    irr = [rng.uniform(0.1, 1.0, (125, 8, 8, 4)) for _ in range(2)]
    for i in range(2):
        for p in range(125):
            irr[i][p] = O.border(irr[i][p])
    valid = [np.ones(125, np.uint8), np.ones(125, np.uint8)]
    n = np.array([0.0, 0.6, 0.8])
    x = np.array([3.0, 3.1, 2.9])                                # inside the fine inner box
    out, w, lvl = O.sample_irradiance_cascade([fine, coarse], irr, valid, x, n)
    assert lvl == 0 and w == 1.0 and np.array_equal(out, O.sample_irradiance(fine, irr[0], valid[0], x, n))
    x = np.array([5.0, 1.0, 3.0])                                # outside the fine box
    out, w, lvl = O.sample_irradiance_cascade([fine, coarse], irr, valid, x, n)
    assert lvl == 1 and np.array_equal(out, O.sample_irradiance(coarse, irr[1], valid[1], x, n))
    x = np.array([2.2, 3.0, 3.0])                                # in the fine volume's transition shell
    out, w, lvl = O.sample_irradiance_cascade([fine, coarse], irr, valid, x, n)
    ef, ec = O.sample_irradiance(fine, irr[0], valid[0], x, n), O.sample_irradiance(coarse, irr[1], valid[1], x, n)
    assert lvl == 0 and 0 < w < 1 and np.allclose(out, w * ef + (1 - w) * ec, rtol=0, atol=1e-15)


def _weight_by_quadrature(lo, hi, sp, x):
    """The cascade weight from the integral that defines mean value coordinates, face by face.

    lambda_j = W_j / sum W with W_j the integral over the surface of phi_j / r over the sphere
    of directions; with d(omega) = h / r^3 dA that is the integral of phi_j h / r^4 over the
    surface (h the signed distance of the face's plane along its outward normal). The hats of
    a face's corners sum to 1 on it, so the inner corners' total is the ratio of the inner
    faces' integrals of h / r^4 to all 12 faces' ones, each integrated here by adaptive 2-D
    quadrature.
    """
    from scipy import integrate
    lo, hi, sp = (np.asarray(v, float) for v in (lo, hi, sp))
    ilo, ihi = lo + sp, hi - sp
    num = den = 0.0
    for inner, (L, H) in ((False, (lo, hi)), (True, (ilo, ihi))):
        for ax in range(3):
            p, q = [k for k in range(3) if k != ax]
            for side in (0, 1):
                n = (1.0 if side else -1.0) * (-1.0 if inner else 1.0)   # outward from the shell
                h = n * ((H if side else L)[ax] - x[ax])
                f = lambda b, a, h=h: h / (h * h + a * a + b * b) ** 2
                val = integrate.dblquad(f, L[p] - x[p], H[p] - x[p], L[q] - x[q], H[q] - x[q],
                                        epsabs=1e-15, epsrel=1e-12)[0]
                den += val
                num += val if inner else 0.0
    return num / den


def test_cascade_weight_equals_the_surface_integral():
    """Generic shell points and points within 1e-7 spacings of an inner face's plane (outside
    the face), where the per-triangle closed form is a difference of nearly equal terms (an
    FP64 evaluation of it is off by 2e-8 at the first point of the large volume); the bar
    is the quadrature's accuracy."""
    cases = []
    dims, origin, sp = (7, 5, 9), np.array([1.0, -2.0, 0.5]), np.array([0.5, 0.5, 0.5])
    cases.append((dims, origin, sp, [[1.2, -1.1, 2.0], [3.7, -0.4, 1.3], [2.0, -0.3, 4.3], [1.25, -1.75, 0.8],
                                     [1.2, -1.5 + 5e-8, 2.2], [2.1, -1.5 - 1.5e-7, 0.65]]))
    dims, origin, sp = (32, 16, 32), np.array([-60.0, -2.0, -64.0]), np.array([4.0, 4.0, 4.0])
    cases.append((dims, origin, sp, [[-58.0, 2.0 + 4e-7, -20.0], [61.5, 10.0, -60.0 - 4e-7], [0.0, 54.0 + 2e-7, 59.0],
                                     [-57.5, -0.5, 3.25], [10.0, 56.0, 50.0]]))
    for dims, origin, sp, pts in cases:
        g = _grid(dims, origin, sp)
        lo, hi = origin, origin + (np.array(dims) - 1) * sp
        for x in map(np.array, pts):
            ref = _weight_by_quadrature(lo, hi, sp, x)
            got = O.cascade_weight(g, x)
            assert abs(got - ref) < 1e-10, (x, got, ref)


def test_flat_inner_box_means_no_transition():
    g = _grid((3, 6, 5), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))      # inner box flat in x
    for x in ([0.5, 2.5, 2.0], [1.0, 0.2, 3.9], [1.7, 4.8, 0.1]):
        assert O.cascade_weight(g, np.array(x)) == 1.0


def test_weight_is_smooth_up_to_the_faces():
    """Mean value coordinates are smooth up to the interior of a face, so approaching an inner
    face (weight 1 on it) or the probe box's face (weight 0) from the shell, (1 - w) / h and
    w / h tend to the normal derivative: at distances 1e-6 .. 1e-10 spacings they agree with
    their value at 1e-5 to first order. A test for x on a face by the angle sum alone (whose
    gap to 2 pi is second order in the distance) reads such points as on the face."""
    dims, origin, sp = (32, 16, 32), np.array([1.0, -2.0, 0.5]), np.array([4.0, 4.0, 4.0])
    g = _grid(dims, origin, sp)
    lo, hi = origin, origin + (np.array(dims) - 1) * sp
    ilo = lo + sp
    foot = np.array([78.7, 0.0, 47.9])
    for face_y, sign, inner in ((ilo[1], -1.0, True), (lo[1], 1.0, False)):
        def gap(h):
            x = foot.copy()
            x[1] = face_y + sign * h
            w = O.cascade_weight(g, x)
            return ((1.0 - w) if inner else w) / h
        ref = gap(1e-5 * sp[1])
        for k in range(6, 11):
            h = 10.0 ** -k * sp[1]
            assert abs(gap(h) / ref - 1.0) < 1e-4, (inner, k, gap(h), ref)


def test_cascade_with_visibility_composes_the_pinned_rules():
    """With probe visibility (Sec. 3.4), every level but the farthest takes the visibility rule
    and the farthest the plain one (Sec. 3.5): inside the fine inner box the result is the
    fine volume's visibility interpolation, in its shell the weight's blend of that and the
    coarse plain interpolation, outside it the coarse plain interpolation; softness 0 is
    the plain cascade."""
    import workloads as W
    h = 0.125
    s = W.Scene()
    s.add(W.BOX, [4.0, 4.0, 4.0, h, 10.0, 10.0], (0.5, 0.5, 0.5))   # a wall at x = 4
    baked = W.bake(s, (64, 64, 64), h)
    sc = O.OracleScene(baked.sdf, h, (0, 0, 0), None)
    fine = O.make_grid((5, 5, 5), (3.0, 3.0, 3.0), (0.5, 0.5, 0.5), 8, 128, 0.01, 300.0, 0.97)   # [3, 5]^3
    coarse = O.make_grid((5, 5, 5), (1.0, 1.0, 1.0), (1.5, 1.5, 1.5), 8, 128, 0.01, 300.0, 0.97)  # [1, 7]^3
    rng = np.random.default_rng(4)
    irr = [rng.uniform(0.1, 1.0, (125, 8, 8, 4)) for _ in range(2)]
    valid = [np.ones(125, np.uint8), np.ones(125, np.uint8)]
    grids, scenes = [fine, coarse], [sc, sc]
    n = np.array([0.0, 0.6, 0.8])
    for x, where in (([3.7, 4.1, 3.9], "inner"), ([3.2, 4.0, 4.3], "shell"), ([6.0, 2.0, 3.0], "outside")):
        x = np.array(x)
        out, w, lvl, m = O.sample_irradiance_cascade_visible(scenes, grids, irr, valid, x, n, 8.0)
        vis_fine = O.sample_irradiance_visible(sc, fine, irr[0], valid[0], x, n, 8.0)
        plain_coarse = O.sample_irradiance(coarse, irr[1], valid[1], x, n)
        if where == "inner":
            assert lvl == 0 and w == 1.0 and np.array_equal(out, vis_fine[0])
            assert np.array_equal(m[0], vis_fine[2]) and np.all(m[1] > 1e30)
        elif where == "shell":
            assert lvl == 0 and 0 < w < 1
            assert np.allclose(out, w * vis_fine[0] + (1 - w) * plain_coarse, rtol=0, atol=1e-15)
        else:
            assert lvl == 1 and np.array_equal(out, plain_coarse) and np.all(m > 1e30)
        plain = O.sample_irradiance_cascade(grids, irr, valid, x, n)
        assert np.array_equal(O.sample_irradiance_cascade_visible(scenes, grids, irr, valid, x, n, 0.0)[0], plain[0])
