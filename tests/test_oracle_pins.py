"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No test here re-types a formula of the oracle: each compares it with a closed
form (plane and sphere distances, the inverse-square law, the multi-bounce
geometric series), an invariant (unit directions, equal-area bands, seam
continuity of the octahedral map, exactness of trilinear interpolation on
linear fields) or brute force (dense ray marching), chosen so that a dropped
term, a wrong sign or index, or a transposed operand fails at least one.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLDEN = (math.sqrt(5.0) - 1.0) / 2.0


def oscene(scene, dims, h, origin=(0.0, 0.0, 0.0), dtype="f32"):
    b = W.bake(scene, dims, h, origin, dtype=dtype)
    return O.OracleScene(b.sdf, b.h, b.origin, b.material), b


def grid_for(dims, origin, spacing, rays, **kw):
    args = dict(max_steps=256, eps_vox=0.01, tmax_vox=200.0, hysteresis=0.97, depth_exponent=50,
                k_bounce=1.0, bias_vox=1.0, sky=(0.0, 0.0, 0.0))
    args.update(kw)
    return O.make_grid(dims, origin, spacing, rays, **args)


def probes_at(positions, active=True):
    st = np.zeros(len(positions), dtype=O.PROBE_DTYPE)
    st["pos"] = np.asarray(positions, dtype=np.float32)
    st["flags"] = 1 if active else 0
    return st


# --------------------------------------------------------------------------- ray set
@pytest.mark.parametrize("n", [1, 2, 7, 64, 256, 1023])
def test_sf_unit_equal_area(n):
    d = np.array([O.sf_dir(i, n) for i in range(n)])
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    # the z coordinates are symmetric about 0 and equally spaced: equal-area bands on the sphere
    assert abs(d[:, 2].sum()) < 1e-10
    edges = np.linspace(-1.0, 1.0, 9)
    counts = np.histogram(d[:, 2], bins=edges)[0]
    assert np.all(np.abs(counts - n / 8.0) <= 1.0)


def test_sf_golden_angle_increment():
    n = 300
    d = np.array([O.sf_dir(i, n) for i in range(n)])
    az = np.arctan2(d[:, 1], d[:, 0])
    inc = np.mod(np.diff(az), 2 * math.pi)
    expect = 2 * math.pi * GOLDEN  # azimuth advances by the golden fraction of a turn (counter-clockwise)
    assert np.allclose(inc, expect, atol=1e-6)


@pytest.mark.parametrize("n,tol", [(64, 0.06), (256, 0.02), (1024, 0.006)])
def test_sf_cosine_quadrature(n, tol):
    # (4 pi / n) sum max(0, u.d_i) approximates the integral of max(0, cos) over the sphere = pi
    rng = np.random.default_rng(3)
    rot = W.frame_rotation(5, 1)
    d = np.array([O.sf_dir(i, n) for i in range(n)]) @ rot.astype(np.float64).T
    for _ in range(20):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        q = 4 * math.pi / n * np.maximum(0.0, d @ u).sum()
        assert abs(q - math.pi) < tol * math.pi


def test_frame_rotation_is_uniform_rotation():
    zs = []
    for f in range(2000):
        r = W.frame_rotation(42, f).astype(np.float64)
        assert np.allclose(r.T @ r, np.eye(3), atol=1e-6)
        assert abs(np.linalg.det(r) - 1.0) < 1e-6
        zs.append(r[:, 2])
    zs = np.array(zs)
    assert np.linalg.norm(zs.mean(axis=0)) < 0.06           # isotropic image of a fixed axis
    assert not np.allclose(W.frame_rotation(42, 0), W.frame_rotation(42, 1))
    assert not np.allclose(W.frame_rotation(42, 0), W.frame_rotation(42, 0, volume=1))
    assert np.array_equal(W.frame_rotation(42, 3), W.frame_rotation(42, 3))


# --------------------------------------------------------------------------- octahedral map
def test_oct_known_points_and_roundtrip():
    assert np.allclose(O.oct_encode([0, 0, 1]), [0.5, 0.5])
    assert np.allclose(O.oct_encode([1, 0, 0]), [1.0, 0.5])
    assert np.allclose(O.oct_encode([-1, 0, 0]), [0.0, 0.5])
    assert np.allclose(O.oct_encode([0, 1, 0]), [0.5, 1.0])
    assert np.allclose(O.oct_encode([0, -1, 0]), [0.5, 0.0])
    for corner in ([0, 0], [1, 0], [0, 1], [1, 1]):
        assert np.allclose(O.oct_decode(corner), [0, 0, -1])
    # upper hemisphere fills the inner diamond, lower hemisphere the four corners
    rng = np.random.default_rng(0)
    for _ in range(2000):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        uv = O.oct_encode(v)
        assert np.all((uv >= 0) & (uv <= 1))
        inner = abs(uv[0] - 0.5) + abs(uv[1] - 0.5) <= 0.5 + 1e-12
        assert inner == (v[2] >= 0) or abs(v[2]) < 1e-12
        assert np.allclose(O.oct_decode(uv), v, atol=1e-12)


def _one_probe_grid():
    return grid_for((1, 1, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 1)


def _sample_map(irr_map, direction):
    g = _one_probe_grid()
    return O.sample_irradiance(g, irr_map[None], np.ones(1, np.uint8), [0.0, 0.0, 0.0], direction)


def _seam_directions(rng, k):
    """Directions on the folds of the octahedral map (lower hemisphere with x = 0 or y = 0)."""
    out = []
    for _ in range(k):
        a, z = rng.uniform(0.05, 1.0), -rng.uniform(0.05, 1.0)
        s = rng.choice([-1.0, 1.0])
        out.append((np.array([s * a, 0.0, z]), 1))   # fold where y changes sign
        out.append((np.array([0.0, s * a, z]), 0))   # fold where x changes sign
    return out


def test_border_makes_octahedral_sampling_continuous():
    rng = np.random.default_rng(11)
    m = np.zeros((O.IRR_T, O.IRR_T, 4))
    m[1:-1, 1:-1, :3] = rng.uniform(0.0, 1.0, (O.IRR_N, O.IRR_N, 3))
    fixed = O.border(m)
    assert np.array_equal(fixed[1:-1, 1:-1], m[1:-1, 1:-1])        # interior untouched
    eps = 1e-9
    for d, axis in _seam_directions(rng, 40):
        dp, dm = d.copy(), d.copy()
        dp[axis] += eps
        dm[axis] -= eps
        a, b = _sample_map(fixed, dp), _sample_map(fixed, dm)
        assert np.allclose(a, b, atol=1e-6), (d, a, b)
    # the pole (0,0,-1) maps to all four corners: every approach agrees
    vals = [_sample_map(fixed, [sx * 1e-9, sy * 1e-9, -1.0]) for sx in (-1, 1) for sy in (-1, 1)]
    assert np.allclose(vals, vals[0], atol=1e-6)
    # without the fixup the same probes see a jump (the test has teeth)
    jumps = [np.abs(_sample_map(m, d + e) - _sample_map(m, d - e)).max()
             for d, axis in _seam_directions(rng, 10) for e in [np.eye(3)[axis] * eps]]
    assert max(jumps) > 1e-3


@pytest.mark.parametrize("n", [1, 2, 6, 14])
def test_border_is_a_copy_of_interior(n):
    rng = np.random.default_rng(n)
    m = np.zeros((n + 2, n + 2, 2))
    m[1:-1, 1:-1] = rng.uniform(size=(n, n, 2))
    f = O.border(m)
    inner = {tuple(v) for v in f[1:-1, 1:-1].reshape(-1, 2)}
    edge = np.concatenate([f[0], f[-1], f[:, 0], f[:, -1]])
    assert all(tuple(v) in inner for v in edge)          # bit-exact copies of interior texels


# --------------------------------------------------------------------------- trilinear sampling
def _linear_scene(axis, offset):
    s = W.Scene()
    if axis == 1:
        s.add(W.PLANE_Y, [offset], (0.5, 0.5, 0.5))
    elif axis == 0:
        s.add(W.BOX, [offset - 500.0, 0, 0, 500.0, 1e4, 1e4], (0.5, 0.5, 0.5))
    else:
        s.add(W.BOX, [0, 0, offset - 500.0, 1e4, 1e4, 500.0], (0.5, 0.5, 0.5))
    return s


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_trilinear_exact_on_linear_fields(axis):
    dims, h, origin = (12, 16, 20), 0.25, (0.5, -1.0, 2.0)
    sc, _ = oscene(_linear_scene(axis, 1.3 + origin[axis]), dims, h, origin)
    rng = np.random.default_rng(axis)
    lo = np.array(origin) + 0.5 * h
    hi = np.array(origin) + (np.array(dims) - 0.5) * h
    for _ in range(300):
        p = rng.uniform(lo, hi)
        assert abs(O.sample_sdf(sc, p) - (p[axis] - 1.3 - origin[axis])) < 2e-6
    # outside the voxel-centre hull the field is clamped to its edge value
    p = (lo + hi) / 2
    p[axis] = origin[axis] - 3.0
    assert abs(O.sample_sdf(sc, p) - (lo[axis] - 1.3 - origin[axis])) < 2e-6


# --------------------------------------------------------------------------- sphere tracing
def test_trace_plane_closed_form():
    s = W.Scene()
    s.add(W.PLANE_Y, [1.0], (0.5, 0.5, 0.5))
    h = 0.125
    sc, _ = oscene(s, (64, 64, 64), h)
    rng = np.random.default_rng(1)
    o = np.array([4.0, 5.0, 4.0])
    for _ in range(200):
        d = rng.normal(size=3)
        d[1] = -abs(d[1])
        d /= np.linalg.norm(d)
        c = -d[1]
        if c < 0.75:
            continue
        ev, t, steps, _ = O.trace(sc, o, d, 0.01, 1e3, 10000)
        tstar = 4.0 / c
        assert ev == O.HIT
        assert tstar - 0.01 * h / c - 1e-9 <= t <= tstar + 1e-9
    ev, t, steps, _ = O.trace(sc, o, [0.0, 1.0, 0.0], 0.01, 1e3, 10000)
    assert ev == O.LEFT_VOLUME and t == 1e3
    ev, t, steps, _ = O.trace(sc, o, [0.0, 1.0, 0.0], 0.01, 2.0, 10000)
    assert ev == O.PAST_LIMIT and steps == 1               # first step of 4 m passes the 2 m limit
    ev, t, steps, _ = O.trace(sc, [4.0, 1.5, 4.0], [1.0, 0.0, 0.0], 0.01, 1e3, 5)
    assert ev == O.EXHAUSTED and steps == 5 and abs(t - 5 * 0.5) < 1e-6


def _ray_sphere(o, d, c, r):
    oc = o - c
    b = np.dot(oc, d)
    disc = b * b - (np.dot(oc, oc) - r * r)
    if disc < 0:
        return None
    return -b - math.sqrt(disc)


def test_trace_sphere_within_bake_bound():
    s = W.Scene()
    c, r, h = np.array([4.0, 4.0, 4.0]), 1.5, 0.125
    s.add(W.SPHERE, list(c) + [r], (0.5, 0.5, 0.5))
    sc, _ = oscene(s, (64, 64, 64), h)
    rng = np.random.default_rng(2)
    err = h * h / (4.0 * (r - math.sqrt(3) * h))  # trilinear error of |x - c| - r near the surface
    n_checked = 0
    for _ in range(400):
        o = c + rng.normal(size=3) * 0.0
        o = c + (lambda v: v / np.linalg.norm(v))(rng.normal(size=3)) * 3.5
        target = c + (lambda v: v / np.linalg.norm(v))(rng.normal(size=3)) * r * 0.8
        d = target - o
        d /= np.linalg.norm(d)
        tstar = _ray_sphere(o, d, c, r)
        if tstar is None:
            continue
        nrm = (o + tstar * d - c) / r
        cos = -np.dot(nrm, d)
        if cos < 0.5:
            continue
        ev, t, steps, _ = O.trace(sc, o, d, 0.01, 1e3, 10000)
        assert ev == O.HIT
        assert abs(t - tstar) <= (0.01 * h + err) / cos + 1e-9
        n_checked += 1
    assert n_checked > 100


def _dense_first_below(sc, o, d, level, tmax, step):
    t = 0.0
    prev = O.sample_sdf(sc, o)
    if prev < level:
        return 0.0
    while t < tmax:
        t1 = t + step
        v = O.sample_sdf(sc, o + t1 * d)
        if v < level:
            a, b = t, t1
            for _ in range(50):
                m = 0.5 * (a + b)
                if O.sample_sdf(sc, o + m * d) < level:
                    b = m
                else:
                    a = m
            return b
        t = t1
    return None


def _exit_t(o, d, lo, hi):
    ts = []
    for a in range(3):
        if d[a] > 0:
            ts.append((hi[a] - o[a]) / d[a])
        elif d[a] < 0:
            ts.append((lo[a] - o[a]) / d[a])
    return min(ts)


def test_trace_matches_dense_march():
    s = W.Scene()
    rng = np.random.default_rng(9)
    centres = []
    for _ in range(4):
        c = rng.uniform(0.6, 2.4, 3)
        centres.append(c)
        s.add(W.SPHERE, list(c) + [rng.uniform(0.2, 0.6)], (0.5, 0.5, 0.5))
    c = rng.uniform(0.8, 2.2, 3)
    centres.append(c)
    s.add(W.BOX, list(c) + list(rng.uniform(0.1, 0.4, 3)), (0.5, 0.5, 0.5))
    s.add(W.CAPSULE, [0.5, 0.5, 2.5, 2.5, 2.0, 0.5, 0.15], (0.5, 0.5, 0.5))
    h = 0.25
    sc, _ = oscene(s, (12, 12, 12), h)
    eps = 0.01
    n_hit = n_miss = 0
    for k in range(120):
        o = rng.uniform(0.2, 2.8, 3)
        if O.sample_sdf(sc, o) < 0.2:
            continue
        if k % 3 == 0:
            d = rng.normal(size=3)
        else:
            d = centres[k % len(centres)] + rng.normal(size=3) * 0.3 - o
        d /= np.linalg.norm(d)
        ev, t, steps, _ = O.trace(sc, o, d, eps, 1e3, 100000)
        first_eps = _dense_first_below(sc, o, d, eps * h, 6.0, 1e-3 * h)
        first_zero = _dense_first_below(sc, o, d, 0.0, 6.0, 1e-3 * h)
        if ev == O.HIT:
            n_hit += 1
            assert first_eps is not None and t >= first_eps - 1e-9
            assert O.sample_sdf(sc, o + t * d) < eps * h
            # a trilinear interpolant is not exactly 1-Lipschitz, so a step may pass the
            # first zero crossing by a small fraction of a voxel, never more
            assert first_zero is None or t <= first_zero + 0.02 * h
        else:
            n_miss += 1
            assert ev == O.LEFT_VOLUME
            t_exit = _exit_t(o, d, np.zeros(3), np.full(3, 12 * h))
            assert first_eps is None or first_eps > t_exit - 1e-9
    assert n_hit > 30 and n_miss > 5


# --------------------------------------------------------------------------- shading
FP16_EXACT_ALBEDO = (0.25, 0.5, 0.75)


def _floor_scene(extra=()):
    s = W.Scene()
    s.add(W.PLANE_Y, [1.0], FP16_EXACT_ALBEDO)
    for t, p in extra:
        s.add(t, p, FP16_EXACT_ALBEDO)
    return s


def test_shade_floor_directional_closed_form():
    sc, _ = oscene(_floor_scene(), (64, 64, 64), 0.125)
    g = grid_for((2, 2, 2), (0.0, 0.0, 0.0), (8.0, 8.0, 8.0), 1, k_bounce=0.0)
    l = np.array([0.3, 0.8, 0.2]) / np.linalg.norm([0.3, 0.8, 0.2])
    E = (2.0, 3.0, 4.0)
    lights = [{"type": "dir", "v": l, "rgb": E}]
    irr, _, valid = O.empty_maps(8)
    rec = O.shade(sc, g, lights, irr, valid, [3.7, 1.0, 4.2], [0.0, -1.0, 0.0])
    expect = np.array(FP16_EXACT_ALBEDO) / math.pi * np.array(E) * l[1]   # rho/pi * E * cos
    assert np.allclose(rec["L"], expect, rtol=1e-9)
    assert rec["lit_mask"] == 1


def test_shade_point_light_inverse_square_and_range():
    sc, _ = oscene(_floor_scene(), (64, 64, 64), 0.125)
    g = grid_for((2, 2, 2), (0.0, 0.0, 0.0), (8.0, 8.0, 8.0), 1, k_bounce=0.0)
    irr, _, valid = O.empty_maps(8)
    x = np.array([3.0, 1.0, 5.0])
    lp = np.array([4.0, 5.0, 4.5])
    I = np.array([10.0, 20.0, 30.0])
    rec = O.shade(sc, g, [{"type": "point", "v": lp, "rgb": I, "range": 1e6}], irr, valid, x, [0, -1, 0])
    dist = np.linalg.norm(lp - x)
    cos = (lp - x)[1] / dist
    expect = np.array(FP16_EXACT_ALBEDO) / math.pi * I * cos / dist ** 2       # inverse-square law
    assert np.allclose(rec["L"], expect, rtol=1e-9)
    far = O.shade(sc, g, [{"type": "point", "v": lp, "rgb": I, "range": 0.9 * dist}], irr, valid, x, [0, -1, 0])
    assert np.all(far["L"] == 0.0) and far["traced_mask"] == 0
    near = O.shade(sc, g, [{"type": "point", "v": lp, "rgb": I, "range": 1.5 * dist}], irr, valid, x, [0, -1, 0])
    assert np.all(0 < near["L"]) and np.all(near["L"] < rec["L"])            # the window only attenuates


def test_shade_shadow_matches_analytic_occluder():
    c, r = np.array([4.0, 2.5, 4.0]), 0.75
    sc, _ = oscene(_floor_scene([(W.SPHERE, list(c) + [r])]), (64, 64, 64), 0.125)
    g = grid_for((2, 2, 2), (0.0, 0.0, 0.0), (8.0, 8.0, 8.0), 1, k_bounce=0.0)
    l = np.array([0.2, 1.0, -0.1]) / np.linalg.norm([0.2, 1.0, -0.1])
    irr, _, valid = O.empty_maps(8)
    checked = lit = 0
    for a in np.linspace(2.0, 6.0, 21):
        for b in np.linspace(2.0, 6.0, 21):
            x = np.array([a, 1.0, b])
            xs = x + np.array([0.0, 0.125, 0.0])
            oc = xs - c
            tc = -np.dot(oc, l)
            closest = np.linalg.norm(oc + tc * l)
            if abs(closest - r) < 0.1:
                continue  # tangent rays: within the bake's resolution
            rec = O.shade(sc, g, [{"type": "dir", "v": l, "rgb": (1, 1, 1)}], irr, valid, x, [0, -1, 0])
            blocked = closest < r and tc > 0
            assert (rec["lit_mask"] == 0) == blocked, (x, closest)
            checked += 1
            lit += not blocked
    assert checked > 300 and 0 < lit < checked


def test_shade_emission_and_indirect():
    s = W.Scene()
    s.add(W.PLANE_Y, [1.0], FP16_EXACT_ALBEDO, emission=(0.5, 1.5, 2.5))
    sc, _ = oscene(s, (32, 32, 32), 0.25)
    g0 = grid_for((2, 2, 2), (0.0, 0.0, 0.0), (8.0, 8.0, 8.0), 1, k_bounce=0.0)
    irr, _, valid = O.empty_maps(8)
    rec = O.shade(sc, g0, [], irr, valid, [4.0, 1.0, 4.0], [0, -1, 0])
    assert np.array_equal(rec["L"], [0.5, 1.5, 2.5])
    # with uniform last-frame maps S and gain k, the bounce adds k * albedo * S
    S = np.array([0.2, 0.4, 0.8])
    irr[..., :3] = S
    valid[:] = 1
    g1 = grid_for((2, 2, 2), (0.0, 0.0, 0.0), (8.0, 8.0, 8.0), 1, k_bounce=0.5)
    rec = O.shade(sc, g1, [], irr, valid, [4.0, 1.0, 4.0], [0, -1, 0])
    assert np.allclose(rec["L"], np.array([0.5, 1.5, 2.5]) + 0.5 * np.array(FP16_EXACT_ALBEDO) * S, rtol=1e-12)


# --------------------------------------------------------------------------- whole update
def _closed_room(emission, albedo, extra=()):
    s = W.room_scene(0, size=8.0, n_spheres=0, n_boxes=0, aperture=0.0, uniform_albedo=albedo,
                     emission=emission, sun=False)
    for t, p in extra:
        s.add(t, p, albedo, emission)
    return s


@pytest.mark.parametrize("rays", [7, 64])
def test_white_furnace(rays):
    Le = (0.5, 1.0, 2.0)
    s = _closed_room(Le, (0.0, 0.0, 0.0), [(W.SPHERE, [3.0, 3.0, 3.0, 1.2]), (W.BOX, [6, 2, 5, 0.7, 1.1, 0.5])])
    sc, _ = oscene(s, (32, 32, 32), 0.25)
    dims, org, sp = (4, 4, 4), (1.0, 1.0, 1.0), (2.0, 2.0, 2.0)
    st = W.probe_states(s, dims, org, sp, 0.25)
    g = grid_for(dims, org, sp, rays, max_steps=64, tmax_vox=56.0)
    for frame in range(2):
        out = O.update(sc, g, [], W.frame_rotation(3, frame), st)
        act = (st["flags"] & 1).astype(bool)
        irr = out["irr"][act][:, 1:-1, 1:-1]
        assert np.allclose(irr[..., :3], Le, rtol=1e-12)
        assert np.all(out["irr"][~act] == 0.0)
        mu, mu2 = out["depth"][act][..., 0], out["depth"][act][..., 1]
        assert np.all(mu2 >= mu * mu * (1 - 1e-12))          # Jensen: E[t^2] >= E[t]^2
        assert np.all(mu > 0) and np.all(mu <= 56.0 * 0.25)


def test_single_ray_texels_take_its_value():
    s = W.room_scene(7)
    sc, _ = oscene(s, (64, 64, 64), 0.125)
    dims, org, sp = (3, 3, 3), (2.0, 2.0, 2.0), (2.0, 2.0, 2.0)
    st = W.probe_states(s, dims, org, sp, 0.125)
    g = grid_for(dims, org, sp, 1, max_steps=64)
    rot = W.frame_rotation(1, 0)
    out = O.update(sc, g, s.lights, rot, st)
    d = rot.astype(np.float64) @ O.sf_dir(0, 1)
    for p in np.flatnonzero(st["flags"] & 1):
        ray = out["rays"][p, 0]
        for b in range(O.IRR_N):
            for a in range(O.IRR_N):
                u = O.oct_decode([(a + 0.5) / O.IRR_N, (b + 0.5) / O.IRR_N])
                tex = out["irr"][p, b + 1, a + 1]
                if np.dot(u, d) > 0:
                    assert np.allclose(tex[:3], ray["L"], rtol=1e-12) and tex[3] == 1.0
                else:
                    assert np.all(tex == 0.0)


def test_hysteresis_limits_and_reject():
    s = W.room_scene(7)
    sc, _ = oscene(s, (64, 64, 64), 0.125)
    dims, org, sp = (3, 3, 3), (2.0, 2.0, 2.0), (2.0, 2.0, 2.0)
    st = W.probe_states(s, dims, org, sp, 0.125)
    rng = np.random.default_rng(0)
    P = st.shape[0]
    prev = (rng.uniform(size=(P, O.IRR_T, O.IRR_T, 4)), rng.uniform(size=(P, O.DEP_T, O.DEP_T, 2)),
            np.ones(P, np.uint8))
    rot = W.frame_rotation(1, 4)
    keep = O.update(sc, grid_for(dims, org, sp, 32, hysteresis=1.0), s.lights, rot, st, prev=prev)
    act = (st["flags"] & 1).astype(bool)
    assert np.array_equal(keep["irr"][act][:, 1:-1, 1:-1, :3], prev[0][act][:, 1:-1, 1:-1, :3])
    assert np.array_equal(keep["depth"][act][:, 1:-1, 1:-1], prev[1][act][:, 1:-1, 1:-1])
    # (no multi-bounce term here: it reads the previous maps, which differ between the two runs)
    fresh = O.update(sc, grid_for(dims, org, sp, 32, hysteresis=0.5, k_bounce=0.0), s.lights, rot, st)
    reset = st.copy()
    reset["flags"] |= W.REJECT_HISTORY
    rejected = O.update(sc, grid_for(dims, org, sp, 32, hysteresis=0.5, k_bounce=0.0), s.lights, rot, reset,
                        prev=prev)
    assert np.array_equal(rejected["irr"][act], fresh["irr"][act])
    assert np.array_equal(rejected["depth"][act], fresh["depth"][act])
    # inactive probes keep whatever they had
    assert np.array_equal(rejected["irr"][~act], prev[0][~act])


def test_multibounce_closed_form():
    Le, rho, hyst = np.array([1.0, 0.5, 0.25]), 0.5, 0.97
    s = _closed_room(tuple(Le), (rho, rho, rho), [(W.BOX, [3.0, 2.0, 5.0, 0.5, 0.5, 0.5])])
    sc, _ = oscene(s, (32, 32, 32), 0.25)
    dims, org, sp = (4, 4, 4), (1.0, 1.0, 1.0), (2.0, 2.0, 2.0)
    st = W.probe_states(s, dims, org, sp, 0.25)
    act = (st["flags"] & 1).astype(bool)
    g = grid_for(dims, org, sp, 32, max_steps=64, tmax_vox=56.0, hysteresis=hyst, k_bounce=1.0)
    S_inf = Le / (1 - rho)
    r = hyst + (1 - hyst) * rho
    prev = None
    for n in range(6):
        out = O.update(sc, g, [], W.frame_rotation(9, n), st, prev=prev, want_rays=False)
        expect = S_inf + (Le - S_inf) * r ** n
        assert np.allclose(out["irr"][act][:, 1:-1, 1:-1, :3], expect, rtol=1e-11), n
        prev = (out["irr"], out["depth"], out["valid"])


def test_depth_moments_hollow_ball_and_misses():
    s = W.Scene()
    c, r, h = (4.0, 4.0, 4.0), 3.0, 0.125
    s.add(W.INV_SPHERE, list(c) + [r], (0.5, 0.5, 0.5))
    sc, _ = oscene(s, (64, 64, 64), h)
    g = grid_for((1, 1, 1), c, (1.0, 1.0, 1.0), 64, max_steps=256)
    out = O.update(sc, g, [], W.frame_rotation(2, 0), probes_at([c]))
    err = h * h / (4 * (r - math.sqrt(3) * h))
    mu, mu2 = out["depth"][0, 1:-1, 1:-1, 0], out["depth"][0, 1:-1, 1:-1, 1]
    assert np.all(mu <= r + 1e-12) and np.all(mu >= r - err - 0.01 * h - 1e-9)
    assert np.all(mu2 <= r * r + 1e-9) and np.all(mu2 >= (r - err - 0.01 * h) ** 2 - 1e-9)
    # rays that leave the volume record the trace limit exactly
    s2 = W.Scene()
    s2.add(W.SPHERE, [0.3, 0.3, 0.3, 0.1], (0.5, 0.5, 0.5))
    sc2, _ = oscene(s2, (64, 64, 64), h)
    g2 = grid_for((1, 1, 1), c, (1.0, 1.0, 1.0), 16, tmax_vox=150.0)
    out2 = O.update(sc2, g2, [], W.frame_rotation(2, 0), probes_at([c]))
    assert np.all(O.is_miss(out2["rays"]["event"]))
    tm = 150.0 * h
    assert np.allclose(out2["depth"][0, 1:-1, 1:-1, 0], tm, rtol=1e-14)
    assert np.allclose(out2["depth"][0, 1:-1, 1:-1, 1], tm * tm, rtol=1e-14)


# --------------------------------------------------------------------------- interpolation rule
def _grid_maps(values):
    P = len(values)
    irr = np.zeros((P, O.IRR_T, O.IRR_T, 4))
    irr[..., :3] = np.asarray(values)[:, None, None, :]
    return irr


def test_sample_rule_constant_and_linear():
    dims, org, sp = (4, 3, 5), (1.0, -2.0, 0.5), (0.5, 1.5, 1.0)
    g = grid_for(dims, org, sp, 1)
    pos = W.probe_grid_positions(dims, org, sp)
    rng = np.random.default_rng(4)
    const = _grid_maps(np.tile([[0.3, 0.6, 0.9]], (len(pos), 1)))
    valid = np.ones(len(pos), np.uint8)
    for _ in range(50):
        x = rng.uniform(-5, 8, 3)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        assert np.allclose(O.sample_irradiance(g, const, valid, x, n), [0.3, 0.6, 0.9], rtol=1e-14)
    coef = np.array([0.7, -0.3, 0.2])
    lin = pos @ coef + 5.0
    maps = _grid_maps(np.stack([lin, 2 * lin, 3 * lin], axis=1))
    lo, hi = np.array(org), np.array(org) + (np.array(dims) - 1) * np.array(sp)
    for _ in range(100):
        x = rng.uniform(lo, hi)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        v = x @ coef + 5.0
        assert np.allclose(O.sample_irradiance(g, maps, valid, x, n), [v, 2 * v, 3 * v], rtol=1e-12)


def test_sample_rule_at_probe_and_validity():
    dims, org, sp = (3, 3, 3), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    g = grid_for(dims, org, sp, 1)
    pos = W.probe_grid_positions(dims, org, sp)
    rng = np.random.default_rng(6)
    maps = np.zeros((27, O.IRR_T, O.IRR_T, 4))
    maps[..., :3] = rng.uniform(size=(27, O.IRR_T, O.IRR_T, 3))
    valid = np.ones(27, np.uint8)
    one = grid_for((1, 1, 1), (0, 0, 0), (1, 1, 1), 1)
    for p in range(27):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        own = O.sample_irradiance(one, maps[p:p + 1], np.ones(1, np.uint8), [0, 0, 0], n)
        assert np.allclose(O.sample_irradiance(g, maps, valid, pos[p], n), own, rtol=1e-14)
    # an invalid probe takes no part, whatever its map holds
    x = np.array([0.4, 0.6, 0.5])
    n = np.array([0.0, 0.0, 1.0])
    base = O.sample_irradiance(g, maps, valid, x, n)
    v2 = valid.copy()
    v2[0] = 0
    m2 = maps.copy()
    m2[0] = 1e6
    alt = O.sample_irradiance(g, m2, v2, x, n)
    assert np.all(alt < 10.0) and not np.allclose(alt, base)
    assert np.all(O.sample_irradiance(g, maps, np.zeros(27, np.uint8), x, n) == 0.0)


# --------------------------------------------------------------------------- gather weights (Eq. 3)
def _texel_dir(a, b, n):
    return np.asarray(O.oct_decode([(a + 0.5) / n, (b + 0.5) / n]))


def test_irradiance_weight_emissive_cap_closed_form():
    """Eq. 3 with direction-dependent radiance: an emissive sphere (albedo 0, radiance Le) seen
    from a probe in an otherwise empty box subtends a cap of half-angle alpha. For a texel whose
    hemisphere holds the whole cap (theta + alpha <= 90 deg, theta = angle between the texel and
    the cap centre) the cosine-weighted mean is Le sin^2(alpha) cos(theta) (the cap's irradiance
    pi Le sin^2 alpha cos theta over the hemisphere's pi); a texel whose hemisphere misses the cap
    is exactly 0. A cos^2 weight would give Le (1 - cos^3 alpha) at theta = 0 (here 0.90 against
    0.66), a flipped lobe non-zero far texels."""
    h, dims = 0.25, (64, 64, 64)
    c0 = np.array([8.0, 8.0, 8.0])
    u0 = _texel_dir(2, 3, O.IRR_N)
    D, alpha, Le = 5.0, math.radians(35.0), 2.0
    sc = O.OracleScene.analytic([W.SPHERE], [[*(c0 + D * u0), D * math.sin(alpha), 0, 0, 0]], [[0, 0, 0]],
                                [[Le, Le, Le]], (0, 0, 0), dims, h)
    g = grid_for((1, 1, 1), tuple(c0), (1, 1, 1), 16384, max_steps=4000, tmax_vox=200.0, eps_vox=1e-4)
    maps = [O.update(sc, g, [], W.frame_rotation(11, f), probes_at([c0]), want_rays=False)["irr"][0]
            for f in range(16)]
    mean = np.mean(maps, axis=0)
    n_full = n_zero = 0
    for b in range(O.IRR_N):
        for a in range(O.IRR_N):
            th = math.acos(float(np.clip(_texel_dir(a, b, O.IRR_N) @ u0, -1.0, 1.0)))
            if th + alpha <= math.pi / 2:
                expect = Le * math.sin(alpha) ** 2 * math.cos(th)
                assert np.allclose(mean[b + 1, a + 1, :3], expect, rtol=2e-3), (a, b, mean[b + 1, a + 1], expect)
                n_full += 1
            elif th - alpha >= math.pi / 2:
                assert all(np.all(m[b + 1, a + 1, :3] == 0.0) for m in maps), (a, b)
                n_zero += 1
    assert n_full >= 6 and n_zero >= 6


def _moment_quadrature(u, p, t_of):
    """int max(0,u.d)^p t(d)^k dd / int max(0,u.d)^p dd for k = 1, 2 by Gauss-Legendre in the
    angle psi from u and the trapezoid rule (spectrally accurate, periodic) in its azimuth."""
    xg, wg = np.polynomial.legendre.leggauss(200)
    psi, wpsi = (xg + 1) * (math.pi / 4), wg * (math.pi / 4)
    phi = np.arange(128) * (2 * math.pi / 128)
    a = np.array([1.0, 0.0, 0.0]) if abs(u[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(u, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(u, e1)
    P, F = np.meshgrid(psi, phi, indexing="ij")
    d = (np.cos(P)[..., None] * u + (np.sin(P) * np.cos(F))[..., None] * e1
         + (np.sin(P) * np.sin(F))[..., None] * e2)
    w = np.cos(P) ** p * np.sin(P) * wpsi[:, None]
    t = t_of(d.reshape(-1, 3)).reshape(P.shape)
    return (w * t).sum() / w.sum(), (w * t * t).sum() / w.sum()


def test_depth_moment_weight_exponent_off_centre_ball():
    """The depth moments' weight max(0, u.d)^p: an off-centre probe in a hollow ball sees the
    wall at t(d) = -(c.d) + sqrt((c.d)^2 - |c|^2 + r^2) (c = probe - centre). Every texel's
    moments equal the quadrature of their defining integrals; with p = 40 or 64 instead of 50
    the quadrature moves by ~3e-3, thirty times the tolerance, and a transposed texel index
    reads another direction of this asymmetric field."""
    h, dims = 0.25, (64, 64, 64)
    C, rb = np.array([8.0, 8.0, 8.0]), 6.0
    off = np.array([3.0, -1.5, 2.0])
    sc = O.OracleScene.analytic([W.INV_SPHERE], [[*C, rb, 0, 0, 0]], [[0.5, 0.5, 0.5]], [[0, 0, 0]], (0, 0, 0),
                                dims, h)

    def t_of(d):
        cd = d @ off
        return -cd + np.sqrt(cd * cd - off @ off + rb * rb)

    g = grid_for((1, 1, 1), tuple(C + off), (1, 1, 1), 4096, max_steps=4000, tmax_vox=200.0, eps_vox=1e-4,
                 depth_exponent=50)
    K = 4
    dep = sum(O.update(sc, g, [], W.frame_rotation(13, f), probes_at([C + off]), want_rays=False)["depth"][0]
              for f in range(K)) / K
    rng = np.random.default_rng(8)
    moved = 0.0
    for j in rng.choice(O.DEP_N * O.DEP_N, 24, replace=False):
        a, b = int(j % O.DEP_N), int(j // O.DEP_N)
        u = _texel_dir(a, b, O.DEP_N)
        m1, m2 = _moment_quadrature(u, 50, t_of)
        assert abs(dep[b + 1, a + 1, 0] - m1) <= 1e-4 * m1, (a, b, dep[b + 1, a + 1], m1)
        assert abs(dep[b + 1, a + 1, 1] - m2) <= 2e-4 * m2, (a, b, dep[b + 1, a + 1], m2)
        for p_wrong in (40, 64):
            moved = max(moved, abs(_moment_quadrature(u, p_wrong, t_of)[0] - m1) / m1)
    assert moved > 30 * 1e-4  # the pin tells a wrong exponent apart


# --------------------------------------------------------------------------- float32 rounding bounds
def _trilinear_np(sdf, h, origin, p, ft):
    """The trilinear sampling rule restated in numpy in dtype ft (no fused multiply-add)."""
    nz, ny, nx = sdf.shape
    v = sdf.astype(ft)
    inv_h = ft(1.0) / ft(h)
    idx, fr = [], []
    for a, n in ((0, nx), (1, ny), (2, nz)):
        g = (p[:, a] - ft(origin[a])) * inv_h - ft(0.5)
        i = np.clip(np.floor(g).astype(np.int64), 0, n - 2)
        idx.append(i)
        fr.append(np.clip(g - i.astype(ft), ft(0), ft(1)).astype(ft))
    (ix, iy, iz), (fx, fy, fz) = idx, fr

    def V(dx, dy, dz):
        return v[iz + dz, iy + dy, ix + dx]

    def lerp(a, b, t):
        return a + t * (b - a)

    x00, x10 = lerp(V(0, 0, 0), V(1, 0, 0), fx), lerp(V(0, 1, 0), V(1, 1, 0), fx)
    x01, x11 = lerp(V(0, 0, 1), V(1, 0, 1), fx), lerp(V(0, 1, 1), V(1, 1, 1), fx)
    return lerp(lerp(x00, x10, fy), lerp(x01, x11, fy), fz)


def _room_rays(seed_rot=7, stride=2):
    import harness as H
    w = H.make_workload(W.PRESETS["room64"])
    sub = np.flatnonzero(w.states["flags"] & 1)[::stride]
    rot = W.frame_rotation(seed_rot, 0)
    out = O.update(H.oracle_scene(w), H.oracle_grid(w), w.lights, rot, w.states, subset=sub)
    R = w.params["rays"]
    dirs = np.array([O.sf_dir(i, R) for i in range(R)]) @ rot.astype(np.float64).T
    o = np.repeat(w.states["pos"][sub].astype(np.float64), R, axis=0)
    return w, out["rays"].reshape(-1), o, np.tile(dirs, (len(sub), 1))


def test_t_cond_bounds_a_float32_trace():
    """The oracle's per-ray t_cond (first-order float32 rounding bound of the hit distance,
    propagated through every step) against an actual float32 sphere trace of the same rays on
    the same baked field: wherever the float32 trace takes the oracle's path (event and step
    count), |t_f32 - t_f64| <= t_cond."""
    w, rays, o, d = _room_rays()
    f32, h = np.float32, w.baked.h
    o32, d32 = o.astype(f32), d.astype(f32)
    eps, tl = f32(w.params["eps_vox"] * h), f32(w.params["tmax_vox"] * h)
    lo = np.array(w.baked.origin, f32)
    hi = lo + np.array(w.baked.sdf.shape[::-1], f32) * f32(h)
    n = len(o)
    t, ev, st = np.zeros(n, f32), np.full(n, O.EXHAUSTED), np.full(n, w.params["max_steps"])
    alive = np.ones(n, bool)
    for s in range(w.params["max_steps"]):
        idx = np.flatnonzero(alive)
        if not len(idx):
            break
        p = o32[idx] + t[idx, None] * d32[idx]
        out = np.any((p < lo) | (p > hi), axis=1)
        ev[idx[out]], st[idx[out]], alive[idx[out]] = O.LEFT_VOLUME, s, False
        idx, p = idx[~out], p[~out]
        sd = _trilinear_np(w.baked.sdf, h, w.baked.origin, p, f32)
        hit = sd < eps
        ev[idx[hit]], st[idx[hit]], alive[idx[hit]] = O.HIT, s + 1, False
        idx, sd = idx[~hit], sd[~hit]
        t[idx] = t[idx] + sd
        past = t[idx] > tl
        ev[idx[past]], st[idx[past]], alive[idx[past]] = O.PAST_LIMIT, s + 1, False
    same = (ev == rays["natural_event"]) & (st == rays["natural_steps"]) & ~O.is_miss(ev)
    assert same.sum() > 0.95 * (~O.is_miss(rays["natural_event"])).sum()
    dt = np.abs(t.astype(np.float64) - rays["t"])[same] / h
    assert np.all(dt <= rays["t_cond"][same]), float((dt / rays["t_cond"][same]).max())


def test_float32_shading_normal_cosine_within_eps_nl():
    """The parity bar's EPS_NL: the light cosine n.l of a shading normal normalised from float32
    central differences (six trilinear samples half a voxel off the hit) stays within EPS_NL of
    the same rule in FP64, at the oracle's hit points of a room for 64 seeded light directions."""
    import harness as H
    w, rays, o, d = _room_rays(stride=3)
    h = w.baked.h
    hit = rays["natural_event"] == O.HIT
    x = (o[hit] + rays["t"][hit, None] * d[hit]).astype(np.float32)

    def normal(x, ft):
        g = []
        for a in range(3):
            e = np.zeros(3, ft)
            e[a] = ft(0.5 * h)
            g.append(_trilinear_np(w.baked.sdf, h, w.baked.origin, (x + e).astype(ft), ft)
                     - _trilinear_np(w.baked.sdf, h, w.baked.origin, (x - e).astype(ft), ft))
        g = np.stack(g, 1)
        return g / np.sqrt((g * g).sum(1))[:, None]

    n32 = normal(x, np.float32).astype(np.float64)
    n64 = normal(x.astype(np.float64), np.float64)
    rng = np.random.default_rng(0)
    L = rng.normal(size=(64, 3))
    L /= np.linalg.norm(L, axis=1)[:, None]
    err = np.abs(n32 @ L.T - n64 @ L.T)
    assert err.max() <= H.EPS_NL, float(err.max())
