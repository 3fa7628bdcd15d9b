"""Irradiance from a cascade of probe volumes (Sec. 3.5) on the GPU against the FP64 oracle
(needs a B300).

Three nested volumes hold random maps (border fixed up, one probe in five without history).
Every box bound and spacing is exact in float, so the finest volume that holds a point, a
discrete decision, must match the oracle's bit for bit. The transition weight is the float
evaluation of the mean value coordinates' face integrals. Its bar is 2e-6: a few units
of float rounding (6e-8 each) over the 12 face terms and the ratio, and nothing cancels
in them. The irradiance's bar adds that weight error times |E_k - E_k+1| to the plain
interpolation's relative 1e-5 of each level (that test's bar in test_gpu_parity.py).
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

W_TOL = 2e-6
REL = 1e-5
# (dims, origin, spacing), finest first; every bound is a float
LEVELS = [((12, 8, 12), (-2.75, -1.5, -3.0), (0.5, 0.5, 0.5)),
          ((16, 8, 16), (-15.0, -4.0, -16.0), (2.0, 2.0, 2.0)),
          ((16, 8, 16), (-64.0, -8.0, -60.0), (8.0, 8.0, 8.0))]


class Cascade:
    def __init__(self, levels, seed=0):
        import torch
        import paper_2007_14394_b300 as S
        self.S, self.torch = S, torch
        rng = np.random.default_rng(seed)
        self.scene = S.create_scene()
        self.vols, self.grids, self.irr, self.valid = [], [], [], []
        for dims, origin, sp in levels:
            v = S.create_volume(S.make_desc(dims, 64, origin, sp, 64), self.scene)
            P = int(np.prod(dims))
            irr = rng.uniform(0.05, 1.0, (P, 8, 8, 4))
            for p in range(P):
                irr[p] = O.border(irr[p])
            irr = irr.astype(np.float32)
            valid = (rng.random(P) < 0.8).astype(np.uint8)
            S.write_state(v, irr, np.zeros((P, 16, 16, 2), np.float32), valid)
            self.vols.append(v)
            self.grids.append(O.make_grid(dims, origin, sp, 64, 64, 0.01, 100.0, 0.97))
            self.irr.append(irr.astype(np.float64))
            self.valid.append(valid)
        torch.cuda.synchronize()

    def sample(self, pts, nrm, vols=None):
        t = self.torch
        n = len(pts)
        out = t.empty((n, 3), dtype=t.float32, device="cuda")
        lvl = t.empty(n, dtype=t.int32, device="cuda")
        w = t.empty(n, dtype=t.float32, device="cuda")
        self.S.sample_irradiance_cascade(self.vols if vols is None else vols, t.from_numpy(pts).cuda(),
                                         t.from_numpy(nrm).cuda(), out, lvl, w)
        return out.cpu().numpy(), lvl.cpu().numpy(), w.cpu().numpy()

    def reference(self, x, n, levels=None):
        k = range(len(self.grids)) if levels is None else levels
        grids, irr, valid = [self.grids[i] for i in k], [self.irr[i] for i in k], [self.valid[i] for i in k]
        out, w, lvl = O.sample_irradiance_cascade(grids, irr, valid, x.astype(np.float64), n.astype(np.float64))
        ek = O.sample_irradiance(grids[lvl], irr[lvl], valid[lvl], x, n)
        ec = O.sample_irradiance(grids[lvl + 1], irr[lvl + 1], valid[lvl + 1], x, n) if lvl + 1 < len(grids) else ek
        return out, w, lvl, ek, ec

    def close(self):
        for v in self.vols:
            self.S.destroy_volume(v)
        self.S.destroy_scene(self.scene)


@pytest.fixture(scope="module")
def cascade(cuda_device):
    c = Cascade(LEVELS)
    yield c
    c.close()


def unit_normals(rng, n):
    v = rng.normal(size=(n, 3))
    return (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)


def box(level):
    dims, origin, sp = level
    lo = np.array(origin)
    return lo, lo + (np.array(dims) - 1) * np.array(sp), np.array(sp)


def edge_points():
    """Points on the boxes' faces, edges and corners, on the inner boxes, beside the inner
    boxes' faces and edges by a few float steps, and outside every box."""
    pts = []
    for level in LEVELS[:2]:
        lo, hi, sp = box(level)
        ilo, ihi = lo + sp, hi - sp
        mid = 0.5 * (lo + hi)
        for c in range(8):                                       # probe box and inner box corners
            pts.append(np.where([c & 1, c & 2, c & 4], hi, lo))
            pts.append(np.where([c & 1, c & 2, c & 4], ihi, ilo))
        for a in range(3):
            for v in (lo[a], hi[a], ilo[a], ihi[a]):             # on each face plane, mid-face
                x = mid.copy()
                x[a] = v
                pts.append(x)
            for v in (ilo[a], ihi[a]):                           # beside an inner face, outside it
                for d in (-3e-6, 4e-7, 2e-5):
                    x = mid.copy()
                    x[a] = v + d * sp[a]
                    x[(a + 1) % 3] = 0.5 * (lo[(a + 1) % 3] + ilo[(a + 1) % 3])
                    pts.append(x)
            x = ilo.copy()                                        # along an inner edge, just outside
            x[a] = mid[a]
            x[(a + 1) % 3] -= 1e-6 * sp[a]
            pts.append(x)
    lo, hi, _ = box(LEVELS[-1])
    pts += [hi + 3.0, lo - 1.0, np.array([hi[0] + 5.0, 0.0, 0.0])]  # outside every box
    return np.array(pts, np.float32)


def check(c, pts, nrm, got, lvl, w):
    bad = []
    for i in range(len(pts)):
        ref, wr, lr, ek, ec = c.reference(pts[i], nrm[i])
        if lvl[i] != lr:
            bad.append((i, "level", lvl[i], lr))
            continue
        if abs(w[i] - wr) > W_TOL:
            bad.append((i, "weight", w[i], wr))
            continue
        scale = np.maximum(np.maximum(np.abs(ek), np.abs(ec)), 1e-3)
        tol = W_TOL * np.abs(ek - ec) + REL * scale
        if np.any(np.abs(got[i] - ref) > tol):
            bad.append((i, "rgb", got[i], ref))
    assert not bad, (len(bad), bad[:5])


def test_cascade_matches_oracle(cascade):
    rng = np.random.default_rng(1)
    parts = []
    for level, n in zip(LEVELS, (1500, 1500, 1000)):            # concentrated around each box's shell
        lo, hi, sp = box(level)
        parts.append(rng.uniform(lo - 0.5 * sp, hi + 0.5 * sp, (n, 3)))
    pts = np.concatenate(parts).astype(np.float32)
    nrm = unit_normals(rng, len(pts))
    got, lvl, w = cascade.sample(pts, nrm)
    shell = (w > 0) & (w < 1)
    print("points", len(pts), "in a transition", int(shell.sum()), "levels", np.bincount(lvl))
    assert shell.sum() > 500 and np.all(np.bincount(lvl, minlength=3) > 300)
    check(cascade, pts, nrm, got, lvl, w)


def test_cascade_edge_points(cascade):
    pts = edge_points()
    nrm = unit_normals(np.random.default_rng(2), len(pts))
    got, lvl, w = cascade.sample(pts, nrm)
    check(cascade, pts, nrm, got, lvl, w)
    for level in LEVELS[:2]:                                     # exact limits
        lo, hi, sp = box(level)
        on_outer = np.any((pts == lo.astype(np.float32)) | (pts == hi.astype(np.float32)), axis=1)
        inside = np.all((pts >= lo) & (pts <= hi), axis=1)
        k = LEVELS.index(level)
        sel = on_outer & inside & (lvl == k)
        assert np.all(w[sel] == 0.0)
        inner = np.all((pts >= lo + sp) & (pts <= hi - sp), axis=1) & (lvl == k)
        assert inner.any() and np.all(w[inner] == 1.0)


def test_single_volume_and_thin_volume(cascade):
    """A one-volume cascade is the plain interpolation bit for bit; a volume with 3 probes along
    an axis has no transition."""
    import paper_2007_14394_b300 as S
    t = cascade.torch
    rng = np.random.default_rng(3)
    lo, hi, sp = box(LEVELS[1])
    pts = rng.uniform(lo - sp, hi + sp, (2000, 3)).astype(np.float32)
    nrm = unit_normals(rng, len(pts))
    got, lvl, w = cascade.sample(pts, nrm, vols=[cascade.vols[1]])
    plain = t.empty((len(pts), 3), dtype=t.float32, device="cuda")
    S.sample_irradiance(cascade.vols[1], t.from_numpy(pts).cuda(), t.from_numpy(nrm).cuda(), plain)
    assert np.array_equal(got, plain.cpu().numpy()) and np.all(lvl == 0) and np.all(w == 1.0)
    thin = Cascade([((3, 6, 5), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)), LEVELS[2]], seed=4)
    try:
        pts = rng.uniform(-0.5, 5.5, (500, 3)).astype(np.float32)
        nrm = unit_normals(rng, len(pts))
        got, lvl, w = thin.sample(pts, nrm)
        assert np.all(w == 1.0)
        check(thin, pts, nrm, got, lvl, w)
    finally:
        thin.close()


def test_cascade_arguments(cascade):
    import paper_2007_14394_b300 as S
    t = cascade.torch
    e = t.empty((0, 3), device="cuda")
    S.sample_irradiance_cascade(cascade.vols, e, e, e)           # empty batch: no launch
    with pytest.raises(S.SdfddgiError):
        S.sample_irradiance_cascade([], e, e, e)
    with pytest.raises(S.SdfddgiError):
        S.sample_irradiance_cascade(cascade.vols * 3, e, e, e)   # 9 > 8 volumes
    with pytest.raises(S.SdfddgiError):
        S.sample_irradiance_cascade([cascade.vols[0], None], e, e, e)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(S.SdfddgiError):
            S.sample_irradiance_cascade(cascade.vols, e, e, e, softness=bad)
    with pytest.raises(S.SdfddgiError):                          # visibility needs the scenes' SDF
        S.sample_irradiance_cascade(cascade.vols, e, e, e, softness=8.0)


def test_cascade512_query_full_size_sampled(cuda_device):
    """The bench's workload and launch: the 4 cascade512 volumes with their random maps, all
    2,073,600 points in one call; 3000 sampled points (and every point whose weight is
    strictly between 0 and 1 among them) checked against the oracle."""
    import torch
    import paper_2007_14394_b300 as S
    import workloads as W
    c = W.CASCADES["cascade512"]
    maps = W.cascade_query_maps(c)
    sc = S.create_scene()
    vols = []
    try:
        for i, v in enumerate(c.volumes):
            vols.append(S.create_volume(S.make_desc(v.probe_dims, v.rays, v.probe_origin, v.probe_spacing,
                                                    v.max_steps, volume_id=i), sc))
            S.write_state(vols[i], maps[i][0], np.zeros((v.n_probes, 16, 16, 2), np.float32), maps[i][1])
        pts, nrm = W.cascade_query_points()
        n = len(pts)
        out = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        lvl = torch.empty(n, dtype=torch.int32, device="cuda")
        wgt = torch.empty(n, dtype=torch.float32, device="cuda")
        S.sample_irradiance_cascade(vols, torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda(), out, lvl, wgt)
        got, lv, w = out.cpu().numpy(), lvl.cpu().numpy(), wgt.cpu().numpy()
        assert np.all(np.isfinite(got)) and np.all((w >= 0) & (w <= 1))
        rng = np.random.default_rng(8)
        sample = rng.choice(n, 3000, replace=False)
        print("levels", np.bincount(lv, minlength=4), "blending", int(((w < 1) & (lv < 3)).sum()))
        grids = [O.make_grid(v.probe_dims, v.probe_origin, v.probe_spacing, v.rays, v.max_steps, v.eps_vox,
                             v.tmax_vox, v.hysteresis) for v in c.volumes]
        irr = [m[0].astype(np.float64) for m in maps]
        valid = [m[1] for m in maps]
        bad = []
        for i in sample:
            x, nn = pts[i].astype(np.float64), nrm[i].astype(np.float64)
            ref, wr, lr = O.sample_irradiance_cascade(grids, irr, valid, x, nn)
            ek = O.sample_irradiance(grids[lr], irr[lr], valid[lr], x, nn)
            ec = O.sample_irradiance(grids[lr + 1], irr[lr + 1], valid[lr + 1], x, nn) if lr < 3 else ek
            scale = np.maximum(np.maximum(np.abs(ek), np.abs(ec)), 1e-3)
            if lv[i] != lr or abs(w[i] - wr) > W_TOL or np.any(np.abs(got[i] - ref) > W_TOL * np.abs(ek - ec) + REL * scale):
                bad.append((int(i), int(lv[i]), lr, float(w[i]), wr))
        assert not bad, (len(bad), bad[:5])
    finally:
        for v in vols:
            S.destroy_volume(v)
        S.destroy_scene(sc)


def test_cascade_with_visibility_matches_oracle(cuda_device):
    """Probe visibility (Sec. 3.4) in every level but the farthest (Sec. 3.5), over the room64
    scene: 3 levels (0.5 m, 1 m, 2.5 m spacing), random maps, the finest level's probes moved
    off their grid positions (probe states). The bar adds the visibility interpolation's
    (relative 1e-4; points whose march takes a rounding-sensitive decision are left out, at
    most 1 %) to the weight's."""
    import torch
    import paper_2007_14394_b300 as S
    import workloads as W
    from harness import DELTA_COS, DELTA_VOX, GpuVolume, make_workload, oracle_scene
    O.set_delta(DELTA_VOX, DELTA_COS)
    w = make_workload(W.PRESETS["room64"])
    gv = GpuVolume(w)
    levels = [((9, 9, 9), (2.0, 2.0, 2.0), (0.5, 0.5, 0.5)), ((8, 8, 8), (0.5, 0.5, 0.5), (1.0, 1.0, 1.0)),
              ((4, 4, 4), (0.25, 0.25, 0.25), (2.5, 2.5, 2.5))]
    rng = np.random.default_rng(11)
    vols, grids, irrs, valids = [], [], [], []
    try:
        for dims, origin, sp in levels:
            v = S.create_volume(S.make_desc(dims, 64, origin, sp, 64, eps=0.01, normal_bias=1.0), gv.scene)
            vols.append(v)
            P = int(np.prod(dims))
            irr = rng.uniform(0.05, 1.0, (P, 8, 8, 4)).astype(np.float32)
            valid = (rng.random(P) < 0.9).astype(np.uint8)
            S.write_state(v, irr, np.zeros((P, 16, 16, 2), np.float32), valid)
            grids.append(O.make_grid(dims, origin, sp, 64, 64, 0.01, 100.0, 0.97, bias_vox=1.0))
            irrs.append(irr.astype(np.float64))
            valids.append(valid)
        d0, o0, s0 = levels[0]
        P0 = int(np.prod(d0))
        st = np.zeros(P0, S.PROBE_STATE_DTYPE)
        idx = np.stack(np.meshgrid(*[np.arange(k) for k in d0], indexing="ij"), -1).transpose(2, 1, 0, 3).reshape(-1, 3)
        st["pos"] = (np.array(o0) + idx * np.array(s0) + rng.uniform(-0.1, 0.1, (P0, 3))).astype(np.float32)
        st["flags"] = 1
        st_dev = torch.from_numpy(st.view(np.uint8).copy()).cuda()
        osc = oracle_scene(w)
        pts = []
        while len(pts) < 600:
            x = rng.uniform(1.5, 6.5, 3) if len(pts) < 400 else rng.uniform(0.4, 7.6, 3)
            if O.sample_sdf(osc, x) > 1.5 * w.baked.h:
                pts.append(x)
        pts = np.array(pts, np.float32)
        nrm = unit_normals(rng, len(pts))
        n = len(pts)
        out = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        lvl = torch.empty(n, dtype=torch.int32, device="cuda")
        wgt = torch.empty(n, dtype=torch.float32, device="cuda")
        S.sample_irradiance_cascade(vols, torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda(), out, lvl, wgt,
                                    softness=8.0, states=[st_dev, None, None])
        got, lv, wg = out.cpu().numpy(), lvl.cpu().numpy(), wgt.cpu().numpy()
        plain = torch.empty_like(out)
        S.sample_irradiance_cascade(vols, torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda(), plain)
        assert np.abs(plain.cpu().numpy() - got).max() > 1e-3        # visibility changes the result
        keep, worst = 0, 0.0
        for i in range(n):
            ref, wr, lr, m = O.sample_irradiance_cascade_visible([osc] * 3, grids, irrs, valids, pts[i].astype(np.float64),
                                                                 nrm[i].astype(np.float64), 8.0,
                                                                 probe_pos=[st["pos"], None, None])
            assert lv[i] == lr and abs(wg[i] - wr) <= W_TOL, (i, lv[i], lr, wg[i], wr)
            if np.any(m[..., 0] < DELTA_VOX) or np.any(m[..., 1] < 1e-4):
                continue
            keep += 1
            # the maps lie in [0.05, 1), so |E_k - E_k+1| < 1
            tol = 1e-4 * max(np.abs(ref).max(), 1e-3) + W_TOL
            worst = max(worst, float(np.abs(got[i] - ref).max() / tol))
        print("visibility cascade: points", n, "compared", keep, "levels", np.bincount(lv, minlength=3),
              "max error / bar", worst)
        assert keep >= 0.99 * n and worst <= 1.0
    finally:
        for v in vols:
            S.destroy_volume(v)
        gv.close()
