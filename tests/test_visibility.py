"""Interpolation with SDF probe visibility (Sec. 3.4) on the GPU against the FP64 oracle
(needs a B300).

Values agree to 1e-4 relative (float32 march, float32 ratios softness * sdf / t). A point
is left out where a probe's march takes a rounding-sensitive decision that matters: a hit
test within 2e-4 voxel of the threshold whose other outcome changes the visibility (the
oracle follows both branches to find out), or a march length within 1e-4 voxel of the
probe's distance. At most 1 % of the points are left out.
"""
import numpy as np
import pytest

import oracle as O
import paper_2007_14394_b300 as S
import workloads as W
from harness import DELTA_COS, DELTA_VOX, GpuVolume, make_workload, oracle_grid, oracle_scene

pytestmark = pytest.mark.gpu

SOFTNESS = 8.0


@pytest.fixture(autouse=True)
def _band(cuda_device):
    O.set_delta(DELTA_VOX, DELTA_COS)


def _gpu_sample(vol, pts, nrm, states=None):
    import torch
    p = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.float32)).cuda()
    n = torch.from_numpy(np.ascontiguousarray(nrm, dtype=np.float32)).cuda()
    out = torch.empty_like(p)
    S.sample_irradiance_visible(vol, p, n, out, SOFTNESS, states=states)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _compare(got, pts, nrm, osc, g, irr, valid, probe_pos=None):
    keep, errs = [], []
    for i in range(len(pts)):
        o, vis, marg = O.sample_irradiance_visible(osc, g, irr, valid, pts[i].astype(np.float64),
                                                   nrm[i].astype(np.float64), SOFTNESS, probe_pos)
        sensitive = np.any(marg[:, 0] < DELTA_VOX) or np.any(marg[:, 1] < 1e-4)
        keep.append(not sensitive)
        if not sensitive:
            errs.append(np.abs(got[i] - o).max() / max(np.abs(o).max(), 1e-6))
    keep = np.array(keep)
    assert keep.mean() >= 0.99, keep.mean()
    print("points", len(pts), "compared", int(keep.sum()), "max rel err", max(errs))
    assert max(errs) <= 1e-4


def _random_free_points(osc, h, lo, hi, n, rng, clearance_vox=1.5):
    pts = []
    while len(pts) < n:
        x = rng.uniform(lo, hi)
        if O.sample_sdf(osc, x) > clearance_vox * h:
            pts.append(x)
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return np.array(pts, dtype=np.float32), nrm.astype(np.float32)


def test_wall_has_no_leak(cuda_device):
    h = 0.125
    s = W.Scene()
    s.add(W.BOX, [4.0, 4.0, 4.0, h, 10.0, 10.0], (0.5, 0.5, 0.5))
    baked = W.bake(s, (64, 64, 64), h)
    sc = S.create_scene()
    S.upload_sdf(sc, baked.sdf, h, (0.0, 0.0, 0.0), material=baked.material)
    S.set_lights(sc, [], (0.0, 0.0, 0.0))
    desc = S.make_desc((2, 2, 2), 8, (3.5, 3.5, 3.5), (1.0, 1.0, 1.0), 128)
    v = S.create_volume(desc, sc)
    A, B = np.array([0.2, 0.4, 0.6]), np.array([1.0, 0.8, 0.6])
    irr = np.zeros((8, 8, 8, 4), np.float32)
    for p in range(8):
        irr[p, ..., :3] = A if p % 2 == 0 else B
    irr[..., 3] = 1.0
    S.write_state(v, irr, np.zeros((8, 16, 16, 2), np.float32), np.ones(8, np.uint8))
    try:
        rng = np.random.default_rng(4)
        pts = np.concatenate([rng.uniform([3.5, 3.5, 3.5], [3.82, 4.5, 4.5], (64, 3)),
                              rng.uniform([4.18, 3.5, 3.5], [4.5, 4.5, 4.5], (64, 3))]).astype(np.float32)
        nrm = np.zeros_like(pts)
        nrm[:64, 0], nrm[64:, 0] = -1.0, 1.0
        got = _gpu_sample(v, pts, nrm)
        assert np.allclose(got[:64], A, rtol=0, atol=1e-6) and np.allclose(got[64:], B, rtol=0, atol=1e-6)
        osc = O.OracleScene(baked.sdf, h, (0, 0, 0), baked.material)
        g = O.make_grid((2, 2, 2), (3.5, 3.5, 3.5), (1.0, 1.0, 1.0), 8, 128, 0.01, 0.0, 0.97, bias_vox=1.0)
        _compare(got, pts, nrm, osc, g, irr.astype(np.float64), np.ones(8, np.uint8))
    finally:
        S.destroy_volume(v)
        S.destroy_scene(sc)


def test_room_after_an_update_matches_oracle(cuda_device):
    w = make_workload(W.PRESETS["room64"])
    gv = GpuVolume(w)
    try:
        gv.update(W.frame_rotation(7, 0), record=False)
        irr, _, valid = gv.state()
        osc, g = oracle_scene(w), oracle_grid(w)
        pts, nrm = _random_free_points(osc, w.baked.h, [0.4, 0.4, 0.4], [7.6, 7.6, 7.6], 400,
                                       np.random.default_rng(5))
        got = _gpu_sample(gv.vol, pts, nrm, states=gv.states_dev)
        pos = w.states["pos"]
        _compare(got, pts, nrm, osc, g, irr.astype(np.float64), valid, probe_pos=pos)
        # without visibility some points would take light through walls and objects
        import torch
        plain = torch.empty((len(pts), 3), device="cuda")
        S.sample_irradiance(gv.vol, torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda(), plain)
        assert np.abs(plain.cpu().numpy() - got).max() > 1e-3
    finally:
        gv.close()


def test_visibility_argument_errors(cuda_device):
    w = make_workload(W.PRESETS["room64"], probe_dims=(2, 2, 2))
    gv = GpuVolume(w)
    try:
        import torch
        p = torch.zeros((4, 3), device="cuda")
        for bad in (0.0, -1.0, float("inf")):
            with pytest.raises(S.SdfddgiError):
                S.sample_irradiance_visible(gv.vol, p, p, p, bad)
    finally:
        gv.close()
