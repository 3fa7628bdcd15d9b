"""The probe update on a scene of analytic SDF primitives (Sec. 3.1) against the FP64
oracle, and the exactness of the cluster culling (needs a B300).

The bar is the float32 parity bar of tests/test_gpu_parity.py. One discrete decision is
new: the material of a hit comes from the nearest primitive. The GPU records its choice,
and the oracle follows it only where its own two nearest distances lie within the
rounding band (2e-4 voxel); anywhere else a different choice is a hard mismatch. Cluster
culling and the sphere trace's bound of twice the last distance leave every query at the
minimum over all primitives, so culled and brute-force scenes give the same maps bit for
bit.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from harness import (DELTA_COS, DELTA_VOX, GpuVolume, assert_bar, border_is_mirror,
                     compare, force_from_records, make_workload, oracle_grid, oracle_scene)

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _band(cuda_device):
    O.set_delta(DELTA_VOX, DELTA_COS)


def run_analytic(w, frames=1, subset=None, seed_rot=7, cluster_size=8):
    gv = GpuVolume(w, analytic=True, cluster_size=cluster_size)
    sc, g = oracle_scene(w, analytic=True), oracle_grid(w)
    sub = np.arange(w.P) if subset is None else np.asarray(subset)
    stats = []
    try:
        for f in range(frames):
            prev = gv.state()
            rot = W.frame_rotation(seed_rot, f)
            gv.update(rot)
            cur = gv.state()
            rec = gv.records_np()
            orc = O.update(sc, g, w.lights, rot, w.states,
                           prev=(prev[0].astype(np.float64), prev[1].astype(np.float64), prev[2]),
                           subset=sub, force=force_from_records(rec[sub]))
            s = compare(w, cur, rec, orc, sub, w.baked.h, rot=rot)
            s["border_irr"] = border_is_mirror(cur[0][sub])
            s["border_depth"] = border_is_mirror(cur[1][sub])
            live = orc["rays"]["event"] >= 0
            hits = live & ~O.is_miss(orc["rays"]["event"])
            s["owner_equal"] = float((rec[sub]["material_owner"][hits] == orc["rays"]["owner"][hits]).mean())
            s["owner_forced"] = int((orc["rays"]["owner"] != orc["rays"]["natural_owner"])[hits].sum())
            stats.append(s)
        assert gv.S.volume_status(gv.vol) == 0
    finally:
        gv.close()
    return stats


def test_room_analytic_parity_two_frames():
    w = make_workload(W.PRESETS["room64"], k_bounce=1.0)
    for f, s in enumerate(run_analytic(w, frames=2)):
        print("analytic room frame", f, s)
        assert_bar(s, f"analytic room frame {f}")
        assert s["owner_equal"] == 1.0


def test_open_analytic_sampled():
    w = make_workload(W.PRESETS["open256"])
    rng = np.random.default_rng(6)
    act = np.flatnonzero(w.states["flags"] & 1)
    sub = np.sort(rng.choice(act, 32, replace=False))
    (s,) = run_analytic(w, subset=sub, seed_rot=11)
    print("analytic open", s)
    assert_bar(s, "analytic open")


@pytest.mark.parametrize("preset", ["room64", "open256"])
def test_cluster_culling_is_exact(preset):
    """Includes points inside several overlapping primitives (the open scene's primitives
    overlap each other and the ground), where every box containing the point must be visited."""
    w = make_workload(W.PRESETS[preset])
    if preset == "open256":  # a quarter of the probes keeps the test short
        w = make_workload(W.PRESETS[preset], probe_dims=(16, 8, 16), probe_spacing=(4.0, 4.0, 4.0))
    maps = []
    for cs in (0, 1, 8, 64):
        gv = GpuVolume(w, analytic=True, cluster_size=cs)
        try:
            gv.update(W.frame_rotation(3, 0))
            maps.append((gv.state(), gv.records_np()))
        finally:
            gv.close()
    for (st, rec), cs in zip(maps[1:], (1, 8, 64)):
        assert all(np.array_equal(a, b) for a, b in zip(st, maps[0][0])), (preset, cs)
        assert np.array_equal(rec, maps[0][1]), (preset, cs)


def test_relocation_and_visibility_on_primitives():
    import torch
    import paper_2007_14394_b300 as S
    w = make_workload(W.PRESETS["room64"], probe_origin=(0.3, 0.35, 0.4), probe_spacing=(1.05, 1.0, 1.02))
    gv = GpuVolume(w, analytic=True)
    sc, g = oracle_scene(w, analytic=True), oracle_grid(w)
    try:
        out = torch.empty(w.P * 16, dtype=torch.uint8, device="cuda")
        S.relocate_probes(gv.vol, out, clearance=3.0, max_offset=0.45)
        got = out.cpu().numpy().view(S.PROBE_STATE_DTYPE)
        ref = O.relocate(sc, g, 3.0, 0.0, 0.45, 0.5, 16)
        conv = (ref["iters"] == 0) | (ref["margin"][:, 0] + 0.5 >= 3.0 - 1e-9)
        err = np.abs(got["pos"].astype(np.float64) - ref["pos"]).max(axis=1) / w.baked.h
        print("analytic relocation: converged", int(conv.sum()), "max err", err[conv].max())
        assert err[conv].max() <= 1e-3
        # visibility-weighted interpolation after an update, at free points
        gv.update(W.frame_rotation(7, 0), record=False)
        irr, _, valid = gv.state()
        rng = np.random.default_rng(9)
        pts, nrm = [], []
        while len(pts) < 200:
            x = rng.uniform(0.4, 7.6, 3)
            if O.sample_sdf(sc, x) > 1.5 * w.baked.h:
                pts.append(x)
        pts = np.array(pts, np.float32)
        nrm = rng.normal(size=(200, 3))
        nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
        p_t, n_t = torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda()
        o_t = torch.empty_like(p_t)
        S.sample_irradiance_visible(gv.vol, p_t, n_t, o_t, 8.0, states=gv.states_dev)
        res = o_t.cpu().numpy().astype(np.float64)
        worst = 0.0
        for i in range(200):
            o, _, m = O.sample_irradiance_visible(sc, g, irr.astype(np.float64), valid, pts[i].astype(np.float64),
                                                  nrm[i].astype(np.float64), 8.0, w.states["pos"])
            if np.any(m[:, 0] < DELTA_VOX) or np.any(m[:, 1] < 1e-4):
                continue
            worst = max(worst, np.abs(res[i] - o).max() / max(np.abs(o).max(), 1e-6))
        print("analytic visibility max rel err", worst)
        assert worst <= 1e-4
    finally:
        gv.close()
