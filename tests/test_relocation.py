"""Probe relocation (Sec. 3.2, UpdateProbePos) on the GPU against the FP64 oracle, and an
update driven by the relocated probes (needs a B300).

Probes whose descent converged (it reached the clearance level) agree with the oracle to
float32 rounding of a few Gauss-Newton steps: 1e-3 voxel, flags equal. A descent that did
not converge is ill-conditioned: it wanders against the displacement limit, or meets a
vanishing gradient inside geometry, and its path depends on rounding (differences of a
few hundredths of a voxel after 16 clamped steps). For such a probe the result is checked
for validity instead of equality: it lies within the displacement limit of its grid
position, its ACTIVE flag agrees with the oracle's SDF at the GPU's position, and its
REJECT_HISTORY flag agrees with its distance from last frame's position. Decisions within
1e-3 voxel (clearance) or 1e-5 m (rejection) of their threshold are rounding-sensitive
and not compared.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
import paper_2007_14394_b300 as S
import workloads as W
from harness import (DELTA_COS, DELTA_VOX, GpuVolume, assert_bar, border_is_mirror,
                     compare, force_from_records, make_workload, oracle_grid, oracle_scene)

pytestmark = pytest.mark.gpu

POS_TOL_VOX = 1e-3


def _check(got, ref, w, label, clearance, max_offset=0.45, min_clearance=0.5, reject=0.0, last=None):
    h = w.baked.h
    gpos = got["pos"].astype(np.float64)
    err = np.abs(gpos - ref["pos"]).max(axis=1) / h
    s_end = ref["margin"][:, 0] + min_clearance                 # the oracle's final SDF, voxels
    conv = (ref["iters"] == 0) | (s_end >= clearance - 1e-9)
    print(label, "moved", int((ref["iters"] > 0).sum()), "of", len(err), "converged", int(conv.sum()),
          "max err (voxels)", err[conv].max())
    assert conv.sum() > 0.8 * len(err)  # this grid is pushed into geometry on purpose
    # converged: equal to the oracle
    assert err[conv].max() <= POS_TOL_VOX, label
    band = (np.abs(ref["margin"][:, 0]) < 1e-3) | (np.abs(ref["margin"][:, 1]) < 1e-5)
    same = got["flags"] == ref["flags"]
    assert np.all((same | band)[conv]), (label, np.flatnonzero(~same & ~band & conv))
    # not converged: a valid outcome of the descent
    home = W.probe_grid_positions(w.params["probe_dims"], w.params["probe_origin"], w.params["probe_spacing"])
    lim = max_offset * np.asarray(w.params["probe_spacing"])
    sc = oracle_scene(w)
    base = home if last is None else np.asarray(last, dtype=np.float64)
    for i in np.flatnonzero(~conv):
        assert np.all(np.abs(gpos[i] - home[i]) <= lim + 1e-5), (label, i)
        s_vox = O.sample_sdf(sc, gpos[i]) / h
        if abs(s_vox - min_clearance) > 1e-3:
            assert bool(got["flags"][i] & 1) == (s_vox > min_clearance), (label, i, s_vox)
        d = np.linalg.norm(gpos[i] - base[i])
        if reject > 0 and abs(d - reject) > 1e-5:
            assert bool(got["flags"][i] & 2) == (d > reject), (label, i, d)


def _relocate(gv, out, last=None, **kw):
    S.relocate_probes(gv.vol, out, last=last, **kw)
    gv.torch.cuda.synchronize()
    return out.cpu().numpy().view(S.PROBE_STATE_DTYPE).copy()


@pytest.fixture
def room(cuda_device):
    # grid shifted toward the walls and into the primitives: many probes need to move
    w = make_workload(W.PRESETS["room64"], probe_origin=(0.3, 0.35, 0.4), probe_spacing=(1.05, 1.0, 1.02))
    gv = GpuVolume(w)
    yield w, gv
    gv.close()


def test_relocation_matches_oracle(room):
    import torch
    w, gv = room
    out = torch.empty(w.P * 16, dtype=torch.uint8, device="cuda")
    kw = dict(clearance=3.0, reject_distance=0.05, max_offset=0.45, min_clearance=0.5, max_iterations=16)
    got = _relocate(gv, out, **kw)
    ref = O.relocate(oracle_scene(w), oracle_grid(w), 3.0, 0.05, 0.45, 0.5, 16)
    assert (ref["iters"] > 0).sum() > 50
    assert np.any(ref["flags"] == 0) and np.any(ref["flags"] == 3) and np.any(ref["flags"] == 1)
    _check(got, ref, w, "grid", 3.0, reject=0.05)


def test_relocation_from_last_positions_in_place(room):
    import torch
    w, gv = room
    out = torch.empty(w.P * 16, dtype=torch.uint8, device="cuda")
    first = _relocate(gv, out, clearance=2.0, max_offset=0.3)
    # next frame: a larger clearance, last frame's states as input, written over them
    got = _relocate(gv, out, last=out, clearance=4.0, reject_distance=0.1, max_offset=0.45)
    ref = O.relocate(oracle_scene(w), oracle_grid(w), 4.0, 0.1, 0.45, 0.5, 16, last_pos=first["pos"])
    _check(got, ref, w, "from last", 4.0, reject=0.1, last=first["pos"])
    assert np.any(ref["flags"] & 2) and np.any((ref["flags"] & 2) == 0)


def test_update_with_relocated_probes_matches_oracle(room):
    import torch
    O.set_delta(DELTA_VOX, DELTA_COS)
    w, gv = room
    out = torch.empty(w.P * 16, dtype=torch.uint8, device="cuda")
    states = _relocate(gv, out, clearance=3.0, max_offset=0.45)
    wr = dataclasses.replace(w, states=states.view(W.PROBE_DTYPE))
    rot = W.frame_rotation(7, 0)
    S.update_probes(gv.vol, 0, rotation=rot, states=out, records=gv.records)
    cur = gv.state()
    rec = gv.records_np()
    orc = O.update(oracle_scene(wr), oracle_grid(wr), wr.lights, rot, wr.states, subset=np.arange(w.P),
                   force=force_from_records(rec))
    s = compare(wr, cur, rec, orc, np.arange(w.P), w.baked.h, rot=rot)
    s["border_irr"] = border_is_mirror(cur[0])
    s["border_depth"] = border_is_mirror(cur[1])
    print("relocated update", s)
    assert_bar(s, "relocated update")
    assert S.volume_status(gv.vol) == 0


def test_relocation_argument_errors(room):
    import torch
    w, gv = room
    out = torch.empty(w.P * 16, dtype=torch.uint8, device="cuda")
    for bad in (dict(max_offset=0.6), dict(max_iterations=65), dict(min_clearance=-1.0),
                dict(clearance=float("nan"))):
        with pytest.raises(S.SdfddgiError):
            S.relocate_probes(gv.vol, out, **bad)
