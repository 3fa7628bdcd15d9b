"""Parity of the CUDA probe update with the FP64 oracle (needs a B300).

Every test drives the library through its C ABI on seeded synthetic inputs and
compares element by element with the oracle run on the same float32 data.
Discrete decisions (sphere-trace termination step, exit event, light visibility)
that the oracle finds within a rounding band of their threshold follow the GPU's
outcome; every such decision is counted, and one outside the band is a hard
mismatch. The bar (float32 path):
  hard mismatches 0; hit/miss agreement >= 99.9% of non-grazing rays;
  hit distance within 1e-3 voxel; irradiance and moments relative error <= 1e-4;
  borders bit-exact mirrors; history flags equal.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
import workloads as W
from harness import (DELTA_VOX, DELTA_COS, GpuVolume, assert_bar, border_is_mirror,
                     compare, f32, f32v, force_from_records, make_workload, oracle_grid, oracle_scene)

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _band(cuda_device):
    O.set_delta(DELTA_VOX, DELTA_COS)


def run_and_compare(w, frames=1, subset=None, seed_rot=7, prev_gpu=None, record_check=False):
    """Runs `frames` GPU updates; each frame is compared with the oracle started from the GPU's
    previous maps (teacher forcing). Returns the list of per-frame statistics."""
    gv = GpuVolume(w)
    sc, g = oracle_scene(w), oracle_grid(w)
    h = w.baked.h
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
            s = compare(w, cur, rec, orc, sub, h, rot=rot)
            s["border_irr"] = border_is_mirror(cur[0][sub])
            s["border_depth"] = border_is_mirror(cur[1][sub])
            stats.append(s)
            if record_check and f == 0:
                # the record writes must not change the computation
                gv.S.write_state(gv.vol, *prev)
                gv.update(rot, record=False)
                again = gv.state()
                s["records_neutral"] = all(np.array_equal(a, b) for a, b in zip(again, cur))
        assert gv.S.volume_status(gv.vol) == 0  # no device-side failure recorded
    finally:
        gv.close()
    return stats


def test_room64_full_parity():
    w = make_workload(W.PRESETS["room64"])
    (s,) = run_and_compare(w, record_check=True)
    print("room64", s)
    assert s["rays"] > 20000
    assert_bar(s, "room64")
    assert s["records_neutral"]


def test_room64_multiframe_multibounce():
    w = make_workload(W.PRESETS["room64"], k_bounce=1.0)
    stats = run_and_compare(w, frames=4)
    for f, s in enumerate(stats):
        print("frame", f, s)
        assert_bar(s, f"frame {f}")


def test_open256_full_size_sampled():
    """The 256^3 open scene at full size and in the bench's launch configuration (two slab
    branches); the oracle checks a seeded sample of probes (active and inactive) in each of
    8 consecutive frames, every frame after the first lit through the previous frame's
    probes (multi-bounce)."""
    w = make_workload(W.PRESETS["open256"])
    rng = np.random.default_rng(5)
    act = np.flatnonzero(w.states["flags"] & 1)
    ina = np.flatnonzero((w.states["flags"] & 1) == 0)
    sub = np.sort(np.concatenate([rng.choice(act, 48, replace=False), ina[:4]]))
    stats = run_and_compare(w, frames=8, subset=sub, seed_rot=11)
    for f, s in enumerate(stats):
        print("open256 frame", f, s)
        assert_bar(s, f"open256 frame {f}")


def test_odd_depth_unequal_sides():
    """An SDF of 64 x 56 x 61 voxels: unequal sides and an odd depth, so the last z-pair of
    the quad store holds one slice; probes fill the cut room."""
    pr = dataclasses.replace(W.PRESETS["room64"], sdf_dims=(64, 56, 61))
    w = make_workload(pr, probe_dims=(6, 5, 6), probe_origin=(0.7, 0.6, 0.5), probe_spacing=(1.1, 1.2, 1.2))
    (s,) = run_and_compare(w)
    print("64x56x61", s)
    assert s["rays"] > 5000
    assert_bar(s, "64x56x61")


@pytest.mark.parametrize("n_lights", [0, 32])
def test_light_counts(n_lights):
    """No light (no shadow task at all) and the most a scene holds, 32 (every value of the
    tasks' 5-bit light index and every bit of the visibility mask)."""
    w = make_workload(W.PRESETS["room64"], probe_dims=(4, 4, 4), probe_origin=(1.2, 1.2, 1.2),
                      probe_spacing=(1.8, 1.8, 1.8))
    rng = np.random.default_rng(n_lights)
    points = [{"type": "point", "v": f32v(rng.uniform(1.0, 7.0, 3)), "rgb": f32v(rng.uniform(0.5, 4.0, 3)),
               "range": f32(rng.uniform(2.0, 6.0))} for _ in range(max(n_lights - 1, 0))]
    w = dataclasses.replace(w, lights=(w.lights[:1] + points) if n_lights else [])
    (s,) = run_and_compare(w)
    print(n_lights, "lights", s)
    assert_bar(s, f"{n_lights} lights")


def test_one_step_budget_and_probes_outside_the_box():
    """A budget of one step (every ray that does not hit at once ends exhausted, shaded where
    it stopped) and active probes outside the volume box (x = -1 and 8.6 m for an 8 m box:
    their rays leave before their first sample)."""
    w = make_workload(W.PRESETS["room64"], max_steps=1, probe_dims=(4, 3, 3), probe_origin=(-1.0, 2.0, 2.0),
                      probe_spacing=(3.2, 2.0, 2.0))
    outside = (w.states["pos"][:, 0] < 0) | (w.states["pos"][:, 0] > 8)
    assert (w.states["flags"][outside] & 1).all() and outside.sum() == 18
    (s,) = run_and_compare(w)
    print("one step", s)
    assert_bar(s, "one step, probes outside")


@pytest.mark.parametrize("rays", [1, 7, 33, 1000, 1024])
def test_ray_counts(rays):
    w = make_workload(W.PRESETS["room64"], rays=rays, probe_dims=(3, 2, 3), probe_origin=(1.5, 2.0, 1.5),
                      probe_spacing=(2.5, 3.0, 2.5))
    (s,) = run_and_compare(w)
    assert_bar(s, f"R={rays}")


@pytest.mark.parametrize("dims", [(1, 1, 1), (5, 1, 3), (1, 7, 1)])
def test_probe_grid_shapes(dims):
    w = make_workload(W.PRESETS["room64"], rays=48, probe_dims=dims, probe_origin=(1.25, 1.75, 2.25),
                      probe_spacing=(1.1, 0.9, 1.3))
    stats = run_and_compare(w, frames=2)
    for s in stats:
        assert_bar(s, str(dims))


def test_fp16_sdf_matches_oracle_on_same_values():
    w = make_workload(W.PRESETS["room64"], sdf_dtype="f16")
    assert w.baked.sdf.dtype == np.float16
    (s,) = run_and_compare(w)
    assert_bar(s, "fp16 sdf")


def test_inactive_and_rejected_probes():
    w = make_workload(W.PRESETS["room64"], rays=32)
    gv = GpuVolume(w)
    try:
        # two frames of history, then a frame with every probe inactive: maps unchanged
        for f in range(2):
            gv.update(W.frame_rotation(1, f))
        before = gv.state()
        off = w.states.copy()
        off["flags"] = 0
        gv.update(W.frame_rotation(1, 2), states=gv.torch.from_numpy(off.view(np.uint8).copy()).cuda())
        after = gv.state()
        assert all(np.array_equal(a, b) for a, b in zip(before, after))
        rec = gv.records_np()
        assert np.all(rec["event"] == 255)
    finally:
        gv.close()
    # a rejected history equals no history (without the bounce term, which reads the old maps)
    w0 = make_workload(W.PRESETS["room64"], rays=32, k_bounce=0.0)
    rej = w0.states.copy()
    rej["flags"] |= W.REJECT_HISTORY
    act = (w0.states["flags"] & 1).astype(bool)
    gv = GpuVolume(w0)
    try:
        rot = W.frame_rotation(1, 3)
        gv.update(W.frame_rotation(1, 0))
        gv.update(rot, states=gv.torch.from_numpy(rej.view(np.uint8).copy()).cuda())
        rejected = gv.state()
        gv.S.reset(gv.vol)
        gv.update(rot)
        fresh = gv.state()
        assert np.array_equal(rejected[0][act], fresh[0][act])
        assert np.array_equal(rejected[1][act], fresh[1][act])
    finally:
        gv.close()


def test_library_rotation_matches_generator():
    w = make_workload(W.PRESETS["room64"], rays=16)
    gv = GpuVolume(w)
    try:
        gv.S.update_probes(gv.vol, 5, rotation=None, states=gv.states_dev)  # seed 0, frame 5
        a = gv.state()
        gv.S.reset(gv.vol)
        gv.update(W.frame_rotation(0, 5), record=False)
        b = gv.state()
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
    finally:
        gv.close()


def test_sample_irradiance_matches_oracle():
    import torch
    w = make_workload(W.PRESETS["room64"], k_bounce=1.0)
    gv = GpuVolume(w)
    try:
        for f in range(2):
            gv.update(W.frame_rotation(2, f), record=False)
        irr, dep, val = gv.state()
        rng = np.random.default_rng(0)
        n = 5000
        pts = rng.uniform(-0.5, 8.5, (n, 3)).astype(np.float32)
        nrm = rng.normal(size=(n, 3))
        nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
        out = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        gv.S.sample_irradiance(gv.vol, torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda(), out)
        got = out.cpu().numpy()
        g = oracle_grid(w)
        ref = np.array([O.sample_irradiance(g, irr.astype(np.float64), val, pts[i], nrm[i]) for i in range(n)])
        err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-6 * np.abs(ref).max())
        assert err.max() <= 1e-5, err.max()
        # empty batch is a no-op
        gv.S.sample_irradiance(gv.vol, torch.empty((0, 3), device="cuda"), torch.empty((0, 3), device="cuda"),
                               torch.empty((0, 3), device="cuda"))
    finally:
        gv.close()
