"""The batched update of several probe volumes in one graph launch (needs a B300).

Sec. 3.5 covers a large scene with cascaded probe volumes of different density, all
updated every frame. A batch records the stages of all its volumes either as parallel
branches of one CUDA graph or, merged, as one launch per stage over every volume. Each
volume must come out exactly as a plain update of that volume with the same launch shapes
would leave it. These tests check that bit for bit over several frames: in both forms, with
both gathers, after scene changes, after the autotuner has chosen schedules and form, and at
the full 4-volume cascade size. At that size the oracle also checks a sample of every
volume's probes.
"""
import numpy as np
import pytest

import oracle as O
import paper_2007_14394_b300 as S
import workloads as W
from harness import (DELTA_COS, DELTA_VOX, REL_TOL, GpuVolume, assert_bar,
                     border_is_mirror, compare, force_from_records, make_cascade, make_workload, oracle_grid,
                     oracle_scene, rel_err)

pytestmark = pytest.mark.gpu

SEED = 3


def room_members():
    """Three volumes over the room64 scene: the preset grid (64 rays, tensor-core gather),
    a small offset grid at 33 rays (SIMT gather) and a coarse grid at 512 rays."""
    pr = W.PRESETS["room64"]
    return [make_workload(pr),
            make_workload(pr, rays=33, probe_dims=(5, 3, 4), probe_origin=(1.1, 1.3, 0.9),
                          probe_spacing=(1.3, 2.1, 1.7)),
            make_workload(pr, rays=512, probe_dims=(3, 3, 3), probe_origin=(1.5, 1.5, 1.5),
                          probe_spacing=(2.5, 2.5, 2.5))]


class Twins:
    """The same volumes twice over one library scene: `batched` updated through a batch,
    `plain` through sdfddgi_update_probes, one call per volume."""

    def __init__(self, ws, with_states=(True, False, True)):
        import torch
        self.torch, self.ws = torch, ws
        w0 = ws[0]
        self.scene = S.create_scene()
        S.upload_sdf(self.scene, w0.baked.sdf, w0.baked.h, w0.baked.origin, material=w0.baked.material)
        S.set_lights(self.scene, w0.lights, w0.sky)
        self.batched = [GpuVolume(w, seed=SEED, scene=self.scene, volume_id=i) for i, w in enumerate(ws)]
        self.plain = [GpuVolume(w, seed=SEED, scene=self.scene, volume_id=i) for i, w in enumerate(ws)]
        self.states = [gv.states_dev if use else None for gv, use in zip(self.batched, with_states)]
        self.batch = S.create_batch([gv.vol for gv in self.batched], self.states)

    def update_batch(self, frame):
        S.update_batch(self.batch, frame)

    def update_plain(self, frame, records=False):
        for gv, st in zip(self.plain, self.states):
            S.update_probes(gv.vol, frame, states=st, records=gv.records if records else None)

    def assert_equal(self, label):
        for i, (a, b) in enumerate(zip(self.batched, self.plain)):
            for x, y, name in zip(a.state(), b.state(), ("irr", "depth", "valid")):
                assert np.array_equal(x, y), (label, i, name)
            assert S.volume_status(a.vol) == 0 and S.volume_status(b.vol) == 0, (label, i)

    def close(self):
        S.destroy_batch(self.batch)
        for gv in self.batched + self.plain:
            gv.close()
        S.destroy_scene(self.scene)


def test_batch_equals_plain_updates_bit_for_bit(cuda_device):
    t = Twins(room_members())
    try:
        for frame in range(4):  # the graph is replayed from frame 2 on (two ping-pong parities)
            t.update_batch(frame)
            t.update_plain(frame)
            t.assert_equal(f"frame {frame}")
        assert np.abs(t.batched[0].state()[0][..., :3]).max() > 0
        for i, w in enumerate(t.ws):
            pb, bps, g, ix, stp, ms = S.batch_schedule(t.batch, i)
            assert (pb, bps, g, ix, stp, ms) == (0, 0, 0, 0, 0, 0.0)
    finally:
        t.close()


def test_batch_follows_scene_changes(cuda_device):
    """A new light set or SDF after the graph was built must reach the next batched frame."""
    t = Twins(room_members())
    try:
        for frame in range(2):
            t.update_batch(frame)
            t.update_plain(frame)
        w0 = t.ws[0]
        brighter = [dict(l, rgb=tuple(2.0 * c for c in l["rgb"])) for l in w0.lights]
        S.set_lights(t.scene, brighter + [{"type": "point", "v": (4.0, 6.0, 4.0), "rgb": (9.0, 8.0, 7.0),
                                           "range": 5.0}], (0.1, 0.2, 0.3))
        t.update_batch(2)
        t.update_plain(2)
        t.assert_equal("after set_lights")
        S.upload_sdf(t.scene, w0.baked.sdf, w0.baked.h, w0.baked.origin, material=w0.baked.material)
        t.update_batch(3)
        t.update_plain(3)
        t.assert_equal("after upload_sdf")
    finally:
        t.close()


def test_batch_explicit_rotations(cuda_device):
    t = Twins(room_members())
    try:
        rots = np.stack([W.frame_rotation(99, 5, i) for i in range(3)])
        S.update_batch(t.batch, 0, rotations=rots)
        for gv, st, r in zip(t.plain, t.states, rots):
            S.update_probes(gv.vol, 0, rotation=r, states=st)
        t.assert_equal("explicit rotations")
        with pytest.raises(S.SdfddgiError):
            S.update_batch(t.batch, 1, rotations=np.full((3, 3, 3), np.nan, np.float32))
    finally:
        t.close()


def test_autotune_keeps_state_and_results(cuda_device):
    t = Twins(room_members())
    try:
        t.update_batch(0)
        t.update_plain(0)
        before = [gv.state() for gv in t.batched]
        S.batch_autotune(t.batch, repeats=2)
        after = [gv.state() for gv in t.batched]
        for b, a in zip(before, after):
            assert all(np.array_equal(x, y) for x, y in zip(b, a))
        for i, w in enumerate(t.ws):
            pb, bps, g, ix, stp, ms = S.batch_schedule(t.batch, i)
            R = w.params["rays"]
            assert pb in (16, 32, 64) + ((R,) if R > 64 else ()), (i, pb, R)  # or a warp per probe
            assert bps in (0, 4) and g in (1, 2) and ix in (1, 2) and ms > 0, (i, pb, bps, g, ms)
            assert stp in (1, 2), (i, stp)  # voxel volumes, plain traces: both step counts tried
            assert g == 2 or w.params["rays"] % 16 == 0
        # the tuned schedule differs from the default one at most in the gather's rounding
        for frame in (1, 2):
            t.update_batch(frame)
            t.update_plain(frame)
            for i, (a, b) in enumerate(zip(t.batched, t.plain)):
                x, y = a.state(), b.state()
                assert np.array_equal(x[2], y[2]), (frame, i)
                assert rel_err(x[0], y[0]).max() <= REL_TOL, (frame, i)
                assert rel_err(x[1], y[1]).max() <= REL_TOL, (frame, i)
    finally:
        t.close()


def merged_members():
    """Volumes the merged form takes (rays per probe multiples of 16: the tensor-core gather
    for all), of uneven sizes and ray counts: the preset grid at 64 rays, an offset grid of 45
    probes at 48 rays (2160 rays: the merged pool pads its part to the next whole batch) and a
    coarse grid at 512 rays."""
    pr = W.PRESETS["room64"]
    return [make_workload(pr),
            make_workload(pr, rays=48, probe_dims=(5, 3, 3), probe_origin=(1.1, 1.3, 0.9),
                          probe_spacing=(1.3, 2.1, 1.7)),
            make_workload(pr, rays=512, probe_dims=(3, 3, 3), probe_origin=(1.5, 1.5, 1.5),
                          probe_spacing=(2.5, 2.5, 2.5))]


def test_merged_batch_equals_plain_updates_bit_for_bit(cuda_device):
    """One launch per stage over all volumes: every volume equals its plain update."""
    t = Twins(merged_members())
    try:
        assert S.batch_form(t.batch) == (S.BATCH_FORM_BRANCHES, 0.0, 0.0)  # untuned automatic form
        S.batch_set_form(t.batch, S.BATCH_FORM_MERGED)
        assert S.batch_form(t.batch)[0] == S.BATCH_FORM_MERGED
        for frame in range(4):
            t.update_batch(frame)
            t.update_plain(frame)
            t.assert_equal(f"merged frame {frame}")
        assert np.abs(t.batched[1].state()[0][..., :3]).max() > 0
        # back to branches mid-stream: the same results
        S.batch_set_form(t.batch, S.BATCH_FORM_BRANCHES)
        t.update_batch(4)
        t.update_plain(4)
        t.assert_equal("branches after merged")
    finally:
        t.close()


def test_merged_form_needs_tensor_core_gathers(cuda_device):
    """A 33-ray volume gathers on the SIMT path, so the batch cannot run merged."""
    t = Twins(room_members())
    try:
        with pytest.raises(S.SdfddgiError, match="tensor-core gather"):
            S.batch_set_form(t.batch, S.BATCH_FORM_MERGED)
        with pytest.raises(S.SdfddgiError):
            S.batch_set_form(t.batch, 7)
        S.batch_autotune(t.batch, repeats=1)
        form, ms_b, ms_m = S.batch_form(t.batch)
        assert form == S.BATCH_FORM_BRANCHES and ms_b > 0 and ms_m == 0.0
    finally:
        t.close()


def test_autotune_times_both_forms(cuda_device):
    t = Twins(merged_members())
    try:
        t.update_batch(0)
        t.update_plain(0)
        before = [gv.state() for gv in t.batched]
        S.batch_autotune(t.batch, repeats=2)
        for b, a in zip(before, [gv.state() for gv in t.batched]):
            assert all(np.array_equal(x, y) for x, y in zip(b, a))
        form, ms_b, ms_m = S.batch_form(t.batch)
        print("frame ms: branches", ms_b, "merged", ms_m, "chosen", form)
        assert ms_b > 0 and ms_m > 0
        assert form == (S.BATCH_FORM_MERGED if ms_m < ms_b else S.BATCH_FORM_BRANCHES)
        for frame in (1, 2):
            t.update_batch(frame)
            t.update_plain(frame)
            for i, (a, b) in enumerate(zip(t.batched, t.plain)):
                x, y = a.state(), b.state()
                assert np.array_equal(x[2], y[2]), (frame, i)
                assert rel_err(x[0], y[0]).max() <= REL_TOL, (frame, i)
                assert rel_err(x[1], y[1]).max() <= REL_TOL, (frame, i)
    finally:
        t.close()


def test_batch_argument_errors(cuda_device):
    w = make_workload(W.PRESETS["room64"], probe_dims=(2, 2, 2))
    a, b = GpuVolume(w), GpuVolume(w)
    try:
        with pytest.raises(S.SdfddgiError, match="share one scene"):
            S.create_batch([a.vol, b.vol])
        with pytest.raises(S.SdfddgiError, match="twice"):
            S.create_batch([a.vol, a.vol])
        bt = S.create_batch([a.vol])
        with pytest.raises(S.SdfddgiError):
            S.batch_schedule(bt, 1)
        with pytest.raises(S.SdfddgiError):
            S.batch_autotune(bt, repeats=0)
        S.destroy_batch(bt)
    finally:
        a.close()
        b.close()


def test_cascade512_full_size_sampled(cuda_device):
    """The 4-volume cascade over the 512^3 binary16 SDF, in the launch configuration the
    bench times: the batch equals the plain updates bit for bit on two frames, and the
    oracle checks a seeded sample of every volume's probes (active and inactive) against
    the plain updates' records."""
    O.set_delta(DELTA_VOX, DELTA_COS)
    c = W.CASCADES["cascade512"]
    ws = make_cascade(c)
    t = Twins(ws, with_states=(True, True, True, True))
    rng = np.random.default_rng(8)
    sc = oracle_scene(ws[0])
    try:
        for frame in range(2):
            prev = [gv.state() for gv in t.plain]
            t.update_batch(frame)
            t.update_plain(frame, records=True)
            t.assert_equal(f"cascade frame {frame}")
            for i, (w, gv) in enumerate(zip(ws, t.plain)):
                act = np.flatnonzero(w.states["flags"] & 1)
                ina = np.flatnonzero((w.states["flags"] & 1) == 0)
                sub = np.sort(np.concatenate([rng.choice(act, min(12, len(act)), replace=False), ina[:2]]))
                rot = W.frame_rotation(SEED, frame, i)
                rec = gv.records_np()
                cur = gv.state()
                orc = O.update(sc, oracle_grid(w), w.lights, rot, w.states,
                               prev=(prev[i][0].astype(np.float64), prev[i][1].astype(np.float64), prev[i][2]),
                               subset=sub, force=force_from_records(rec[sub]))
                s = compare(w, cur, rec, orc, sub, w.baked.h, rot=rot)
                s["border_irr"] = border_is_mirror(cur[0][sub])
                s["border_depth"] = border_is_mirror(cur[1][sub])
                print("cascade volume", i, "frame", frame, s)
                assert_bar(s, f"cascade volume {i} frame {frame}")
        # the merged form at full size: one launch per stage over the four volumes
        S.batch_set_form(t.batch, S.BATCH_FORM_MERGED)
        for frame in (2, 3):
            t.update_batch(frame)
            t.update_plain(frame)
            t.assert_equal(f"cascade merged frame {frame}")
    finally:
        t.close()
