"""Slab branches of one update (needs a B300).

An update can run its probes as z-slabs of the probe grid, each slab's traces, shading and
gather a chain of its own on one of two streams, so that one slab's kernels fill the SMs
while another's pools drain to their last long rays. That is a schedule, not a change of
arithmetic: the maps, the validity and every ray's record must equal the serial update's
bit for bit. That includes the multi-bounce lookups near slab boundaries (they read the
whole volume's last maps, Sec. 3.3), inactive probes, both gathers, uneven splits, the
full open256 size the bench runs, and the fall-back to one slab while stage events are set.
"""
import numpy as np
import pytest
import torch

import paper_2007_14394_b300 as S
import workloads as W
from harness import GpuVolume, make_workload

pytestmark = pytest.mark.gpu


class Pair:
    """The same volume twice: `serial` with one slab, `split` with `slabs` slabs; over one
    library scene, or (analytic) each over its own identical scene of primitives."""

    def __init__(self, w, slabs, flags=0, analytic=False):
        self.w = w
        self.scene = None
        if analytic:
            self.serial = GpuVolume(w, seed=5, flags=flags, analytic=True)
            self.split = GpuVolume(w, seed=5, flags=flags, analytic=True)
        else:
            self.scene = S.create_scene()
            S.upload_sdf(self.scene, w.baked.sdf, w.baked.h, w.baked.origin, material=w.baked.material)
            S.set_lights(self.scene, w.lights, w.sky)
            self.serial = GpuVolume(w, seed=5, flags=flags, scene=self.scene)
            self.split = GpuVolume(w, seed=5, flags=flags, scene=self.scene)
        S.set_slabs(self.serial.vol, 1)
        S.set_slabs(self.split.vol, slabs)

    def step(self, frame, record=True):
        rot = W.frame_rotation(9, frame)
        self.serial.update(rot, record=record)
        self.split.update(rot, record=record)

    def assert_equal(self, label, records=True):
        for x, y, name in zip(self.serial.state(), self.split.state(), ("irr", "depth", "valid")):
            assert np.array_equal(x, y), (label, name)
        if records:
            torch.cuda.synchronize()
            assert torch.equal(self.serial.records, self.split.records), (label, "records")
        assert S.volume_status(self.serial.vol) == 0 and S.volume_status(self.split.vol) == 0, label

    def close(self):
        self.serial.close()
        self.split.close()
        if self.scene is not None:
            S.destroy_scene(self.scene)


@pytest.mark.parametrize("rays,dims,slabs", [
    (64, (8, 8, 8), 2),     # tensor-core gather, even split
    (64, (8, 8, 8), 3),     # uneven: 2, 3, 3 z-layers
    (48, (6, 5, 7), 4),     # 1, 2, 2, 2 z-layers; slab sizes not multiples of the gather's 19 probes
    (33, (5, 3, 6), 4),     # SIMT gather (R not a multiple of 16)
])
def test_slabs_equal_the_serial_update_bit_for_bit(cuda_device, rays, dims, slabs):
    w = make_workload(W.PRESETS["room64"], rays=rays, probe_dims=dims, probe_origin=(0.7, 0.6, 0.5),
                      probe_spacing=(0.9, 0.95, 0.9), k_bounce=0.9, hysteresis=0.5)
    assert (w.states["flags"] & 1).sum() < len(w.states)  # some probes sit in geometry (inactive)
    pr = Pair(w, slabs)
    try:
        assert S.volume_slabs(pr.split.vol) == slabs and S.volume_slabs(pr.serial.vol) == 1
        for frame in range(3):  # frames 1 and 2 light hits from the last maps (multi-bounce)
            pr.step(frame)
            pr.assert_equal(f"frame {frame}")
        assert np.abs(pr.split.state()[0][..., :3]).max() > 0
    finally:
        pr.close()


def test_small_and_large_shadow_pools_agree_bit_for_bit(cuda_device):
    """A launch of fewer than 2^19 rays runs its shadow pool as the small-pool kernel (24 CTAs
    per SM, two trace steps between votes), a larger one as the large-pool kernel: the serial
    update here has 2^19 rays (large pool), each of its two slabs 2^18 (small pool)."""
    w = make_workload(W.PRESETS["room64"], rays=128, probe_dims=(16, 16, 16), probe_origin=(0.6, 0.55, 0.6),
                      probe_spacing=(0.45, 0.45, 0.45), k_bounce=0.9, hysteresis=0.5)
    assert 16 ** 3 * 128 == 1 << 19
    pr = Pair(w, 2)
    try:
        for frame in range(2):
            pr.step(frame)
            pr.assert_equal(f"frame {frame}")
        assert np.abs(pr.split.state()[0][..., :3]).max() > 0
    finally:
        pr.close()


@pytest.mark.parametrize("form", ["binary16 SDF, bf16 gather", "relaxed traces", "analytic primitives"])
def test_slabs_equal_serial_in_every_form(cuda_device, form):
    """The other forms of the update run through the same slab branches."""
    preset, flags, analytic = {
        "binary16 SDF, bf16 gather": ("room64_fp16", S.FLAG_BLEND_BF16, False),
        "relaxed traces": ("room64", S.FLAG_RELAXED_PRIMARY | S.FLAG_RELAXED_SHADOW, False),
        "analytic primitives": ("room64", 0, True),
    }[form]
    w = make_workload(W.PRESETS[preset], k_bounce=0.9, hysteresis=0.5)
    pr = Pair(w, 3, flags=flags, analytic=analytic)
    try:
        for frame in range(2):
            pr.step(frame)
            pr.assert_equal(f"{form}, frame {frame}")
    finally:
        pr.close()


def test_open256_auto_slabs_equal_serial(cuda_device):
    """The bench's workload and launch configuration (automatic: two slabs) against one slab."""
    w = make_workload(W.PRESETS["open256"])
    pr = Pair(w, 0)
    try:
        assert S.volume_slabs(pr.split.vol) == 2
        for frame in range(2):
            pr.step(frame)
            pr.assert_equal(f"open256 frame {frame}")
    finally:
        pr.close()


def test_slab_arguments_and_stage_events(cuda_device):
    w = make_workload(W.PRESETS["room64"])
    gv = GpuVolume(w)
    try:
        assert S.volume_slabs(gv.vol) == 1  # 512 probes x 64 rays: below the automatic threshold
        for bad in (-1, S.MAX_SLABS + 1):
            with pytest.raises(S.SdfddgiError) as err:
                S.set_slabs(gv.vol, bad)
            assert err.value.code == S.ERR_INVALID_ARG
        S.set_slabs(gv.vol, 4)
        assert S.volume_slabs(gv.vol) == 4
        events = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        for e in events:
            e.record()
        S.set_stage_events(gv.vol, events)
        assert S.volume_slabs(gv.vol) == 1  # stage timing runs serially
        gv.update(W.frame_rotation(1, 0), record=False)
        torch.cuda.synchronize()
        assert events[0].elapsed_time(events[5]) > 0
        S.set_stage_events(gv.vol, [])
        assert S.volume_slabs(gv.vol) == 4
    finally:
        gv.close()


def test_slab_updates_captured_in_a_graph(cuda_device):
    """Two slab-branched updates captured into a CUDA graph (their fork and join become graph
    edges) and replayed twice equal a twin volume updated directly, bit for bit."""
    w = make_workload(W.PRESETS["room64"], k_bounce=0.9, hysteresis=0.5)
    a = GpuVolume(w, seed=5)
    b = GpuVolume(w, seed=5)
    try:
        for gv in (a, b):
            S.set_slabs(gv.vol, 2)
        rots = [W.frame_rotation(3, f) for f in range(2)]
        for gv in (a, b):  # buffers and one-time set-up before any capture
            gv.update(rots[1], record=False)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for r in rots:  # two updates: the ping-pong parity is back where it was
                S.update_probes(a.vol, 0, rotation=r, states=a.states_dev, stream=s)
        for rep in range(2):
            g.replay()
            for r in rots:
                b.update(r, record=False)
            torch.cuda.synchronize()
            for x, y, name in zip(a.state(), b.state(), ("irr", "depth", "valid")):
                assert np.array_equal(x, y), (rep, name)
        assert np.abs(b.state()[0][..., :3]).max() > 0
        assert S.volume_status(a.vol) == 0
    finally:
        a.close()
        b.close()
