"""The allocation-free update entry point against the regular one (needs a B300).

sdfddgi_update_probes_noalloc exists for callers that may not allocate device memory
while they run (an engine that reserves all GPU memory at start-up, a plug-in inside
another framework's memory manager, a real-time frame loop where an allocation could
stall). It takes every buffer from the caller and keeps its scratch in a fixed device
array. It runs the same kernels as sdfddgi_update_probes, so its maps and ray records
must equal that entry point's bit for bit. This file is named so that pytest collects it
after every other test file.
"""

import numpy as np
import pytest

import paper_2007_14394_b300 as S
import workloads as W
from harness import GpuVolume, make_workload

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 32 << 20


def scratch_needed(sdf_dims, sdf_elem, P, R, n_lights):
    """The header's statement of the scratch an update needs (each part rounded to 256 B)."""
    nx, ny, nz = sdf_dims
    up = lambda x: (x + 255) // 256 * 256  # noqa: E731
    rays = P * R
    parts = [(nx + 2) * (ny + 2) * (nz + 2 + nz % 2) * 4 * sdf_elem, rays * 4, rays * 4, rays * 16, rays * 16, rays * 16, rays * 4,
             rays * 4, rays * 16 * max(n_lights, 1), 32, 944 * R + 928, 32768 * ((R + 15) // 16),
             rays * 4 * max(n_lights, 1), rays * 4]
    return sum(up(x) for x in parts)


class NoAllocRun:
    """The caller's buffers of one volume: the scene on the device and two sets of maps."""

    def __init__(self, w, gv):
        import torch
        self.torch, self.w, self.gv = torch, w, gv
        P, R = w.P, w.params["rays"]
        self.sdf = torch.from_numpy(w.baked.sdf).cuda()
        self.material = torch.from_numpy(w.baked.material).cuda()
        self.maps = [self._zeros() for _ in range(2)]
        self.records = torch.empty(P * R * 32, dtype=torch.uint8, device="cuda")

    def _zeros(self):
        t, P = self.torch, self.w.P
        return (t.zeros((P, 8, 8, 4), dtype=t.float32, device="cuda"),
                t.zeros((P, 16, 16, 2), dtype=t.float32, device="cuda"), t.zeros(P, dtype=t.uint8, device="cuda"))

    def update(self, frame, rot):
        """One call; the maps written become the next call's history."""
        w = self.w
        S.update_probes_noalloc(self.gv.desc, self.sdf, w.baked.h, w.baked.origin, w.lights, w.sky, self.maps[0],
                                self.maps[1], frame=frame, rotation=rot, material=self.material,
                                states=self.gv.states_dev, records=self.records)
        self.maps.reverse()
        return self.maps[0]

    def state(self):
        self.torch.cuda.synchronize()
        return [t.cpu().numpy() for t in self.maps[0]], self.records.cpu().numpy()


def assert_equal_to_update_probes(w, flags=0, frames=2, seed_rot=7):
    """Both entry points over `frames` consecutive frames (the second reads the first's maps as
    history): maps, validity and per-ray records equal bit for bit."""
    gv = GpuVolume(w, flags=flags)
    try:
        run = NoAllocRun(w, gv)
        for frame in range(frames):
            rot = W.frame_rotation(seed_rot, frame)
            gv.update(rot, record=True)
            ref, ref_rec = gv.state(), gv.records.cpu().numpy()
            run.update(frame, rot)
            got, got_rec = run.state()
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), frame
            assert np.array_equal(got_rec, ref_rec), frame
            assert np.abs(ref[0][..., :3]).max() > 0  # the comparison is not between two empty maps
        assert S.volume_status(gv.vol) == 0
    finally:
        gv.close()


def test_noalloc_equals_update_probes_on_two_consecutive_calls(cuda_device):
    """room64 at 64 rays: the tensor-core gather on both sides."""
    assert_equal_to_update_probes(make_workload(W.PRESETS["room64"]))


def test_noalloc_precision_form_and_relaxed_traces(cuda_device):
    """A binary16 SDF with the bf16 gather, and both over-relaxed traces, as volume flags."""
    assert_equal_to_update_probes(make_workload(W.PRESETS["room64"], sdf_dtype="f16"), flags=S.FLAG_BLEND_BF16)
    assert_equal_to_update_probes(make_workload(W.PRESETS["room64"], rays=48),
                                  flags=S.FLAG_RELAXED_PRIMARY | S.FLAG_RELAXED_SHADOW, frames=1)


def test_noalloc_just_under_its_scratch_limit(cuda_device):
    """7x6x6 probes at 1024 rays over the 64^3 room need 29.0 MiB of the 32 MiB; one more probe
    row (7x7x6) does not fit and is rejected before any device work."""
    pr = W.PRESETS["room64"]
    w = make_workload(pr, rays=1024, probe_dims=(7, 6, 6), probe_origin=(0.6, 0.6, 0.7), probe_spacing=(1.1, 1.3, 1.3))
    need = scratch_needed(pr.sdf_dims, 4, w.P, 1024, len(w.lights))
    assert 28 << 20 < need <= SCRATCH_BYTES
    assert_equal_to_update_probes(w, frames=1)
    w7 = make_workload(pr, rays=1024, probe_dims=(7, 7, 6), probe_origin=(0.6, 0.6, 0.7), probe_spacing=(1.1, 1.1, 1.3))
    assert scratch_needed(pr.sdf_dims, 4, w7.P, 1024, len(w7.lights)) > SCRATCH_BYTES
    gv = GpuVolume(w7)
    try:
        run = NoAllocRun(w7, gv)
        with pytest.raises(S.SdfddgiError) as err:
            run.update(0, W.frame_rotation(7, 0))
        assert err.value.code == S.ERR_INVALID_ARG and "scratch" in str(err.value)
    finally:
        gv.close()


def test_noalloc_allocates_nothing(cuda_device):
    """After the first call on the device (which looks up the scratch array), further calls
    leave the device's free memory and torch's allocator exactly as they were."""
    import torch
    w = make_workload(W.PRESETS["room64"])
    gv = GpuVolume(w)
    try:
        run = NoAllocRun(w, gv)
        run.update(0, W.frame_rotation(3, 0))
        torch.cuda.synchronize()
        free0, alloc0, res0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
        for frame in range(1, 5):
            run.update(frame, W.frame_rotation(3, frame))
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == res0
    finally:
        gv.close()


def test_noalloc_rejects_an_update_beyond_its_scratch(cuda_device):
    import torch
    big = torch.zeros((256, 256, 256), dtype=torch.float32, device="cuda")  # 256 MiB of quads needed
    desc = S.make_desc((2, 2, 2), 16, (1.0, 1.0, 1.0), (2.0, 2.0, 2.0), 32)
    maps = [(torch.zeros((8, 8, 8, 4), device="cuda"), torch.zeros((8, 16, 16, 2), device="cuda"),
             torch.zeros(8, dtype=torch.uint8, device="cuda")) for _ in range(2)]
    with pytest.raises(S.SdfddgiError) as err:
        S.update_probes_noalloc(desc, big, 0.25, (0.0, 0.0, 0.0), [], (0, 0, 0), maps[0], maps[1])
    assert err.value.code == S.ERR_INVALID_ARG and "scratch" in str(err.value)
