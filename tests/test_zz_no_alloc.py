"""The allocation-free update entry point against the regular one (needs a B300).

sdfddgi_update_probes_noalloc exists for callers that may not allocate device memory
while they run (an engine that reserves all GPU memory at start-up, a plug-in inside
another framework's memory manager, a real-time frame loop where an allocation could
stall). It takes every buffer from the caller and keeps its scratch in a fixed device
array. This file is named so that pytest collects it after every other test file.
"""
import numpy as np
import pytest

import paper_2007_14394_b300 as S
import workloads as W
from harness import REL_TOL, GpuVolume, make_workload, rel_err

pytestmark = pytest.mark.gpu


def test_noalloc_matches_update_probes_on_two_consecutive_calls(cuda_device):
    import torch
    w = make_workload(W.PRESETS["room64"])
    gv = GpuVolume(w)
    P = w.P
    sdf = torch.from_numpy(w.baked.sdf).cuda()
    material = torch.from_numpy(w.baked.material).cuda()

    def maps():
        return (torch.zeros((P, 8, 8, 4), dtype=torch.float32, device="cuda"),
                torch.zeros((P, 16, 16, 2), dtype=torch.float32, device="cuda"),
                torch.zeros(P, dtype=torch.uint8, device="cuda"))

    prev, cur = maps(), maps()
    try:
        for frame in range(2):  # the second call reads the first call's maps as history
            rot = W.frame_rotation(7, frame)
            gv.update(rot, record=False)
            ref = gv.state()
            S.update_probes_noalloc(gv.desc, sdf, w.baked.h, w.baked.origin, w.lights, w.sky, prev, cur,
                                    frame=frame, rotation=rot, material=material, states=gv.states_dev)
            torch.cuda.synchronize()
            got = [t.cpu().numpy() for t in cur]
            assert np.array_equal(got[2], ref[2]), frame
            assert rel_err(got[0], ref[0]).max() <= REL_TOL, frame
            assert rel_err(got[1], ref[1]).max() <= REL_TOL, frame
            assert np.abs(ref[0][..., :3]).max() > 0  # the comparison is not between two empty maps
            prev, cur = cur, prev
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
