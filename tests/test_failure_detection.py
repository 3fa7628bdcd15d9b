"""Failure detection on the GPU without a fault (needs a B300).

The tensor-core gather's waits are bounded. A test-only volume flag leaves the first
chunk's weight copy out, so a wait that nothing will satisfy runs out (about 0.2 s). The
kernel then records the failure bit, stops its other roles and CTAs, waits for its own
copies in flight and releases its tensor memory. The host reads the failure through
sdfddgi_volume_status, which answers SDFDDGI_ERR_TIMEOUT once and clears it. Updates in
between skip the gather, and the context stays usable: a normal volume on the same scene
then updates to the same maps as a volume that never saw a failure.
"""
import time

import numpy as np
import pytest

import workloads as W
from harness import GpuVolume, make_workload

pytestmark = pytest.mark.gpu


def test_gather_wait_runs_out_and_is_reported(cuda_device):
    import torch
    import paper_2007_14394_b300 as S
    w = make_workload(W.PRESETS["room64"])
    for flags in (0, S.FLAG_BLEND_BF16):
        stalled = GpuVolume(w, flags=flags | S.FLAG_TEST_GATHER_STALL)
        good = GpuVolume(w, flags=flags, scene=stalled.scene)
        ref = GpuVolume(w, flags=flags)
        try:
            t0 = time.perf_counter()
            stalled.update(W.frame_rotation(5, 0), record=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            with pytest.raises(S.SdfddgiError) as err:
                S.volume_status(stalled.vol)
            assert err.value.code == S.ERR_TIMEOUT, err.value
            assert dt < 5.0, dt                                   # bounded, not hung
            assert S.volume_status(stalled.vol) == 0              # read once, then cleared
            # the context is still usable: an update on the same scene matches a clean volume's
            for v in (good, ref):
                v.update(W.frame_rotation(5, 0), record=False)
            torch.cuda.synchronize()
            assert S.volume_status(good.vol) == 0 and S.volume_status(ref.vol) == 0
            a, b = good.state(), ref.state()
            assert all(np.array_equal(x, y) for x, y in zip(a, b))
            assert a[2].any()                                     # maps were written
        finally:
            ref.close()
            good.close()
            stalled.close()
