"""An SDF holding non-finite values (needs a B300; runs inside the bounds-checked build).

Nothing in the upload rejects NaN or infinite distances, so the update must stay inside its
buffers when they occur. In the sphere traces a NaN distance makes t NaN, and the negated
stop test (not t <= the stop distance) ends the trace as leaving the volume instead of
sampling at a NaN point. A +inf distance passes the limit. A -inf distance is a hit. A hit
whose gradient is not finite takes the reversed ray direction as its normal. The test runs
in the bounds-checked build (tests/test_checked_build.py names this file, which pytest does not
collect by itself, and starts it with SDFDDGI_CHECKED=1),
where an index outside its buffer is recorded and skipped rather than used, so a mistake
here shows as SDFDDGI_ERR_BOUNDS, never as a memory fault.
"""
import dataclasses
import os

import numpy as np
import pytest

import paper_2007_14394_b300 as S
import workloads as W
from harness import GpuVolume, make_workload

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("SDFDDGI_CHECKED") != "1",
                                 reason="runs in the bounds-checked build (tests/test_checked_build.py)")]


def test_nonfinite_sdf_values_stay_in_bounds(cuda_device):
    w = make_workload(W.PRESETS["room64"])
    sdf = w.baked.sdf.copy()
    nz, ny, nx = sdf.shape
    sdf[:, :, nx // 3] = np.nan      # a plane of NaN the probes' rays cross
    sdf[nz // 2, :, :] = np.inf      # a plane of +inf
    sdf[:, 3 * ny // 4, :] = -np.inf  # a plane of -inf: the rays reaching it hit
    bad = dataclasses.replace(w, baked=dataclasses.replace(w.baked, sdf=sdf))
    gv = GpuVolume(bad)
    try:
        for frame in range(3):
            gv.update(W.frame_rotation(5, frame), record=frame == 2)
        assert S.volume_status(gv.vol) == 0  # no index left its buffer
        irr, dep, _ = gv.state()
        assert np.isfinite(irr).all() and np.isfinite(dep).all()
        rec = gv.records_np()
        live = rec["event"] != 255
        assert live.any() and np.isfinite(rec["L"][live]).all()
    finally:
        gv.close()
