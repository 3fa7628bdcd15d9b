"""The update with over-relaxed traces (SDFDDGI_FLAG_RELAXED_PRIMARY / _SHADOW; the
accelerated sphere tracing of Sec. 3.3) against the FP64 oracle tracing the same way (needs a
B300).

The bar is the float32 parity bar of tests/test_gpu_parity.py. The relaxed trace adds one
discrete decision per step, whether the new sample's sphere overlaps the previous one's
(or the step left the box). The oracle follows the GPU's recorded path through such tests
where they lie within the rounding band (2e-4 voxel); any other disagreement is a hard
mismatch. The plain update is unchanged by the flags' existence (its parity tests run as
before). Relaxed shadow rays take fewer steps than plain ones on the open scene, where they
run far through free space toward the lights.
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


def run_relaxed(w, flags, frames=1, subset=None, seed_rot=7):
    import paper_2007_14394_b300 as S
    gv = GpuVolume(w, flags=flags)
    om_p = S.RELAX_OMEGA if flags & S.FLAG_RELAXED_PRIMARY else 1.0
    om_s = S.RELAX_OMEGA if flags & S.FLAG_RELAXED_SHADOW else 1.0
    sc, g = oracle_scene(w), oracle_grid(w, omega_primary=om_p, omega_shadow=om_s)
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
            live = rec[sub]["event"] != 255
            s["primary_steps"] = int(rec[sub]["steps"][live].sum())
            s["shadow_steps"] = int(rec[sub]["shadow_steps"][live].sum())
            stats.append(s)
        assert S.volume_status(gv.vol) == 0
    finally:
        gv.close()
    return stats


def test_room_relaxed_parity_two_frames():
    import paper_2007_14394_b300 as S
    w = make_workload(W.PRESETS["room64"], k_bounce=1.0)
    for f, s in enumerate(run_relaxed(w, S.FLAG_RELAXED_PRIMARY | S.FLAG_RELAXED_SHADOW, frames=2)):
        print("relaxed room frame", f, s)
        assert_bar(s, f"relaxed room frame {f}")


def test_open_relaxed_sampled_and_fewer_shadow_steps():
    import paper_2007_14394_b300 as S
    w = make_workload(W.PRESETS["open256"])
    rng = np.random.default_rng(6)
    act = np.flatnonzero(w.states["flags"] & 1)
    sub = np.sort(rng.choice(act, 32, replace=False))
    steps = {}
    for label, flags in (("both", S.FLAG_RELAXED_PRIMARY | S.FLAG_RELAXED_SHADOW), ("shadow", S.FLAG_RELAXED_SHADOW),
                         ("plain", 0)):
        (s,) = run_relaxed(w, flags, subset=sub, seed_rot=11)
        print("relaxed open", label, s)
        assert_bar(s, f"relaxed open {label}")
        steps[label] = (s["primary_steps"], s["shadow_steps"])
    print("(primary, shadow) steps:", steps)
    assert steps["shadow"][0] == steps["plain"][0]     # primary traces untouched by the shadow flag
    assert steps["shadow"][1] < 0.9 * steps["plain"][1]
