"""The precision form (binary16 SDF rounded toward zero, float32 stepping, bf16 x bf16
tensor-core gather with float32 accumulation) against the FP64 oracle, beside the float32
path on the same GPU (needs a B300).

Both are compared with the oracle's own, unforced run on the float32 scene -- the
reference -- and the per-output errors are reported: irradiance RMSE and maximum relative
error, depth-moment maximum error (voxels), hit/miss agreement. The float32 path must stay
at rounding level; the precision form's errors are reported, and bounded only loosely.
"""
import numpy as np
import pytest

import oracle as O
import paper_2007_14394_b300 as S
import workloads as W
from harness import DELTA_COS, DELTA_VOX, GpuVolume, make_workload, oracle_grid, oracle_scene

pytestmark = pytest.mark.gpu


def errors(gpu_state, gpu_rec, ref, h):
    irr_g, dep_g, _ = gpu_state
    act = ref["valid"].astype(bool)
    ig, io = irr_g[act][:, 1:-1, 1:-1, :3].astype(np.float64), ref["irr"][act][:, 1:-1, 1:-1, :3]
    dg, do = dep_g[act][:, 1:-1, 1:-1].astype(np.float64), ref["depth"][act][:, 1:-1, 1:-1]
    rays = ref["rays"][act]
    live = rays["event"] >= 0
    miss_o = O.is_miss(rays["natural_event"])
    miss_g = np.isin(gpu_rec[act]["event"], (0, 2))
    scale = float(np.abs(io).mean())
    return {
        "irr_rmse_rel": float(np.sqrt(((ig - io) ** 2).mean()) / scale),
        "irr_max_rel": float((np.abs(ig - io) / np.maximum(np.abs(io), 1e-3 * scale)).max()),
        "depth_mean_max_err_vox": float(np.abs(dg[..., 0] - do[..., 0]).max() / h),
        "depth_mean_rmse_vox": float(np.sqrt(((dg[..., 0] - do[..., 0]) ** 2).mean()) / h),
        "hit_agreement": float((miss_g == miss_o)[live].mean()),
    }


def test_precision_form_error_table(cuda_device):
    O.set_delta(DELTA_VOX, DELTA_COS)
    w32 = make_workload(W.PRESETS["room64"])
    w16 = make_workload(W.PRESETS["room64"], sdf_dtype="f16")
    rot = W.frame_rotation(7, 0)
    ref = O.update(oracle_scene(w32), oracle_grid(w32), w32.lights, rot, w32.states)  # unforced FP64 truth
    h = w32.baked.h
    table = {}
    for name, w, flags in (("float32 path", w32, 0), ("precision form", w16, S.FLAG_BLEND_BF16)):
        gv = GpuVolume(w, flags=flags)
        try:
            gv.update(rot)
            table[name] = errors(gv.state(), gv.records_np(), ref, h)
        finally:
            gv.close()
    print("\nper-output error vs the FP64 oracle (room64, one frame):")
    for name, e in table.items():
        print(f"  {name:15s} " + "  ".join(f"{k}={v:.3g}" for k, v in e.items()))
    f32, prec = table["float32 path"], table["precision form"]
    assert f32["irr_rmse_rel"] < 1e-4 and f32["hit_agreement"] >= 0.999
    assert f32["depth_mean_max_err_vox"] < 0.1
    # the precision form: bf16 keeps 8 significant bits, binary16 moves surfaces by < 1 ulp toward them
    assert prec["irr_rmse_rel"] < 2e-2 and prec["irr_max_rel"] < 0.3
    assert prec["hit_agreement"] >= 0.98
    assert prec["irr_rmse_rel"] > f32["irr_rmse_rel"]  # the form is really in use


def test_precision_form_error_table_open256(cuda_device):
    """The same table on the open256 workload (the bench's), one frame from no history, for a
    seeded sample of 64 active probes, in the bench's launch configuration (two slab branches)."""
    O.set_delta(DELTA_VOX, DELTA_COS)
    w32 = make_workload(W.PRESETS["open256"])
    w16 = make_workload(W.PRESETS["open256"], sdf_dtype="f16")
    rng = np.random.default_rng(21)
    sub = np.sort(rng.choice(np.flatnonzero(w32.states["flags"] & 1), 64, replace=False))
    rot = W.frame_rotation(11, 0)
    ref = O.update(oracle_scene(w32), oracle_grid(w32), w32.lights, rot, w32.states, subset=sub)
    keep = np.zeros(w32.P, bool)
    keep[sub] = True
    ref = dict(ref, valid=ref["valid"] * keep)  # compare the sampled probes only
    rays = np.zeros((w32.P, w32.params["rays"]), dtype=O.RAY_DTYPE)
    rays["event"] = -1
    rays[sub] = ref["rays"]
    ref["rays"] = rays
    h = w32.baked.h
    table = {}
    for name, w, flags in (("float32 path", w32, 0), ("precision form", w16, S.FLAG_BLEND_BF16)):
        gv = GpuVolume(w, flags=flags)
        try:
            gv.update(rot)
            table[name] = errors(gv.state(), gv.records_np(), ref, h)
        finally:
            gv.close()
    print("\nper-output error vs the FP64 oracle (open256, 64 sampled probes, one frame):")
    for name, e in table.items():
        print(f"  {name:15s} " + "  ".join(f"{k}={v:.3g}" for k, v in e.items()))
    f32, prec = table["float32 path"], table["precision form"]
    assert f32["irr_rmse_rel"] < 1e-4 and f32["hit_agreement"] >= 0.999
    assert prec["irr_rmse_rel"] < 5e-2 and prec["hit_agreement"] >= 0.98
    assert prec["irr_rmse_rel"] > f32["irr_rmse_rel"]


def test_bf16_gather_close_to_float32_gather(cuda_device):
    """Same inputs, same traces: the bf16 gather differs from the float32 one only by the
    rounding of weights and values to 8 significant bits."""
    w = make_workload(W.PRESETS["room64"])
    rot = W.frame_rotation(3, 0)
    out = {}
    for flags in (0, S.FLAG_BLEND_BF16):
        gv = GpuVolume(w, flags=flags)
        try:
            gv.update(rot, record=False)
            out[flags] = gv.state()
        finally:
            gv.close()
    a, b = out[0], out[S.FLAG_BLEND_BF16]
    act = a[2].astype(bool)
    ia, ib = a[0][act][:, 1:-1, 1:-1, :3], b[0][act][:, 1:-1, 1:-1, :3]
    rel = np.abs(ia - ib) / np.maximum(np.abs(ia), 1e-3 * np.abs(ia).mean())
    assert 0 < rel.max() < 0.05
    assert np.array_equal(a[2], b[2])
