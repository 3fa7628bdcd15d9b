"""The FP64 validation reduction on the device (needs a B300).

Two scenes have an exact answer for every interior irradiance texel, whatever the ray set
and its rotation, because Eq. 3 is self-normalised (Sec. 3.3):
  - white furnace: a closed room whose surfaces all have emission Le and albedo 0: every ray
    brings Le, so every texel is Le;
  - closed-room multi-bounce: emission Le, albedo rho, no lights, coefficient k = 1,
    hysteresis h: s_0 = Le and s_n = S + (Le - S) r^n with S = Le / (1 - rho) and
    r = h + (1 - h) rho.
The library's reduction measures the float32 maps against these values in FP64 on the
device; each result is also checked against the same statistics formed here in numpy from
the maps read back, and the float32 maps are held to the parity bar's 1e-4 (observed far
below it).
"""
import dataclasses

import numpy as np
import pytest

import workloads as W
from harness import GpuVolume, make_workload

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4


def closed_room(emission, albedo, hysteresis=0.97, rays=64, n_spheres=2, n_boxes=1):
    """8 m closed room (no ceiling opening, no sun) with `n_spheres` spheres and `n_boxes`
    boxes, every surface of the same emission and albedo; 4^3 probes 2 m apart; 32^3 float32
    SDF. The material volume stores binary16, so the emission and albedo given here are
    values binary16 holds exactly."""
    pr = dataclasses.replace(
        W.PRESETS["room64"], world=8.0, sdf_dims=(32, 32, 32), h=0.25, probe_dims=(4, 4, 4),
        probe_origin=(1.0, 1.0, 1.0), probe_spacing=(2.0, 2.0, 2.0), rays=rays, max_steps=64,
        hysteresis=hysteresis, k_bounce=1.0, seed=3,
        scene_args=dict(n_spheres=n_spheres, n_boxes=n_boxes, aperture=0.0, uniform_albedo=tuple(albedo),
                        emission=tuple(emission), sun=False))
    return make_workload(pr)


def host_stats(irr, states, ref):
    """The reduction's statistics formed on the host in FP64 from maps read back."""
    act = (states["flags"] & 1).astype(bool) if states is not None else np.ones(len(irr), bool)
    e = irr[act][:, 1:-1, 1:-1, :3].reshape(-1, 3).astype(np.float64)
    fin = np.all(np.isfinite(e), axis=1)
    e = e[fin]
    d = (e - np.asarray(ref, np.float64)) / np.asarray(ref, np.float64)
    return {"count": len(e), "mean": e.mean(axis=0), "max_rel": np.abs(d).max(axis=0),
            "rms_rel": np.sqrt((d * d).mean(axis=0)), "nonfinite": int((~fin).sum())}


def assert_matches_host(dev, host):
    assert dev["count"] == host["count"] and dev["nonfinite"] == host["nonfinite"]
    np.testing.assert_allclose(dev["mean"], host["mean"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(dev["max_rel"], host["max_rel"], rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(dev["rms_rel"], host["rms_rel"], rtol=1e-9, atol=1e-300)


def test_white_furnace_reduction(cuda_device):
    Le = np.array([0.3125, 0.6875, 1.875], np.float32)
    w = closed_room(Le, (0.0, 0.0, 0.0))
    gv = GpuVolume(w)
    try:
        gv.update(W.frame_rotation(5, 0))
        n_act = int((w.states["flags"] & 1).sum())
        dev = gv.S.irradiance_deviation(gv.vol, Le, states=gv.states_dev)
        again = gv.S.irradiance_deviation(gv.vol, Le, states=gv.states_dev)
        print("furnace", dev)
        assert dev == again  # a fixed summation order
        assert dev["count"] == n_act * 36 and dev["nonfinite"] == 0
        assert max(dev["max_rel"]) <= REL_TOL
        irr = gv.state()[0]
        assert_matches_host(dev, host_stats(irr, w.states, Le))
        # without states every probe counts; the inactive ones (inside the spheres and the box)
        # were never updated and hold zeros, a deviation of exactly 1
        all_p = gv.S.irradiance_deviation(gv.vol, Le)
        assert all_p["count"] == w.P * 36
        assert_matches_host(all_p, host_stats(irr, None, Le))
        if n_act < w.P:
            assert max(all_p["max_rel"]) == 1.0
        # a non-finite texel is counted apart and left out of the statistics
        irr2, dep, val = gv.state()
        p0 = int(np.flatnonzero(w.states["flags"] & 1)[0])
        irr2[p0, 3, 4, 1] = np.nan
        gv.S.write_state(gv.vol, irr2, dep, val)
        bad = gv.S.irradiance_deviation(gv.vol, Le, states=gv.states_dev)
        assert bad["nonfinite"] == 1 and bad["count"] == n_act * 36 - 1
        assert_matches_host(bad, host_stats(irr2, w.states, Le))
        assert gv.S.volume_status(gv.vol) == 0
    finally:
        gv.close()


def test_closed_room_multibounce_reduction(cuda_device):
    Le = np.array([1.0, 0.5, 0.25], np.float32)
    rho, h = np.float32(0.5), np.float32(0.97)
    # no interior primitives: a probe inside one has no history, and a hit beside it can take
    # its multi-bounce lookup from fewer probes or none, which the closed form does not model
    # (the FP64 oracle shows the same: 9.1e-4 off on one texel with two spheres and a box)
    w = closed_room(Le, (rho, rho, rho), hysteresis=h, n_spheres=0, n_boxes=0)
    gv = GpuVolume(w)
    S_inf = Le.astype(np.float64) / (1.0 - float(rho))
    r = float(h) + (1.0 - float(h)) * float(rho)
    try:
        for n in range(6):
            gv.update(W.frame_rotation(9, n))
            expect = S_inf + (Le.astype(np.float64) - S_inf) * r ** n
            ref = expect.astype(np.float32)
            dev = gv.S.irradiance_deviation(gv.vol, ref, states=gv.states_dev)
            print("closed room frame", n, dev)
            assert dev["count"] == int((w.states["flags"] & 1).sum()) * 36 and dev["nonfinite"] == 0
            # the reference is the float32 rounding of the closed form: at most half an ulp of it
            bound = REL_TOL + 2.0 ** -24
            assert max(dev["max_rel"]) <= bound, n
            assert_matches_host(dev, host_stats(gv.state()[0], w.states, ref))
        assert gv.S.volume_status(gv.vol) == 0
    finally:
        gv.close()
