"""Shared set-up for the parity tests: one seeded workload fed to both the CUDA
library (through its C ABI) and the FP64 oracle, with every parameter rounded to
float32 first so that both sides read identical data, and the comparison
statistics of the parity bar.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import oracle as O
import workloads as W

DELTA_VOX = 2e-4      # width of the rounding band of distance decisions, voxels
DELTA_COS = 1e-4      # width of the rounding band of light-gating decisions
T_TOL_VOX = 1e-3      # hit-distance tolerance, voxels
REL_TOL = 1e-4        # float32 irradiance / moment relative tolerance


def f32(x):
    return float(np.float32(x))


def f32v(v):
    return tuple(f32(x) for x in v)


@dataclass
class Workload:
    preset: W.Preset
    scene: W.Scene
    baked: W.Baked
    states: np.ndarray
    lights: list
    sky: tuple
    params: dict

    @property
    def P(self):
        return len(self.states)


def make_workload(preset: W.Preset, seed=None, sdf_dtype=None, **overrides) -> Workload:
    """Builds the preset's scene, bake, probe states and float32 parameters.
    overrides: any of rays, max_steps, eps_vox, hysteresis, k_bounce, depth_exponent, bias_vox,
    tmax_vox, probe_dims, probe_origin, probe_spacing."""
    scene = preset.scene(seed)
    baked = W.bake(scene, preset.sdf_dims, preset.h, (0.0, 0.0, 0.0), dtype=sdf_dtype or preset.sdf_dtype)
    p = dict(rays=preset.rays, max_steps=preset.max_steps, eps_vox=preset.eps_vox, hysteresis=preset.hysteresis,
             k_bounce=preset.k_bounce, depth_exponent=preset.depth_exponent, bias_vox=preset.bias_vox,
             tmax_vox=preset.tmax_vox, probe_dims=preset.probe_dims, probe_origin=preset.probe_origin,
             probe_spacing=preset.probe_spacing)
    p.update(overrides)
    for k in ("eps_vox", "hysteresis", "k_bounce", "bias_vox", "tmax_vox"):
        p[k] = f32(p[k])
    p["probe_origin"] = f32v(p["probe_origin"])
    p["probe_spacing"] = f32v(p["probe_spacing"])
    states = W.probe_states(scene, p["probe_dims"], p["probe_origin"], p["probe_spacing"], preset.h)
    lights = [{"type": l["type"], "v": f32v(l["v"]), "rgb": f32v(l["rgb"]), "range": f32(l.get("range", 0.0))}
              for l in scene.lights]
    return Workload(preset, scene, baked, states, lights, f32v(scene.sky), p)


# ------------------------------------------------------------------------- oracle side
def oracle_scene(w: Workload) -> O.OracleScene:
    return O.OracleScene(w.baked.sdf, w.baked.h, w.baked.origin, w.baked.material)


def oracle_grid(w: Workload) -> O.Grid:
    p = w.params
    return O.make_grid(p["probe_dims"], p["probe_origin"], p["probe_spacing"], p["rays"], p["max_steps"],
                       p["eps_vox"], p["tmax_vox"], p["hysteresis"], p["depth_exponent"], p["k_bounce"],
                       p["bias_vox"], w.sky)


def force_from_records(rec: np.ndarray) -> np.ndarray:
    f = np.zeros(rec.shape, dtype=O.FORCE_DTYPE)
    f["event"] = rec["event"].astype(np.int32)
    f["steps"] = rec["steps"].astype(np.int32)
    f["lit_mask"] = rec["lit_mask"]
    return f


# ------------------------------------------------------------------------- GPU side
class GpuVolume:
    """A scene + probe volume in the CUDA library, built from a Workload."""

    def __init__(self, w: Workload, seed: int = 0):
        import torch
        import paper_2007_14394_b300 as S
        self.S, self.torch, self.w = S, torch, w
        p = w.params
        self.scene = S.create_scene()
        S.upload_sdf(self.scene, w.baked.sdf, w.baked.h, w.baked.origin, material=w.baked.material)
        S.set_lights(self.scene, w.lights, w.sky)
        self.desc = S.make_desc(p["probe_dims"], p["rays"], p["probe_origin"], p["probe_spacing"], p["max_steps"],
                                p["depth_exponent"], p["eps_vox"], p["tmax_vox"], p["hysteresis"], p["k_bounce"],
                                p["bias_vox"], seed=seed)
        self.vol = S.create_volume(self.desc, self.scene)
        self.states_dev = torch.from_numpy(w.states.view(np.uint8).copy()).cuda()
        self.records = torch.empty(w.P * p["rays"] * 32, dtype=torch.uint8, device="cuda")

    def update(self, rotation, record=True, states=None):
        st = self.states_dev if states is None else states
        self.S.update_probes(self.vol, 0, rotation=rotation, states=st, records=self.records if record else None)

    def records_np(self) -> np.ndarray:
        self.torch.cuda.synchronize()
        return self.records.cpu().numpy().view(self.S.RAY_RECORD_DTYPE).reshape(self.w.P, self.w.params["rays"])

    def state(self):
        P = self.w.P
        irr = np.empty((P, 8, 8, 4), np.float32)
        dep = np.empty((P, 16, 16, 2), np.float32)
        val = np.empty(P, np.uint8)
        self.S.read_state(self.vol, irr, dep, val)
        return irr, dep, val

    def close(self):
        self.S.destroy_volume(self.vol)
        self.S.destroy_scene(self.scene)


# ------------------------------------------------------------------------- comparison
def rel_err(g, o):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    floor = 1e-6 * max(float(np.abs(o).max()), 1e-30)
    return np.abs(g - o) / np.maximum(np.abs(o), floor)


def compare(w: Workload, gpu_state, gpu_rec, orc, subset, h_vox: float):
    """Statistics of one update over `subset` probes. gpu_rec: [P,R] records; orc: oracle output
    (forced by the GPU's records) for `subset`."""
    irr_g, dep_g, val_g = gpu_state
    rays_o = orc["rays"]
    rec = gpu_rec[subset]
    act = rays_o["event"] >= 0
    n_rays = int(act.sum())
    st = {"rays": n_rays}
    st["hard"] = int((rays_o["hard"][act] > 0).sum())
    st["forced"] = int((rays_o["forced"][act] > 0).sum())
    miss_g = np.isin(rec["event"], (0, 2))
    miss_o = O.is_miss(rays_o["natural_event"])
    grazing = rays_o["margin_primary"] < DELTA_VOX
    st["class_agree_all"] = float((miss_g == miss_o)[act].mean()) if n_rays else 1.0
    ok = act & ~grazing
    st["class_agree_nongrazing"] = float((miss_g == miss_o)[ok].mean()) if ok.any() else 1.0
    st["grazing_frac"] = float(grazing[act].mean()) if n_rays else 0.0
    same_path = act & (rays_o["hard"] == 0)
    dt = np.abs(rec["t"].astype(np.float64) - rays_o["t"]) / h_vox
    st["t_err_vox_max"] = float(dt[same_path].max()) if same_path.any() else 0.0
    st["event_equal"] = bool(np.array_equal(rec["event"][act].astype(np.int32), rays_o["event"][act]))
    st["steps_equal"] = bool(np.array_equal(rec["steps"][act].astype(np.int32), rays_o["steps"][act]))
    st["lit_equal"] = bool(np.array_equal(rec["lit_mask"][act], rays_o["lit_mask"][act]))
    Lerr = rel_err(rec["L"][same_path], rays_o["L"][same_path]) if same_path.any() else np.zeros(1)
    st["ray_L_rel_max"] = float(Lerr.max())
    ig, io = irr_g[subset][:, 1:-1, 1:-1, :3], orc["irr"][subset][:, 1:-1, 1:-1, :3]
    dg, do = dep_g[subset][:, 1:-1, 1:-1], orc["depth"][subset][:, 1:-1, 1:-1]
    st["irr_rel_max"] = float(rel_err(ig, io).max()) if ig.size else 0.0
    st["depth_rel_max"] = float(rel_err(dg, do).max()) if dg.size else 0.0
    st["alpha_equal"] = bool(np.array_equal(irr_g[subset][..., 3], orc["irr"][subset][..., 3]))
    st["valid_equal"] = bool(np.array_equal(val_g[subset], orc["valid"][subset]))
    return st


def border_is_mirror(maps: np.ndarray) -> bool:
    """Every border texel of every map bit-equals the interior texel the octahedral fold
    places next to it: the maps sample continuously across the seams (checked on the
    oracle side with a direction-space continuity test)."""
    import oracle
    fixed = np.stack([oracle.border(m.astype(np.float64)) for m in maps])
    return bool(np.array_equal(fixed.astype(np.float32), maps))
