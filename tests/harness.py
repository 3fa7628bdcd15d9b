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
T_COND_FACTOR = 8.0   # a larger hit-distance difference must be within this multiple of the ray's rounding bound
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


def make_cascade(c: W.Cascade, seed=None) -> list:
    """One Workload per member volume of a cascade, all sharing one scene and one bake."""
    first = make_workload(c.base, seed)
    out = [first]
    for pr in c.volumes[1:]:
        p = dict(first.params, rays=pr.rays, probe_dims=pr.probe_dims, probe_origin=f32v(pr.probe_origin),
                 probe_spacing=f32v(pr.probe_spacing))
        states = W.probe_states(first.scene, p["probe_dims"], p["probe_origin"], p["probe_spacing"], pr.h)
        out.append(Workload(pr, first.scene, first.baked, states, first.lights, first.sky, p))
    return out


# ------------------------------------------------------------------------- oracle side
def oracle_scene(w: Workload, analytic: bool = False) -> O.OracleScene:
    """The oracle's scene: the baked volume, or (analytic) the primitives themselves over the
    same box, with the voxel size as the unit."""
    if analytic:
        t, prm = w.scene.arrays()
        return O.OracleScene.analytic(t, prm, w.scene.albedo, w.scene.emission, w.baked.origin,
                                      w.preset.sdf_dims, w.baked.h)
    return O.OracleScene(w.baked.sdf, w.baked.h, w.baked.origin, w.baked.material)


def oracle_grid(w: Workload, omega_primary: float = 1.0, omega_shadow: float = 1.0) -> O.Grid:
    p = w.params
    return O.make_grid(p["probe_dims"], p["probe_origin"], p["probe_spacing"], p["rays"], p["max_steps"],
                       p["eps_vox"], p["tmax_vox"], p["hysteresis"], p["depth_exponent"], p["k_bounce"],
                       p["bias_vox"], w.sky, omega_primary=omega_primary, omega_shadow=omega_shadow)


def force_from_records(rec: np.ndarray) -> np.ndarray:
    f = np.zeros(rec.shape, dtype=O.FORCE_DTYPE)
    f["event"] = rec["event"].astype(np.int32)
    f["steps"] = rec["steps"].astype(np.int32)
    f["lit_mask"] = rec["lit_mask"]
    f["owner"] = rec["material_owner"].astype(np.int32)
    return f


def texel_geometry(rays: int, rot, exponent: int):
    """Per map (irradiance [6,6], depth [14,14]): the oracle-side weights w [n,n,R] of every interior
    texel for every ray (max(0, u.d) and max(0, u.d)^p, Eq. 3 and the moment weight) and their
    sums [n,n]. A texel whose sum lies inside the rounding band of the cosine cutoff (irradiance)
    or of float32 underflow of cos^p (depth) makes 'no ray reached it' rounding-sensitive."""
    d = np.array([O.sf_dir(i, rays) for i in range(rays)]) @ np.asarray(rot, np.float64).T
    out = []
    for n, e in ((O.IRR_N, 1), (O.DEP_N, exponent)):
        u = np.array([[O.oct_decode([(a + 0.5) / n, (b + 0.5) / n]) for a in range(n)] for b in range(n)])
        w_ = np.maximum(u @ d.T, 0.0) ** e
        out.append((w_, w_.sum(axis=-1)))
    return out


def illcond_effect(geo, dvals, active):
    """First-order effect on each texel mean m_j = sum_i w_ij v_i / sum_i w_ij of per-ray value
    differences dvals [P,R,C] (nonzero only on the counted ill-conditioned rays):
    sum_i w_ij |dv_i| / sum_i w_ij, shape [P,n,n,C]."""
    w_, sw = geo
    P = dvals.shape[0]
    out = np.zeros((P,) + sw.shape + (dvals.shape[-1],))
    safe = np.where(sw > 0, sw, 1.0)
    for p in np.flatnonzero(active):
        if dvals[p].any():
            out[p] = np.einsum("abr,rc->abc", w_, dvals[p]) / safe[..., None]
    return out


# ------------------------------------------------------------------------- GPU side
class GpuVolume:
    """A scene + probe volume in the CUDA library, built from a Workload. With `scene`, the
    volume is made over that existing library scene (not owned) instead of a new one."""

    def __init__(self, w: Workload, seed: int = 0, flags: int = 0, scene=None, volume_id: int = 0,
                 analytic: bool = False, cluster_size: int = 8):
        import torch
        import paper_2007_14394_b300 as S
        self.S, self.torch, self.w = S, torch, w
        p = w.params
        self.own_scene = scene is None
        if scene is None:
            scene = S.create_scene()
            if analytic:  # the primitives themselves over the baked volume's box, unit = voxel size
                t, prm = w.scene.arrays()
                lo = np.asarray(w.baked.origin, dtype=np.float64)
                hi = lo + np.asarray(w.preset.sdf_dims) * w.baked.h
                S.upload_primitives(scene, t, prm, w.scene.albedo, w.scene.emission, lo, hi, w.baked.h,
                                    cluster_size)
            else:
                S.upload_sdf(scene, w.baked.sdf, w.baked.h, w.baked.origin, material=w.baked.material)
            S.set_lights(scene, w.lights, w.sky)
        self.scene = scene
        self.desc = S.make_desc(p["probe_dims"], p["rays"], p["probe_origin"], p["probe_spacing"], p["max_steps"],
                                p["depth_exponent"], p["eps_vox"], p["tmax_vox"], p["hysteresis"], p["k_bounce"],
                                p["bias_vox"], seed=seed, volume_id=volume_id, flags=flags)
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
        if self.own_scene:
            self.S.destroy_scene(self.scene)


# ------------------------------------------------------------------------- comparison
def rel_err(g, o):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    floor = 1e-6 * max(float(np.abs(o).max()), 1e-30)
    return np.abs(g - o) / np.maximum(np.abs(o), floor)


IRR_SW_BAND = 1e-5     # irradiance texels whose cosine sum is below this are rounding-sensitive
DEP_SW_BAND = 1e-30    # depth texels whose cos^p sum is below this underflow in float32
ILLCOND_FACTOR = 2.0   # safety factor on the first-order effect of an ill-conditioned ray's hit distance
FORCED_FRAC_MAX = 1e-3      # rays whose discrete decisions the oracle followed inside the rounding band
T_ILLCOND_RATE = 1e-4       # hits whose distance may differ by more than T_TOL_VOX (at least one per sample)
# The shading normal is normalised from differences of float32 trilinear samples one voxel
# apart. Each sample carries a few roundings of corner values up to ~2 voxels, so a normal
# component is good to ~1e-6 and a light's cosine n.l to EPS_NL. Where a light grazes the
# surface that absolute error is a large relative one. The oracle reports dL/d(n.l) per ray
# (summed over its visible lights); tests/test_oracle_pins.py pins EPS_NL against a float32
# restatement of the normal on seeded surface points.
EPS_NL = 2e-6


def compare(w: Workload, gpu_state, gpu_rec, orc, subset, h_vox: float, rot=None):
    """Statistics of one update over `subset` probes. gpu_rec: [P,R] records; orc: oracle output
    (told the GPU's discrete decisions) for `subset`; rot: the frame rotation.

    Hit distances: the oracle keeps its own. A hit whose distances differ by more than
    T_TOL_VOX is ill-conditioned when the difference is within T_COND_FACTOR times the
    oracle's first-order float32 rounding bound of that trace (t_cond), and a hard mismatch
    otherwise. Texels: relative error <= REL_TOL on every texel, except where a texel's value
    is sensitive beyond a tenth of that to (a) the distance difference of an ill-conditioned
    hit (the oracle's own dL/dt times the difference for the radiance, the difference itself
    for the moments) or (b) the float32 rounding EPS_NL of the cosine of a light that grazes
    the surface (the oracle's own dL/d(n.l)). Those texels are counted, and held to REL_TOL
    plus that first-order effect."""
    irr_g, dep_g, val_g = gpu_state
    rays_o = orc["rays"]
    rec = gpu_rec[subset]
    act = rays_o["event"] >= 0
    n_rays = int(act.sum())
    st = {"rays": n_rays}
    st["hard_decisions"] = int((rays_o["hard"][act] > 0).sum())
    st["forced"] = int((rays_o["forced"][act] > 0).sum())
    st["forced_frac"] = st["forced"] / n_rays if n_rays else 0.0
    miss_g = np.isin(rec["event"], (0, 2))
    miss_o = O.is_miss(rays_o["natural_event"])
    grazing = rays_o["margin_primary"] < DELTA_VOX
    st["class_agree_all"] = float((miss_g == miss_o)[act].mean()) if n_rays else 1.0
    ok = act & ~grazing
    st["class_agree_nongrazing"] = float((miss_g == miss_o)[ok].mean()) if ok.any() else 1.0
    st["grazing_frac"] = float(grazing[act].mean()) if n_rays else 0.0
    hit = act & ~O.is_miss(rays_o["event"]) & (rays_o["hard"] == 0)
    dt = np.where(hit, np.abs(rec["t"].astype(np.float64) - rays_o["t"]) / h_vox, 0.0)
    illcond = hit & (dt > T_TOL_VOX)
    t_hard = illcond & (dt > T_COND_FACTOR * rays_o["t_cond"])
    st["hits"] = int(hit.sum())
    st["t_within_tol_frac"] = float((dt[hit] <= T_TOL_VOX).mean()) if hit.any() else 1.0
    st["t_illcond"] = int(illcond.sum())
    st["t_hard"] = int(t_hard.sum())
    st["t_err_vox_max"] = float(dt[hit].max()) if hit.any() else 0.0
    st["t_err_vox_max_wellcond"] = float(dt[hit & ~illcond].max()) if (hit & ~illcond).any() else 0.0
    st["t_illcond_max_ratio"] = (float((dt / np.maximum(rays_o["t_cond"], 1e-300))[illcond].max())
                                 if illcond.any() else 0.0)
    st["t_illcond_allowed"] = max(1, int(T_ILLCOND_RATE * st["hits"]))
    st["hard"] = st["hard_decisions"] + st["t_hard"]
    same = act & (rays_o["hard"] == 0)
    st["event_equal"] = bool(np.array_equal(rec["event"][act].astype(np.int32), rays_o["event"][act]))
    st["steps_equal"] = bool(np.array_equal(rec["steps"][act].astype(np.int32), rays_o["steps"][act]))
    st["lit_equal"] = bool(np.array_equal(rec["lit_mask"][act], rays_o["lit_mask"][act]))
    wc = same & ~illcond
    st["ray_L_rel_max"] = float(rel_err(rec["L"][wc], rays_o["L"][wc]).max()) if wc.any() else 0.0
    ig, io = irr_g[subset][:, 1:-1, 1:-1, :3], orc["irr"][subset][:, 1:-1, 1:-1, :3]
    dg, do = dep_g[subset][:, 1:-1, 1:-1], orc["depth"][subset][:, 1:-1, 1:-1]
    keep_i = np.ones(ig.shape[1:3], bool)
    keep_d = np.ones(dg.shape[1:3], bool)
    geo = None
    if rot is not None:
        geo = texel_geometry(w.params["rays"], rot, w.params["depth_exponent"])
        keep_i, keep_d = geo[0][1] >= IRR_SW_BAND, geo[1][1] >= DEP_SW_BAND
    st["texels_banded"] = int((~keep_i).sum() + (~keep_d).sum())
    # first-order effect of the ill-conditioned rays' distance differences on their values
    tmax = w.params["tmax_vox"] * h_vox
    that = np.minimum(rays_o["t"], tmax)
    dt_w = np.where(illcond, dt * h_vox, 0.0)
    dvals = (np.abs(rays_o["dLdt"]) * dt_w[..., None], np.stack([dt_w, 2.0 * that * dt_w], axis=-1))
    dshade = np.where(act[..., None], EPS_NL * np.abs(rays_o["dLdcos"]), 0.0)
    for name, g_map, o_map, keep, k in (("irr", ig, io, keep_i, 0), ("depth", dg, do, keep_d, 1)):
        eff_t, eff_s = np.zeros_like(o_map), np.zeros_like(o_map)
        if geo is not None and illcond.any():
            eff_t = ILLCOND_FACTOR * illcond_effect(geo[k], dvals[k], act.any(axis=1))
        if geo is not None and k == 0 and dshade.any():
            eff_s = illcond_effect(geo[k], dshade, act.any(axis=1))
        g_k, o_k = g_map[:, keep], o_map[:, keep]
        et, es = eff_t[:, keep], eff_s[:, keep]
        re = rel_err(g_k, o_k)
        touched = et > 0.1 * REL_TOL * np.abs(o_k)
        grazing_l = (es > 0.1 * REL_TOL * np.abs(o_k)) & ~touched
        plain = ~touched & ~grazing_l
        floor = 1e-6 * max(float(np.abs(o_k).max()), 1e-30) if o_k.size else 1.0
        tol_rel = REL_TOL + (et + es) / np.maximum(np.abs(o_k), floor)
        st[f"{name}_rel_max_all"] = float(re.max()) if re.size else 0.0
        st[f"{name}_rel_max"] = float(re[plain].max()) if plain.any() else 0.0
        st[f"{name}_touched_texels"] = int(touched.sum())
        st[f"{name}_touched_rel_max"] = float(re[touched].max()) if touched.any() else 0.0
        st[f"{name}_grazing_light_texels"] = int(grazing_l.sum())
        st[f"{name}_grazing_light_rel_max"] = float(re[grazing_l].max()) if grazing_l.any() else 0.0
        st[f"{name}_tol_ratio_max"] = float((re / tol_rel).max()) if re.size else 0.0
        st[f"{name}_over_1e4"] = int((re > REL_TOL).sum())
        st[f"{name}_over_1e4_frac"] = float((re > REL_TOL).mean()) if re.size else 0.0
    ag, ao = irr_g[subset][:, 1:-1, 1:-1, 3], orc["irr"][subset][:, 1:-1, 1:-1, 3]
    st["alpha_equal"] = bool(np.array_equal(ag[:, keep_i], ao[:, keep_i]))
    st["valid_equal"] = bool(np.array_equal(val_g[subset], orc["valid"][subset]))
    return st


def border_is_mirror(maps: np.ndarray) -> bool:
    """Every border texel of every map bit-equals the interior texel the octahedral fold
    places next to it: the maps sample continuously across the seams (checked on the
    oracle side with a direction-space continuity test)."""
    import oracle
    fixed = np.stack([oracle.border(m.astype(np.float64)) for m in maps])
    return bool(np.array_equal(fixed.astype(np.float32), maps))


def assert_bar(s, label=""):
    assert s["hard"] == 0, (label, s)
    assert s["forced_frac"] <= FORCED_FRAC_MAX, (label, s)
    assert s["class_agree_nongrazing"] >= 0.999, (label, s)
    assert s["t_illcond"] <= s["t_illcond_allowed"], (label, s)
    # relative 1e-4 on every texel; the counted texels that an ill-conditioned hit distance or a
    # grazing light reaches within 1e-4 plus the oracle's own first-order effect of it
    assert s["irr_rel_max"] <= REL_TOL and s["irr_tol_ratio_max"] <= 1.0, (label, s)
    assert s["depth_rel_max"] <= REL_TOL and s["depth_tol_ratio_max"] <= 1.0, (label, s)
    assert s["alpha_equal"] and s["valid_equal"], (label, s)
    assert s["border_irr"] and s["border_depth"], (label, s)
