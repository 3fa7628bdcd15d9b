"""The learned form: training pairs from the plain update, training and evaluation of
the probe denoiser. Every step of the method runs in the library's kernels through
its C ABI; torch only holds device buffers and gathers minibatches.

Pairs (one per scene seed, a room scene of the 64^3 kind with its 8 x 8 x 8 probes):
  history  `history_frames` plain updates at 1024 rays with hysteresis 0, so that the
           multi-bounce term has converged (each frame adds one bounce);
  input    one 32-ray update from that history, hysteresis 0;
  target   the mean of `target_frames` 1024-ray updates from the same history,
           hysteresis 0 (the converged irradiance the network should reach);
  plain R  one R-ray update from the same history, hysteresis 0, for each R of
           `plain_rays` (the baselines the learned 32-ray update is compared with; the
           ray count at which the plain update reaches the learned update's error is
           read off their errors).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import (DENOISE_SIMT_BF16, DENOISE_TENSOR, create_scene, create_volume, destroy_scene, destroy_volume,
               denoise, denoiser_train_step, make_desc, probe_maps, read_state, set_lights, update_probes,
               upload_sdf, write_state)


@dataclass
class PairSet:
    """Device tensors of n grids of P probes each (grid-major)."""
    dims: tuple
    n: int
    irr: object         # [n, P, 8, 8, 4] 32-ray input
    depth: object       # [n, P, 16, 16, 2]
    valid: object       # [n, P]
    states: object      # [n, P * 16] bytes
    target: object      # [n, P, 8, 8, 4]
    plain: dict         # rays -> [n, P, 8, 8, 4]
    active: object      # [n, P] bool

    @property
    def plain256(self):
        return self.plain[256]

    def maps(self, idx=None):
        """ProbeMaps of all grids, or of the grids `idx` gathered into fresh buffers."""
        import torch
        if idx is None:
            t = (self.irr, self.depth, self.valid, self.states, self.target)
            n = self.n
        else:
            i = torch.as_tensor(idx, device=self.irr.device, dtype=torch.long)
            t = tuple(x.index_select(0, i) for x in (self.irr, self.depth, self.valid, self.states, self.target))
            n = len(idx)
        return probe_maps(self.dims, n, t[0], t[1], t[2], t[3]), t


def make_pairs(preset, seeds, rays_in=32, rays_target=1024, target_frames=4, history_frames=24,
               plain_rays=(256,), device="cuda"):
    import torch
    import workloads as W
    pr = preset
    dims = pr.probe_dims
    P = int(np.prod(dims))
    n = len(seeds)
    irr = torch.empty((n, P, 8, 8, 4), device=device)
    depth = torch.empty((n, P, 16, 16, 2), device=device)
    valid = torch.empty((n, P), dtype=torch.uint8, device=device)
    states = torch.empty((n, P * 16), dtype=torch.uint8, device=device)
    target = torch.empty((n, P, 8, 8, 4), device=device)
    plain = {r: torch.empty((n, P, 8, 8, 4), device=device) for r in plain_rays}
    active = torch.empty((n, P), dtype=torch.bool, device=device)
    for j, seed in enumerate(seeds):
        scene = pr.scene(seed)
        baked = W.bake(scene, pr.sdf_dims, pr.h, (0.0, 0.0, 0.0), dtype=pr.sdf_dtype)
        st = W.probe_states(scene, dims, pr.probe_origin, pr.probe_spacing, pr.h)
        sc = create_scene()
        vols = []
        try:
            upload_sdf(sc, baked.sdf, baked.h, baked.origin, material=baked.material)
            set_lights(sc, scene.lights, scene.sky)
            st_dev = torch.from_numpy(st.view(np.uint8).copy()).to(device)

            def volume(rays):
                d = make_desc(dims, rays, pr.probe_origin, pr.probe_spacing, pr.max_steps, pr.depth_exponent,
                              pr.eps_vox, pr.tmax_vox, 0.0, pr.k_bounce, pr.bias_vox, seed=seed)
                v = create_volume(d, sc)
                vols.append(v)
                return v

            hist = volume(rays_target)
            for f in range(history_frames):
                update_probes(hist, f, states=st_dev)
            H = (torch.empty((P, 8, 8, 4), device=device), torch.empty((P, 16, 16, 2), device=device),
                 torch.empty(P, dtype=torch.uint8, device=device))
            read_state(hist, *H)
            acc = torch.zeros((P, 8, 8, 4), device=device)
            cur = tuple(torch.empty_like(x) for x in H)
            for f in range(target_frames):
                write_state(hist, *H)
                update_probes(hist, 1000 + f, states=st_dev)
                read_state(hist, *cur)
                acc += cur[0]
            target[j] = acc / target_frames
            runs = [(rays_in, None, 2000)] + [(r, plain[r], 3000 + r) for r in plain_rays]
            for rays, dst, frame in runs:
                v = volume(rays)
                write_state(v, *H)
                update_probes(v, frame, states=st_dev)
                read_state(v, *cur)
                if dst is None:
                    irr[j], depth[j], valid[j] = cur
                else:
                    dst[j] = cur[0]
            states[j] = st_dev
            active[j] = torch.from_numpy((st["flags"] & 1).astype(bool)).to(device)
            torch.cuda.synchronize()
        finally:
            for v in vols:
                destroy_volume(v)
            destroy_scene(sc)
    return PairSet(tuple(dims), n, irr, depth, valid, states, target, plain, active)


def rmse(a, b, active) -> float:
    """Root mean square difference over the interior rgb texels of active probes."""
    x = a[..., 1:7, 1:7, :3]
    y = b[..., 1:7, 1:7, :3]
    m = active[..., None, None, None].expand_as(x)
    d = (x - y)[m]
    return float(d.double().pow(2).mean().sqrt())


def train(d, data: PairSet, steps=2000, batch_grids=8, lr=3e-4, seed=0, log_every=0):
    """Adam on random minibatches of whole grids; the learning rate rises linearly over the
    first 5 % of the steps, then decays as a cosine to lr / 20. Returns the loss history
    (one value per logged step)."""
    import torch
    rng = np.random.default_rng(seed)
    loss = torch.zeros(1, device=data.irr.device)
    hist = []
    for s in range(steps):
        idx = rng.choice(data.n, size=min(batch_grids, data.n), replace=False)
        maps, t = data.maps(idx)
        warm = min(1.0, (s + 1) / max(1.0, 0.05 * steps))
        a = warm * lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * s / max(1, steps))))
        denoiser_train_step(d, maps, t[4], a, loss, mode=DENOISE_SIMT_BF16)
        if log_every and (s % log_every == 0 or s == steps - 1):
            hist.append((s, float(loss.item())))
    return hist


def evaluate(d, data: PairSet, mode=DENOISE_TENSOR) -> dict:
    """Irradiance RMSE against the converged target: plain 32-ray, denoised 32-ray (in
    `mode`), plain 256-ray."""
    import torch
    maps, _ = data.maps()
    out = torch.empty_like(data.irr)
    denoise(d, maps, out, mode)
    torch.cuda.synchronize()
    r = {"plain32": rmse(data.irr, data.target, data.active),
         "denoised32": rmse(out, data.target, data.active),
         "grids": data.n}
    for rays, maps in sorted(data.plain.items()):
        r[f"plain{rays}"] = rmse(maps, data.target, data.active)
    return r


def equal_error_rays(r: dict, rays_in: int = 32) -> float | None:
    """The ray count at which the plain update's error equals the denoised update's,
    interpolated linearly in log(error) against log(rays) between the measured plain ray
    counts (None outside their range)."""
    pts = sorted([(rays_in, r["plain32"])] + [(int(k[5:]), v) for k, v in r.items()
                                             if k.startswith("plain") and k != "plain32"])
    e = r["denoised32"]
    for (r0, e0), (r1, e1) in zip(pts, pts[1:]):
        if e1 <= e <= e0 and e0 > e1:
            f = (math.log(e0) - math.log(e)) / (math.log(e0) - math.log(e1))
            return float(math.exp(math.log(r0) + f * (math.log(r1) - math.log(r0))))
    return None
