#!/usr/bin/env python3
"""Throughput of the SDFDDGI per-frame probe update on one B300 (or N replicas).

One step = one probe-volume update of the 256^3 open-scene workload (32x16x32
probes, 256 rays/probe, <=128 sphere-trace steps, sun + 16 point lights with SDF
shadow rays, multi-bounce from the previous frame, both octahedral maps with
hysteresis, border fixup). value = probe-rays traced per second (active probes x
rays), device-timed with CUDA events around each update on its stream, L2 flushed
between timed steps. Under torchrun every rank updates its own copy of the
workload (weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "probe-rays/s & ms per probe-volume update; learned vs plain rays at equal RMSE"
UNIT = "probe-rays/s"
WORKLOAD = "open256"
L2_FLUSH_BYTES = 512 << 20
KERNELS_PER_UPDATE = 4  # primary trace, hit preparation, shadow trace, gather


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def workload_config(pr: W.Preset, rays_traced: int):
    return {"workload": f"{pr.name}: {pr.description}", "probes": pr.n_probes, "rays_per_probe": pr.rays,
            "sdf": "x".join(map(str, pr.sdf_dims)) + f" {pr.sdf_dtype}", "max_steps": pr.max_steps,
            "active_rays_per_step": rays_traced, "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
            "seed": pr.seed}


def build_inputs(pr: W.Preset):
    scene = pr.scene()
    baked = W.bake(scene, pr.sdf_dims, pr.h, (0.0, 0.0, 0.0), dtype=pr.sdf_dtype)
    states = W.probe_states(scene, pr.probe_dims, pr.probe_origin, pr.probe_spacing, pr.h)
    return scene, baked, states


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.dev = device_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(device_index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.strip()]
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, name in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(rec: np.ndarray, sdf_elem: int, n_probes: int, n_active: int) -> dict:
    """Bytes the algorithm gathers in one update, from the step counts it actually took:
    8 corners per SDF sample over the primary trace, the shadow traces and the 6 normal samples;
    8 material corners (16 B) per shaded hit; 8 probes x 4 texels (16 B) for the bounce term;
    previous-map reads and current-map writes (3 KiB each per probe) and the probe state."""
    live = rec["event"] != 255
    shaded = live & ((rec["event"] == 1) | (rec["event"] == 3))
    samples = int(rec["steps"][live].sum()) + int(rec["shadow_steps"][live].sum()) + 6 * int(shaded.sum())
    b = samples * 8 * sdf_elem + int(shaded.sum()) * (8 * 16 + 8 * 4 * 16) + n_probes * (2 * 3072 + 16)
    return {"bytes": b, "sdf_samples": samples, "shaded": int(shaded.sum()), "rays": int(live.sum())}


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2007_14394_b300 as S

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pr = W.PRESETS[args.workload]
    scene, baked, states = build_inputs(pr)
    P, R = pr.n_probes, pr.rays
    n_active = int((states["flags"] & 1).sum())
    rays_per_step = n_active * R

    sc = S.create_scene()
    S.upload_sdf(sc, baked.sdf, baked.h, baked.origin, material=baked.material)
    S.set_lights(sc, scene.lights, scene.sky)
    desc = S.make_desc(pr.probe_dims, R, pr.probe_origin, pr.probe_spacing, pr.max_steps, pr.depth_exponent,
                       pr.eps_vox, pr.tmax_vox, pr.hysteresis, pr.k_bounce, pr.bias_vox, seed=pr.seed)
    vol = S.create_volume(desc, sc)
    states_dev = torch.from_numpy(states.view(np.uint8).copy()).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # one recorded update (outside any timed region) for the algorithmic byte count
    records = torch.empty(P * R * 32, dtype=torch.uint8, device=dev)
    S.update_probes(vol, 0, states=states_dev, records=records)
    torch.cuda.synchronize()
    rec = records.cpu().numpy().view(S.RAY_RECORD_DTYPE)
    algo = algorithmic_bytes(rec, 4 if pr.sdf_dtype == "f32" else 2, P, n_active)
    del records
    S.reset(vol)

    frame = 0
    for _ in range(args.warmup):
        S.update_probes(vol, frame, states=states_dev)
        frame += 1
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = Clocks(local_rank)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))                       # evict the SDF and maps from L2 (not timed)
        starts[k].record(stream)
        S.update_probes(vol, frame, states=states_dev, stream=stream)
        ends[k].record(stream)
        frame += 1
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    per_step = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dev_ms = float(sum(per_step))

    # end to end through the C ABI with host buffers: pinned probe states in, both maps out
    host_states = torch.from_numpy(states.view(np.uint8).copy()).pin_memory()
    h_irr = torch.empty(P * 8 * 8 * 4, dtype=torch.float32).pin_memory()
    h_dep = torch.empty(P * 16 * 16 * 2, dtype=torch.float32).pin_memory()
    h_val = torch.empty(P, dtype=torch.uint8).pin_memory()
    st_np = host_states.numpy().view(S.PROBE_STATE_DTYPE)
    e_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        e_s[k].record(stream)
        S.update_probes(vol, frame, states=st_np, stream=stream)
        S.lib.sdfddgi_read_state(vol, h_irr.data_ptr(), h_dep.data_ptr(), h_val.data_ptr(), 0,
                                 S._stream(stream))
        e_e[k].record(stream)
        frame += 1
    torch.cuda.synchronize()
    barrier()
    e2e_ms = float(sum(s.elapsed_time(e) for s, e in zip(e_s, e_e)))

    if world > 1:
        t = torch.tensor([dev_ms, e2e_ms, wall], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        dev_ms, e2e_ms, wall = (float(x) for x in t.tolist())

    ms = dev_ms / args.steps
    value = world * rays_per_step * args.steps / (dev_ms / 1e3)
    e2e_value = world * rays_per_step * args.steps / (e2e_ms / 1e3)
    peak, peak_kind = peaks()
    achieved = algo["bytes"] / (ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded scene, baked on the host)", "config": workload_config(pr, rays_per_step),
        "gpu_launches": KERNELS_PER_UPDATE * args.steps,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": P * 16,
                "d2h_bytes_per_step": P * (8 * 8 * 4 * 4 + 16 * 16 * 2 * 4 + 1), "ms_per_step": e2e_ms / args.steps},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "probe_update_kernel<float>",
                     "algorithmic_bytes_per_launch": algo["bytes"], "sdf_samples_per_launch": algo["sdf_samples"],
                     "peak_source": f"{peak_kind} hbm_gbs"},
        "wall_s_timed_loop": wall,
        "step_ms": {"min": min(per_step), "median": statistics.median(per_step), "max": max(per_step)},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(pr, scene, baked, states, budget_s=args.cpu_budget)
    S.destroy_volume(vol)
    S.destroy_scene(sc)
    return line


def oracle_sample(pr, scene, baked, states, n_probes, seed=0, frame=0, threads=0):
    """Times the oracle's update of a seeded sample of active probes; returns (seconds, rays)."""
    import oracle as O
    act = np.flatnonzero(states["flags"] & 1)
    rng = np.random.default_rng(seed)
    sub = np.sort(rng.choice(act, min(n_probes, len(act)), replace=False))
    osc = O.OracleScene(baked.sdf, baked.h, baked.origin, baked.material)
    g = O.make_grid(pr.probe_dims, pr.probe_origin, pr.probe_spacing, pr.rays, pr.max_steps, pr.eps_vox,
                    pr.tmax_vox, pr.hysteresis, pr.depth_exponent, pr.k_bounce, pr.bias_vox, scene.sky)
    rot = W.frame_rotation(pr.seed, frame)
    t0 = time.perf_counter()
    O.update(osc, g, scene.lights, rot, states, subset=sub, want_rays=False, n_threads=threads)
    return time.perf_counter() - t0, len(sub) * pr.rays


def cpu_baseline(pr, scene, baked, states, budget_s=15.0):
    cores = os.cpu_count() or 1
    n_active = int((states["flags"] & 1).sum())
    calib = max(4, cores)
    dt, rays = oracle_sample(pr, scene, baked, states, calib)       # calibrate the sample size
    n = int(max(4, min(n_active, budget_s / max(dt, 1e-3) * calib)))
    dt, rays = oracle_sample(pr, scene, baked, states, n, seed=1)
    return {"value": rays / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} random active probes of {pr.name} (frame 0, {pr.rays} rays each), "
                      f"{dt:.1f} s on {cores} OpenMP threads"}


def run_reference(args):
    pr = W.PRESETS[args.workload]
    scene, baked, states = build_inputs(pr)
    cores = os.cpu_count() or 1
    n_active = int((states["flags"] & 1).sum())
    dt, _ = oracle_sample(pr, scene, baked, states, max(4, cores))
    per_step_budget = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    n = int(max(4, min(n_active, (per_step_budget / max(dt, 1e-3)) * max(4, cores))))
    for k in range(args.warmup):
        oracle_sample(pr, scene, baked, states, n, seed=100 + k, frame=k)
    times, rays = [], 0
    for k in range(args.steps):
        dt, r = oracle_sample(pr, scene, baked, states, n, seed=200 + k, frame=args.warmup + k)
        times.append(dt)
        rays += r
    tot = sum(times)
    value = rays / tot
    ms = tot / args.steps * (n_active / n) * 1e3
    sample = f"{n} random active probes of {pr.name} per step (of {n_active}); ms_per_step extrapolated linearly"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded scene, baked on the host)",
            "config": workload_config(pr, n_active * pr.rays),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(W.PRESETS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
