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
KERNELS_PER_UPDATE = 7  # texel weights, primary, hit preparation, shadow, finalize, weight image, gather
MERGED_KERNELS = 7  # a merged batch frame: the same seven stages, each one launch over every volume


def max_over_ranks(values, world: int, device=None):
    """Each value's maximum over the ranks (the slowest rank's time); the values unchanged at
    world size 1. NCCL reduces a tensor on `device`, gloo one in host memory."""
    values = [float(v) for v in values]
    if world <= 1:
        return values
    import torch
    import torch.distributed as dist
    on = device if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor(values, dtype=torch.float64, device=on)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(world: int, units_per_rank_step: float, steps: int, ms_total: float) -> float:
    """Units per second of the whole job: every rank processes units_per_rank_step per step
    (weak scaling), over the slowest rank's total time in milliseconds."""
    return world * units_per_rank_step * steps / (ms_total / 1e3)


def kernels_per_update(slabs: int) -> int:
    """Kernel launches of one update run as `slabs` slab branches (tensor-core gather): the
    directions, the weights and the weight image once, then five stage kernels per slab."""
    return KERNELS_PER_UPDATE if slabs <= 1 else 3 + 5 * slabs


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def l2_read_peak(S, dev) -> float:
    """The L2 read bandwidth (GB/s), the second ceiling of the gathers: the library's
    microbenchmark over a 32 MiB buffer (L2-resident), the best of three timed sweeps."""
    import torch
    buf = torch.zeros((32 << 20) // 4, dtype=torch.float32, device=dev)
    best = max(S.l2_read_bandwidth(buf, reps=50) for _ in range(3))
    del buf
    return best


def source_hash(patterns) -> str:
    """Hash of the files matching the glob patterns (repository-relative)."""
    import glob
    import hashlib
    h = hashlib.sha256()
    files = sorted({f for pat in patterns for f in glob.glob(os.path.join(ROOT, pat))})
    for f in files:
        h.update(os.path.relpath(f, ROOT).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(stage: str, workload: str):
    """DRAM bytes per launch of `stage` from the committed ncu capture of `workload`
    (profiles/traffic_<workload>.json), or None when a source it covers changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", f"traffic_{workload}.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("source_hash") != source_hash(t.get("sources", [])):
        return None
    return t["dram_bytes_per_launch"].get(stage)


def tensor_peak():
    """Dense bf16 tensor peak (TFLOP/s), burst: the measured one, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1800.0, "fallback"


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
    """SM clock and throttle reasons sampled through NVML every few ms during the timed region."""
    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40, "sw_power_cap": 0x4}

    def __init__(self, device_index: int, period_s: float = 0.005):
        import threading
        self.samples, self.reasons, self.max_mhz = [], set(), None
        self._stop = threading.Event()
        self._thread = None
        self._proc, self.source = None, None
        try:
            import pynvml
            pynvml.nvmlInit()
            self._nv = pynvml
            self._h = pynvml.nvmlDeviceGetHandleByIndex(device_index)
            self.max_mhz = float(pynvml.nvmlDeviceGetMaxClockInfo(self._h, pynvml.NVML_CLOCK_SM))
        except Exception:  # no NVML binding: nvidia-smi every 100 ms instead
            self._nv = None
            self._start_smi(device_index)
            return
        self._period = period_s
        self.source = "NVML, 5 ms period"
        self._thread = threading.Thread(target=self._run, daemon=True)
        self._thread.start()

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def _start_smi(self, device_index):
        import subprocess
        try:
            self._proc = subprocess.Popen(["nvidia-smi", "-i", str(device_index), f"--query-gpu={self.Q}",
                                           "--format=csv,noheader,nounits", "-lms", "10"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._first = self._proc.stdout.readline()  # the sampler is running before the timed region
            self.source = "nvidia-smi, 10 ms period"
        except OSError:
            self._proc = None

    def _stop_smi(self):
        self._proc.terminate()
        try:
            out, _ = self._proc.communicate(timeout=5)
        except Exception:
            self._proc.kill()
            out, _ = self._proc.communicate()
        names = ["hw_slowdown", "sw_thermal_slowdown", "hw_thermal_slowdown", "sw_power_cap"]
        for row in out.strip().splitlines():
            f = [x.strip() for x in row.split(",")]
            try:
                self.samples.append(float(f[0]))
                self.max_mhz = max(self.max_mhz or 0.0, float(f[1]))
                for k, name in enumerate(names):
                    if f[2 + k].lower() == "active":
                        self.reasons.add(name)
            except (ValueError, IndexError):
                continue

    def _run(self):
        nv = self._nv
        while not self._stop.is_set():
            try:
                self.samples.append(float(nv.nvmlDeviceGetClockInfo(self._h, nv.NVML_CLOCK_SM)))
                get = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                    nv.nvmlDeviceGetCurrentClocksThrottleReasons
                mask = get(self._h)
                for name, bit in self.REASONS.items():
                    if mask & bit:
                        self.reasons.add(name)
            except Exception:
                pass
            self._stop.wait(self._period)

    def stop(self):
        if self._proc is not None:
            self._stop_smi()
        elif self._thread is not None:
            self._stop.set()
            self._thread.join()
        if not self.samples:
            return None
        return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(self.samples), "source": self.source}


def stage_work(rec: np.ndarray, sdf_elem: int, n_probes: int, rays: int, n_active: int) -> dict:
    """Algorithmic work of each stage of one update, from the step counts the update took.
    SDF sample = 8 trilinear corners of sdf_elem bytes. Per stage:
      primary -- its SDF samples + the 8-byte result of every ray;
      prep    -- per shaded hit 6 normal samples, 8 material corners (16 B), 8 probes x 4 texels
                 (16 B) of last frame's irradiance, and 64 B of shading data written;
      shadow  -- its SDF samples + per task the 4-byte task, the hit's 20 bytes and the result;
      gather  -- floating-point work of Eq. 3: 2 flops per (texel, ray, channel) over the 36 x 3
                 irradiance and 196 x 2 moment outputs of every active probe."""
    live = rec["event"] != 255
    shaded = live & ((rec["event"] == 1) | (rec["event"] == 3))
    prim = int(rec["steps"][live].sum())
    shad = int(rec["shadow_steps"][live].sum())
    hits = int(shaded.sum())
    corner = 8 * sdf_elem
    return {
        "primary": {"bytes": prim * corner + int(live.sum()) * 8, "sdf_samples": prim},
        "prep": {"bytes": hits * (6 * corner + 8 * 16 + 8 * 4 * 16 + 64), "sdf_samples": 6 * hits},
        "shadow": {"bytes": shad * corner, "sdf_samples": shad},
        "gather": {"flops": 2 * rays * (36 * 3 + 196 * 2) * n_active},
        "rays": int(live.sum()), "hits": hits,
    }


def fp32_peak_tflops(clock_mhz: float) -> float:
    """FP32 FMA peak from unit counts and clock: 148 SMs x 128 FP32 lanes x 2 flops per cycle."""
    return 148 * 128 * 2 * clock_mhz * 1e6 / 1e12


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
                       pr.eps_vox, pr.tmax_vox, pr.hysteresis, pr.k_bounce, pr.bias_vox, seed=pr.seed,
                       flags=S.FLAG_BLEND_BF16 if pr.blend == "bf16" else 0)
    vol = S.create_volume(desc, sc)
    S.set_slabs(vol, args.slabs)
    states_dev = torch.from_numpy(states.view(np.uint8).copy()).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # one recorded update (outside any timed region) for the algorithmic byte count
    records = torch.empty(P * R * 32, dtype=torch.uint8, device=dev)
    S.update_probes(vol, 0, states=states_dev, records=records)
    torch.cuda.synchronize()
    rec = records.cpu().numpy().view(S.RAY_RECORD_DTYPE)
    work = stage_work(rec, 4 if pr.sdf_dtype == "f32" else 2, P, R, n_active)
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
    slabs = S.volume_slabs(vol)  # the library's automatic schedule: slab branches for an update this size
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

    # stage times: the same updates with stage events, which run them serially (one slab), so
    # that every stage kernel is timed alone on the update's stream
    n_s = max(10, min(args.steps, 200))
    stage_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(n_s)]
    for evs in stage_ev:
        for e in evs:
            e.record(stream)
    torch.cuda.synchronize()
    for k in range(n_s):
        flush.fill_(float(k))
        S.set_stage_events(vol, stage_ev[k])
        S.update_probes(vol, frame, states=states_dev, stream=stream)
        frame += 1
    torch.cuda.synchronize()
    S.set_stage_events(vol, [])
    stage_ms = {name: sum(evs[i].elapsed_time(evs[i + 1]) for evs in stage_ev) / n_s
                for i, name in enumerate(S.STAGES)}
    serial_ms = sum(evs[0].elapsed_time(evs[5]) for evs in stage_ev) / n_s

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
    e2e_serial_ms = float(sum(s.elapsed_time(e) for s, e in zip(e_s, e_e)))

    # the same, pipelined as a caller shipping every frame's maps would run it: frame k's maps
    # are copied out (read_state_async, the volume's copy stream) while frame k+1 updates;
    # one interval over all steps (no L2 flush: the 256 MiB SDF copy alone exceeds L2)
    done = [torch.cuda.Event() for _ in range(args.steps)]
    p_s, p_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(args.warmup):
        S.update_probes(vol, frame, states=st_np, stream=stream)
        S.read_state_async(vol, h_irr, h_dep, h_val, stream=stream)
        frame += 1
    torch.cuda.synchronize()
    barrier()
    p_s.record(stream)
    for k in range(args.steps):
        S.update_probes(vol, frame, states=st_np, stream=stream)
        S.read_state_async(vol, h_irr, h_dep, h_val, stream=stream, done_event=done[k])
        frame += 1
    stream.wait_event(done[-1])
    p_e.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = float(p_s.elapsed_time(p_e))

    # the same update with over-relaxed traces (a variant; the headline is the plain path)
    relaxed = {}
    for label, fl in (("relaxed_shadow", S.FLAG_RELAXED_SHADOW),
                      ("relaxed_primary_and_shadow", S.FLAG_RELAXED_SHADOW | S.FLAG_RELAXED_PRIMARY)):
        rdesc = S.make_desc(pr.probe_dims, R, pr.probe_origin, pr.probe_spacing, pr.max_steps, pr.depth_exponent,
                            pr.eps_vox, pr.tmax_vox, pr.hysteresis, pr.k_bounce, pr.bias_vox, seed=pr.seed,
                            flags=(S.FLAG_BLEND_BF16 if pr.blend == "bf16" else 0) | fl)
        rvol = S.create_volume(rdesc, sc)
        n_r = max(10, min(args.steps, 200))
        for k in range(args.warmup):
            S.update_probes(rvol, k, states=states_dev, stream=stream)
        r_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(n_r)]
        for evs in r_ev:
            for e in evs:
                e.record(stream)
        torch.cuda.synchronize()
        for k in range(n_r):
            flush.fill_(float(k))
            S.set_stage_events(rvol, r_ev[k])
            S.update_probes(rvol, args.warmup + k, states=states_dev, stream=stream)
        torch.cuda.synchronize()
        S.set_stage_events(rvol, [])
        assert S.volume_status(rvol) == 0
        r_stage = {name: sum(evs[i].elapsed_time(evs[i + 1]) for evs in r_ev) / n_r for i, name in enumerate(S.STAGES)}
        r_ms = sum(evs[0].elapsed_time(evs[5]) for evs in r_ev) / n_r
        relaxed[label] = {"ms_per_update": r_ms, "primary_ms": r_stage["primary"], "shadow_ms": r_stage["shadow"],
                          "updates": n_r}
        S.destroy_volume(rvol)

    # the precision form on the same workload: a binary16 SDF (rounded toward zero when baked) and
    # the bf16 x bf16 tensor-core gather; same schedule, same timing rules (its per-output errors
    # against the FP64 oracle are measured by tests/test_precision_form.py)
    precision = None
    if pr.sdf_dtype == "f32" and pr.blend == "f32":
        baked16 = W.bake(scene, pr.sdf_dims, pr.h, (0.0, 0.0, 0.0), dtype="f16")
        sc16 = S.create_scene()
        S.upload_sdf(sc16, baked16.sdf, baked16.h, baked16.origin, material=baked16.material)
        S.set_lights(sc16, scene.lights, scene.sky)
        pdesc = S.make_desc(pr.probe_dims, R, pr.probe_origin, pr.probe_spacing, pr.max_steps, pr.depth_exponent,
                            pr.eps_vox, pr.tmax_vox, pr.hysteresis, pr.k_bounce, pr.bias_vox, seed=pr.seed,
                            flags=S.FLAG_BLEND_BF16)
        pvol = S.create_volume(pdesc, sc16)
        S.set_slabs(pvol, args.slabs)
        for k in range(args.warmup):
            S.update_probes(pvol, k, states=states_dev, stream=stream)
        n_p = max(10, min(args.steps, 200))
        pe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_p)]
        torch.cuda.synchronize()
        for k in range(n_p):
            flush.fill_(float(k))
            pe[k][0].record(stream)
            S.update_probes(pvol, args.warmup + k, states=states_dev, stream=stream)
            pe[k][1].record(stream)
        torch.cuda.synchronize()
        p_ms = statistics.median(a.elapsed_time(b) for a, b in pe)
        p_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(n_p)]
        for evs in p_ev:
            for e in evs:
                e.record(stream)
        torch.cuda.synchronize()
        for k in range(n_p):
            flush.fill_(float(k))
            S.set_stage_events(pvol, p_ev[k])
            S.update_probes(pvol, args.warmup + n_p + k, states=states_dev, stream=stream)
        torch.cuda.synchronize()
        S.set_stage_events(pvol, [])
        assert S.volume_status(pvol) == 0
        p_stage = {name: sum(evs[i].elapsed_time(evs[i + 1]) for evs in p_ev) / n_p for i, name in enumerate(S.STAGES)}
        precision = {"form": "binary16 SDF (rounded toward zero), float32 stepping, bf16 x bf16 tensor-core gather "
                             "with float32 accumulation",
                     "ms_per_update": p_ms, "value": rays_per_step / (p_ms / 1e3), "unit": UNIT,
                     "float32_ms_per_update": statistics.median(per_step),
                     "serial_stage_ms": p_stage, "updates": n_p,
                     "errors": "per-output errors against the FP64 oracle: tests/test_precision_form.py"}
        S.destroy_volume(pvol)
        S.destroy_scene(sc16)

    dev_ms, e2e_ms, e2e_serial_ms, wall = max_over_ranks([dev_ms, e2e_ms, e2e_serial_ms, wall], world, dev)

    ms = dev_ms / args.steps
    value = whole_job_rate(world, rays_per_step, args.steps, dev_ms)
    e2e_value = whole_job_rate(world, rays_per_step, args.steps, e2e_ms)
    hbm, peak_kind = peaks()
    l2 = l2_read_peak(S, dev)
    sm_mhz = float((clk or {}).get("sm_max_mhz") or 2032.0)
    stages = {}
    for name in S.STAGES:
        ms_k = stage_ms[name]
        if name == "gather" and R % 16 == 0:  # the tensor-core gather (3 x tf32 products)
            ach = work[name]["flops"] / (ms_k / 1e3) / 1e12
            bf16, bf16_kind = tensor_peak()
            peak_k = bf16 * 1.1 / 2.25
            stages[name] = {"ms": ms_k, "bound": "tensor", "achieved": ach, "peak": peak_k, "unit": "TFLOP/s",
                            "frac": ach / peak_k, "flops_per_launch": work[name]["flops"],
                            "peak_source": f"{bf16_kind} bf16 burst x nominal tf32/bf16 (1.1/2.25)",
                            "note": "includes the per-ray finalize and the weight-image pack"}
        elif name == "gather":
            ach = work[name]["flops"] / (ms_k / 1e3) / 1e12
            peak_k = fp32_peak_tflops(sm_mhz)
            stages[name] = {"ms": ms_k, "bound": "alu", "achieved": ach, "peak": peak_k, "unit": "TFLOP/s",
                            "frac": ach / peak_k, "flops_per_launch": work[name]["flops"],
                            "peak_source": f"derived: 148 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz"}
        elif name in work:
            ach = work[name]["bytes"] / (ms_k / 1e3) / 1e9
            stages[name] = {"ms": ms_k, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                            "frac": ach / hbm, "bytes_per_launch": work[name]["bytes"],
                            "sdf_samples_per_launch": work[name]["sdf_samples"],
                            "peak_source": f"{peak_kind} hbm_gbs",
                            "l2_peak": l2, "l2_frac": ach / l2,
                            "l2_peak_source": "measured here: sdfddgi_l2_read_bandwidth, 32 MiB L2-resident "
                                              "buffer, 16-byte loads bypassing L1"}
        else:
            stages[name] = {"ms": ms_k}
    dominant = max((n for n in S.STAGES if n in work), key=lambda n: stage_ms[n])
    roof = dict(stages[dominant])
    roof.update({"kernel": dominant, "traffic": measured_traffic(dominant, args.workload)})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if pr.blend == "f32" and pr.sdf_dtype == "f32" else f"{pr.sdf_dtype} sdf, {pr.blend} gather",
        "data": "synthetic (seeded scene, baked on the host)", "config": workload_config(pr, rays_per_step),
        "gpu_launches": kernels_per_update(slabs) * args.steps,
        "schedule": {"slabs": slabs, "serial_ms_per_update": serial_ms, "stage_updates": n_s,
                     "note": "value: updates as the library runs them by default (slab branches); stages and "
                             "roofline: the same updates run serially with stage events, L2 flushed"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": P * 16,
                "d2h_bytes_per_step": P * (8 * 8 * 4 * 4 + 16 * 16 * 2 * 4 + 1), "ms_per_step": e2e_ms / args.steps,
                "how": "update_probes with page-locked host probe states, then read_state_async of both maps and "
                       "validity into page-locked host memory; frame k's read overlaps frame k+1's update; one "
                       "CUDA-event interval over all steps, ending when the last read is done"},
        "e2e_serial": {"value": whole_job_rate(world, rays_per_step, args.steps, e2e_serial_ms), "unit": UNIT,
                       "ms_per_step": e2e_serial_ms / args.steps,
                       "how": "the same calls with the synchronous read_state, each step timed alone, L2 flushed "
                              "between steps"},
        "roofline": roof,
        "stages": stages,
        "precision_form": precision,
        "relaxed_trace_variants": dict(relaxed, omega=S.RELAX_OMEGA,
                                       note="SDFDDGI_FLAG_RELAXED_* volumes, same workload, stage events (serial); "
                                            "plain serial path: " + f"{serial_ms:.4f} ms"),
        "wall_s_timed_loop": wall,
        "step_ms": {"min": min(per_step), "median": statistics.median(per_step), "max": max(per_step)},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(pr, scene, baked, states, budget_s=args.cpu_budget)
    S.destroy_volume(vol)
    S.destroy_scene(sc)
    return line


def run_batch(args, rank, world, local_rank):
    """A cascade of volumes (Sec. 3.5) as one batch: one CUDA-graph launch per frame after the
    autotuner has chosen each volume's schedule, against the same volumes updated by one plain
    launch each (default schedules). One step = one frame of every volume."""
    import torch
    import paper_2007_14394_b300 as S

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c = W.CASCADES[args.workload]
    base = c.base
    scene = c.scene()
    baked = W.bake(scene, base.sdf_dims, base.h, (0.0, 0.0, 0.0), dtype=base.sdf_dtype)
    states = [W.probe_states(scene, v.probe_dims, v.probe_origin, v.probe_spacing, v.h) for v in c.volumes]
    n_active = [int((st["flags"] & 1).sum()) for st in states]
    rays_per_step = sum(a * v.rays for a, v in zip(n_active, c.volumes))

    sc = S.create_scene()
    S.upload_sdf(sc, baked.sdf, baked.h, baked.origin, material=baked.material)
    S.set_lights(sc, scene.lights, scene.sky)
    vols, states_dev = [], []
    for i, v in enumerate(c.volumes):
        desc = S.make_desc(v.probe_dims, v.rays, v.probe_origin, v.probe_spacing, v.max_steps, v.depth_exponent,
                           v.eps_vox, v.tmax_vox, v.hysteresis, v.k_bounce, v.bias_vox, seed=v.seed, volume_id=i)
        vols.append(S.create_volume(desc, sc))
        states_dev.append(torch.from_numpy(states[i].view(np.uint8).copy()).to(dev))
    batch = S.create_batch(vols, states_dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # one recorded plain update per volume (outside any timed region) for the algorithmic work
    work = []
    for i, v in enumerate(c.volumes):
        records = torch.empty(v.n_probes * v.rays * 32, dtype=torch.uint8, device=dev)
        S.update_probes(vols[i], 0, states=states_dev[i], records=records)
        torch.cuda.synchronize()
        rec = records.cpu().numpy().view(S.RAY_RECORD_DTYPE)
        work.append(stage_work(rec, 4 if base.sdf_dtype == "f32" else 2, v.n_probes, v.rays, n_active[i]))
        del records
        S.reset(vols[i])
    t_tune = time.perf_counter()
    S.batch_autotune(batch, repeats=3, stream=stream)
    t_tune = time.perf_counter() - t_tune
    schedules = [dict(zip(("pool_batch", "blocks_per_sm", "gather", "index", "steps", "tuned_ms"), S.batch_schedule(batch, i)))
                 for i in range(len(vols))]
    form, tuned_branches, tuned_merged = S.batch_form(batch)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(step_fn, frame0):
        for k in range(args.warmup):
            step_fn(frame0 + k)
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            step_fn(frame0 + args.warmup + k)
            ends[k].record(stream)
        torch.cuda.synchronize()
        barrier()
        return [s.elapsed_time(e) for s, e in zip(starts, ends)]

    def plain(frame):
        for i in range(len(vols)):
            S.update_probes(vols[i], frame, states=states_dev[i], stream=stream)

    clocks = Clocks(local_rank)
    t0 = time.perf_counter()
    per_step = timed(lambda f: S.update_batch(batch, f, stream=stream), 0)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    seq_step = timed(plain, 10_000)
    # both forms of the frame, each timed the same way (the headline runs the autotuner's)
    forms = {}
    for name, f in (("branches", S.BATCH_FORM_BRANCHES), ("merged", S.BATCH_FORM_MERGED)):
        try:
            S.batch_set_form(batch, f)
        except S.SdfddgiError as err:
            forms[name] = {"unavailable": str(err)}
            continue
        forms[name] = {"ms_per_step": statistics.median(timed(lambda fr: S.update_batch(batch, fr, stream=stream),
                                                              30_000 + 1000 * f))}
    S.batch_set_form(batch, S.BATCH_FORM_AUTO)
    forms.update({"chosen": "merged" if form == S.BATCH_FORM_MERGED else "branches",
                  "autotune_ms": {"branches": tuned_branches, "merged": tuned_merged},
                  "what": "median step of each form; branches: one graph branch of stage kernels per volume; "
                          "merged: one launch per stage over all volumes, the trace pools spanning every volume"})

    # end to end: probe states in from pinned host memory, every volume's maps out
    host_states = [torch.from_numpy(st.view(np.uint8).copy()).pin_memory() for st in states]
    outs = [(torch.empty(v.n_probes * 8 * 8 * 4, dtype=torch.float32).pin_memory(),
             torch.empty(v.n_probes * 16 * 16 * 2, dtype=torch.float32).pin_memory(),
             torch.empty(v.n_probes, dtype=torch.uint8).pin_memory()) for v in c.volumes]

    def e2e_step(frame):
        for d, h in zip(states_dev, host_states):
            d.copy_(h, non_blocking=True)
        S.update_batch(batch, frame, stream=stream)
        for vol, (a, b, cc) in zip(vols, outs):
            S.lib.sdfddgi_read_state(vol, a.data_ptr(), b.data_ptr(), cc.data_ptr(), 0, S._stream(stream))
    e2e_step_ms = timed(e2e_step, 20_000)

    dev_ms, seq_ms, e2e_ms = float(sum(per_step)), float(sum(seq_step)), float(sum(e2e_step_ms))
    dev_ms, seq_ms, e2e_ms, wall = max_over_ranks([dev_ms, seq_ms, e2e_ms, wall], world, dev)
    ms = dev_ms / args.steps
    value = whole_job_rate(world, rays_per_step, args.steps, dev_ms)
    hbm, peak_kind = peaks()
    frame_bytes = sum(w[k]["bytes"] for w in work for k in ("primary", "prep", "shadow"))
    ach = frame_bytes / (ms / 1e3) / 1e9
    roof = {"kernel": "frame (all stages of all volumes in one graph launch)", "bound": "hbm", "achieved": ach,
            "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "bytes_per_launch": frame_bytes,
            "peak_source": f"{peak_kind} hbm_gbs", "traffic": None,
            "note": "trace/prep/shadow gathered bytes of every volume over the whole frame's time"}
    P_all = sum(v.n_probes for v in c.volumes)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"{base.sdf_dtype} sdf, f32 gather", "data": "synthetic (seeded scene, baked on the host)",
        "config": {"workload": f"{c.name}: {c.description}", "volumes": [
            {"probes": v.n_probes, "rays_per_probe": v.rays, "active_probes": a, **sch}
            for v, a, sch in zip(c.volumes, n_active, schedules)],
            "sdf": "x".join(map(str, base.sdf_dims)) + f" {base.sdf_dtype}", "max_steps": base.max_steps,
            "active_rays_per_step": rays_per_step, "seed": base.seed,
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)", "autotune_s": t_tune},
        "gpu_launches": (MERGED_KERNELS if form == S.BATCH_FORM_MERGED else KERNELS_PER_UPDATE * len(vols)) * args.steps,
        "forms": forms,
        "sequential": {"ms_per_step": seq_ms / args.steps, "value": whole_job_rate(world, rays_per_step, args.steps, seq_ms),
                       "what": "one plain update_probes launch per volume, default schedules, same stream"},
        "e2e": {"value": whole_job_rate(world, rays_per_step, args.steps, e2e_ms), "unit": UNIT,
                "h2d_bytes_per_step": P_all * 16,
                "d2h_bytes_per_step": P_all * (8 * 8 * 4 * 4 + 16 * 16 * 2 * 4 + 1),
                "ms_per_step": e2e_ms / args.steps},
        "roofline": roof,
        "wall_s_timed_loop": wall,
        "step_ms": {"min": min(per_step), "median": statistics.median(per_step), "max": max(per_step)},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cascade_cpu_baseline(c, scene, baked, states, budget_s=args.cpu_budget)
    S.destroy_batch(batch)
    for v in vols:
        S.destroy_volume(v)
    S.destroy_scene(sc)
    return line


CASCADE_QUERY = "cascade512_query"


def touched_map_bytes(c, pts, level, weight):
    """Irradiance-map and history bytes of the distinct probes the points interpolate from (the
    8 probes of the point's cell in its level, and in the next level where it blends)."""
    total = 0
    for i, v in enumerate(c.volumes):
        use = (level == i) | ((level == i - 1) & (weight < 1.0))
        if not use.any():
            continue
        d, o, sp = np.array(v.probe_dims), np.array(v.probe_origin), np.array(v.probe_spacing)
        g = np.clip((pts[use] - o) / sp, 0, d - 1)
        b = np.clip(np.floor(g).astype(np.int64), 0, np.maximum(d - 2, 0))
        ids = []
        for k in range(8):
            q = np.minimum(b + [(k >> a) & 1 for a in range(3)], d - 1)
            ids.append((q[:, 2] * d[1] + q[:, 1]) * d[0] + q[:, 0])
        total += np.unique(np.concatenate(ids)).size * (8 * 8 * 16 + 1)
    return total


def run_cascade_query(args, rank, world, local_rank):
    """Irradiance queries against a cascade of volumes (Sec. 3.5): the four volumes of the
    cascade512 workload (finest first, their maps random), 2,073,600 points per step; each
    point takes the finest volume holding it, blended toward the next across that volume's
    border with the mean-value-coordinate weight."""
    import torch
    import paper_2007_14394_b300 as S

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c = W.CASCADES["cascade512"]
    sc = S.create_scene()
    vols, host_maps = [], W.cascade_query_maps(c)
    for i, v in enumerate(c.volumes):
        desc = S.make_desc(v.probe_dims, v.rays, v.probe_origin, v.probe_spacing, v.max_steps, volume_id=i)
        vols.append(S.create_volume(desc, sc))
        irr, valid = host_maps[i]
        S.write_state(vols[i], irr, np.zeros((v.n_probes, 16, 16, 2), np.float32), valid)
    n = W.QUERY_POINTS
    pts, nrm = W.cascade_query_points(n)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    p_d, n_d = torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev)
    out = torch.empty((n, 3), dtype=torch.float32, device=dev)
    lvl = torch.empty(n, dtype=torch.int32, device=dev)
    wgt = torch.empty(n, dtype=torch.float32, device=dev)
    S.sample_irradiance_cascade(vols, p_d, n_d, out, lvl, wgt, stream=stream)
    torch.cuda.synchronize()
    level, weight = lvl.cpu().numpy(), wgt.cpu().numpy()
    blend = (weight < 1.0) & (level < len(vols) - 1)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(step_fn):
        for _ in range(args.warmup):
            step_fn()
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            step_fn()
            ends[k].record(stream)
        torch.cuda.synchronize()
        barrier()
        return [a.elapsed_time(b) for a, b in zip(starts, ends)]

    clocks = Clocks(local_rank)
    per_step = timed(lambda: S.sample_irradiance_cascade(vols, p_d, n_d, out, stream=stream))
    clk = clocks.stop()
    # end to end: points and normals in from pinned host memory, the irradiance out
    hp, hn = torch.from_numpy(pts).pin_memory(), torch.from_numpy(nrm).pin_memory()
    ho = torch.empty((n, 3), dtype=torch.float32).pin_memory()

    def e2e_step():
        p_d.copy_(hp, non_blocking=True)
        n_d.copy_(hn, non_blocking=True)
        S.sample_irradiance_cascade(vols, p_d, n_d, out, stream=stream)
        ho.copy_(out, non_blocking=True)
    e2e_ms = timed(e2e_step)
    ms, e2e = float(np.mean(per_step)), float(np.mean(e2e_ms))
    ms, e2e = max_over_ranks([ms, e2e], world, dev)
    hbm, peak_kind = peaks()
    alg = n * (24 + 12) + touched_map_bytes(c, pts, level, weight)
    ach = alg / (ms / 1e3) / 1e9
    line = {
        "metric": "irradiance queries/s through a cascade of probe volumes", "value": whole_job_rate(world, n, 1, ms),
        "unit": "points/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (random maps, seeded points)",
        "config": {"workload": f"{CASCADE_QUERY}: {n} points (1920x1080) against the 4 volumes of cascade512 "
                               "(8^3, 16^3 @2 m; 32x8x32 @4 m; 64x16x64 @2 m)",
                   "points": n, "levels": np.bincount(level, minlength=len(vols)).tolist(),
                   "blending_points": int(blend.sum()),
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
        "gpu_launches": args.steps,
        "e2e": {"value": whole_job_rate(world, n, 1, e2e), "unit": "points/s", "h2d_bytes_per_step": n * 24,
                "d2h_bytes_per_step": n * 12, "ms_per_step": e2e},
        "roofline": {"kernel": "cascade_kernel", "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                     "frac": ach / hbm, "bytes_per_launch": alg, "peak_source": f"{peak_kind} hbm_gbs",
                     "traffic": measured_traffic("cascade", CASCADE_QUERY),
                     "note": "36 B per point plus the maps of the distinct probes touched. The kernel is bound "
                             "by FP32 issue, not memory: each blending point's weight is 48 closed-form "
                             "face-edge terms (4 arctangents per lane of a warp)"},
        "step_ms": {"min": min(per_step), "median": statistics.median(per_step), "max": max(per_step)},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cascade_query_cpu_baseline(c, host_maps, pts, nrm, args.cpu_budget)
    for v in vols:
        S.destroy_volume(v)
    S.destroy_scene(sc)
    return line


def cascade_query_cpu_baseline(c, host_maps, pts, nrm, budget_s):
    import oracle as O
    grids = [O.make_grid(v.probe_dims, v.probe_origin, v.probe_spacing, v.rays, v.max_steps, v.eps_vox, v.tmax_vox,
                         v.hysteresis) for v in c.volumes]
    irr = [m[0].astype(np.float64) for m in host_maps]
    valid = [m[1] for m in host_maps]
    t0, k = time.perf_counter(), 0
    while time.perf_counter() - t0 < budget_s and k < len(pts):
        O.sample_irradiance_cascade(grids, irr, valid, pts[k].astype(np.float64), nrm[k].astype(np.float64))
        k += 1
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": f"the first {k} of the step's points, one oracle call each ({dt:.1f} s)"}


VISIBILITY_QUERY = "visibility256_query"
RELOCATE = "relocate256"


def surface_points(baked, lo, hi, n, seed):
    """n seeded shading-like points: uniform in the box [lo, hi] where the nearest voxel's SDF lies
    between half a voxel and two voxels (a shell over the surfaces), each with the unit gradient
    of the baked SDF there as its normal (central differences of the neighbouring voxels)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = baked.sdf.shape
    sdf = baked.sdf.astype(np.float32)
    pts, nrm = np.empty((0, 3)), np.empty((0, 3))
    while len(pts) < n:
        c = rng.uniform(lo, hi, (8 * n, 3))
        g = np.clip(np.floor((c - np.asarray(baked.origin)) / baked.h).astype(np.int64), 1, [nx - 2, ny - 2, nz - 2])
        v = sdf[g[:, 2], g[:, 1], g[:, 0]]
        keep = (v > 0.5 * baked.h) & (v <= 2.0 * baked.h)
        g, c = g[keep], c[keep]
        grad = np.stack([sdf[g[:, 2], g[:, 1], g[:, 0] + 1] - sdf[g[:, 2], g[:, 1], g[:, 0] - 1],
                         sdf[g[:, 2], g[:, 1] + 1, g[:, 0]] - sdf[g[:, 2], g[:, 1] - 1, g[:, 0]],
                         sdf[g[:, 2] + 1, g[:, 1], g[:, 0]] - sdf[g[:, 2] - 1, g[:, 1], g[:, 0]]], axis=1)
        ln = np.linalg.norm(grad, axis=1)
        ok = ln > 0
        pts = np.concatenate([pts, c[ok]])
        nrm = np.concatenate([nrm, grad[ok] / ln[ok, None]])
    return pts[:n].astype(np.float32), nrm[:n].astype(np.float32)


def run_point_query(args, rank, world, local_rank):
    """Interpolation with SDF probe visibility (Sec. 3.4) at 1920x1080 points of open256: each
    point weighs its 8 probes by a soft SDF shadow march toward each; the maps are those of 4
    updates of the open256 volume. Or (relocate256) probe relocation (Sec. 3.2) of the open256
    grid: a descent on the SDF per probe."""
    import torch
    import paper_2007_14394_b300 as S

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pr = W.PRESETS["open256"]
    scene, baked, states = build_inputs(pr)
    sc = S.create_scene()
    S.upload_sdf(sc, baked.sdf, baked.h, baked.origin, material=baked.material)
    S.set_lights(sc, scene.lights, scene.sky)
    desc = S.make_desc(pr.probe_dims, pr.rays, pr.probe_origin, pr.probe_spacing, pr.max_steps, pr.depth_exponent,
                       pr.eps_vox, pr.tmax_vox, pr.hysteresis, pr.k_bounce, pr.bias_vox, seed=pr.seed)
    vol = S.create_volume(desc, sc)
    states_dev = torch.from_numpy(states.view(np.uint8).copy()).to(dev)
    for f in range(4):
        S.update_probes(vol, f, states=states_dev)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(step_fn):
        for _ in range(args.warmup):
            step_fn()
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            step_fn()
            ends[k].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in zip(starts, ends)]

    hbm, peak_kind = peaks()
    lo = np.asarray(pr.probe_origin, np.float64)
    hi = lo + (np.asarray(pr.probe_dims) - 1) * np.asarray(pr.probe_spacing)
    if args.workload == VISIBILITY_QUERY:
        softness = 8.0
        n = W.QUERY_POINTS
        pts, nrm = surface_points(baked, lo, hi, n, seed=13)
        p_d, n_d = torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev)
        out = torch.empty((n, 3), dtype=torch.float32, device=dev)
        clocks = Clocks(local_rank)
        per_step = timed(lambda: S.sample_irradiance_visible(vol, p_d, n_d, out, softness, states_dev, stream=stream))
        clk = clocks.stop()
        hp, hn = torch.from_numpy(pts).pin_memory(), torch.from_numpy(nrm).pin_memory()
        ho = torch.empty((n, 3), dtype=torch.float32).pin_memory()

        def e2e_step():
            p_d.copy_(hp, non_blocking=True)
            n_d.copy_(hn, non_blocking=True)
            S.sample_irradiance_visible(vol, p_d, n_d, out, softness, states_dev, stream=stream)
            ho.copy_(out, non_blocking=True)
        e2e_ms = timed(e2e_step)
        units, unit, kernel = n, "points/s", "sample_visible_kernel"
        fixed = n * (24 + 12 + 8 * (16 + 4 * 16 + 1))  # point, normal, result; per probe its state, 4 texels, flag
        h2d, d2h = n * 24, n * 12
        what = (f"{VISIBILITY_QUERY}: {n} seeded shading points (1920x1080) in the probe box of open256, 0.5 to 2 "
                f"voxels off the surfaces, normals from the SDF's gradient, softness {softness}; maps of 4 updates")
        cpu = visibility_cpu_baseline(pr, baked, states, vol, pts, nrm, softness, args.cpu_budget) \
            if rank == 0 and world == 1 and not args.no_cpu_baseline else None
    else:
        n = pr.n_probes
        out = torch.empty(n * 16, dtype=torch.uint8, device=dev)
        clocks = Clocks(local_rank)
        per_step = timed(lambda: S.relocate_probes(vol, out, stream=stream))
        clk = clocks.stop()
        ho = torch.empty(n * 16, dtype=torch.uint8).pin_memory()

        def e2e_step():
            S.relocate_probes(vol, out, stream=stream)
            ho.copy_(out, non_blocking=True)
        e2e_ms = timed(e2e_step)
        units, unit, kernel = n, "probes/s", "relocate_kernel"
        fixed = n * 16  # each probe's new state
        h2d, d2h = 0, n * 16
        what = f"{RELOCATE}: relocation of the {n} probes of open256 (clearance 2 voxels, at most 16 descent steps)"
        cpu = relocate_cpu_baseline(pr, baked, args.cpu_budget) \
            if rank == 0 and world == 1 and not args.no_cpu_baseline else None
    ms, e2e = float(np.mean(per_step)), float(np.mean(e2e_ms))
    ms, e2e = max_over_ranks([ms, e2e], world, dev)
    ach = fixed / (ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": whole_job_rate(world, units, 1, ms), "unit": unit, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded scene and points, baked on the host)",
        "config": {"workload": what, "units": units,
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
        "gpu_launches": args.steps,
        "e2e": {"value": whole_job_rate(world, units, 1, e2e), "unit": unit, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e},
        "roofline": {"kernel": kernel, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                     "frac": ach / hbm, "bytes_per_launch": fixed, "peak_source": f"{peak_kind} hbm_gbs",
                     "traffic": None,
                     "note": "a lower bound: the bytes counted are the fixed ones per unit; the SDF samples of the "
                             "marches or descent steps (their counts are not exposed) come on top"},
        "step_ms": {"min": min(per_step), "median": statistics.median(per_step), "max": max(per_step)},
        "clocks": clk,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    S.destroy_volume(vol)
    S.destroy_scene(sc)
    return line


def visibility_cpu_baseline(pr, baked, states, vol, pts, nrm, softness, budget_s):
    """The oracle's visibility-weighted interpolation, one point per call, on the same maps."""
    import oracle as O
    import paper_2007_14394_b300 as S
    osc = O.OracleScene(baked.sdf, baked.h, baked.origin, baked.material)
    g = O.make_grid(pr.probe_dims, pr.probe_origin, pr.probe_spacing, pr.rays, pr.max_steps, pr.eps_vox,
                    pr.tmax_vox, pr.hysteresis, pr.depth_exponent, pr.k_bounce, pr.bias_vox)
    P = pr.n_probes
    irr = np.empty((P, 8, 8, 4), np.float32)
    dep = np.empty((P, 16, 16, 2), np.float32)
    val = np.empty(P, np.uint8)
    S.read_state(vol, irr, dep, val)
    irr64 = irr.astype(np.float64)
    pos = states["pos"].astype(np.float32)
    t0, k = time.perf_counter(), 0
    while time.perf_counter() - t0 < budget_s and k < len(pts):
        O.sample_irradiance_visible(osc, g, irr64, val, pts[k].astype(np.float64), nrm[k].astype(np.float64),
                                    softness, probe_pos=pos)
        k += 1
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": f"the first {k} of the step's points, one oracle call each ({dt:.1f} s)"}


def relocate_cpu_baseline(pr, baked, budget_s):
    """The oracle's relocation of the whole grid, repeated for about budget_s seconds."""
    import oracle as O
    osc = O.OracleScene(baked.sdf, baked.h, baked.origin, baked.material)
    g = O.make_grid(pr.probe_dims, pr.probe_origin, pr.probe_spacing, pr.rays, pr.max_steps, pr.eps_vox,
                    pr.tmax_vox, pr.hysteresis, pr.depth_exponent, pr.k_bounce, pr.bias_vox)
    t0, k = time.perf_counter(), 0
    while time.perf_counter() - t0 < budget_s and k < 64:
        O.relocate(osc, g, 2.0, 0.0)
        k += 1
    dt = time.perf_counter() - t0
    return {"value": k * pr.n_probes / dt, "unit": "probes/s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"{k} relocations of the whole grid ({pr.n_probes} probes), {dt:.1f} s"}


ANALYTIC = {"open256_analytic": "open256", "room64_analytic": "room64"}


def run_analytic(args, rank, world, local_rank):
    """The preset's scene as analytic SDF primitives (Sec. 3.1) instead of a voxel volume: the
    update with the paper's cluster culling (8 primitives per cluster, queries along a trace
    bounded by twice the last distance), against the same update with culling off (one cluster:
    the plain loop over all primitives, the paper's baseline) and against the voxel volume."""
    import torch
    import paper_2007_14394_b300 as S

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pr = W.PRESETS[ANALYTIC[args.workload]]
    scene, baked, states = build_inputs(pr)
    P, R = pr.n_probes, pr.rays
    n_active = int((states["flags"] & 1).sum())
    rays_per_step = n_active * R
    t, prm = scene.arrays()
    hi = np.asarray(pr.sdf_dims, dtype=np.float64) * pr.h
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    states_dev = torch.from_numpy(states.view(np.uint8).copy()).to(dev)
    desc = S.make_desc(pr.probe_dims, R, pr.probe_origin, pr.probe_spacing, pr.max_steps, pr.depth_exponent,
                       pr.eps_vox, pr.tmax_vox, pr.hysteresis, pr.k_bounce, pr.bias_vox, seed=pr.seed)

    def measure(setup, steps, with_stages=False, with_clocks=False):
        sc = S.create_scene()
        setup(sc)
        S.set_lights(sc, scene.lights, scene.sky)
        vol = S.create_volume(desc, sc)
        for k in range(args.warmup):
            S.update_probes(vol, k, states=states_dev, stream=stream)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        stage_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(steps)]
        for evs in stage_ev:
            for e in evs:
                e.record(stream)
        torch.cuda.synchronize()
        clocks = Clocks(local_rank) if with_clocks else None
        for k in range(steps):
            flush.fill_(float(k))
            if with_stages:
                S.set_stage_events(vol, stage_ev[k])
            ev[k][0].record(stream)
            S.update_probes(vol, args.warmup + k, states=states_dev, stream=stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks else None
        S.set_stage_events(vol, [])
        ms = [a.elapsed_time(b) for a, b in ev]
        stages = None
        if with_stages:
            stages = {name: sum(e[i].elapsed_time(e[i + 1]) for e in stage_ev) / steps for i, name in enumerate(S.STAGES)}
        assert S.volume_status(vol) == 0
        S.destroy_volume(vol)
        S.destroy_scene(sc)
        return ms, stages, clk

    def prims(cluster_size):
        return lambda sc: S.upload_primitives(sc, t, prm, scene.albedo, scene.emission, (0.0, 0.0, 0.0), hi, pr.h,
                                              cluster_size)

    ms_c, stages, clk = measure(prims(8), args.steps, with_stages=True, with_clocks=True)
    ms_b, _, _ = measure(prims(0), max(3, args.steps // 4))
    ms_v, _, _ = measure(lambda sc: S.upload_sdf(sc, baked.sdf, baked.h, baked.origin, material=baked.material),
                         max(3, args.steps // 4))
    ms = float(np.mean(ms_c))
    (ms,) = max_over_ranks([ms], world, dev)
    dominant = max(("primary", "prep", "shadow"), key=lambda n: stages[n])
    line = {
        "metric": METRIC, "value": whole_job_rate(world, rays_per_step, 1, ms), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded scene of analytic primitives)",
        "config": dict(workload_config(pr, rays_per_step), workload=f"{args.workload}: the {pr.name} scene as "
                       f"{len(t)} analytic primitives, clusters of 8", primitives=len(t)),
        "gpu_launches": KERNELS_PER_UPDATE * args.steps,
        "clusters": {"ms_per_update": ms, "brute_force_ms_per_update": float(np.mean(ms_b)),
                     "speedup": float(np.mean(ms_b)) / ms,
                     "note": "culling on (8 primitives per cluster, traces bounded by twice the last distance) "
                             "vs one cluster holding every primitive (the plain loop)"},
        "voxel_ms_per_update": float(np.mean(ms_v)),
        "stages_ms": stages,
        "roofline": {"kernel": dominant, "bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
                     "traffic": None, "note": "primitive queries run from L1 (the primitives take a few KiB); "
                                              "no byte or flop model is reported for them"},
        "e2e": None,
        "clocks": clk,
    }
    return line


LEARNED = "learned32"
DENOISER_FLOPS_PER_PROBE = 2 * 36 * (9 * 35 * 64 + 9 * 64 * 48 + 9 * 48 * 3)  # 3 convs over 36 interior texels


def run_learned(args, rank, world, local_rank):
    """The learned form: the denoiser trained on pairs the plain update makes on 64 room
    scenes, its error on 8 held-out scenes against plain updates of several ray counts,
    and the frame time at 32 x 16 x 32 probes of the open scene: a 32-ray update plus the
    tensor-core denoiser against plain updates at the ray count of equal error and at 256."""
    import torch
    import paper_2007_14394_b300 as S
    from paper_2007_14394_b300 import learned as L

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    room = W.PRESETS["room64"]
    plain_rays = (48, 64, 96, 128, 192, 256)
    t0 = time.perf_counter()
    train = L.make_pairs(room, list(range(1, 65)), plain_rays=plain_rays)
    held = L.make_pairs(room, list(range(1001, 1009)), plain_rays=plain_rays)
    t_pairs = time.perf_counter() - t0
    depth_scale = 4.0
    d = S.create_denoiser(W.denoiser_init(0), depth_scale)
    t0 = time.perf_counter()
    hist = L.train(d, train, steps=args.train_steps, batch_grids=8, lr=3e-4, log_every=max(1, args.train_steps // 8))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    err = L.evaluate(d, held)
    err_train = L.evaluate(d, train)
    r_eq = L.equal_error_rays(err)

    # frame times on the open scene's 32 x 16 x 32 grid
    pr = W.PRESETS["open256"]
    scene, baked, states = build_inputs(pr)
    n_active = int((states["flags"] & 1).sum())
    sc = S.create_scene()
    S.upload_sdf(sc, baked.sdf, baked.h, baked.origin, material=baked.material)
    S.set_lights(sc, scene.lights, scene.sky)
    states_dev = torch.from_numpy(states.view(np.uint8).copy()).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def volume(rays):
        desc = S.make_desc(pr.probe_dims, rays, pr.probe_origin, pr.probe_spacing, pr.max_steps, pr.depth_exponent,
                           pr.eps_vox, pr.tmax_vox, pr.hysteresis, pr.k_bounce, pr.bias_vox, seed=pr.seed)
        return S.create_volume(desc, sc)

    def timed(step_fn):
        for k in range(args.warmup):
            step_fn(k)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            step_fn(args.warmup + k)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    v32 = volume(32)
    dn_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    dn_ms = []

    def learned_frame(f):
        S.update_probes(v32, f, states=states_dev, stream=stream)
        dn_ev[0].record(stream)
        S.denoise_volume(d, v32, states_dev, stream=stream)
        dn_ev[1].record(stream)

    clocks = Clocks(local_rank)
    learned_steps = []
    for k in range(args.warmup):
        learned_frame(k)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        learned_frame(args.warmup + k)
        b.record(stream)
        torch.cuda.synchronize()
        learned_steps.append(a.elapsed_time(b))
        dn_ms.append(dn_ev[0].elapsed_time(dn_ev[1]))
    clk = clocks.stop()
    plain_ms = {}
    for rays in sorted({256, int(math.ceil(r_eq)) if r_eq else 256}):
        v = volume(rays)
        plain_ms[rays] = statistics.median(timed(lambda f: S.update_probes(v, f, states=states_dev, stream=stream)))
        S.destroy_volume(v)
    learned_ms = statistics.median(learned_steps)
    (learned_ms,) = max_over_ranks([learned_ms], world, dev)
    denoise_ms = statistics.median(dn_ms)
    P = pr.n_probes
    tc_peak, tc_kind = tensor_peak()
    ach = DENOISER_FLOPS_PER_PROBE * n_active / (denoise_ms / 1e3) / 1e12
    eq_rays = r_eq if r_eq else None
    value = whole_job_rate(world, n_active * eq_rays, 1, learned_ms) if eq_rays else None
    line = {
        "metric": METRIC, "value": value, "unit": "equal-error probe-rays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": learned_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 update, bf16 x bf16 -> f32 denoiser",
        "data": "synthetic (seeded scenes, baked on the host; pairs made by the plain update)",
        "config": {"workload": f"{LEARNED}: 32-ray update + denoiser at {pr.probe_dims} probes of {pr.name}; "
                               "trained on 64 room64 seeds (1..64), evaluated on 8 held-out seeds (1001..1008)",
                   "probes": P, "active_probes": n_active, "train_steps": args.train_steps, "batch_grids": 8,
                   "lr": 3e-4, "depth_scale": depth_scale,
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
        "gpu_launches": (kernels_per_update(S.volume_slabs(v32)) + 2) * args.steps,
        "rmse_heldout": err, "rmse_train": err_train, "equal_error_rays": r_eq,
        "ms": {"learned32_frame": learned_ms, "denoise": denoise_ms, "update32": learned_ms - denoise_ms,
               **{f"plain{r}": t for r, t in plain_ms.items()}},
        "training": {"pairs_s": t_pairs, "train_s": t_train, "loss": hist},
        "roofline": {"kernel": "denoise_tc_kernel", "bound": "tensor", "achieved": ach, "peak": tc_peak,
                     "unit": "TFLOP/s", "frac": ach / tc_peak, "flops_per_launch": DENOISER_FLOPS_PER_PROBE * n_active,
                     "peak_source": f"{tc_kind} bf16 burst", "traffic": measured_traffic("denoise", LEARNED)},
        "clocks": clk,
    }
    S.destroy_volume(v32)
    S.destroy_scene(sc)
    S.destroy_denoiser(d)
    return line


def cascade_cpu_baseline(c, scene, baked, states, budget_s=10.0):
    """The oracle on a seeded sample of every volume's active probes, about budget_s seconds in
    all; the frame time is extrapolated linearly in the probe counts."""
    cores = os.cpu_count() or 1
    per_vol = budget_s / len(c.volumes)
    frame_s, rays, samples = 0.0, 0, []
    for i, (v, st) in enumerate(zip(c.volumes, states)):
        n_act = int((st["flags"] & 1).sum())
        dt, _ = oracle_sample(v, scene, baked, st, max(4, cores), volume=i)
        n = int(max(4, min(n_act, max(4, cores) * per_vol / max(dt, 1e-3))))
        dt, r = oracle_sample(v, scene, baked, st, n, seed=1, volume=i)
        frame_s += dt * n_act / n
        rays += n_act * v.rays
        samples.append(f"{n}/{n_act}")
    return {"value": rays / frame_s, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"seeded active probes per volume {', '.join(samples)} of {c.name}, one frame each; "
                      f"frame time extrapolated linearly", "ms_per_step": 1e3 * frame_s}


def oracle_sample(pr, scene, baked, states, n_probes, seed=0, frame=0, threads=0, volume=0):
    """Times the oracle's update of a seeded sample of active probes; returns (seconds, rays)."""
    import oracle as O
    act = np.flatnonzero(states["flags"] & 1)
    rng = np.random.default_rng(seed)
    sub = np.sort(rng.choice(act, min(n_probes, len(act)), replace=False))
    osc = O.OracleScene(baked.sdf, baked.h, baked.origin, baked.material)
    g = O.make_grid(pr.probe_dims, pr.probe_origin, pr.probe_spacing, pr.rays, pr.max_steps, pr.eps_vox,
                    pr.tmax_vox, pr.hysteresis, pr.depth_exponent, pr.k_bounce, pr.bias_vox, scene.sky)
    rot = W.frame_rotation(pr.seed, frame, volume)
    t0 = time.perf_counter()
    O.update(osc, g, scene.lights, rot, states, subset=sub, want_rays=False, n_threads=threads)
    return time.perf_counter() - t0, len(sub) * pr.rays


def cpu_baseline(pr, scene, baked, states, budget_s=10.0):
    """The oracle as it stands, on all host cores: consecutive frames of the whole workload
    (each frame starting from the oracle's own previous maps) until about budget_s seconds."""
    import oracle as O
    cores = os.cpu_count() or 1
    osc = O.OracleScene(baked.sdf, baked.h, baked.origin, baked.material)
    g = O.make_grid(pr.probe_dims, pr.probe_origin, pr.probe_spacing, pr.rays, pr.max_steps, pr.eps_vox,
                    pr.tmax_vox, pr.hysteresis, pr.depth_exponent, pr.k_bounce, pr.bias_vox, scene.sky)
    n_active = int((states["flags"] & 1).sum())
    prev, frames, t_total = None, 0, 0.0
    while t_total < budget_s and frames < 64:
        t0 = time.perf_counter()
        out = O.update(osc, g, scene.lights, W.frame_rotation(pr.seed, frames), states, prev=prev, want_rays=False,
                       n_threads=cores)
        t_total += time.perf_counter() - t0
        prev = (out["irr"], out["depth"], out["valid"])
        frames += 1
    # one core, on a seeded sample of the active probes sized for about a third of the budget
    per_probe_1core = t_total / frames / n_active * cores
    n1 = int(max(8, min(n_active, budget_s / 3 / max(per_probe_1core, 1e-9))))
    sub = np.sort(np.random.default_rng(3).choice(np.flatnonzero(states["flags"] & 1), n1, replace=False))
    t0 = time.perf_counter()
    O.update(osc, g, scene.lights, W.frame_rotation(pr.seed, frames), states, prev=prev, subset=sub, want_rays=False,
             n_threads=1)
    t1 = time.perf_counter() - t0
    return {"value": frames * n_active * pr.rays / t_total, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{frames} consecutive full frames of {pr.name} ({n_active} active probes x {pr.rays} rays), "
                      f"{t_total:.1f} s on {cores} OpenMP threads",
            "ms_per_step": 1e3 * t_total / frames,
            "one_core": {"value": n1 * pr.rays / t1, "unit": UNIT, "cores": 1,
                         "sample": f"{n1} seeded active probes of frame {frames} x {pr.rays} rays, {t1:.1f} s "
                                   "on 1 thread"}}


def run_reference(args):
    pr = W.PRESETS[args.workload]
    scene, baked, states = build_inputs(pr)
    cores = os.cpu_count() or 1
    n_active = int((states["flags"] & 1).sum())
    dt, _ = oracle_sample(pr, scene, baked, states, max(4, cores))
    per_step_budget = max(0.05, 60.0 / max(1, args.steps + args.warmup))
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
    ms = tot / args.steps * 1e3  # what was timed: one step is the oracle over a sample of the probes
    sample = (f"one step = the oracle's update of {n} seeded random active probes of {pr.name} (of {n_active}) x "
              f"{pr.rays} rays on {cores} OpenMP threads; ms_per_step is that sample's time, and "
              "ms_per_frame_extrapolated scales it linearly to the whole frame")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "ms_per_frame_extrapolated": ms * n_active / n,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded scene, baked on the host)",
            "config": workload_config(pr, n_active * pr.rays),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=sorted(W.PRESETS) + sorted(W.CASCADES) + [LEARNED] + sorted(ANALYTIC) + [CASCADE_QUERY]
                    + [VISIBILITY_QUERY, RELOCATE])
    ap.add_argument("--train-steps", type=int, default=24000, help="training steps of the learned32 workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--slabs", type=int, default=0,
                    help="slab branches per update of the open256 volume (0: the library's automatic choice)")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if args.workload in W.CASCADES or args.workload in (LEARNED, CASCADE_QUERY, VISIBILITY_QUERY, RELOCATE) \
                or args.workload in ANALYTIC:
            ap.error("the reference arm times single-volume workloads")
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    run = (run_batch if args.workload in W.CASCADES else run_learned if args.workload == LEARNED
           else run_analytic if args.workload in ANALYTIC else run_cascade_query if args.workload == CASCADE_QUERY
           else run_point_query if args.workload in (VISIBILITY_QUERY, RELOCATE) else run_ours)
    line = run(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
