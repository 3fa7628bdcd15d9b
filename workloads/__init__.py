"""Seeded synthetic inputs for the SDFDDGI probe update (tests, bench, smoke).

This module serves the CUDA path and the oracle alike, so it holds no step of
the probe update itself: only scene construction (analytic primitives and
their bake into a voxel signed-distance volume plus a material volume), probe
grids and probe states, lights, the named workload presets, and the per-frame
random rotation of the ray set (a counter-based generator, splitmix64 feeding
Shoemake's uniform random rotation, that the library also implements from the
same published definitions for callers that do not pass a rotation).

Scene recipes follow the paper's setting of a scene made of SDF primitives
(Sec. 3.1) at the sizes of the five named workloads (``PRESETS``).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bake.c")
_LIB = os.path.join(_HERE, "libbake.so")
_lock = threading.Lock()
_lib = None

SPHERE, BOX, CAPSULE, PLANE_Y, INV_SPHERE = 0, 1, 2, 3, 4
PROBE_DTYPE = np.dtype([("pos", "f4", (3,)), ("flags", "u4")])
ACTIVE, REJECT_HISTORY = 1, 2


def build(force: bool = False) -> str:
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_SRC) > os.path.getmtime(_LIB)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.wl_eval.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
            lib.wl_bake.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_int, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
            _lib = lib
    return _lib


# ---------------------------------------------------------------------------- scenes
@dataclass
class Scene:
    """Analytic primitives with per-primitive albedo/emission, lights and sky."""
    types: list = field(default_factory=list)
    params: list = field(default_factory=list)      # 8 doubles each
    albedo: list = field(default_factory=list)      # rgb
    emission: list = field(default_factory=list)    # rgb
    lights: list = field(default_factory=list)      # dicts {type, v, rgb, range}
    sky: tuple = (0.0, 0.0, 0.0)

    def add(self, t, params, albedo, emission=(0.0, 0.0, 0.0)):
        p = list(map(float, params)) + [0.0] * (8 - len(params))
        self.types.append(int(t))
        self.params.append(p)
        self.albedo.append(tuple(map(float, albedo)))
        self.emission.append(tuple(map(float, emission)))

    def arrays(self):
        return (np.ascontiguousarray(self.types, dtype=np.int32),
                np.ascontiguousarray(self.params, dtype=np.float64).reshape(-1, 8))

    def eval(self, pts) -> tuple[np.ndarray, np.ndarray]:
        """Exact union SDF and owning primitive at world points [n,3]."""
        pts = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 3))
        t, p = self.arrays()
        sdf = np.empty(len(pts))
        own = np.empty(len(pts), dtype=np.int32)
        _load().wl_eval(len(t), t.ctypes.data, p.ctypes.data, len(pts), pts.ctypes.data, sdf.ctypes.data,
                        own.ctypes.data)
        return sdf, own


@dataclass
class Baked:
    sdf: np.ndarray            # [nz,ny,nx] float32 or float16 (RTZ)
    material: np.ndarray       # [nz,ny,nx,8] float16: albedo rgb, 0, emission rgb, 0
    h: float
    origin: tuple
    sdf64: np.ndarray | None = None


def bake(scene: Scene, dims, h: float, origin=(0.0, 0.0, 0.0), dtype="f32", keep64=False,
         n_threads: int = 0) -> Baked:
    nx, ny, nz = (int(d) for d in dims)
    t, p = scene.arrays()
    org = np.ascontiguousarray(origin, dtype=np.float64)
    n = nx * ny * nz
    sdf64 = np.empty((nz, ny, nx)) if keep64 else None
    sdf32 = np.empty((nz, ny, nx), dtype=np.float32) if dtype == "f32" else None
    sdf16 = np.empty((nz, ny, nx), dtype=np.uint16) if dtype == "f16" else None
    owner = np.empty(n, dtype=np.int32)
    _load().wl_bake(nx, ny, nz, float(h), org.ctypes.data, len(t), t.ctypes.data, p.ctypes.data,
                    sdf64.ctypes.data if sdf64 is not None else None,
                    sdf32.ctypes.data if sdf32 is not None else None,
                    sdf16.ctypes.data if sdf16 is not None else None, owner.ctypes.data, int(n_threads))
    table = np.zeros((len(t), 8), dtype=np.float64)
    table[:, 0:3] = np.asarray(scene.albedo)
    table[:, 4:7] = np.asarray(scene.emission)
    material = table.astype(np.float16)[owner].reshape(nz, ny, nx, 8)
    sdf = sdf32 if sdf32 is not None else sdf16.view(np.float16)
    return Baked(sdf=sdf, material=material, h=float(h), origin=tuple(map(float, origin)), sdf64=sdf64)


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def room_scene(seed: int, size: float = 8.0, wall: float = 0.25, n_spheres: int = 4, n_boxes: int = 3,
               aperture: float = 3.0, uniform_albedo=None, emission=(0.0, 0.0, 0.0), sun=True) -> Scene:
    """Box room of side `size` with walls of thickness `wall`, `n_spheres` spheres
    (r ~ U[0.5, 2]) and `n_boxes` axis-aligned boxes (half-extents ~ U[0.25, 1.5])
    with centres uniform in the interior, per-primitive albedo ~ U[0.5, 0.9] per
    channel. A square opening of side `aperture` in the ceiling lets the single
    directional light in (aperture 0 closes the room completely).
    `uniform_albedo`/`emission` give every surface the same material (furnace and
    multi-bounce scenes)."""
    rng = np.random.default_rng(seed)
    s = Scene()

    def alb():
        return tuple(uniform_albedo) if uniform_albedo is not None else tuple(rng.uniform(0.5, 0.9, 3))

    c, hw = size / 2, wall / 2
    s.add(BOX, [c, hw, c, c, hw, c], alb(), emission)                 # floor
    s.add(BOX, [hw, c, c, hw, c, c], alb(), emission)                 # wall -x
    s.add(BOX, [size - hw, c, c, hw, c, c], alb(), emission)          # wall +x
    s.add(BOX, [c, c, hw, c, c, hw], alb(), emission)                 # wall -z
    s.add(BOX, [c, c, size - hw, c, c, hw], alb(), emission)          # wall +z
    yc = size - hw
    if aperture <= 0:
        s.add(BOX, [c, yc, c, c, hw, c], alb(), emission)             # closed ceiling
    else:
        a0, a1 = c - aperture / 2, c + aperture / 2
        s.add(BOX, [c, yc, a0 / 2, c, hw, a0 / 2], alb(), emission)
        s.add(BOX, [c, yc, (a1 + size) / 2, c, hw, (size - a1) / 2], alb(), emission)
        s.add(BOX, [a0 / 2, yc, c, a0 / 2, hw, aperture / 2], alb(), emission)
        s.add(BOX, [(a1 + size) / 2, yc, c, (size - a1) / 2, hw, aperture / 2], alb(), emission)
    lo, hi = wall, size - wall
    for _ in range(n_spheres):
        s.add(SPHERE, list(rng.uniform(lo, hi, 3)) + [rng.uniform(0.5, 2.0)], alb(), emission)
    for _ in range(n_boxes):
        s.add(BOX, list(rng.uniform(lo, hi, 3)) + list(rng.uniform(0.25, 1.5, 3)), alb(), emission)
    if sun:
        s.lights.append({"type": "dir", "v": _unit([0.25, 1.0, 0.15]), "rgb": (3.0, 2.9, 2.7), "range": 0.0})
    return s


def open_scene(seed: int, size: float = 64.0, n_prims: int = 200, ground: float = 1.0, n_points: int = 16,
               point_y=(2.0, 10.0), sky=(0.25, 0.35, 0.55)) -> Scene:
    """Open world of side `size`: a ground half-space at y = `ground`, `n_prims`
    spheres / axis-aligned boxes / randomly oriented capsules (type uniform, size
    log-uniform in [0.2, 8] m) resting on the ground, a sun and `n_points` point
    lights with finite range, constant sky radiance."""
    rng = np.random.default_rng(seed)
    s = Scene(sky=tuple(sky))
    s.add(PLANE_Y, [ground], tuple(rng.uniform(0.5, 0.9, 3)))
    for _ in range(n_prims):
        kind = int(rng.integers(0, 3))
        size_m = math.exp(rng.uniform(math.log(0.2), math.log(8.0)))
        x, z = rng.uniform(0.0, size, 2)
        alb = tuple(rng.uniform(0.5, 0.9, 3))
        if kind == SPHERE:
            r = size_m / 2
            s.add(SPHERE, [x, ground + r, z, r], alb)
        elif kind == BOX:
            e = size_m / 2 * rng.uniform(0.4, 1.0, 3)
            s.add(BOX, [x, ground + e[1], z, e[0], e[1], e[2]], alb)
        else:
            r = size_m * rng.uniform(0.08, 0.2)
            half = max(size_m / 2 - r, 0.0)
            u = _unit(rng.normal(size=3))
            cy = ground + abs(u[1]) * half + r
            a = np.array([x, cy, z]) - u * half
            b = np.array([x, cy, z]) + u * half
            s.add(CAPSULE, list(a) + list(b) + [r], alb)
    s.lights.append({"type": "dir", "v": _unit([0.35, 0.8, 0.25]), "rgb": (2.6, 2.4, 2.0), "range": 0.0})
    for _ in range(n_points):
        pos = (rng.uniform(2.0, size - 2.0), rng.uniform(*point_y), rng.uniform(2.0, size - 2.0))
        tint = rng.uniform(0.6, 1.0, 3)
        s.lights.append({"type": "point", "v": pos, "rgb": tuple(rng.uniform(20.0, 80.0) * tint),
                         "range": float(rng.uniform(8.0, 16.0))})
    return s


# ---------------------------------------------------------------------------- probes
def probe_grid_positions(dims, origin, spacing) -> np.ndarray:
    """World positions [P,3] of the probe grid, x fastest (index = (z*ny + y)*nx + x)."""
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    idx = np.stack([x, y, z], axis=-1).reshape(-1, 3).astype(np.float64)
    return np.asarray(origin, dtype=np.float64) + idx * np.asarray(spacing, dtype=np.float64)


def probe_states(scene: Scene, dims, origin, spacing, h: float, min_clearance_vox: float = 0.5) -> np.ndarray:
    """Probe states at the grid positions; a probe is active when the exact scene
    distance at its position exceeds `min_clearance_vox` voxels."""
    pos = probe_grid_positions(dims, origin, spacing)
    sdf, _ = scene.eval(pos)
    st = np.zeros(len(pos), dtype=PROBE_DTYPE)
    st["pos"] = pos.astype(np.float32)
    st["flags"] = np.where(sdf > min_clearance_vox * h, ACTIVE, 0).astype(np.uint32)
    return st


# ---------------------------------------------------------------------------- frame rotation
_M64 = (1 << 64) - 1


def _splitmix64(state: int):
    state = (state + 0x9E3779B97F4A7C15) & _M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return state, z ^ (z >> 31)


def frame_rotation(seed: int, frame: int, volume: int = 0) -> np.ndarray:
    """float32 (3,3) rotation of frame `frame`: three uniforms u1,u2,u3 in [0,1) from
    splitmix64 started at seed*G + frame*A + volume*B (mod 2^64), mapped to a unit
    quaternion by Shoemake's method, then to a row-major matrix."""
    state = (seed * 0x9E3779B97F4A7C15 + frame * 0xBF58476D1CE4E5B9 + volume * 0x94D049BB133111EB) & _M64
    u = []
    for _ in range(3):
        state, z = _splitmix64(state)
        u.append((z >> 11) * (1.0 / 9007199254740992.0))
    u1, u2, u3 = u
    a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
    x, y = a * math.sin(2.0 * math.pi * u2), a * math.cos(2.0 * math.pi * u2)
    z, w = b * math.sin(2.0 * math.pi * u3), b * math.cos(2.0 * math.pi * u3)
    m = np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])
    return m.astype(np.float32)


# ---------------------------------------------------------------------------- presets
@dataclass
class Preset:
    name: str
    description: str
    world: float
    sdf_dims: tuple
    h: float
    probe_dims: tuple
    probe_origin: tuple
    probe_spacing: tuple
    rays: int
    max_steps: int
    eps_vox: float = 0.01
    hysteresis: float = 0.97
    depth_exponent: int = 50
    k_bounce: float = 0.9
    bias_vox: float = 1.0
    frames: int = 1
    sdf_dtype: str = "f32"
    blend: str = "f32"
    seed: int = 7
    scene_kind: str = "room"
    scene_args: dict = field(default_factory=dict)

    @property
    def n_probes(self) -> int:
        return int(np.prod(self.probe_dims))

    @property
    def tmax_vox(self) -> float:
        """Trace length limit: the volume's diagonal, in voxels."""
        return float(math.sqrt(sum(d * d for d in self.sdf_dims)))

    def scene(self, seed: int | None = None) -> Scene:
        seed = self.seed if seed is None else seed
        if self.scene_kind == "room":
            return room_scene(seed, size=self.world, **self.scene_args)
        return open_scene(seed, size=self.world, **self.scene_args)


PRESETS = {
    "room64": Preset(
        "room64", "8x8x8 probes over a 64^3 float32 SDF of a box room with 4 spheres and 3 boxes, "
        "1 directional light, 64 rays/probe, <=64 steps, eps 0.01 voxel, hysteresis 0.97, one frame",
        world=8.0, sdf_dims=(64, 64, 64), h=0.125, probe_dims=(8, 8, 8), probe_origin=(0.5, 0.5, 0.5),
        probe_spacing=(1.0, 1.0, 1.0), rays=64, max_steps=64, frames=1, seed=7, scene_kind="room"),
    "open256": Preset(
        "open256", "32x16x32 probes over a 256^3 float32 SDF of 200 primitives on a ground plane, sun + 16 "
        "point lights, 256 rays/probe, <=128 steps, 8 frames with multi-bounce",
        world=64.0, sdf_dims=(256, 256, 256), h=0.25, probe_dims=(32, 16, 32), probe_origin=(1.0, 2.0, 1.0),
        probe_spacing=(2.0, 2.0, 2.0), rays=256, max_steps=128, frames=8, seed=11, scene_kind="open"),
    "open256_quarter": Preset(
        "open256_quarter", "the open256 scene and SDF with the first 8 of its 32 probe layers (32x16x8 probes): "
        "the same kernels on a quarter of the probes, for profiler captures (the SDF copies still exceed L2)",
        world=64.0, sdf_dims=(256, 256, 256), h=0.25, probe_dims=(32, 16, 8), probe_origin=(1.0, 2.0, 1.0),
        probe_spacing=(2.0, 2.0, 2.0), rays=256, max_steps=128, frames=8, seed=11, scene_kind="open"),
    "room64_fp16": Preset(
        "room64_fp16", "room64 with a float16 SDF (rounded toward zero), float32 stepping, bf16 blend",
        world=8.0, sdf_dims=(64, 64, 64), h=0.125, probe_dims=(8, 8, 8), probe_origin=(0.5, 0.5, 0.5),
        probe_spacing=(1.0, 1.0, 1.0), rays=64, max_steps=64, frames=1, seed=7, scene_kind="room",
        sdf_dtype="f16", blend="bf16"),
}


@dataclass
class Cascade:
    """Several probe volumes over one scene (Sec. 3.5 cascades), updated together as a
    batch. Every member is a Preset with the same scene fields; member i is volume id i."""
    name: str
    description: str
    volumes: tuple

    @property
    def base(self) -> Preset:
        return self.volumes[0]

    @property
    def n_rays(self) -> int:
        return sum(v.n_probes * v.rays for v in self.volumes)

    def scene(self, seed: int | None = None) -> Scene:
        return self.base.scene(seed)


def _cascade_member(name, probe_dims, probe_origin, probe_spacing, rays) -> Preset:
    return Preset(name, f"{probe_dims} probes at {probe_spacing[0]} m, {rays} rays/probe", world=128.0,
                  sdf_dims=(512, 512, 512), h=0.25, probe_dims=probe_dims, probe_origin=probe_origin,
                  probe_spacing=probe_spacing, rays=rays, max_steps=128, frames=8, seed=11, scene_kind="open",
                  scene_args={"n_prims": 2000}, sdf_dtype="f16")


# Four concentric volumes of uneven sizes and ray counts around the centre of a 128 m open
# world (512^3 binary16 SDF of 2000 primitives, h = 0.25 m, sun + 16 point lights);
# 6,553,600 probe rays per frame in all.
CASCADES = {
    "cascade512": Cascade(
        "cascade512", "4 volumes over one 512^3 float16 SDF of 2000 primitives: 8^3 @512 rays, 16^3 @256, "
        "32x8x32 @128, 64x16x64 @64; <=128 steps, sun + 16 point lights",
        volumes=(
            _cascade_member("cascade512.0", (8, 8, 8), (57.0, 2.0, 57.0), (2.0, 2.0, 2.0), 512),
            _cascade_member("cascade512.1", (16, 16, 16), (49.0, 2.0, 49.0), (2.0, 2.0, 2.0), 256),
            _cascade_member("cascade512.2", (32, 8, 32), (2.0, 2.0, 2.0), (4.0, 4.0, 4.0), 128),
            _cascade_member("cascade512.3", (64, 16, 64), (1.0, 2.0, 1.0), (2.0, 2.0, 2.0), 64),
        )),
}


# ---------------------------------------------------------------------------- learned form
# Layer shapes of the probe denoiser's parameter vector, in order (weights [tap][in][out]).
DENOISER_SHAPES = (("w1", (9, 35, 64)), ("b1", (64,)), ("w2", (9, 64, 48)), ("b2", (48,)),
                   ("w3", (9, 48, 3)), ("b3", (3,)))


def denoiser_init(seed: int, last_scale: float = 0.0) -> np.ndarray:
    """Seeded initial parameters (float32 [49219]): He-uniform weights, U(-sqrt(6/fan_in),
    +sqrt(6/fan_in)) with fan_in = 9 x input channels, the last layer scaled by `last_scale`
    (0 by default: the initial network is the identity, its residual zero); zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in DENOISER_SHAPES:
        if name.startswith("w"):
            lim = math.sqrt(6.0 / (9 * shape[1]))
            w = rng.uniform(-lim, lim, shape)
            parts.append(w * (last_scale if name == "w3" else 1.0))
        else:
            parts.append(np.zeros(shape))
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)


# Irradiance queries against the cascade512 volumes (Sec. 3.5): one 1080p frame's shading points.
QUERY_POINTS = 1920 * 1080


def cascade_query_points(n: int = QUERY_POINTS, seed: int = 5):
    """Shading points as a camera at the 128 m world's centre sees them: horizontal distance
    log-uniform over 0.5..62 m, azimuth uniform, height uniform over 2.5..31.5 m (the volumes'
    slab, inset 0.5 m); unit normals uniform on the sphere. float32 [n, 3] each."""
    rng = np.random.default_rng(seed)
    r = np.exp(rng.uniform(np.log(0.5), np.log(62.0), n))
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    pts = np.stack([64.0 + r * np.cos(phi), rng.uniform(2.5, 31.5, n), 64.0 + r * np.sin(phi)], axis=1)
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return pts.astype(np.float32), nrm.astype(np.float32)


def cascade_query_maps(c: Cascade, seed: int = 7):
    """Per volume: irradiance maps uniform in [0.05, 1) (float32 [P, 8, 8, 4]) and history
    flags (uint8 [P], 9 in 10 set)."""
    rng = np.random.default_rng(seed)
    out = []
    for v in c.volumes:
        irr = rng.uniform(0.05, 1.0, (v.n_probes, 8, 8, 4)).astype(np.float32)
        out.append((irr, (rng.random(v.n_probes) < 0.9).astype(np.uint8)))
    return out
