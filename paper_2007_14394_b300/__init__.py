"""Python binding of the SDFDDGI probe-update library (libsdfddgi.so, CUDA sm_103a).

Argument marshalling only: every step of the probe update runs in the library's
CUDA kernels; PyTorch supplies device memory and streams. The functions keep the
C names without the ``sdfddgi_`` prefix (see include/sdfddgi.h for the contract
of each). There is no CPU fallback: importing this package fails loudly when the
compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# SDFDDGI_CHECKED=1 in the environment loads the bounds-checked build instead (libsdfddgi_checked.so)
LIB_PATH = os.path.join(_PKG, "libsdfddgi_checked.so" if os.environ.get("SDFDDGI_CHECKED") == "1" else "libsdfddgi.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_STATE, ERR_BOUNDS = 0, -1, -2, -3, -4, -5, -6
F32, F16 = 0, 1
LIGHT_DIRECTIONAL, LIGHT_POINT = 0, 1
PROBE_ACTIVE, PROBE_REJECT_HISTORY = 1, 2
FLAG_BLEND_BF16 = 1  # volume flag: the precision form of the gather (bf16 tensor-core products)
FLAG_RELAXED_SHADOW = 2   # volume flag: over-relaxed shadow traces (RELAX_OMEGA)
FLAG_RELAXED_PRIMARY = 4  # volume flag: over-relaxed primary traces
RELAX_OMEGA = float(np.float32(1.6))  # the relaxation factor of FLAG_RELAXED_TRACE (float32 1.6)
BATCH_FORM_AUTO, BATCH_FORM_BRANCHES, BATCH_FORM_MERGED = 0, 1, 2  # sdfddgi_batch_set_form
FLAG_TEST_GATHER_STALL = 1 << 30  # volume flag for failure tests: the gather's bounded waits run out
MAX_LIGHTS, MAX_RAYS, MAX_STEPS = 32, 1024, 65535
IRR_SIDE, DEPTH_SIDE = 8, 16
EVENT_LEFT_VOLUME, EVENT_HIT, EVENT_PAST_LIMIT, EVENT_EXHAUSTED, EVENT_NO_RAY = 0, 1, 2, 3, 255


class SdfddgiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sdfddgi error {code}: {msg}")
        self.code = code


class Light(C.Structure):
    _fields_ = [("type", C.c_int32), ("v", C.c_float * 3), ("rgb", C.c_float * 3), ("range", C.c_float)]


class Relocation(C.Structure):
    _fields_ = [("clearance", C.c_float), ("reject_distance", C.c_float), ("max_offset", C.c_float),
                ("min_clearance", C.c_float), ("max_iterations", C.c_int32)]


class ProbeMaps(C.Structure):
    _fields_ = [("dims", C.c_int32 * 3), ("n_grids", C.c_int32), ("irr", C.c_void_p), ("depth", C.c_void_p),
                ("valid", C.c_void_p), ("states", C.c_void_p)]


class ProbeState(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("flags", C.c_uint32)]


class VolumeDesc(C.Structure):
    _fields_ = [("dims", C.c_int32 * 3), ("rays_per_probe", C.c_int32), ("origin", C.c_float * 3),
                ("spacing", C.c_float * 3), ("max_steps", C.c_int32), ("depth_exponent", C.c_int32),
                ("eps", C.c_float), ("t_max", C.c_float), ("hysteresis", C.c_float), ("multibounce_k", C.c_float),
                ("normal_bias", C.c_float), ("seed", C.c_uint32), ("volume_id", C.c_uint32), ("flags", C.c_uint32)]


PROBE_STATE_DTYPE = np.dtype([("pos", "f4", (3,)), ("flags", "u4")])
RAY_RECORD_DTYPE = np.dtype([("t", "f4"), ("L", "f4", (3,)), ("lit_mask", "u4"), ("shadow_steps", "u4"),
                             ("steps", "u2"), ("event", "u1"), ("reserved0", "u1"), ("material_owner", "u4")])
PRIMITIVE_DTYPE = np.dtype([("type", "i4"), ("params", "f4", (7,)), ("albedo", "f4", (3,)),
                            ("emission", "f4", (3,)), ("pad", "f4", (2,))])
PRIM_SPHERE, PRIM_BOX, PRIM_CAPSULE, PRIM_PLANE_Y, PRIM_INV_SPHERE = 0, 1, 2, 3, 4
assert RAY_RECORD_DTYPE.itemsize == 32 and PROBE_STATE_DTYPE.itemsize == 16 and PRIMITIVE_DTYPE.itemsize == 64


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2007_14394_b300/build.py` "
                          "(the CUDA library is required; there is no fallback)")
    lib = C.CDLL(LIB_PATH)
    vp, i32, u32, i64 = C.c_void_p, C.c_int32, C.c_uint32, C.c_int64
    sig = {
        "sdfddgi_last_error": ([], C.c_char_p),
        "sdfddgi_create_scene": ([C.POINTER(vp)], C.c_int),
        "sdfddgi_destroy_scene": ([vp], None),
        "sdfddgi_upload_sdf": ([vp, vp, C.POINTER(i32), C.c_float, C.POINTER(C.c_float), i32, vp, i32, vp], C.c_int),
        "sdfddgi_set_lights": ([vp, C.POINTER(Light), i32, C.POINTER(C.c_float)], C.c_int),
        "sdfddgi_create_volume": ([C.POINTER(VolumeDesc), vp, C.POINTER(vp)], C.c_int),
        "sdfddgi_destroy_volume": ([vp], None),
        "sdfddgi_volume_probe_count": ([vp, C.POINTER(i64)], C.c_int),
        "sdfddgi_frame_rotation": ([u32, u32, u32, C.POINTER(C.c_float)], C.c_int),
        "sdfddgi_update_probes": ([vp, u32, vp, vp, i32, vp, vp], C.c_int),
        "sdfddgi_sample_irradiance": ([vp, vp, vp, i64, vp, vp], C.c_int),
        "sdfddgi_get_maps": ([vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)], C.c_int),
        "sdfddgi_read_state": ([vp, vp, vp, vp, i32, vp], C.c_int),
        "sdfddgi_write_state": ([vp, vp, vp, vp, i32, vp], C.c_int),
        "sdfddgi_reset": ([vp, vp], C.c_int),
        "sdfddgi_set_stage_events": ([vp, C.POINTER(vp), i32], C.c_int),
        "sdfddgi_set_slabs": ([vp, i32], C.c_int),
        "sdfddgi_read_state_async": ([vp, vp, vp, vp, vp, vp], C.c_int),
        "sdfddgi_volume_slabs": ([vp, C.POINTER(i32)], C.c_int),
        "sdfddgi_update_probes_noalloc": ([C.POINTER(VolumeDesc), vp, C.POINTER(i32), C.c_float, C.POINTER(C.c_float),
                                           i32, vp, C.POINTER(Light), i32, C.POINTER(C.c_float), u32, vp, vp,
                                           vp, vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "sdfddgi_volume_status": ([vp, C.POINTER(u32)], C.c_int),
        "sdfddgi_upload_primitives": ([vp, vp, i32, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_float, i32],
                                      C.c_int),
        "sdfddgi_relocate_probes": ([vp, C.POINTER(Relocation), vp, vp, vp], C.c_int),
        "sdfddgi_sample_irradiance_visible": ([vp, vp, vp, i64, C.c_float, vp, vp, vp], C.c_int),
        "sdfddgi_sample_irradiance_cascade": ([vp, C.c_int32, vp, vp, i64, C.c_float, vp, vp, vp, vp, vp], C.c_int),
        "sdfddgi_denoiser_status": ([vp, C.POINTER(u32)], C.c_int),
        "sdfddgi_create_denoiser": ([C.POINTER(C.c_float), C.c_float, C.POINTER(vp)], C.c_int),
        "sdfddgi_destroy_denoiser": ([vp], None),
        "sdfddgi_denoiser_params": ([vp, vp, vp], C.c_int),
        "sdfddgi_denoise": ([vp, C.POINTER(ProbeMaps), vp, i32, vp], C.c_int),
        "sdfddgi_denoise_volume": ([vp, vp, vp, i32, vp], C.c_int),
        "sdfddgi_denoiser_gradients": ([vp, C.POINTER(ProbeMaps), vp, i32, vp, vp, vp], C.c_int),
        "sdfddgi_denoiser_adam": ([vp, vp, C.c_float, vp], C.c_int),
        "sdfddgi_denoiser_train_step": ([vp, C.POINTER(ProbeMaps), vp, i32, C.c_float, vp, vp], C.c_int),
        "sdfddgi_create_batch": ([C.POINTER(vp), C.POINTER(vp), i32, C.POINTER(vp)], C.c_int),
        "sdfddgi_destroy_batch": ([vp], None),
        "sdfddgi_update_batch": ([vp, u32, vp, vp], C.c_int),
        "sdfddgi_batch_autotune": ([vp, i32, vp], C.c_int),
        "sdfddgi_batch_schedule": ([vp, i32, C.POINTER(i32), C.POINTER(C.c_float)], C.c_int),
        "sdfddgi_batch_set_form": ([vp, i32], C.c_int),
        "sdfddgi_batch_form": ([vp, C.POINTER(i32), C.POINTER(C.c_float)], C.c_int),
        "sdfddgi_l2_read_bandwidth": ([vp, C.c_size_t, i32, C.POINTER(C.c_float), vp], C.c_int),
        "sdfddgi_irradiance_deviation": ([vp, vp, C.POINTER(C.c_float), C.POINTER(C.c_double), vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()
EXPORTED = ("last_error", "create_scene", "destroy_scene", "upload_sdf", "set_lights", "create_volume",
            "destroy_volume", "volume_probe_count", "frame_rotation", "update_probes", "update_probes_noalloc",
            "sample_irradiance", "set_stage_events", "get_maps", "read_state", "write_state", "reset",
            "create_batch", "destroy_batch", "update_batch", "batch_autotune", "batch_schedule",
            "batch_set_form", "batch_form",
            "create_denoiser", "destroy_denoiser", "denoiser_params", "denoise", "denoise_volume",
            "denoiser_gradients", "denoiser_adam", "denoiser_train_step", "volume_status", "denoiser_status",
            "relocate_probes", "sample_irradiance_visible", "upload_primitives", "sample_irradiance_cascade",
            "set_slabs", "volume_slabs", "read_state_async", "irradiance_deviation")
MAX_SLABS = 4
DENOISER_PARAMS = 49219
DENOISE_TENSOR, DENOISE_SIMT_BF16, DENOISE_SIMT_FP32 = 0, 1, 2
STAGES = ("weights", "primary", "prep", "shadow", "gather")  # intervals between the stage events


def set_stage_events(volume, events) -> None:
    """events: [] to stop, or 6 torch.cuda.Event(enable_timing=True) recorded once already."""
    n = len(events)
    arr = (C.c_void_p * max(n, 1))(*[e.cuda_event for e in events])
    _check(lib.sdfddgi_set_stage_events(volume, arr, n))


def set_slabs(volume, slabs: int) -> None:
    """Slab branches per update of `volume`: 0 automatic, 1 serial, up to MAX_SLABS."""
    _check(lib.sdfddgi_set_slabs(volume, int(slabs)))


def read_state_async(volume, irr, depth, valid, stream=None, done_event=None) -> None:
    """Copies the current maps into irr/depth/valid (torch tensors, page-locked host or device
    memory, or None) on the volume's copy stream, after the work enqueued on `stream`; records
    `done_event` (a torch.cuda.Event, or None) after the copies. Returns at once."""
    ptr = lambda t: None if t is None else t.data_ptr()
    ev = None
    if done_event is not None:
        if not done_event.cuda_event:  # torch creates the CUDA event at its first record
            done_event.record()
        ev = done_event.cuda_event
    _check(lib.sdfddgi_read_state_async(volume, ptr(irr), ptr(depth), ptr(valid), _stream(stream), ev))


def volume_slabs(volume) -> int:
    """The number of slabs the next update of `volume` runs as."""
    n = C.c_int32()
    _check(lib.sdfddgi_volume_slabs(volume, C.byref(n)))
    return n.value


def last_error() -> str:
    return lib.sdfddgi_last_error().decode()


def _check(rc: int) -> None:
    if rc != OK:
        raise SdfddgiError(rc, last_error())


# ------------------------------------------------------------------ marshalling helpers
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(address, on_device) of a torch tensor or numpy array (contiguous)."""
    if x is None:
        return None, 0
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), int(x.is_cuda)
    a = np.asarray(x)
    if not a.flags.c_contiguous:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data, 0


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _floats(v, n):
    return (C.c_float * n)(*[float(x) for x in v])


# ------------------------------------------------------------------ C entry points
def create_scene() -> C.c_void_p:
    h = C.c_void_p()
    _check(lib.sdfddgi_create_scene(C.byref(h)))
    return h


def destroy_scene(scene) -> None:
    lib.sdfddgi_destroy_scene(scene)


def upload_sdf(scene, sdf, voxel_size: float, origin, material=None, stream=None) -> None:
    """sdf: [nz,ny,nx] float32/float16 (torch or numpy); material: [nz,ny,nx,8] float16 or None."""
    shape = tuple(sdf.shape)
    if len(shape) != 3:
        raise ValueError("sdf must be 3-D [nz, ny, nx]")
    name = str(sdf.dtype)
    dtype = F32 if name.endswith("float32") else F16 if name.endswith("float16") else None
    if dtype is None:
        raise ValueError(f"sdf dtype {sdf.dtype} is neither float32 nor float16")
    p, dev = _ptr(sdf)
    m, mdev = _ptr(material)
    if material is not None:
        if tuple(material.shape) != shape + (8,) or not str(material.dtype).endswith("float16"):
            raise ValueError("material must be float16 [nz, ny, nx, 8]")
        if mdev != dev:
            raise ValueError("sdf and material must both be host or both be device arrays")
    dims = (C.c_int32 * 3)(shape[2], shape[1], shape[0])
    _check(lib.sdfddgi_upload_sdf(scene, p, dims, float(voxel_size), _floats(origin, 3), dtype, m, dev,
                                  _stream(stream)))


def set_lights(scene, lights, sky=(0.0, 0.0, 0.0)) -> None:
    """lights: sequence of dicts {type: 'dir'|'point', v, rgb, range}."""
    n = len(lights)
    arr = (Light * max(n, 1))()
    for i, l in enumerate(lights):
        arr[i].type = LIGHT_DIRECTIONAL if l["type"] in ("dir", LIGHT_DIRECTIONAL) else LIGHT_POINT
        arr[i].v = _floats(l["v"], 3)
        arr[i].rgb = _floats(l["rgb"], 3)
        arr[i].range = float(l.get("range", 0.0))
    _check(lib.sdfddgi_set_lights(scene, arr, n, _floats(sky, 3)))


def make_desc(dims, rays_per_probe, origin, spacing, max_steps, depth_exponent=50, eps=0.01, t_max=0.0,
              hysteresis=0.97, multibounce_k=0.9, normal_bias=1.0, seed=0, volume_id=0, flags=0) -> VolumeDesc:
    return VolumeDesc((C.c_int32 * 3)(*[int(x) for x in dims]), int(rays_per_probe), _floats(origin, 3),
                      _floats(spacing, 3), int(max_steps), int(depth_exponent), float(eps), float(t_max),
                      float(hysteresis), float(multibounce_k), float(normal_bias), int(seed), int(volume_id),
                      int(flags))


def create_volume(desc: VolumeDesc, scene) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib.sdfddgi_create_volume(C.byref(desc), scene, C.byref(h)))
    return h


def destroy_volume(volume) -> None:
    lib.sdfddgi_destroy_volume(volume)


def volume_probe_count(volume) -> int:
    n = C.c_int64()
    _check(lib.sdfddgi_volume_probe_count(volume, C.byref(n)))
    return n.value


def frame_rotation(seed: int, frame: int, volume_id: int = 0) -> np.ndarray:
    out = (C.c_float * 9)()
    _check(lib.sdfddgi_frame_rotation(int(seed), int(frame), int(volume_id), out))
    return np.array(out[:], dtype=np.float32).reshape(3, 3)


def update_probes(volume, frame: int, rotation=None, states=None, records=None, stream=None) -> None:
    """rotation: None or (3,3) float32 host array; states: None, numpy PROBE_STATE_DTYPE [P] (host) or a
    device tensor of P*16 bytes; records: None or a device tensor of P*R*32 bytes."""
    rot = None
    if rotation is not None:
        rot = np.ascontiguousarray(np.asarray(rotation, dtype=np.float32).reshape(9))
    sp, sdev = _ptr(states)
    rp, rdev = _ptr(records)
    if records is not None and not rdev:
        raise ValueError("records must be a device tensor")
    _check(lib.sdfddgi_update_probes(volume, int(frame), rot.ctypes.data if rot is not None else None, sp, sdev,
                                     rp, _stream(stream)))


def sample_irradiance(volume, points, normals, out, stream=None) -> None:
    """points, normals, out: device float32 tensors [n, 3]."""
    n = int(points.shape[0]) if points is not None else 0
    for t in (points, normals, out):
        if t is not None and (not _is_torch(t) or not t.is_cuda or str(t.dtype) != "torch.float32"):
            raise ValueError("points/normals/out must be CUDA float32 tensors")
    _check(lib.sdfddgi_sample_irradiance(volume, _ptr(points)[0], _ptr(normals)[0], n, _ptr(out)[0],
                                         _stream(stream)))


def get_maps(volume):
    """Raw device addresses (irr, depth, valid) of the current maps."""
    a, b, c = C.c_void_p(), C.c_void_p(), C.c_void_p()
    _check(lib.sdfddgi_get_maps(volume, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def read_state(volume, irr, depth, valid, stream=None) -> None:
    """Copies the current maps into irr [P,8,8,4] f32, depth [P,16,16,2] f32, valid [P] u8 (host or device)."""
    (ip, idev), (dp, ddev), (vp_, vdev) = _ptr(irr), _ptr(depth), _ptr(valid)
    if not (idev == ddev == vdev):
        raise ValueError("read_state: all three arrays must be host or all device")
    _check(lib.sdfddgi_read_state(volume, ip, dp, vp_, idev, _stream(stream)))


def write_state(volume, irr, depth, valid, stream=None) -> None:
    (ip, idev), (dp, ddev), (vp_, vdev) = _ptr(irr), _ptr(depth), _ptr(valid)
    if not (idev == ddev == vdev):
        raise ValueError("write_state: all three arrays must be host or all device")
    _check(lib.sdfddgi_write_state(volume, ip, dp, vp_, idev, _stream(stream)))


def reset(volume, stream=None) -> None:
    _check(lib.sdfddgi_reset(volume, _stream(stream)))


def update_probes_noalloc(desc: VolumeDesc, sdf, voxel_size: float, origin, lights, sky, prev, cur, frame: int = 0,
                          rotation=None, material=None, states=None, records=None, stream=None) -> None:
    """The update for callers that cannot allocate device memory (see include/sdfddgi.h): every
    buffer is the caller's. sdf [nz,ny,nx] float32/float16 and material [nz,ny,nx,8] float16 are
    device tensors; prev and cur are (irr [P,8,8,4] f32, depth [P,16,16,2] f32, valid [P] u8)
    device tensors; states None or a device tensor of P*16 bytes; records None or P*R*32 bytes."""
    shape = tuple(sdf.shape)
    name = str(sdf.dtype)
    dtype = F32 if name.endswith("float32") else F16 if name.endswith("float16") else None
    if dtype is None or len(shape) != 3:
        raise ValueError("sdf must be a 3-D float32 or float16 device tensor")
    # the library cannot see buffer sizes: check every one against desc before the call
    P = int(desc.dims[0]) * int(desc.dims[1]) * int(desc.dims[2])
    R = int(desc.rays_per_probe)
    if len(prev) != 3 or len(cur) != 3:
        raise ValueError("prev and cur are (irr, depth, valid)")
    for label, (irr, dep, val) in (("prev", prev), ("cur", cur)):
        for t, n, kind in ((irr, P * IRR_SIDE * IRR_SIDE * 4, "float32"), (dep, P * DEPTH_SIDE * DEPTH_SIDE * 2, "float32"),
                           (val, P, "uint8")):
            if t is None or not _is_torch(t) or not str(t.dtype).endswith(kind) or t.numel() != n:
                raise ValueError(f"update_probes_noalloc: {label} maps must be {kind} tensors of "
                                 f"{P}x(8*8*4, 16*16*2, 1) elements for {P} probes")
    if material is not None and (tuple(material.shape) != (*shape, 8) or not str(material.dtype).endswith("float16")):
        raise ValueError(f"update_probes_noalloc: material must be float16 of shape {(*shape, 8)}")
    for t, n, label in ((states, P * 16, "states"), (records, P * R * 32, "records")):
        if t is not None and (not _is_torch(t) or t.numel() * t.element_size() != n):
            raise ValueError(f"update_probes_noalloc: {label} must hold {n} bytes")
    spans = [(t.data_ptr(), t.numel() * t.element_size()) for t in (*cur, *prev)]
    for i in range(3):
        for j in range(i + 1, 6):
            (a, na), (b, nb) = spans[i], spans[j]
            if a < b + nb and b < a + na:
                raise ValueError("update_probes_noalloc: the cur maps share memory with prev or with each other")
    for t in (sdf, material, states, records, *prev, *cur):
        if t is not None and not (_is_torch(t) and t.is_cuda):
            raise ValueError("update_probes_noalloc: every buffer must be a CUDA tensor")
    n = len(lights)
    arr = (Light * max(n, 1))()
    for i, l in enumerate(lights):
        arr[i].type = LIGHT_DIRECTIONAL if l["type"] in ("dir", LIGHT_DIRECTIONAL) else LIGHT_POINT
        arr[i].v = _floats(l["v"], 3)
        arr[i].rgb = _floats(l["rgb"], 3)
        arr[i].range = float(l.get("range", 0.0))
    rot = None
    if rotation is not None:
        rot = np.ascontiguousarray(np.asarray(rotation, dtype=np.float32).reshape(9))
    dims = (C.c_int32 * 3)(shape[2], shape[1], shape[0])
    _check(lib.sdfddgi_update_probes_noalloc(
        C.byref(desc), _ptr(sdf)[0], dims, float(voxel_size), _floats(origin, 3), dtype, _ptr(material)[0], arr, n,
        _floats(sky, 3), int(frame), rot.ctypes.data if rot is not None else None, _ptr(states)[0],
        _ptr(prev[0])[0], _ptr(prev[1])[0], _ptr(prev[2])[0], _ptr(cur[0])[0], _ptr(cur[1])[0], _ptr(cur[2])[0],
        _ptr(records)[0], _stream(stream)))


def create_batch(volumes, states=None) -> C.c_void_p:
    """volumes: handles of one scene; states: None or one entry per volume, None or a device tensor of
    P_i * 16 bytes (read at every update_batch)."""
    n = len(volumes)
    vols = (C.c_void_p * n)(*[v.value if isinstance(v, C.c_void_p) else v for v in volumes])
    sts = None
    if states is not None:
        if len(states) != n:
            raise ValueError("one states entry per volume")
        ptrs = []
        for s in states:
            p, dev = _ptr(s)
            if s is not None and not dev:
                raise ValueError("batch states must be device tensors")
            ptrs.append(p)
        sts = (C.c_void_p * n)(*ptrs)
    h = C.c_void_p()
    _check(lib.sdfddgi_create_batch(vols, sts, n, C.byref(h)))
    h._states = tuple(states) if states is not None else ()  # read at every update_batch: kept alive
    return h


def destroy_batch(batch) -> None:
    lib.sdfddgi_destroy_batch(batch)


def update_batch(batch, frame: int, rotations=None, stream=None) -> None:
    """rotations: None (each volume's frame_rotation of `frame`) or float32 [n][3][3] host array."""
    rot = None
    if rotations is not None:
        rot = np.ascontiguousarray(np.asarray(rotations, dtype=np.float32).reshape(-1))
    _check(lib.sdfddgi_update_batch(batch, int(frame), rot.ctypes.data if rot is not None else None,
                                    _stream(stream)))


def batch_autotune(batch, repeats: int = 3, stream=None) -> None:
    _check(lib.sdfddgi_batch_autotune(batch, int(repeats), _stream(stream)))


def batch_schedule(batch, i: int):
    """(pool_batch, blocks_per_sm, gather, index, steps, tuned_ms) of volume i."""
    out = (C.c_int32 * 5)()
    ms = C.c_float()
    _check(lib.sdfddgi_batch_schedule(batch, int(i), out, C.byref(ms)))
    return out[0], out[1], out[2], out[3], out[4], ms.value


def batch_set_form(batch, form: int) -> None:
    """BATCH_FORM_AUTO (the autotuner's choice), BATCH_FORM_BRANCHES or BATCH_FORM_MERGED."""
    _check(lib.sdfddgi_batch_set_form(batch, int(form)))


def batch_form(batch):
    """(form of the next frame, autotuned ms per frame of the branches form, of the merged form)."""
    f = C.c_int32()
    ms = (C.c_float * 2)()
    _check(lib.sdfddgi_batch_form(batch, C.byref(f), ms))
    return f.value, ms[0], ms[1]


# ------------------------------------------------------------------ the learned form
def _dev_ptr(t, what):
    if t is None:
        return None
    p, dev = _ptr(t)
    if not dev:
        raise ValueError(f"{what} must be a device tensor")
    return p


def probe_maps(dims, n_grids, irr, depth, valid, states=None) -> ProbeMaps:
    """Device tensors irr [P,8,8,4] f32, depth [P,16,16,2] f32, valid [P] u8, states None or P*16 bytes.
    The view holds the tensors' device addresses and keeps the tensors alive while it lives."""
    m = ProbeMaps((C.c_int32 * 3)(*[int(x) for x in dims]), int(n_grids), _dev_ptr(irr, "irr"),
                  _dev_ptr(depth, "depth"), _dev_ptr(valid, "valid"), _dev_ptr(states, "states"))
    m._tensors = (irr, depth, valid, states)  # the addresses stay valid as long as the view
    return m


def create_denoiser(params, depth_scale: float) -> C.c_void_p:
    a = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
    if a.size != DENOISER_PARAMS:
        raise ValueError(f"expected {DENOISER_PARAMS} parameters")
    h = C.c_void_p()
    _check(lib.sdfddgi_create_denoiser(a.ctypes.data_as(C.POINTER(C.c_float)), float(depth_scale), C.byref(h)))
    return h


def destroy_denoiser(d) -> None:
    lib.sdfddgi_destroy_denoiser(d)


def denoiser_params(d, write=None) -> np.ndarray:
    """Returns the current parameters (float32); with `write`, sets them first (resets Adam)."""
    if write is not None:
        w = np.ascontiguousarray(np.asarray(write, dtype=np.float32).reshape(-1))
        if w.size != DENOISER_PARAMS:
            raise ValueError(f"expected {DENOISER_PARAMS} parameters")
        _check(lib.sdfddgi_denoiser_params(d, None, w.ctypes.data))
    out = np.empty(DENOISER_PARAMS, np.float32)
    _check(lib.sdfddgi_denoiser_params(d, out.ctypes.data, None))
    return out


def denoise(d, maps: ProbeMaps, out, mode=DENOISE_TENSOR, stream=None) -> None:
    _check(lib.sdfddgi_denoise(d, C.byref(maps), _dev_ptr(out, "out"), int(mode), _stream(stream)))


def denoise_volume(d, volume, states=None, mode=DENOISE_TENSOR, stream=None) -> None:
    _check(lib.sdfddgi_denoise_volume(d, volume, _dev_ptr(states, "states"), int(mode), _stream(stream)))


def denoiser_gradients(d, maps: ProbeMaps, target, grad, loss, mode=DENOISE_SIMT_BF16, stream=None) -> None:
    _check(lib.sdfddgi_denoiser_gradients(d, C.byref(maps), _dev_ptr(target, "target"), int(mode),
                                          _dev_ptr(grad, "grad"), _dev_ptr(loss, "loss"), _stream(stream)))


def denoiser_adam(d, grad, lr: float, stream=None) -> None:
    _check(lib.sdfddgi_denoiser_adam(d, _dev_ptr(grad, "grad"), float(lr), _stream(stream)))


def denoiser_train_step(d, maps: ProbeMaps, target, lr: float, loss=None, mode=DENOISE_SIMT_BF16,
                        stream=None) -> None:
    _check(lib.sdfddgi_denoiser_train_step(d, C.byref(maps), _dev_ptr(target, "target"), int(mode), float(lr),
                                           _dev_ptr(loss, "loss"), _stream(stream)))


def volume_status(volume) -> int:
    """Failure bits recorded by the volume's updates since the last call (cleared);
    raises SdfddgiError: SDFDDGI_ERR_TIMEOUT if a tensor-core wait gave up, SDFDDGI_ERR_BOUNDS if
    the bounds-checked build met an index outside its buffer."""
    f = C.c_uint32()
    _check(lib.sdfddgi_volume_status(volume, C.byref(f)))
    return f.value


def irradiance_deviation(volume, ref_rgb, states=None, stream=None) -> dict:
    """FP64 deviation of the current irradiance maps' interior texels from `ref_rgb` (the
    furnace or closed-room value): states None (every probe) or a device tensor of P*16 bytes
    (active probes only). Returns count, mean[3], max_rel[3], rms_rel[3], nonfinite."""
    ref = (C.c_float * 3)(*[float(x) for x in ref_rgb])
    out = (C.c_double * 11)()
    _check(lib.sdfddgi_irradiance_deviation(volume, _dev_ptr(states, "states"), ref, out, _stream(stream)))
    o = list(out)
    return {"count": int(o[0]), "mean": o[1:4], "max_rel": o[4:7], "rms_rel": o[7:10], "nonfinite": int(o[10])}


def l2_read_bandwidth(buf, reps: int = 20, stream=None) -> float:
    """GB/s read from the device tensor `buf` (kept in L2: e.g. 32 MiB) by 16-byte loads that
    bypass L1, over `reps` sweeps after one untimed sweep. Synchronises the stream."""
    g = C.c_float()
    nbytes = int(buf.numel() * buf.element_size())
    _check(lib.sdfddgi_l2_read_bandwidth(_dev_ptr(buf, "buf"), nbytes, int(reps), C.byref(g), _stream(stream)))
    return float(g.value)


def denoiser_status(d) -> int:
    f = C.c_uint32()
    _check(lib.sdfddgi_denoiser_status(d, C.byref(f)))
    return f.value


def relocate_probes(volume, out, clearance=2.0, reject_distance=0.0, max_offset=0.45, min_clearance=0.5,
                    max_iterations=16, last=None, stream=None) -> None:
    """Probe relocation (Sec. 3.2) into `out` (device tensor of P*16 bytes); `last`: None or
    the last frame's states (device, may be `out`)."""
    r = Relocation(float(clearance), float(reject_distance), float(max_offset), float(min_clearance),
                   int(max_iterations))
    _check(lib.sdfddgi_relocate_probes(volume, C.byref(r), _dev_ptr(last, "last"), _dev_ptr(out, "out"),
                                       _stream(stream)))


def sample_irradiance_visible(volume, points, normals, out, softness=8.0, states=None, stream=None) -> None:
    """Interpolation with SDF probe visibility (Sec. 3.4); points, normals, out: device float [n, 3]."""
    n = int(points.numel() // 3) if _is_torch(points) else int(np.asarray(points).size // 3)
    _check(lib.sdfddgi_sample_irradiance_visible(volume, _dev_ptr(points, "points"), _dev_ptr(normals, "normals"), n,
                                                 float(softness), _dev_ptr(states, "states"), _dev_ptr(out, "out"),
                                                 _stream(stream)))


def sample_irradiance_cascade(volumes, points, normals, out, level=None, weight=None, softness=0.0, states=None,
                              stream=None) -> None:
    """Irradiance from a cascade of volumes (Sec. 3.5), finest first; points, normals, out: device
    float [n, 3]; level (int32 [n]) and weight (float [n]): None or device tensors. softness > 0
    weights the probes of every level but the farthest by their visibility (Sec. 3.4); states:
    None or one entry per volume, each None or that volume's device probe states."""
    vols = list(volumes)
    arr = (C.c_void_p * max(len(vols), 1))(*vols)
    st = None
    if states is not None:
        st = (C.c_void_p * max(len(vols), 1))(*[_dev_ptr(x, "states") for x in states])
    n = int(points.numel() // 3) if _is_torch(points) else int(np.asarray(points).size // 3)
    _check(lib.sdfddgi_sample_irradiance_cascade(arr, len(vols), _dev_ptr(points, "points"),
                                                 _dev_ptr(normals, "normals"), n, float(softness), st,
                                                 _dev_ptr(out, "out"), _dev_ptr(level, "level"),
                                                 _dev_ptr(weight, "weight"), _stream(stream)))


def upload_primitives(scene, types, params, albedo, emission, lo, hi, unit: float, cluster_size: int = 8) -> None:
    """The scene as a union of analytic primitives (Sec. 3.1): types [n], params [n, >=7 or fewer]
    (float32), albedo / emission [n, 3]; the box lo..hi bounds every trace, `unit` is the length
    of one voxel for the voxel-unit parameters; cluster_size 0 disables the cluster culling."""
    n = len(types)
    arr = np.zeros(n, dtype=PRIMITIVE_DTYPE)
    arr["type"] = np.asarray(types, dtype=np.int32)
    par = np.asarray(params, dtype=np.float32).reshape(n, -1)
    arr["params"][:, :min(7, par.shape[1])] = par[:, :7]
    arr["albedo"] = np.asarray(albedo, dtype=np.float32).reshape(n, 3)
    arr["emission"] = np.asarray(emission, dtype=np.float32).reshape(n, 3)
    _check(lib.sdfddgi_upload_primitives(scene, arr.ctypes.data, n, _floats(lo, 3), _floats(hi, 3), float(unit),
                                         int(cluster_size)))
