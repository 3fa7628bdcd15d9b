"""FP64 CPU oracle of the SDFDDGI per-frame probe update (ctypes wrapper).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the CUDA library never
does, and the two share no code. The arithmetic lives in ``oracle.c`` (plain C,
double precision, Sec. 3.3 and Eq. 3 of Hu et al., arXiv 2007.14394); this file
only builds it, marshals numpy arrays and converts records.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

IRR_N, DEP_N = 6, 14
IRR_T, DEP_T = IRR_N + 2, DEP_N + 2
LEFT_VOLUME, HIT, PAST_LIMIT, EXHAUSTED = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (double precision, no FMA contraction, OpenMP)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Volume(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("sdf_dtype", C.c_int32),
                ("h", C.c_double), ("origin", C.c_double * 3),
                ("sdf", C.c_void_p), ("material", C.c_void_p), ("prims", C.c_void_p),
                ("n_prims", C.c_int32), ("pad", C.c_int32)]


PRIM_DTYPE = np.dtype([("type", "i4"), ("pad", "i4"), ("p", "f8", (7,)), ("albedo", "f8", (3,)),
                       ("emission", "f8", (3,))])


class Light(C.Structure):
    _fields_ = [("type", C.c_int32), ("pad", C.c_int32), ("v", C.c_double * 3),
                ("rgb", C.c_double * 3), ("range", C.c_double)]


class Grid(C.Structure):
    _fields_ = [("dims", C.c_int32 * 3), ("rays", C.c_int32),
                ("origin", C.c_double * 3), ("spacing", C.c_double * 3),
                ("max_steps", C.c_int32), ("depth_exponent", C.c_int32),
                ("eps_vox", C.c_double), ("tmax_vox", C.c_double), ("hysteresis", C.c_double),
                ("k_bounce", C.c_double), ("bias_vox", C.c_double), ("sky", C.c_double * 3),
                ("omega_primary", C.c_double), ("omega_shadow", C.c_double)]


RAY_DTYPE = np.dtype([("t", "f8"), ("L", "f8", (3,)), ("margin_primary", "f8"),
                      ("margin_shadow", "f8"), ("margin_decision", "f8"), ("event", "i4"),
                      ("steps", "i4"), ("natural_event", "i4"), ("natural_steps", "i4"),
                      ("lit_mask", "u4"), ("natural_lit_mask", "u4"), ("traced_mask", "u4"),
                      ("shadow_steps", "i4"), ("forced", "i4"), ("hard", "i4"),
                      ("t_cond", "f8"), ("dLdt", "f8", (3,)),
                      ("dLdcos", "f8", (3,)), ("owner", "i4"), ("natural_owner", "i4"), ("margin_owner", "f8")])
FORCE_DTYPE = np.dtype([("event", "i4"), ("steps", "i4"), ("lit_mask", "u4"), ("owner", "i4")])


def is_miss(event):
    """A ray is a miss when it left the volume or passed the trace limit."""
    event = np.asarray(event)
    return (event == LEFT_VOLUME) | (event == PAST_LIMIT)


PROBE_DTYPE = np.dtype([("pos", "f4", (3,)), ("flags", "u4")])


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            lib.oracle_sf_dir.argtypes = [C.c_int32, C.c_int32, dp]
            lib.oracle_oct_encode.argtypes = [dp, dp]
            lib.oracle_oct_decode.argtypes = [dp, dp]
            lib.oracle_sample_sdf.argtypes = [C.POINTER(Volume), dp]
            lib.oracle_sample_sdf.restype = C.c_double
            lib.oracle_trace.argtypes = [C.POINTER(Volume), dp, dp, C.c_double, C.c_double, C.c_int32,
                                         dp, C.POINTER(C.c_int32), dp]
            lib.oracle_trace.restype = C.c_int32
            lib.oracle_trace_relaxed.argtypes = [C.POINTER(Volume), dp, dp, C.c_double, C.c_double, C.c_int32,
                                                 C.c_double, dp, C.POINTER(C.c_int32), dp]
            lib.oracle_trace_relaxed.restype = C.c_int32
            lib.oracle_border.argtypes = [dp, C.c_int32, C.c_int32]
            lib.oracle_sample_irradiance.argtypes = [C.POINTER(Grid), dp, C.c_void_p, dp, dp, dp]
            lib.oracle_shade.argtypes = [C.POINTER(Volume), C.POINTER(Grid), C.POINTER(Light), C.c_int32,
                                         dp, C.c_void_p, dp, dp, C.c_void_p, C.c_void_p]
            lib.oracle_set_delta.argtypes = [C.c_double, C.c_double]
            lib.oracle_update.argtypes = [C.POINTER(Volume), C.POINTER(Grid), C.POINTER(Light), C.c_int32,
                                          C.POINTER(C.c_float), C.c_void_p, dp, dp, C.c_void_p,
                                          dp, dp, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                          C.c_int32]
            lib.oracle_update.restype = C.c_int32
            lib.oracle_sample_irradiance_visible.argtypes = [C.POINTER(Volume), C.POINTER(Grid), dp, C.c_void_p,
                                                             C.c_void_p, C.c_double, dp, dp, dp, dp, dp]
            lib.oracle_analytic_sdf.argtypes = [C.POINTER(Volume), dp, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
            lib.oracle_analytic_sdf.restype = C.c_double
            lib.oracle_mvc.argtypes = [dp, C.c_int32, C.c_void_p, C.c_int32, dp, dp]
            lib.oracle_mvc.restype = C.c_int32
            lib.oracle_cascade_weight.argtypes = [C.POINTER(Grid), dp]
            lib.oracle_cascade_weight.restype = C.c_double
            lib.oracle_sample_irradiance_cascade.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, dp, dp,
                                                             dp, C.POINTER(C.c_double), C.POINTER(C.c_int32)]
            lib.oracle_sample_irradiance_cascade_visible.argtypes = [
                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_double, dp, dp, dp,
                C.POINTER(C.c_double), C.POINTER(C.c_int32), dp]
            lib.oracle_relocate.argtypes = [C.POINTER(Volume), C.POINTER(Grid), C.POINTER(Relocation), C.c_void_p,
                                            dp, C.c_void_p, C.c_void_p, C.c_void_p]
            lib.oracle_record_sizes.argtypes = [C.c_int32]
            lib.oracle_record_sizes.restype = C.c_int32
            assert lib.oracle_record_sizes(0) == RAY_DTYPE.itemsize, "or_ray layout differs from RAY_DTYPE"
            assert lib.oracle_record_sizes(1) == FORCE_DTYPE.itemsize, "or_force layout differs from FORCE_DTYPE"
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vec(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3))


# ----------------------------------------------------------------- scene marshalling
class OracleScene:
    """Keeps the numpy arrays alive that an ``or_volume`` points into."""

    def __init__(self, sdf: np.ndarray, h: float, origin, material: np.ndarray | None = None):
        if sdf.dtype == np.float32:
            dtype_code = 0
        elif sdf.dtype == np.float16:
            dtype_code = 1
        else:
            raise TypeError("sdf must be float32 or float16")
        self.sdf = np.ascontiguousarray(sdf)
        nz, ny, nx = self.sdf.shape
        self.material = None
        if material is not None:
            m = np.ascontiguousarray(material)
            if m.dtype != np.float16 or m.shape != (nz, ny, nx, 8):
                raise ValueError("material must be float16 [nz][ny][nx][8]")
            self.material = m
        self.vol = Volume(nx, ny, nz, dtype_code, float(h), (C.c_double * 3)(*[float(x) for x in origin]),
                          self.sdf.ctypes.data, self.material.ctypes.data if self.material is not None else None,
                          None, 0, 0)

    @classmethod
    def analytic(cls, types, params, albedo, emission, origin, dims, h: float) -> "OracleScene":
        """The union of analytic primitives (float32 parameters promoted exactly); the box
        origin + [0, dims * h] bounds the traces and h is the unit of voxel parameters."""
        self = cls.__new__(cls)
        n = len(types)
        prims = np.zeros(n, dtype=PRIM_DTYPE)
        prims["type"] = np.asarray(types, dtype=np.int32)
        prims["p"] = np.asarray(params, dtype=np.float32).reshape(n, -1)[:, :7].astype(np.float64)
        prims["albedo"] = np.asarray(albedo, dtype=np.float32).astype(np.float64)
        prims["emission"] = np.asarray(emission, dtype=np.float32).astype(np.float64)
        self.prims = prims
        self.sdf = np.zeros(1, np.float32)
        self.material = None
        nx, ny, nz = (int(d) for d in dims)
        self.vol = Volume(nx, ny, nz, 0, float(h), (C.c_double * 3)(*[float(x) for x in origin]),
                          self.sdf.ctypes.data, None, prims.ctypes.data, n, 0)
        return self


def make_lights(lights) -> tuple:
    """lights: list of dicts {type: 'dir'|'point', v, rgb, range}."""
    n = len(lights)
    arr = (Light * max(n, 1))()
    for i, l in enumerate(lights):
        arr[i].type = 0 if l["type"] == "dir" else 1
        arr[i].v = (C.c_double * 3)(*[float(x) for x in l["v"]])
        arr[i].rgb = (C.c_double * 3)(*[float(x) for x in l["rgb"]])
        arr[i].range = float(l.get("range", 0.0))
    return arr, n


def make_grid(dims, origin, spacing, rays, max_steps, eps_vox, tmax_vox, hysteresis,
              depth_exponent=50, k_bounce=1.0, bias_vox=1.0, sky=(0.0, 0.0, 0.0), omega_primary=1.0,
              omega_shadow=1.0) -> Grid:
    return Grid((C.c_int32 * 3)(*[int(x) for x in dims]), int(rays),
                (C.c_double * 3)(*[float(x) for x in origin]), (C.c_double * 3)(*[float(x) for x in spacing]),
                int(max_steps), int(depth_exponent), float(eps_vox), float(tmax_vox), float(hysteresis),
                float(k_bounce), float(bias_vox), (C.c_double * 3)(*[float(x) for x in sky]), float(omega_primary),
                float(omega_shadow))


# ----------------------------------------------------------------- elementary functions
def sf_dir(i: int, n: int) -> np.ndarray:
    out = np.zeros(3)
    _load().oracle_sf_dir(int(i), int(n), _dp(out))
    return out


def oct_encode(v) -> np.ndarray:
    out = np.zeros(2)
    _load().oracle_oct_encode(_dp(_vec(v)), _dp(out))
    return out


def oct_decode(uv) -> np.ndarray:
    out = np.zeros(3)
    _load().oracle_oct_decode(_dp(np.ascontiguousarray(np.asarray(uv, dtype=np.float64).reshape(2))), _dp(out))
    return out


def sample_sdf(scene: OracleScene, p) -> float:
    return float(_load().oracle_sample_sdf(C.byref(scene.vol), _dp(_vec(p))))


def set_delta(delta_vox: float = 2e-4, delta_cos: float = 1e-4) -> None:
    """Widths of the rounding-sensitive band used when following another side's decisions."""
    _load().oracle_set_delta(float(delta_vox), float(delta_cos))


def trace(scene: OracleScene, o, d, eps_vox: float, tlimit: float, max_steps: int, omega: float = 1.0):
    """Returns (event, t, steps, margin_vox); omega > 1: the over-relaxed trace."""
    t = C.c_double()
    m = C.c_double()
    s = C.c_int32()
    if omega > 1.0:
        cls = _load().oracle_trace_relaxed(C.byref(scene.vol), _dp(_vec(o)), _dp(_vec(d)), float(eps_vox),
                                           float(tlimit), int(max_steps), float(omega), C.byref(t), C.byref(s),
                                           C.byref(m))
    else:
        cls = _load().oracle_trace(C.byref(scene.vol), _dp(_vec(o)), _dp(_vec(d)), float(eps_vox),
                                   float(tlimit), int(max_steps), C.byref(t), C.byref(s), C.byref(m))
    return int(cls), t.value, s.value, m.value


def border(map_: np.ndarray) -> np.ndarray:
    """Border fixup of a copy of an (n+2, n+2, C) map."""
    m = np.ascontiguousarray(map_, dtype=np.float64).copy()
    T, T2, Cn = m.shape
    assert T == T2
    _load().oracle_border(_dp(m), T - 2, Cn)
    return m


def sample_irradiance(grid: Grid, irr: np.ndarray, valid: np.ndarray, x, nrm) -> np.ndarray:
    irr = np.ascontiguousarray(irr, dtype=np.float64)
    valid = np.ascontiguousarray(valid, dtype=np.uint8)
    out = np.zeros(3)
    _load().oracle_sample_irradiance(C.byref(grid), _dp(irr), valid.ctypes.data, _dp(_vec(x)),
                                     _dp(_vec(nrm)), _dp(out))
    return out


def shade(scene: OracleScene, grid: Grid, lights, prev_irr: np.ndarray, prev_valid: np.ndarray, x, d):
    """Radiance leaving hit point x along -d; returns the ray record (numpy void)."""
    larr, n = make_lights(lights)
    prev_irr = np.ascontiguousarray(prev_irr, dtype=np.float64)
    prev_valid = np.ascontiguousarray(prev_valid, dtype=np.uint8)
    rec = np.zeros(1, dtype=RAY_DTYPE)
    rec["margin_shadow"] = 1e300
    rec["margin_decision"] = 1e300
    _load().oracle_shade(C.byref(scene.vol), C.byref(grid), larr, n, _dp(prev_irr), prev_valid.ctypes.data,
                         _dp(_vec(x)), _dp(_vec(d)), None, rec.ctypes.data)
    return rec[0]


# ----------------------------------------------------------------- the update
def empty_maps(n_probes: int):
    """Zero previous maps (no history): irr [P,8,8,4], depth [P,16,16,2], valid [P]."""
    return (np.zeros((n_probes, IRR_T, IRR_T, 4)), np.zeros((n_probes, DEP_T, DEP_T, 2)),
            np.zeros(n_probes, dtype=np.uint8))


def update(scene: OracleScene, grid: Grid, lights, rot: np.ndarray, probes: np.ndarray,
           prev=None, subset=None, want_rays: bool = True, n_threads: int = 0, force=None):
    """One probe update. Returns dict(irr, depth, valid, rays).

    rot: float32 (3,3) frame rotation; probes: PROBE_DTYPE [P]; prev: (irr, depth, valid)
    or None for no history; subset: probe indices to update (others keep prev).
    force: None or FORCE_DTYPE [len(subset), R] decisions to follow inside the rounding band.
    rays: RAY_DTYPE [len(subset), R] when want_rays.
    """
    P = int(np.prod(list(grid.dims)))
    probes = np.ascontiguousarray(probes)
    assert probes.dtype == PROBE_DTYPE and probes.shape == (P,)
    if prev is None:
        prev = empty_maps(P)
    pi, pd, pv = (np.ascontiguousarray(prev[0], dtype=np.float64), np.ascontiguousarray(prev[1], dtype=np.float64),
                  np.ascontiguousarray(prev[2], dtype=np.uint8))
    assert pi.shape == (P, IRR_T, IRR_T, 4) and pd.shape == (P, DEP_T, DEP_T, 2) and pv.shape == (P,)
    ci, cd, cv = pi.copy(), pd.copy(), pv.copy()
    rot32 = np.ascontiguousarray(np.asarray(rot, dtype=np.float32).reshape(9))
    if subset is None:
        sub_arr, n_sub = None, P
    else:
        sub_arr = np.ascontiguousarray(np.asarray(subset, dtype=np.int32))
        n_sub = len(sub_arr)
    rays = np.zeros((n_sub, grid.rays), dtype=RAY_DTYPE) if want_rays else None
    if force is not None:
        force = np.ascontiguousarray(force)
        assert force.dtype == FORCE_DTYPE and force.shape == (n_sub, grid.rays)
    larr, nl = make_lights(lights)
    rc = _load().oracle_update(C.byref(scene.vol), C.byref(grid), larr, nl,
                               rot32.ctypes.data_as(C.POINTER(C.c_float)), probes.ctypes.data,
                               _dp(pi), _dp(pd), pv.ctypes.data, _dp(ci), _dp(cd), cv.ctypes.data,
                               sub_arr.ctypes.data if sub_arr is not None else None, n_sub,
                               force.ctypes.data if force is not None else None,
                               rays.ctypes.data if rays is not None else None, int(n_threads))
    if rc != 0:
        raise ValueError("oracle_update: invalid arguments")
    return {"irr": ci, "depth": cd, "valid": cv, "rays": rays}


# ----------------------------------------------------------------- probe relocation
class Relocation(C.Structure):
    _fields_ = [("clearance_vox", C.c_double), ("reject_dist", C.c_double), ("max_offset", C.c_double),
                ("min_clearance_vox", C.c_double), ("max_iters", C.c_int32), ("pad", C.c_int32)]


def relocate(scene: "OracleScene", grid: Grid, clearance_vox: float, reject_dist: float, max_offset: float = 0.45,
             min_clearance_vox: float = 0.5, max_iters: int = 16, last_pos=None) -> dict:
    """Probe relocation (Sec. 3.2); returns pos [P,3], flags [P], iters [P], margin [P,2]."""
    P = int(np.prod(list(grid.dims)))
    rp = Relocation(float(clearance_vox), float(reject_dist), float(max_offset), float(min_clearance_vox),
                    int(max_iters), 0)
    last = None if last_pos is None else np.ascontiguousarray(np.asarray(last_pos, dtype=np.float32).reshape(P, 3))
    pos = np.zeros((P, 3))
    flags = np.zeros(P, np.uint32)
    iters = np.zeros(P, np.int32)
    margin = np.zeros((P, 2))
    _load().oracle_relocate(C.byref(scene.vol), C.byref(grid), C.byref(rp),
                            last.ctypes.data if last is not None else None, _dp(pos), flags.ctypes.data,
                            iters.ctypes.data, _dp(margin))
    return {"pos": pos, "flags": flags, "iters": iters, "margin": margin}


def sample_irradiance_visible(scene: "OracleScene", grid: Grid, irr: np.ndarray, valid: np.ndarray, x, nrm,
                              softness: float, probe_pos=None):
    """Interpolation with SDF probe visibility (Sec. 3.4); returns (rgb, vis[8], margins[8, 2])."""
    irr = np.ascontiguousarray(irr, dtype=np.float64)
    valid = np.ascontiguousarray(valid, dtype=np.uint8)
    pp = None if probe_pos is None else np.ascontiguousarray(np.asarray(probe_pos, dtype=np.float32))
    out, vis, marg = np.zeros(3), np.zeros(8), np.zeros(16)
    _load().oracle_sample_irradiance_visible(C.byref(scene.vol), C.byref(grid), _dp(irr), valid.ctypes.data,
                                             pp.ctypes.data if pp is not None else None, float(softness),
                                             _dp(_vec(x)), _dp(_vec(nrm)), _dp(out), _dp(vis), _dp(marg))
    return out, vis, marg.reshape(8, 2)


def analytic_sdf(scene: "OracleScene", p):
    """(distance, owner index, second-smallest distance) of an analytic scene at p."""
    own = C.c_int32()
    sec = C.c_double()
    d = _load().oracle_analytic_sdf(C.byref(scene.vol), _dp(_vec(p)), C.byref(own), C.byref(sec))
    return d, own.value, sec.value


# ----------------------------------------------------------------- cascade blending
def mvc(verts, tris, x):
    """Mean value coordinates of x over a closed triangle mesh; returns (lambda, on_mesh)."""
    v = np.ascontiguousarray(np.asarray(verts, dtype=np.float64).reshape(-1, 3))
    t = np.ascontiguousarray(np.asarray(tris, dtype=np.int32).reshape(-1, 3))
    lam = np.zeros(len(v))
    on = _load().oracle_mvc(_dp(v), len(v), t.ctypes.data, len(t), _dp(_vec(x)), _dp(lam))
    return lam, bool(on)


def cascade_weight(grid: Grid, x) -> float:
    return _load().oracle_cascade_weight(C.byref(grid), _dp(_vec(x)))


def sample_irradiance_cascade(grids, irrs, valids, x, nrm):
    """Cascade interpolation (Sec. 3.5) over grids[0] (finest) .. grids[-1]; returns (rgb, w, level)."""
    n = len(grids)
    irrs = [np.ascontiguousarray(a, dtype=np.float64) for a in irrs]
    valids = [np.ascontiguousarray(a, dtype=np.uint8) for a in valids]
    gp = (C.c_void_p * n)(*[C.cast(C.pointer(g), C.c_void_p) for g in grids])
    ip = (C.c_void_p * n)(*[a.ctypes.data for a in irrs])
    vp = (C.c_void_p * n)(*[a.ctypes.data for a in valids])
    out = np.zeros(3)
    w = C.c_double()
    lvl = C.c_int32()
    _load().oracle_sample_irradiance_cascade(gp, ip, vp, n, _dp(_vec(x)), _dp(_vec(nrm)), _dp(out), C.byref(w),
                                             C.byref(lvl))
    return out, w.value, lvl.value


def sample_irradiance_cascade_visible(scenes, grids, irrs, valids, x, nrm, softness, probe_pos=None):
    """Cascade interpolation with probe visibility in every level but the farthest (Sec. 3.4,
    3.5); scenes: one OracleScene per level; probe_pos: None or per level None / float32 [P, 3].
    Returns (rgb, w, level, margins [2, 8, 2]) (levels k and k + 1)."""
    n = len(grids)
    irrs = [np.ascontiguousarray(a, dtype=np.float64) for a in irrs]
    valids = [np.ascontiguousarray(a, dtype=np.uint8) for a in valids]
    pps = [None if probe_pos is None or probe_pos[i] is None
           else np.ascontiguousarray(np.asarray(probe_pos[i], dtype=np.float32)) for i in range(n)]
    sp = (C.c_void_p * n)(*[C.cast(C.pointer(sc.vol), C.c_void_p) for sc in scenes])
    gp = (C.c_void_p * n)(*[C.cast(C.pointer(g), C.c_void_p) for g in grids])
    ip = (C.c_void_p * n)(*[a.ctypes.data for a in irrs])
    vp = (C.c_void_p * n)(*[a.ctypes.data for a in valids])
    pp = (C.c_void_p * n)(*[None if a is None else a.ctypes.data for a in pps])
    out, marg = np.zeros(3), np.zeros(32)
    w = C.c_double()
    lvl = C.c_int32()
    _load().oracle_sample_irradiance_cascade_visible(sp, gp, ip, vp, pp, n, float(softness), _dp(_vec(x)),
                                                     _dp(_vec(nrm)), _dp(out), C.byref(w), C.byref(lvl), _dp(marg))
    return out, w.value, lvl.value, marg.reshape(2, 8, 2)
