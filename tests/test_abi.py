"""The C ABI without a GPU: the library loads, exports every declared entry point,
validates arguments before touching the device, and its rotation generator agrees
with the input generator's implementation of the same published definitions."""
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sdfddgi.h")


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2007_14394_b300 as S
    return S


def test_builder_loads_without_the_package():
    # build() must not import the package (which needs the library it is about to build):
    # with the package made unimportable, the builder still loads
    code = ("import sys; sys.modules['paper_2007_14394_b300'] = None; import __graft_entry__ as g; "
            "b = g._load_builder(); print(b.LIB.endswith('libsdfddgi.so'))")
    out = subprocess.check_output([sys.executable, "-c", code], cwd=ROOT, text=True)
    assert out.strip() == "True"


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SDFDDGI_API\s+[\w\s\*]+?\b(sdfddgi_\w+)\s*\(", text)))


def test_header_declares_boundary():
    names = declared_symbols()
    for need in ("sdfddgi_create_volume", "sdfddgi_upload_sdf", "sdfddgi_set_lights", "sdfddgi_update_probes",
                 "sdfddgi_sample_irradiance"):
        assert need in names


def test_library_exports_every_declared_symbol(S):
    out = subprocess.check_output(["nm", "-D", "--defined-only", S.LIB_PATH], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    # nothing else of the library leaks out under the sdfddgi_ prefix
    assert {n for n in exported if n.startswith("sdfddgi_")} == set(declared_symbols())
    for name in S.EXPORTED:
        assert hasattr(S.lib, "sdfddgi_" + name)


@pytest.mark.parametrize("seed,frame,vol", [(0, 0, 0), (7, 3, 0), (11, 1234, 2), (2**32 - 1, 2**32 - 1, 5)])
def test_rotation_generator_agrees(S, seed, frame, vol):
    a = S.frame_rotation(seed, frame, vol)
    b = W.frame_rotation(seed, frame, vol)
    ulp = np.spacing(np.abs(b).astype(np.float32))
    assert np.all(np.abs(a - b) <= ulp)


def test_argument_errors_before_device_work(S):
    import ctypes as C
    rc = S.lib.sdfddgi_set_lights(None, None, 0, None)
    assert rc == S.ERR_INVALID_ARG and "scene" in S.last_error()
    rc = S.lib.sdfddgi_create_volume(None, None, C.byref(C.c_void_p()))
    assert rc == S.ERR_INVALID_ARG
    rc = S.lib.sdfddgi_update_probes(None, 0, None, None, 0, None, None)
    assert rc == S.ERR_INVALID_ARG
    rc = S.lib.sdfddgi_frame_rotation(0, 0, 0, None)
    assert rc == S.ERR_INVALID_ARG
    rc = S.lib.sdfddgi_sample_irradiance(None, None, None, 0, None, None)
    assert rc == S.ERR_INVALID_ARG
    with pytest.raises(S.SdfddgiError):
        S.get_maps(None)


def test_batch_argument_errors_before_device_work(S):
    import ctypes as C
    out = C.c_void_p(1)
    rc = S.lib.sdfddgi_create_batch(None, None, 1, C.byref(out))
    assert rc == S.ERR_INVALID_ARG and out.value is None
    vols = (C.c_void_p * 2)(None, None)
    for n in (0, 9):
        assert S.lib.sdfddgi_create_batch(vols, None, n, C.byref(out)) == S.ERR_INVALID_ARG
        assert "n must be" in S.last_error()
    assert S.lib.sdfddgi_create_batch(vols, None, 2, C.byref(out)) == S.ERR_INVALID_ARG
    assert "NULL" in S.last_error()
    assert S.lib.sdfddgi_update_batch(None, 0, None, None) == S.ERR_INVALID_ARG
    assert S.lib.sdfddgi_batch_autotune(None, 3, None) == S.ERR_INVALID_ARG
    assert S.lib.sdfddgi_batch_schedule(None, 0, (C.c_int32 * 5)(), None) == S.ERR_INVALID_ARG
    S.lib.sdfddgi_destroy_batch(None)


def test_l2_bandwidth_argument_errors_before_device_work(S):
    """The L2 read microbenchmark rejects a missing buffer or output, a size that is not a
    multiple of 16 bytes and a repeat count outside 1..1000 before any device call."""
    import ctypes as C
    g = C.c_float(1.0)
    assert S.lib.sdfddgi_l2_read_bandwidth(None, 1 << 20, 10, C.byref(g), None) == S.ERR_INVALID_ARG
    assert g.value == 0.0
    fake = C.c_void_p(1 << 20)  # never dereferenced: the checks come first
    assert S.lib.sdfddgi_l2_read_bandwidth(fake, 1000, 10, C.byref(g), None) == S.ERR_INVALID_ARG
    assert S.lib.sdfddgi_l2_read_bandwidth(fake, 1 << 20, 0, C.byref(g), None) == S.ERR_INVALID_ARG
    assert S.lib.sdfddgi_l2_read_bandwidth(fake, 1 << 20, 10, None, None) == S.ERR_INVALID_ARG
    assert "l2_read_bandwidth" in S.last_error()


def test_noalloc_argument_errors_before_device_work(S):
    """The allocation-free update checks everything it can see before touching the device:
    flags it does not run, probe counts past int32, non-finite rotations, output maps that
    share memory with the inputs, and updates beyond its fixed scratch. The pointers below
    are never dereferenced: each call returns at its argument check."""
    import ctypes as C
    fake = [C.c_void_p(0x100000 * (k + 1)) for k in range(8)]  # distinct, far-apart stand-in addresses
    dims = (C.c_int32 * 3)(64, 64, 64)
    org = (C.c_float * 3)(0.0, 0.0, 0.0)

    def call(desc, rotation=None, cur=None, dims_=dims):
        cur = cur or (fake[4], fake[5], fake[6])
        rot = (C.c_float * 9)(*rotation) if rotation is not None else None
        return S.lib.sdfddgi_update_probes_noalloc(C.byref(desc), fake[0], dims_, 0.125, org, S.F32, None, None, 0,
                                                   None, 0, rot, None, fake[1], fake[2], fake[3], *cur, None, None)

    ok = S.make_desc((4, 4, 4), 64, (1.0, 1.0, 1.0), (2.0, 2.0, 2.0), 64)
    bad_flags = S.make_desc((4, 4, 4), 64, (1.0, 1.0, 1.0), (2.0, 2.0, 2.0), 64, flags=S.FLAG_TEST_GATHER_STALL)
    assert call(bad_flags) == S.ERR_INVALID_ARG and "flags" in S.last_error()
    huge = S.make_desc((65536, 65536, 2), 1, (1.0, 1.0, 1.0), (2.0, 2.0, 2.0), 64)
    assert call(huge) == S.ERR_INVALID_ARG and "2^31" in S.last_error()
    many_rays = S.make_desc((512, 512, 2), 1024, (1.0, 1.0, 1.0), (2.0, 2.0, 2.0), 64)
    assert call(many_rays) == S.ERR_INVALID_ARG and "2^27" in S.last_error()
    assert call(ok, rotation=[1, 0, 0, 0, float("nan"), 0, 0, 0, 1]) == S.ERR_INVALID_ARG
    assert "rotation" in S.last_error()
    assert call(ok, cur=(fake[1], fake[5], fake[6])) == S.ERR_INVALID_ARG  # cur_irr is prev_irr
    assert "overlap" in S.last_error()
    assert call(ok, cur=(fake[4], fake[4], fake[6])) == S.ERR_INVALID_ARG  # cur_depth is cur_irr
    big = (C.c_int32 * 3)(512, 512, 512)
    assert call(ok, dims_=big) == S.ERR_INVALID_ARG and "scratch" in S.last_error()


def test_noalloc_binding_checks_buffer_sizes(S):
    """The binding checks every caller buffer against the volume description, since the C ABI
    cannot see their sizes; this needs no device (the checks come first)."""
    import torch
    desc = S.make_desc((2, 2, 2), 16, (1.0, 1.0, 1.0), (2.0, 2.0, 2.0), 32)
    sdf = torch.zeros((8, 8, 8))

    def maps(P=8):
        return (torch.zeros((P, 8, 8, 4)), torch.zeros((P, 16, 16, 2)), torch.zeros(P, dtype=torch.uint8))

    with pytest.raises(ValueError, match="cur maps"):
        S.update_probes_noalloc(desc, sdf, 0.25, (0, 0, 0), [], (0, 0, 0), maps(), maps(7))
    with pytest.raises(ValueError, match="prev maps"):
        bad = maps()
        S.update_probes_noalloc(desc, sdf, 0.25, (0, 0, 0), [], (0, 0, 0), (bad[0].double(), bad[1], bad[2]), maps())
    with pytest.raises(ValueError, match="records"):
        S.update_probes_noalloc(desc, sdf, 0.25, (0, 0, 0), [], (0, 0, 0), maps(), maps(),
                                records=torch.zeros(8 * 16 * 32 - 1, dtype=torch.uint8))
    with pytest.raises(ValueError, match="material"):
        S.update_probes_noalloc(desc, sdf, 0.25, (0, 0, 0), [], (0, 0, 0), maps(), maps(),
                                material=torch.zeros((8, 8, 8, 4), dtype=torch.float16))
    same = maps()
    with pytest.raises(ValueError, match="share memory"):
        S.update_probes_noalloc(desc, sdf, 0.25, (0, 0, 0), [], (0, 0, 0), same, same)
    with pytest.raises(ValueError, match="CUDA"):  # right sizes, host tensors
        S.update_probes_noalloc(desc, sdf, 0.25, (0, 0, 0), [], (0, 0, 0), maps(), maps())


def test_checked_build_exports_the_same_symbols(S):
    """The bounds-checked variant (built by build() beside the plain library) exports exactly the
    declared entry points, so that either loads under the same binding."""
    lib = os.path.join(ROOT, "paper_2007_14394_b300", "libsdfddgi_checked.so")
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line and "sdfddgi_" in line}
    assert exported == set(declared_symbols())


def test_irradiance_deviation_argument_errors_before_device_work(S):
    """The FP64 validation reduction rejects a missing volume, reference or output and a
    reference that is not finite and positive before any device call, and zeroes `out`."""
    import ctypes as C
    ref = (C.c_float * 3)(1.0, 1.0, 1.0)
    out = (C.c_double * 11)(*([7.0] * 11))
    assert S.lib.sdfddgi_irradiance_deviation(None, None, ref, out, None) == S.ERR_INVALID_ARG
    assert "irradiance_deviation" in S.last_error()
    fake = C.c_void_p(1 << 20)  # never dereferenced: the checks come first
    assert S.lib.sdfddgi_irradiance_deviation(fake, None, None, out, None) == S.ERR_INVALID_ARG
    assert S.lib.sdfddgi_irradiance_deviation(fake, None, ref, None, None) == S.ERR_INVALID_ARG
    for bad in ((0.0, 1.0, 1.0), (1.0, -2.0, 1.0), (1.0, 1.0, float("nan")), (float("inf"), 1.0, 1.0)):
        r = (C.c_float * 3)(*bad)
        assert S.lib.sdfddgi_irradiance_deviation(fake, None, r, out, None) == S.ERR_INVALID_ARG
        assert "ref_rgb" in S.last_error()
