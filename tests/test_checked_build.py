"""The bounds-checked build of the library (needs a B300).

libsdfddgi_checked.so is compiled with SDFDDGI_CHECKED: the update's data-dependent
accesses (SDF and material samples, the multi-bounce map lookup, per-ray arrays reached
through task payloads, the gather's ray values) check their index, and an index outside
its buffer sets a bit of the volume's failure word, reported by sdfddgi_volume_status as
SDFDDGI_ERR_BOUNDS, instead of being used. With no memory sanitizer run, the checked
library is the memory-safety evidence of the update path beside small cases and oracle
parity. The parity tests below run against it in a separate process (the
environment variable SDFDDGI_CHECKED=1 selects the library); each asserts a clean failure
word after its updates, and their maps must still meet the float32 parity bar.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_is_clean_on_parity_workloads(cuda_device):
    lib = os.path.join(ROOT, "paper_2007_14394_b300", "libsdfddgi_checked.so")
    assert os.path.exists(lib), "build it with: python paper_2007_14394_b300/build.py --checked"
    env = dict(os.environ, SDFDDGI_CHECKED="1")
    probe = subprocess.run([sys.executable, "-c", "import paper_2007_14394_b300 as S; print(S.LIB_PATH)"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert probe.stdout.strip() == lib, probe.stderr
    # room64 (full grid, then 4 multi-bounce frames), 0 and 32 lights, an odd-sized SDF, a one-step
    # budget with probes outside the box, the binary16 SDF, relocated probes, the batched form,
    # and an SDF holding NaN and infinite distances
    sel = ("test_room64_full_parity or test_room64_multiframe_multibounce or test_light_counts or "
           "test_odd_depth_unequal_sides or test_one_step_budget or test_fp16_sdf or "
           "test_update_with_relocated_probes or test_batch_equals_plain_updates or "
           "test_nonfinite_sdf_values_stay_in_bounds")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu", "-k", sel,
           "tests/test_gpu_parity.py", "tests/test_relocation.py", "tests/test_batch.py", "tests/checked_nonfinite_sdf.py"]
    run = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    tail = run.stdout[-3000:] + run.stderr[-2000:]
    assert run.returncode == 0, tail
    assert " passed" in run.stdout and "failed" not in run.stdout and "skipped" not in run.stdout, tail
