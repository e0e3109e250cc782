"""The bounds-checked debug build of the library (build(debug=True): every
global write of the simulation kernels, the order kernel's segment and
staging reads and the shared-memory halo writes are checked; a violation is
recorded as SIM_ERR_BOUNDS in the stream's error word and skipped) runs
parity cases on small and ragged shapes, both tile shapes, the row kernel,
sparse, reset and linear modes, per-crossing times and the group without a
violation and with the oracle's events - in a child process that loads the
debug library through EVSIM_LIBRARY."""
import os
import subprocess
import sys

import pytest

from paper_2209_04634_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = ["test_gpu_parity.py::test_ragged_shapes",
         "test_gpu_parity.py::test_mode_matrix",
         "test_gpu_parity.py::test_rows_of_multi_crossings",
         "test_gpu_parity.py::test_large_flow_beyond_the_shared_halo",
         "test_gpu_rows.py::test_ragged_shapes",
         "test_gpu_rows.py::test_quiet_moving_and_mixed_rows",
         "test_gpu_crossing_time.py",
         "test_group.py::test_group_members_in_either_tile_shape_match_the_oracle"]


def test_debug_build_compiles_the_checks_in():
    src = open(os.path.join(ROOT, "paper_2209_04634_gb300", "csrc", "internal.h")).read()
    assert "EVSIM_BOUNDS_CHECK" in src
    assert "-DEVSIM_BOUNDS_CHECK" not in " ".join(build.FLAGS)  # release builds: no checks


@pytest.mark.gpu
def test_parity_cases_pass_on_the_bounds_checked_build():
    lib = build.build(debug=True)
    env = dict(os.environ, EVSIM_LIBRARY=lib)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"]
    cmd += [os.path.join(ROOT, "tests", c) for c in CASES]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
