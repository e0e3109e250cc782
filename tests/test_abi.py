"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/evsim.h declares.  Runs without a GPU: only argument validation and
error paths are exercised (no kernel is launched)."""
import ctypes
import os
import re

import pytest

from paper_2209_04634_gb300 import build, evsim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(sim\w*)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return evsim.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["sim_create", "sim_push_frame", "sim_pop_events", "sim_destroy",
                     "sim_strerror"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_binding_covers_every_declared_function():
    bound = {n for n, _, _ in evsim.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_library_is_built_for_sm_103a(lib):
    # the build recipe targets sm_103a only
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.LIB)


def test_strerror_and_version(lib):
    assert lib.sim_strerror(0) == b"ok"
    assert b"overflow" in lib.sim_strerror(evsim.SIM_ERR_EVENT_OVERFLOW)
    assert lib.sim_strerror(12345) == b"unknown error"
    assert lib.sim_version().count(b".") == 2


def _cfg(lib, w=64, h=48):
    c = evsim.sim_config()
    assert lib.sim_config_default(ctypes.byref(c), w, h) == 0
    return c


@pytest.mark.parametrize("field,value", [
    ("width", 0), ("height", -3), ("width", 9000), ("pixel_format", 2), ("mode", 7),
    ("intensity", 5), ("ref_mode", 3), ("substeps", 65), ("substeps", -1),
    ("c_pos_q16", 0), ("c_neg_q16", 11), ("c_pos_q16", 1 << 30), ("event_capacity", -5),
    ("event_time", 2), ("event_time", -1),
])
def test_create_rejects_bad_config_before_touching_the_device(lib, field, value):
    c = _cfg(lib)
    setattr(c, field, value)
    h = ctypes.c_void_p()
    assert lib.sim_create(ctypes.byref(c), ctypes.byref(h)) == evsim.SIM_ERR_ARG
    assert not h.value


def test_crossing_times_need_a_reference(lib):
    """Per-crossing event times are defined for the dense and sparse methods
    only (the difference-frame method has no reference to cross)."""
    c = _cfg(lib)
    c.mode = evsim.SIM_DIFF
    c.event_time = evsim.SIM_TIME_CROSSING
    h = ctypes.c_void_p()
    assert lib.sim_create(ctypes.byref(c), ctypes.byref(h)) == evsim.SIM_ERR_ARG
    assert not h.value


def test_linear_accumulate_threshold_floor(lib):
    c = _cfg(lib)
    c.intensity = evsim.SIM_LINEAR
    c.c_pos_q16 = c.c_neg_q16 = 510  # below (255 * 65536) / 32766
    h = ctypes.c_void_p()
    assert lib.sim_create(ctypes.byref(c), ctypes.byref(h)) == evsim.SIM_ERR_ARG


def test_null_arguments(lib):
    assert lib.sim_create(None, None) == evsim.SIM_ERR_ARG
    assert lib.sim_push_frame(None, None, 0, None, 0, 0) == evsim.SIM_ERR_ARG
    n = ctypes.c_int64(0)
    assert lib.sim_pop_events(None, None, 0, ctypes.byref(n), 0) == evsim.SIM_ERR_ARG
    assert lib.sim_destroy(None) == evsim.SIM_ERR_ARG
    assert lib.sim_sync(None) == evsim.SIM_ERR_ARG


def test_create_without_a_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    c = _cfg(lib)
    h = ctypes.c_void_p()
    assert lib.sim_create(ctypes.byref(c), ctypes.byref(h)) == evsim.SIM_ERR_NO_DEVICE


def test_autotune_arguments_and_table_file(lib, tmp_path):
    """Argument errors of the autotuner and its table file round trip (no
    kernel runs)."""
    cfg, _ = evsim.make_config(64, 32)
    assert lib.sim_autotune(ctypes.byref(cfg), 1, None, None) == evsim.SIM_ERR_ARG
    assert lib.sim_autotune(ctypes.byref(cfg), 65, None, None) == evsim.SIM_ERR_ARG
    assert lib.sim_autotune(None, 8, None, None) == evsim.SIM_ERR_ARG
    cfg.tile_height = 5
    h = ctypes.c_void_p()
    assert lib.sim_create(ctypes.byref(cfg), ctypes.byref(h)) == evsim.SIM_ERR_ARG
    src = tmp_path / "tune.txt"
    src.write_text("64 32 1 0 8 0 0 0 0 8 0 10.000 9.000 11.000\n"
                   "640 480 1 1 0 8 0 0 1 16 1 900.000 950.000 0.000\n"
                   "1280 720 3 1 10 0 0 0 0 1 0 900.000 950.000 400.000\n")
    assert lib.sim_autotune_load(str(src).encode()) == evsim.SIM_OK
    out = tmp_path / "out.txt"
    assert lib.sim_autotune_save(str(out).encode()) == evsim.SIM_OK
    text = out.read_text()
    assert "64 32 1 0 8 0 0 0 0 8 0 10.000 9.000 11.000" in text
    assert "640 480 1 1 0 8 0 0 1 16 1 900.000 950.000 0.000" in text
    assert "1280 720 3 1 10 0 0 0 0 1 0 900.000 950.000 400.000" in text
    bad = tmp_path / "bad.txt"
    bad.write_text("64 32 1 0 8 0 0 0 0 12 0 1 1 1\n")  # tile height must be 1, 8 or 16
    assert lib.sim_autotune_load(str(bad).encode()) == evsim.SIM_ERR_ARG
    assert lib.sim_autotune_load(str(tmp_path / "missing.txt").encode()) == evsim.SIM_ERR_ARG
    assert lib.sim_autotune_load(None) == evsim.SIM_ERR_ARG


def test_checkpoint_argument_errors(lib):
    n = ctypes.c_int64(0)
    assert lib.sim_state_size(None, ctypes.byref(n)) == evsim.SIM_ERR_ARG
    assert lib.sim_get_state(None, None, 0) == evsim.SIM_ERR_ARG
    assert lib.sim_set_state(None, None, 0) == evsim.SIM_ERR_ARG


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "evsim.h"

int main(void) {
  sim_config c;
  sim_t* s = NULL;
  if (sim_config_default(&c, 64, 48) != SIM_OK) return 1;
  if (c.mode != SIM_DENSE || c.event_time != SIM_TIME_SUBSTEP) return 2;
  c.event_time = 7;                                   /* rejected before any device work */
  if (sim_create(&c, &s) != SIM_ERR_ARG || s != NULL) return 3;
  c.event_time = SIM_TIME_CROSSING;
  c.mode = SIM_DIFF;
  if (sim_create(&c, &s) != SIM_ERR_ARG) return 4;
  if (sim_destroy(NULL) != SIM_ERR_ARG) return 5;
  if (strcmp(sim_strerror(SIM_OK), "ok") != 0) return 6;
  if (sizeof(sim_event) != 8) return 7;
  printf("%s\n", sim_version());
  return 0;
}
"""


def test_header_is_plain_c_and_links_from_c(lib, tmp_path):
    """include/evsim.h compiles as strict C99 (no C++ in the public header) and
    a C program links against the library and calls it through the ABI."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(build.LIB)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                        "-L", libdir, "-levsim", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.strip().count(".") == 2


def test_threshold_conversion_matches_the_oracles(lib):
    # the library's float -> Q16 threshold conversion and the oracle's own
    # (computed independently) agree, ties included
    import oracle
    vals = [0.0, 0.15, 0.2, 0.03, 2.0, 10.0, 20.0, -0.2, -2.0, 1.0 / 65536, 1e-7]
    vals += [(k + 0.5) / 65536 for k in range(0, 40)]  # exact ties: round half even
    vals += [(k + 0.5) / 65536 for k in range(13100, 13120)]
    for c in vals:
        assert evsim.q16(c) == oracle.q16(c), c
    assert lib.sim_threshold_q16(float("nan")) == evsim.SIM_ERR_ARG
    assert lib.sim_threshold_q16(float("inf")) == evsim.SIM_ERR_ARG
    assert lib.sim_threshold_q16(16384.0) == evsim.SIM_ERR_ARG  # 2^30 in Q16
    assert lib.sim_threshold_q16(16383.99) > 0
