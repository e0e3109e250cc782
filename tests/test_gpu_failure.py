"""Failure detection on the device without a GPU fault: the library's bounded
waits (the order kernel's look-back on a predecessor chunk, a group tile's
wait for its earlier frames) give up after their poll limit when the awaited
word is never published, the kernel returns, the host reads
SIM_ERR_DEVICE_TIMEOUT from the stream's error word, and the context stays
usable (a simulation afterwards still equals the oracle)."""
import ctypes

import numpy as np
import pytest

from paper_2209_04634_gb300 import evsim, synth

from .helpers import assert_same_events, gpu_run, oracle_run


def _wait(which, publish, limit):
    st = ctypes.c_int32(123)
    rc = evsim.load().sim_selftest_bounded_wait(which, publish, limit, ctypes.byref(st))
    return rc, st.value


def test_bounded_wait_rejects_bad_arguments_without_a_device():
    lib = evsim.load()
    st = ctypes.c_int32(0)
    for args in ((2, 0, 10), (0, 2, 10), (0, 0, 0), (1, 0, (1 << 22) + 1)):
        assert lib.sim_selftest_bounded_wait(*args, ctypes.byref(st)) == evsim.SIM_ERR_ARG
    assert lib.sim_selftest_bounded_wait(0, 0, 10, None) == evsim.SIM_ERR_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("which", [0, 1])
def test_unpublished_wait_times_out_and_the_context_survives(which):
    rc, st = _wait(which, 0, 2000)
    assert rc == evsim.SIM_OK and st == evsim.SIM_ERR_DEVICE_TIMEOUT
    rc, st = _wait(which, 1, 2000)
    assert rc == evsim.SIM_OK and st == evsim.SIM_OK
    seq = synth.blob_translation(frames=4, width=96, height=64)
    g = gpu_run(seq, evsim.SIM_DENSE)
    assert_same_events(g["events"], oracle_run(seq, evsim.SIM_DENSE)["events"], "after a timeout")
    assert np.array_equal(g["R"], oracle_run(seq, evsim.SIM_DENSE)["R"])
