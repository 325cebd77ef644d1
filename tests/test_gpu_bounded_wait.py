"""The bounded wait of the resident sweep kernel, run on the GPU.

The resident kernel's CTAs wait for their neighbour planes' counters with a
routine that gives up after a limit (the kernel then reports QSLBM_ETIMEOUT)
instead of spinning for ever.  qslbm_check_bounded_wait runs that routine on a
counter that nothing sets: it must give up after about its limit and leave the
context usable; on a counter that is already set it must return at once.
"""
import ctypes as C

import pytest

from paper_2211_09370_gb300 import _lib
from paper_2211_09370_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _wait(limit_s, counter_set):
    L = _lib.load()
    gave_up, waited = C.c_int32(-1), C.c_double(-1.0)
    rc = L.qslbm_check_bounded_wait(limit_s, counter_set, C.byref(gave_up), C.byref(waited))
    assert rc == _lib.OK, L.qslbm_last_error()
    return gave_up.value, waited.value


def test_wait_on_unset_counter_gives_up_after_its_limit():
    gave_up, waited = _wait(0.05, 0)
    assert gave_up == 1
    assert 0.05 <= waited < 1.0
    # the context still works: a small solve runs after the timed-out wait
    with _lib.Solver(W.small_pipe(nx=12, ny=12, nz=4, diameter=8.0, n_mag=4)) as s:
        s.step(2)
        assert s.observables()["nan_flag"] == 0


def test_wait_on_set_counter_returns_at_once():
    gave_up, waited = _wait(0.5, 1)
    assert gave_up == 0
    assert waited < 0.01
