"""Stopping a run without faulting the GPU: a wall-clock deadline checked on the
device at every flatness check, and an abort request raised from another host
thread.  Either way the run returns a status, the walker state stays
consistent, and resuming gives exactly the trajectory of an uninterrupted run.
"""
import threading
import time

import numpy as np
import pytest

import paper_1302_2320_gb300 as wl

pytestmark = pytest.mark.gpu

ALLOW = (wl.WL_OK, wl.WL_ENOTCONVERGED, wl.WL_ETIMEOUT, wl.WL_EABORTED)


def _same(a, b, ells):
    for ell in ells:
        ga, gb = a.line_state(ell), b.line_state(ell)
        for key in ga:
            assert np.array_equal(ga[key], gb[key]), (ell, key)


def test_deadline_stops_run_and_resume_is_exact():
    budget = 3_000_000
    ref = wl.Handle("square", 32, seed=11, check_interval=1000, move_budget=budget, mapping=8)
    assert ref.run(1e-6, 0.8) == wl.WL_ENOTCONVERGED
    h = wl.Handle("square", 32, seed=11, check_interval=1000, move_budget=budget, mapping=8,
                  timeout_ms=30)
    assert h.run(1e-6, 0.8, allow=ALLOW) == wl.WL_ETIMEOUT
    assert h.stats()["moves"] < ref.stats()["moves"]
    h.set_option("timeout_ms", 0)
    assert h.run(1e-6, 0.8, allow=ALLOW) == wl.WL_ENOTCONVERGED
    _same(h, ref, [1, 100, 256, 512])
    assert h.stats()["moves"] == ref.stats()["moves"]


def test_abort_from_another_thread_and_resume_is_exact():
    budget = 4_000_000
    ref = wl.Handle("square", 32, seed=12, check_interval=1000, move_budget=budget, mapping=8)
    ref.run(1e-6, 0.8)
    h = wl.Handle("square", 32, seed=12, check_interval=1000, move_budget=budget, mapping=8)
    h.set_option("move_budget", 1)
    h.run(1e-6, 0.8)                       # allocates and initialises
    h.set_option("move_budget", budget)
    timer = threading.Timer(0.05, h.abort)
    timer.start()
    t0 = time.time()
    rc = h.run(1e-6, 0.8, allow=ALLOW)     # ctypes releases the GIL during the call
    timer.join()
    assert rc == wl.WL_EABORTED, (rc, time.time() - t0)
    assert h.run(1e-6, 0.8, allow=ALLOW) == wl.WL_ENOTCONVERGED
    _same(h, ref, [1, 100, 256, 512])
