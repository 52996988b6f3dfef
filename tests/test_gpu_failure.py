"""Failure detection on the GPU without a fault: the library's bounded waits
run on conditions that never come (an mbarrier nobody arrives on, a grid
barrier whose target is never reached, a work-queue counter that stays
short), give up after their poll limit and report through the status word
(the queue wait also raises the abort word that stops a fused launch); the
context stays usable afterwards."""
import time

import numpy as np
import pytest

from paper_2206_01683_b300 import fishlbm, inputs

pytestmark = pytest.mark.gpu


def test_bounded_waits_give_up_and_report():
    t0 = time.time()
    mbar, grid, status, queue = fishlbm.selftest_waits(limit=4096)
    assert mbar and grid and status and queue
    assert time.time() - t0 < 60
    # the device is still usable: a domain steps and matches a fresh one
    X, dV = inputs.fibonacci_sphere(100, 3.0, (8.0, 8.0, 8.0))
    out = []
    for _ in range(2):
        d = fishlbm.Domain([fishlbm.env_desc((16, 16, 16), 0.7)], deterministic=True)
        d.set_markers(np.float32(X), np.tile(np.float32([0.01, 0, 0]), (100, 1)), np.float32(dV))
        d.step(5)
        out.append(d.get_body_force_torque())
    assert np.array_equal(out[0], out[1]) and np.all(np.isfinite(out[0]))


def test_selftest_rejects_a_zero_limit():
    with pytest.raises(fishlbm.FgError) as ei:
        fishlbm.selftest_waits(limit=0)
    assert ei.value.status == fishlbm.FG_ERR_INVALID
