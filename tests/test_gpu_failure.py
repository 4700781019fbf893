"""Failure detection on the GPU without a fault: a bounded wait that nothing
satisfies (the PCG kernels' flag-wait routine, on words no other party writes)
runs out, reports PPN_ERR_TIMEOUT to the host, and leaves the device usable."""

import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_21013_gb300")
from ppn_inputs import tiny_scene  # noqa: E402

PPN_ERR_TIMEOUT = 9


def test_wait_that_nothing_satisfies_reports_timeout_and_device_stays_usable():
    assert P.ppn.probe_bounded_wait(152, 4096, preset=True) == 0  # words already at the stamp
    t0 = time.perf_counter()
    assert P.ppn.probe_bounded_wait(152, 4096, preset=False) == PPN_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    # the context is intact: a scene steps normally afterwards
    spec = tiny_scene(cells=(2, 2, 2), seed=3)
    sc = P.Scene.from_spec(spec, precision=P.PREC_MIXED)
    rc, x, _ = sc.step(P.MODE_PPN, 1e-6)
    assert rc == 0 and np.isfinite(x).all()
