"""Serving loop (continuous batching over resident scenes) through the C ABI.

Each scene's results in the mix must equal its results alone: every kernel
treats scenes independently and every reduction is per scene in a fixed
order, so the expected difference is zero; the assertion allows the stated
tolerance (FP64: relative 1e-12, mixed: relative 1e-6 of the displacement).
"""

import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_21013_gb300")
from ppn_inputs import cube_scene, tiny_scene, twisting_beam_scene  # noqa: E402

TOL = {P.PREC_FP64: 1e-12, P.PREC_MIXED: 1e-6}


def scene_set():
    return [
        (cube_scene(4, E=1e5, dt=1 / 60, seed=0), P.MODE_PPN),
        (twisting_beam_scene(4, 4, 10, h=0.02, E=1e5, nu=0.45, omega=40.0, dt=0.1, seed=1), P.MODE_PPN),
        (twisting_beam_scene(5, 5, 14, h=0.02, E=1e6, nu=0.45, omega=8.0, dt=1 / 30, seed=2), P.MODE_PN),
        (cube_scene(5, E=1e5, nu=0.4, dt=1 / 60, seed=3), P.MODE_PDN),
        (tiny_scene(cells=(2, 2, 1), seed=4), P.MODE_NEWTON),
        (twisting_beam_scene(4, 4, 12, h=0.02, E=1e5, nu=0.45, omega=30.0, dt=0.05, seed=5), P.MODE_PDN),
    ]


def alone(spec, mode, steps, prec, tol):
    sc = P.Scene.from_spec(spec, precision=prec)
    out = []
    for n in range(steps):
        sc.set_targets(spec.targets_at(n))
        rc, x, _ = sc.step(mode, tol)
        assert rc == 0
        out.append(x)
    sc.close()
    return out


@pytest.mark.parametrize("prec", [P.PREC_FP64, P.PREC_MIXED])
def test_results_in_the_mix_equal_results_alone(prec):
    steps = 3
    tol = 1e-6 if prec == P.PREC_FP64 else 1e-4  # FP32 steps stall below ~1e-5 relative
    scenes = scene_set()
    ref = [alone(spec, mode, steps, prec, tol) for spec, mode in scenes]
    srv = P.Server(precision=prec, max_batch=4)  # fewer slots than scenes: requests queue
    ids = [srv.add_scene(spec) for spec, _ in scenes]
    tickets = []
    # the first step of every scene now, the rest while those are running
    for (spec, mode), sid in zip(scenes, ids):
        tickets.append((sid, 0, srv.submit(sid, mode, tol, spec.targets_at(0))))
    time.sleep(0.01)
    for n in range(1, steps):
        for (spec, mode), sid in zip(scenes, ids):
            tickets.append((sid, n, srv.submit(sid, mode, tol, spec.targets_at(n))))
    times = []
    for sid, n, t in tickets:
        done, rc, x, st, tm = srv.poll(t, sid)
        assert done and rc == 0
        k = ids.index(sid)
        spec = scenes[k][0]
        disp = np.abs(ref[k][n] - spec.rest).max()
        assert np.abs(x - ref[k][n]).max() <= TOL[prec] * disp
        times.append(tm)
    # continuous batching: several scenes shared the batch, and requests that
    # arrived while others ran were admitted before those finished
    assert max(tm["batch_max"] for tm in times) >= 2
    assert any(a["t_start_ms"] < b["t_done_ms"] and a["t_submit_ms"] > b["t_start_ms"]
               for a in times for b in times)
    s = srv.stats()
    assert s["completed"] == len(tickets) and s["p99_ms"] >= s["p50_ms"] > 0 and s["steps_per_s"] > 0
    srv.close()


def test_admission_by_hbm_footprint():
    spec = cube_scene(5, seed=7)
    probe = P.Scene.from_spec(spec, precision=P.PREC_MIXED)
    nbytes = probe.info()["device_bytes"]
    probe.close()
    total = torch.cuda.get_device_properties(0).total_memory
    srv = P.Server(hbm_fraction=1.5 * nbytes / total, precision=P.PREC_MIXED)
    a = srv.add_scene(spec)
    with pytest.raises(P.PPNError) as e:
        srv.add_scene(spec)  # a second copy exceeds the cap
    assert e.value.status == P.ppn.PPN_ERR_ADMISSION
    assert srv.stats()["rejected_scenes"] == 1
    # requests keep running on the admitted scene; removing it frees the budget
    t = srv.submit(a, P.MODE_PPN, 1e-5, spec.targets_at(0))
    done, rc, _, _, _ = srv.poll(t, a)
    assert done and rc == 0
    srv.remove_scene(a)
    b = srv.add_scene(spec)
    assert srv.stats()["resident_scenes"] == 1 and b != a
    srv.close()
