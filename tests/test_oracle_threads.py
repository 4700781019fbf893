"""The oracle's parallel loops (independent elements and SpMV rows) give the same
results at any thread count: a PPN step of a violent beam is bitwise equal with one
thread and with several."""

import numpy as np

from oracle import oracle as O
from ppn_inputs import twisting_beam_scene


def test_oracle_results_do_not_depend_on_threads():
    spec = twisting_beam_scene(4, 4, 10, h=0.02, E=1e5, nu=0.45, omega=40.0, dt=0.1, seed=1)
    out = []
    orig = O.num_threads()
    for n in (1, 4):
        O.set_num_threads(n)
        o = O.Scene.from_spec(spec)
        xs = []
        for k in range(2):
            o.set_targets(spec.targets_at(k))
            rc, x, st = o.step(O.PPN, 1e-6)
            assert rc == 0
            xs.append((x, st["newton_iters"], st["total_cg_iters"]))
        out.append(xs)
    O.set_num_threads(orig)
    for (xa, na, ca), (xb, nb, cb) in zip(*out):
        assert na == nb and ca == cb
        assert np.array_equal(xa, xb)
