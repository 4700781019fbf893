"""Pins of the oracle's per-attempt records (Algorithm 1, Sec. 4): the selected lists,
the tie counts and the recorded iteration gradients agree with a brute-force evaluation
of the selection rule r_e = ||S^e g||_inf > delta on the recorded gradient."""

import numpy as np

from oracle import oracle as O
from ppn_inputs import twisting_beam_scene


def test_recorded_selections_follow_the_rule_on_the_recorded_gradient():
    spec = twisting_beam_scene(4, 4, 10, h=0.02, E=1e5, nu=0.45, omega=40.0, dt=0.1, seed=3)
    p = O.default_params()
    p.tie_band = 5e-2  # wide enough that ties occur
    o = O.Scene.from_spec(spec, p)
    o.set_record(True)
    tets = o.tets()
    seen_ties = 0
    retries = 0
    for n in range(3):
        o.set_targets(spec.targets_at(n))
        rc, x, st = o.step(O.PPN, 1e-6)
        assert rc == 0
        att = o.attempts()
        its = o.iter_stats()
        already = np.zeros(spec.n_tets, bool)
        cur = -1
        ties_total = 0
        for i, a in enumerate(att):
            if a["newton_iter"] != cur:
                already[:] = False
                cur = a["newton_iter"]
            sel = o.attempt_selection(i)
            if a["attempt"] == 0:
                assert sel.size == 0 and a["n_ties"] == 0
                continue
            retries += 1
            g = o.iteration_gradient(a["newton_iter"])
            r = np.abs(g[tets]).max(axis=(1, 2))
            d = a["delta"]
            expect = np.nonzero((r > d) & ~already)[0]
            assert np.array_equal(sel, expect)
            assert a["n_new_projected"] == sel.size
            # ties of the round that selected (rounds that selected nothing add theirs too)
            assert a["n_ties"] >= int(((np.abs(r - d) <= 5e-2 * d) & ~already).sum())
            ties_total += a["n_ties"]
            already[sel] = True
        # every round's ties are in the step total; the iteration records count the projections
        assert st["n_ties"] >= ties_total
        seen_ties += st["n_ties"]
        assert sum(it["n_new_projected"] for it in its) == st["total_projections"]
        # the gradient of the first iteration is the gradient at the step's initial iterate
        g0 = o.iteration_gradient(0)
        assert np.isclose(np.linalg.norm(g0), its[0]["grad_norm2"], rtol=1e-12)
    assert retries > 0 and seen_ties > 0
