"""Algorithm 1's selection on the GPU against the oracle (Sec. 4).

The element key is r_e = ||S^e g||_inf and a round selects the elements not yet
projected with r_e > delta.  These tests check, through the C ABI:
  - the selected set of every PPN retry of every Newton iteration of several
    violent FP64 steps equals the oracle's, attempt by attempt, away from ties,
    also at non-default tightening / release rates (alpha, beta) of Sec. 5.2's
    ablation;
  - ties (|r_e - delta| <= tie_band delta, 1e-12 in FP64 and 1e-5 in the mixed
    mode) are counted, by the selection kernel and by the oracle alike;
  - in the mixed mode the first retry selects the oracle's set away from ties.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_21013_gb300")
from oracle import oracle as O  # noqa: E402
from ppn_inputs import twisting_beam_scene  # noqa: E402


def violent(seed, omega=40.0):
    return twisting_beam_scene(4, 4, 10, h=0.02, E=1e5, nu=0.45, omega=omega, dt=0.1, seed=seed)


def params_pair(alpha=0.5, beta=2.0):
    pg, po = P.ppn_default_params(), O.default_params()
    pg.alpha, pg.beta = alpha, beta
    po.alpha, po.beta = alpha, beta
    return pg, po


def run_recorded(spec, steps, tol, prec, pg=None, po=None):
    g = P.Scene.from_spec(spec, params=pg, precision=prec)
    g.set_record_selection(True)
    o = O.Scene.from_spec(spec, po)
    o.set_record(True)
    rec = []
    for n in range(steps):
        tg = spec.targets_at(n)
        g.set_targets(tg)
        o.set_targets(tg)
        rc, x, st = g.step(P.MODE_PPN, tol)
        rco, xo, sto = o.step(O.PPN, tol)
        ag, ao = g.attempts(), o.attempts()
        rec.append(dict(rc=rc, x=x, st=st, ag=ag, selg=[g.attempt_selection(i) for i in range(len(ag))],
                        gg=[g.iteration_gradient(k) for k in range(st["newton_iters"] + 1)],
                        rco=rco, xo=xo, sto=sto, ao=ao, selo=[o.attempt_selection(i) for i in range(len(ao))],
                        go=[o.iteration_gradient(k) for k in range(sto["newton_iters"] + 1)]))
    g.close()
    return rec


def keys(tets, grad):
    """r_e = ||S^e g||_inf of every tet."""
    return np.abs(grad[tets]).max(axis=(1, 2))


CASES = [(1, 40.0, 0.5, 2.0), (3, 40.0, 0.5, 2.0), (4, 20.0, 0.5, 2.0), (1, 40.0, 0.25, 1.0), (3, 40.0, 0.9, 16.0)]


@pytest.mark.parametrize("seed,omega,alpha,beta", CASES)
def test_every_retry_selects_exactly_on_the_gpu_iterate(seed, omega, alpha, beta):
    # Every PPN retry of every Newton iteration of four violent FP64 steps: the oracle's
    # selection applied to the GPU's own gradient of that iteration, at the GPU's delta,
    # with the GPU's earlier selections of the iteration as the projected set, gives the
    # GPU's selected set bit for bit (the decisions are FP64 comparisons of the same
    # values on both sides).  Ties at that delta are reported.
    spec = violent(seed, omega)
    pg, po = params_pair(alpha, beta)
    o = O.Scene.from_spec(spec, po)
    tets = o.tets()
    rec = run_recorded(spec, 4, 1e-6, P.PREC_FP64, pg, po)
    retries = 0
    for n, r in enumerate(rec):
        assert r["rc"] == 0
        already, it_prev = np.zeros(spec.n_tets, np.uint8), -1
        for a, sg in zip(r["ag"], r["selg"]):
            if a["newton_iter"] != it_prev:
                already[:] = 0
                it_prev = a["newton_iter"]
            if a["attempt"] == 0:
                assert len(sg) == 0
                continue
            retries += 1
            grad = r["gg"][a["newton_iter"]]
            sel_o, n_o = o.select(grad, a["delta"], already)
            assert np.array_equal(np.nonzero(sel_o)[0], sg), f"step {n} iteration {a['newton_iter']}"
            assert a["n_new_projected"] == n_o == len(sg)
            rk = keys(tets, grad)
            ties = int(((np.abs(rk - a["delta"]) <= 1e-12 * a["delta"]) & (already == 0)).sum())
            assert a["n_ties"] >= ties
            already[sg] = 1
    assert retries >= 5


@pytest.mark.parametrize("seed,omega,alpha,beta", CASES)
def test_selected_sets_follow_the_oracle_run(seed, omega, alpha, beta):
    # The GPU run against the oracle's own run of the same steps.  Attempt by attempt
    # (the same Newton iteration, solve number and verdict) the selected sets are equal,
    # as long as the two runs solve alike.  The PCG stops at a relative residual of 1e-4,
    # so a solve that takes one CG iteration more on one side (a rounding difference at
    # the stopping test) moves that side's Newton iterate by up to ~1e-4 of the step;
    # from there the runs follow different inexact-Newton paths to the same solution,
    # and the rest of the step is compared by its result only.  Before that, the
    # gradients differ by rounding (the keys near convergence, small sums of large terms,
    # by up to ~1e-6 of themselves, and delta = alpha ||g||_inf with them): an element
    # whose key lies within max(1e-6, 4 x the relative difference of the two deltas) of
    # delta on the oracle's iterate may flip, which also ends the comparison.
    spec = violent(seed, omega)
    pg, po = params_pair(alpha, beta)
    tets = O.Scene.from_spec(spec, po).tets()
    rec = run_recorded(spec, 4, 1e-6, P.PREC_FP64, pg, po)
    exact = 0
    for n, r in enumerate(rec):
        assert r["rc"] == r["rco"] == 0
        disp = np.abs(r["xo"] - spec.rest).max()
        assert np.abs(r["x"] - r["xo"]).max() <= 1e-5 * disp
        assert abs(r["st"]["newton_iters"] - r["sto"]["newton_iters"]) <= 1
        flipped = False
        for a, b, sg, so in zip(r["ag"], r["ao"], r["selg"], r["selo"]):
            assert (a["newton_iter"], a["attempt"], a["ind"]) == (b["newton_iter"], b["attempt"], b["ind"]), \
                f"step {n}: the runs took different solves before any selection differed"
            if a["attempt"] == 0:
                if a["cg_iters"] != b["cg_iters"]:
                    flipped = True
                    break
                continue
            drift = abs(a["delta"] / b["delta"] - 1.0)
            if drift > 1e-4:
                flipped = True
                break
            if np.array_equal(sg, so):
                exact += 1
                if drift < 1e-10:
                    assert a["n_ties"] == b["n_ties"]
                if a["cg_iters"] != b["cg_iters"]:
                    flipped = True
                    break
                continue
            band = max(1e-6, 4.0 * drift)
            near = np.abs(keys(tets, r["go"][b["newton_iter"]]) - b["delta"]) <= band * b["delta"]
            diff = np.setxor1d(sg, so)
            assert near[diff].all(), f"step {n} iteration {a['newton_iter']}: {diff} not near delta"
            flipped = True
            break
        if not flipped:
            assert len(r["ag"]) == len(r["ao"])
    assert exact >= 5


def test_mixed_first_retry_selects_the_oracle_set():
    # the first Newton iteration starts from the same state on both sides: the FP64
    # gradient of the mixed path differs from the oracle's by the rounding of the
    # FP32-stored D_m^-1, well inside the mixed tie band 1e-5
    spec = violent(5)
    rec = run_recorded(spec, 1, 1e-5, P.PREC_MIXED)[0]
    ag, ao = rec["ag"], rec["ao"]
    assert ag[0]["ind"] and ao[0]["ind"]
    a, b = ag[1], ao[1]
    assert (a["newton_iter"], a["attempt"]) == (b["newton_iter"], b["attempt"]) == (0, 1)
    assert a["delta"] == pytest.approx(b["delta"], rel=1e-6)
    sg, so = rec["selg"][1], rec["selo"][1]
    assert len(so) > 0
    assert len(np.setxor1d(sg, so)) <= a["n_ties"]


@pytest.mark.parametrize("prec", [P.PREC_FP64, P.PREC_MIXED])
def test_selection_kernel_counts_ties(prec):
    spec = twisting_beam_scene(7, 6, 13, h=0.02, E=1e5, nu=0.45, omega=5.0, dt=1 / 30, seed=26)
    g = P.Scene.from_spec(spec, precision=prec)
    o = O.Scene.from_spec(spec)
    tets = o.tets()
    rng = np.random.default_rng(27)
    grad = rng.standard_normal((spec.n_verts, 3))
    grad[spec.fixed] = 0
    band = 1e-12 if prec == P.PREC_FP64 else 1e-5
    delta = 1.5
    # vertices placed just inside and just outside the band around delta
    free = np.setdiff1d(np.arange(spec.n_verts), spec.fixed)
    picks = rng.choice(free, 8, replace=False)
    for k, f in zip(picks, (0.0, 0.5, -0.5, 0.9, -0.9, 2.0, -2.0, 4.0)):
        grad[k] = 0.0
        grad[k, 1] = delta * (1.0 + f * band)
    r = np.abs(grad[tets]).max(axis=(1, 2))
    already = (rng.random(spec.n_tets) < 0.2).astype(np.uint8)
    sel, n, n_ties = g.probe_select(grad, delta, already, with_ties=True)
    sel_o, n_o = o.select(grad, delta, already)
    # the strict test decides the set; the band only counts
    assert np.array_equal(sel, sel_o) and n == n_o
    expect = int(((np.abs(r - delta) <= band * delta) & (already == 0)).sum())
    assert n_ties == expect and expect > 0
    # a wider band set by the caller
    p = P.ppn_default_params()
    p.tie_band = 1e-2
    g2 = P.Scene.from_spec(spec, params=p, precision=prec)
    _, _, n_ties2 = g2.probe_select(grad, delta, already, with_ties=True)
    assert n_ties2 == int(((np.abs(r - delta) <= 1e-2 * delta) & (already == 0)).sum())
    # select-all and fallback requests count no ties
    assert g.probe_select(grad, -1.0, with_ties=True)[2] == 0
    assert g.probe_select(grad, 1e-13, with_ties=True)[2] == 0
    g.close()
    g2.close()


def test_recording_is_off_by_default_and_rejects_bad_indices():
    spec = violent(1)
    g = P.Scene.from_spec(spec, precision=P.PREC_FP64)
    g.set_targets(spec.targets_at(0))
    g.step(P.MODE_PPN, 1e-6)
    with pytest.raises(P.PPNError):
        g.attempt_selection(0)
    g.set_record_selection(True)
    g.step(P.MODE_PPN, 1e-6)
    n = len(g.attempts())
    assert g.attempt_selection(n - 1) is not None
    with pytest.raises(P.PPNError):
        g.attempt_selection(n)
    g.close()
