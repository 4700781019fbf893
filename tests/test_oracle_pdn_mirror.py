"""Pins of the oracle's two variants the paper compares PPN against: PDN
(project-on-demand Newton, Sec. 2.2 and Sec. 5.1) and eigenvalue mirroring
(Sec. 5.2), against the paper's toy matrices, spectral identities and the
control flow of the countdown."""

import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from ppn_inputs import cube_scene, twisting_beam_scene

HERE = os.path.dirname(os.path.abspath(__file__))
TOY = json.load(open(os.path.join(HERE, "golden", "toy_matrices.json")))
EPS = TOY["eps"]


def test_mirror_on_the_papers_toy_matrices():
    A = np.array(TOY["A"], float)
    Q = np.array(TOY["Q_equals_A_plus_B_plus_C"], float)
    # mirroring replaces a negative eigenvalue by its magnitude; clamping by eps
    assert np.allclose(O.project(A, EPS, O.PROJ_MIRROR)[0], np.diag([1.0, 2.0]), atol=1e-14)
    assert np.allclose(O.project(A, EPS, O.PROJ_CLAMP)[0], np.diag([EPS, 2.0]), atol=1e-14)
    assert np.allclose(O.project(Q, EPS, O.PROJ_MIRROR)[0], np.diag([9.0, 5.0]), atol=1e-13)


def test_mirrored_spectrum_and_reconstruction():
    rng = np.random.default_rng(3)
    for n in (2, 5, 12):
        M = rng.standard_normal((n, n))
        H = 0.5 * (M + M.T)
        Hh, dH = O.project(H, EPS, O.PROJ_MIRROR)
        w = np.linalg.eigvalsh(H)
        assert np.allclose(np.sort(np.linalg.eigvalsh(Hh)), np.sort(np.maximum(np.abs(w), EPS)),
                           atol=1e-12 * np.abs(w).max())
        assert np.allclose(Hh - H, dH, atol=1e-13)
        # the eigenvectors are kept: Hh commutes with H
        assert np.abs(Hh @ H - H @ Hh).max() <= 1e-11 * np.abs(w).max() ** 2


def test_mirror_of_a_negated_spd_matrix_is_the_matrix():
    rng = np.random.default_rng(4)
    M = rng.standard_normal((12, 12))
    S = M @ M.T + np.eye(12)
    Hh, _ = O.project(-S, EPS, O.PROJ_MIRROR)
    assert np.allclose(Hh, S, atol=1e-11 * np.abs(S).max())
    # on an SPD matrix both projections are the identity map
    for kind in (O.PROJ_CLAMP, O.PROJ_MIRROR):
        assert np.abs(O.project(S, EPS, kind)[1]).max() <= 1e-11 * np.abs(S).max()


def violent_beam(seed=1):
    return twisting_beam_scene(4, 4, 10, h=0.02, E=1e5, nu=0.45, omega=40.0, dt=0.1, seed=seed)


def run(spec, mode, steps, tol=1e-6, params=None):
    sc = O.Scene.from_spec(spec, params)
    out = []
    for n in range(steps):
        sc.set_targets(spec.targets_at(n))
        rc, x, st = sc.step(mode, tol)
        out.append((rc, x, st, sc.iter_stats(), sc.attempts()))
    return sc, out


def test_pdn_is_newton_when_no_indefiniteness():
    spec = cube_scene(4, E=1e5, dt=1.0 / 240)
    _, a = run(spec, O.NEWTON, 3)
    _, b = run(spec, O.PDN, 3)
    for (ra, xa, _, _, _), (rb, xb, sb, _, _) in zip(a, b):
        assert ra == rb == 0
        assert sb["total_projections"] == 0
        assert np.array_equal(xa, xb)


def test_pdn_countdown_after_an_indefinite_solve():
    spec = cube_scene(4, E=1e5, dt=1.0 / 240)
    p = O.default_params()
    p.newton_max_iter = 8
    sc = O.Scene.from_spec(spec, p)
    # only the first, unprojected solve of the first iteration reports ind
    sc.set_solve_hook(lambda k, a, n: 1 if (k, a) == (0, 0) else -1)
    sc.set_targets(spec.targets_at(0))
    sc.step(O.PDN, 1e-15)
    its = sc.iter_stats()
    att = sc.attempts()
    nt = spec.n_tets
    assert len(its) == 8
    # iteration 0: unprojected solve, then every element projected and solved again
    a0 = [a for a in att if a["newton_iter"] == 0]
    assert [a["n_new_projected"] for a in a0] == [0, nt] and its[0]["pcg_attempts"] == 2
    assert its[0]["n_projected_total"] == nt
    # the next pdn_countdown = 4 iterations assemble projected without trying unprojected
    for k in range(1, 1 + p.pdn_countdown):
        assert its[k]["pcg_attempts"] == 1 and its[k]["n_projected_total"] == nt
    # then PDN tries the unprojected matrix again
    for k in range(1 + p.pdn_countdown, 8):
        assert its[k]["n_projected_total"] == 0


def test_pdn_projects_all_or_nothing_and_descends_on_a_violent_scene():
    spec = violent_beam()
    _, pdn = run(spec, O.PDN, 4)
    _, pn = run(spec, O.PN, 4)
    nt = spec.n_tets
    tot_pdn = tot_pn = 0
    for (rc, _, st, its, _), (_, _, st_pn, _, _) in zip(pdn, pn):
        assert rc == 0
        tot_pdn += st["total_projections"]
        tot_pn += st_pn["total_projections"]
        for it in its:
            assert it["n_projected_total"] in (0, nt)
            assert it["dir_deriv"] < 0 and it["energy_new"] <= it["energy"]
    assert 0 < tot_pdn <= tot_pn


@pytest.mark.parametrize("mode", [O.PN, O.PPN, O.PDN])
def test_mirroring_gives_descent_steps(mode):
    # every accepted step decreases the potential, also where mirroring converges
    # slowly (the paper reports it worse than clamping in dynamics, Sec. 5.2)
    p = O.default_params()
    p.projection = O.PROJ_MIRROR
    _, out = run(violent_beam(seed=2), mode, 3, params=p)
    for rc, _, _, its, _ in out:
        assert rc in (0, 4)  # converged, or the Newton iteration cap
        for it in its:
            assert it["dir_deriv"] < 0 and it["energy_new"] <= it["energy"]
    milder = twisting_beam_scene(4, 4, 10, h=0.02, E=1e5, nu=0.45, omega=10.0, dt=0.1, seed=2)
    _, out = run(milder, mode, 3, params=p)
    assert all(rc == 0 for rc, *_ in out)
