"""Pins of the oracle's time step: Newton / PN / PPN (Algorithm 1) against
closed forms, a dense brute-force Newton, and the control flow of Algorithm 1.
"""

import math

import numpy as np
import pytest

from oracle import oracle as O
from ppn_inputs import cube_scene, tiny_scene, twisting_beam_scene


def violent_beam(seed=1):
    # small beam twisted fast: the unprojected Hessian turns indefinite within a few steps
    return twisting_beam_scene(4, 4, 10, h=0.02, E=1e5, nu=0.45, omega=40.0, dt=0.1, seed=seed)


def run(spec, mode, steps, tol=1e-6, params=None, sc=None):
    sc = sc or O.Scene.from_spec(spec, params)
    out = []
    for n in range(steps):
        sc.set_targets(spec.targets_at(n))
        rc, x, st = sc.step(mode, tol)
        out.append((rc, x, st, sc.iter_stats(), sc.attempts()))
    return sc, out


def test_free_fall_is_exact():
    spec = tiny_scene(cells=(2, 1, 1), seed=0, fixed_face=False)
    p = O.default_params()
    p.pcg_rel_tol = 1e-14
    sc = O.Scene.from_spec(spec, p)
    g = np.array(spec.gravity)
    dt = spec.dt
    rc, x1, _ = sc.step(O.PPN, 1e-12)
    assert rc == 0
    assert np.allclose(x1, spec.rest + dt * dt * g, rtol=0, atol=1e-12)
    rc, x2, _ = sc.step(O.PPN, 1e-12)
    _, v2 = sc.get_state()
    assert np.allclose(x2, spec.rest + 3 * dt * dt * g, rtol=0, atol=1e-12)
    assert np.allclose(v2, 2 * dt * g, rtol=0, atol=1e-10)


def dense_newton(sc, spec, mode, tol, target, c=1e-4):
    """Textbook Newton with exact dense solves and LAPACK projections."""
    x_n, _ = sc.get_state()
    xhat = sc.xhat()
    x = x_n.copy()
    x[spec.fixed] = target
    m = sc.lumped_mass()
    free = np.ones(spec.n_verts, bool)
    free[spec.fixed] = False
    fm = np.repeat(free, 3)
    tets = sc.tets()
    g0 = None
    iters = 0
    for k in range(100):
        g = sc.gradient(x, xhat)
        gn = np.linalg.norm(g)
        if g0 is None:
            g0 = gn
        if gn <= tol * g0:
            break
        _, _, He = sc.element_eval(x)
        N = 3 * spec.n_verts
        Hd = np.zeros((N, N))
        for e in range(spec.n_tets):
            Hl = He[e]
            if mode == O.PN:
                w, Q = np.linalg.eigh(Hl)
                Hl = (Q * np.maximum(w, 1e-8)) @ Q.T
            idx = (3 * tets[e][:, None] + np.arange(3)[None, :]).reshape(-1)
            Hd[np.ix_(idx, idx)] += Hl
        Hd += np.diag(np.repeat(m / spec.dt ** 2, 3))
        Hff = Hd[np.ix_(fm, fm)]
        assert np.linalg.eigvalsh(0.5 * (Hff + Hff.T)).min() > 0, "brute force needs SPD"
        dx = np.zeros(N)
        dx[fm] = np.linalg.solve(Hff, -g.reshape(-1)[fm])
        dx = dx.reshape(-1, 3)
        E0 = sc.energy(x, xhat)
        dd = float((g * dx).sum())
        gamma = 1.0
        while sc.energy(x + gamma * dx, xhat) > E0 + c * gamma * dd:
            gamma *= 0.5
        x = x + gamma * dx
        iters += 1
    return x, iters


@pytest.mark.parametrize("mode", [O.NEWTON, O.PN, O.PPN])
def test_matches_dense_brute_force_newton(mode):
    spec = tiny_scene(cells=(1, 2, 1), E=2e3, seed=2)
    p = O.default_params()
    p.pcg_rel_tol = 1e-14
    sc = O.Scene.from_spec(spec, p)
    ref = O.Scene.from_spec(spec, p)
    tol = 1e-6 if mode == O.PN else 1e-9  # PN converges only linearly
    for n in range(3):
        xb, itb = dense_newton(ref, spec, O.PN if mode == O.PN else O.NEWTON, tol,
                               spec.targets_at(n))
        ref.set_state(xb, (xb - ref.get_state()[0]) / spec.dt)
        sc.set_targets(spec.targets_at(n))
        rc, x, st = sc.step(mode, tol)
        assert rc == 0
        assert abs(st["newton_iters"] - itb) <= 1
        scale = np.abs(xb - spec.rest).max()
        assert np.abs(x - xb).max() <= 1e-7 * scale


@pytest.mark.parametrize("mode", [O.NEWTON, O.PN, O.PPN])
def test_every_step_is_a_descent_step(mode):
    spec = violent_beam()
    _, out = run(spec, mode, 4)
    for rc, _, _, its, _ in out:
        assert rc == 0
        for it in its:
            assert it["dir_deriv"] < 0
            assert it["energy_new"] <= it["energy"]


def test_ppn_is_newton_when_no_indefiniteness():
    spec = cube_scene(4, E=1e5, dt=1.0 / 240)
    _, a = run(spec, O.NEWTON, 3)
    _, b = run(spec, O.PPN, 3)
    for (ra, xa, sa, _, _), (rb, xb, sb, _, _) in zip(a, b):
        assert ra == rb == 0
        assert sb["total_projections"] == 0
        assert np.array_equal(xa, xb)


def test_ppn_uses_projection_on_violent_scene_and_projects_less_than_pn():
    spec = violent_beam()
    _, ppn = run(spec, O.PPN, 4)
    _, pn = run(spec, O.PN, 4)
    proj_ppn = sum(o[2]["total_projections"] for o in ppn)
    proj_pn = sum(o[2]["total_projections"] for o in pn)
    assert proj_ppn > 0
    assert proj_ppn < 0.25 * proj_pn


def test_ppn_degenerates_to_pn_with_tiny_alpha():
    # with alpha so small that the first tightening falls below eps_delta, the
    # first retry projects every element: the system is PN's, bit for bit
    spec = tiny_scene(cells=(1, 2, 1), E=2e3, seed=3)
    p = O.default_params()
    p.alpha = 1e-15
    p.newton_max_iter = 1
    pn = O.Scene.from_spec(spec, p)
    ppn = O.Scene.from_spec(spec, p)
    ppn.set_solve_hook(lambda k, a, n: 1 if a == 0 else -1)
    _, x_pn, _ = pn.step(O.PN, 1e-12)
    _, x_ppn, st = ppn.step(O.PPN, 1e-12)
    att = ppn.attempts()
    assert att[1]["n_new_projected"] == spec.n_tets and att[1]["delta"] <= 1e-12
    assert np.array_equal(x_pn, x_ppn)


def test_delta_schedule_follows_algorithm_1():
    spec = violent_beam(seed=4)
    p = O.default_params()
    sc = O.Scene.from_spec(spec, p)
    script = {(0, 0): 1, (0, 1): 1, (0, 2): 1, (1, 0): 1}
    sc.set_solve_hook(lambda k, a, n: script.get((k, a), 0 if (k, a) in [(0, 3), (1, 1)] else -1))
    sc.set_targets(spec.targets_at(0))
    xhat = sc.xhat()
    x0, _ = sc.get_state()
    x0[spec.fixed] = spec.targets_at(0)
    rc, _, _ = sc.step(O.PPN, 1e-6)
    att = sc.attempts()
    its = sc.iter_stats()
    g0 = sc.gradient(x0, xhat)
    ginf = np.abs(g0).max()
    tets = sc.tets()
    r = np.array([np.abs(g0[t]).max() for t in tets])
    a0 = [a for a in att if a["newton_iter"] == 0]
    assert a0[0]["attempt"] == 0 and math.isinf(a0[0]["delta"])
    # each recorded retry uses delta = alpha^j ||g||_inf for increasing j, and the
    # projected set is exactly {e : r_e > delta} (cumulative, monotone)
    js, cum = [], 0
    for a in a0[1:]:
        j = math.log(a["delta"] / ginf) / math.log(p.alpha)
        assert abs(j - round(j)) < 1e-9
        js.append(round(j))
        cum += a["n_new_projected"]
        assert cum == int((r > a["delta"]).sum())
    assert js == sorted(js) and js[0] == 1 and len(set(js)) == len(js)
    # after the successful solve delta is relaxed by beta
    assert its[0]["delta"] == pytest.approx(p.beta * a0[-1]["delta"], rel=1e-15)
    # the next iteration starts from the relaxed delta, not from infinity
    a1 = [a for a in att if a["newton_iter"] == 1]
    assert len(a1) >= 2 and a1[1]["delta"] <= its[0]["delta"]


def test_eps_delta_fallback_projects_everything():
    # Two clamped layers: the tets between them touch only Dirichlet vertices, so
    # their residual is exactly zero and only the eps_delta rule can select them.
    from ppn_inputs.scenes import SceneSpec, _face
    base = tiny_scene(cells=(2, 2, 3), E=1e4, seed=5)
    nx, ny, nz = base.meta["dims"]
    fixed = np.union1d(_face(nx, ny, nz, 2, 0), _face(nx, ny, nz, 2, 1)).astype(np.int32)
    spec = SceneSpec("two_layers", base.rest, base.tets, fixed, base.E, base.nu, base.rho, base.dt)
    p = O.default_params()
    p.newton_max_iter = 1
    sc = O.Scene.from_spec(spec, p)
    x = spec.rest + 0.3 * 0.1 * np.random.default_rng(0).standard_normal(spec.rest.shape)
    x[fixed] = spec.rest[fixed]
    sc.set_state(x, np.zeros_like(x))
    sc.set_solve_hook(lambda k, a, n: 1)  # the solver never reports success
    rc, _, _ = sc.step(O.PPN, 1e-6)
    its = sc.iter_stats()
    att = sc.attempts()
    assert its[0]["n_projected_total"] == spec.n_tets
    assert att[-1]["delta"] <= p.eps_delta and att[-1]["n_new_projected"] > 0
    assert att[-2]["delta"] > p.eps_delta
    assert its[0]["fallback"] in (1, 2, 3)
    assert its[0]["dir_deriv"] < 0


def test_paper_stopping_criterion():
    spec = violent_beam(seed=6)
    p = O.default_params()
    p.tol_kind = 1
    sc = O.Scene.from_spec(spec, p)
    sc.set_targets(spec.targets_at(0))
    rc, _, st = sc.step(O.PPN, 1e-3)
    its = sc.iter_stats()
    assert rc == 0
    assert its[-1]["gamma"] > 0


def test_checkpoint_resume_is_bitwise():
    spec = violent_beam(seed=7)
    sc, out = run(spec, O.PPN, 3)
    x, v = sc.get_state()
    sc2 = O.Scene.from_spec(spec)
    sc2.set_state(x, v)
    sc.set_targets(spec.targets_at(3))
    sc2.set_targets(spec.targets_at(3))
    _, xa, _ = sc.step(O.PPN, 1e-6)
    _, xb, _ = sc2.step(O.PPN, 1e-6)
    assert np.array_equal(xa, xb)


def test_scene_at_rest_stops_at_the_rounding_floor():
    # A stiff cube settles on its fixed face.  Near rest the energy differences of a
    # Newton step fall below the FP64 resolution of the energy sum, which the Armijo
    # slack absorbs, and once at rest g(x_n) is rounding noise, so only the floor
    # ||g|| <= 1e-12 ||s|| can end the Newton loop.
    spec = cube_scene(4, E=2e6, nu=0.4, dt=1 / 30, seed=0)
    sc = O.Scene.from_spec(spec)
    for n in range(60):
        sc.set_targets(spec.targets_at(n))
        rc, _, st = sc.step(O.PPN, 1e-4)
        assert rc == 0 and st["newton_iters"] <= 2
    assert st["newton_iters"] == 0  # already at rest: converged before any solve
    x_rest, v_rest = sc.get_state()
    # without the floor the relative test alone cannot stop, and without the slack
    # the line search cannot certify the tiny decrease
    p = O.default_params()
    p.grad_floor = 0.0
    p.newton_max_iter = 6
    sc.set_params(p)
    sc.set_targets(spec.targets_at(60))
    rc, _, st = sc.step(O.PPN, 1e-4)
    assert rc == 4 and st["newton_iters"] == 6
    p = O.default_params()
    p.ls_slack = 0.0
    p.grad_floor = 0.0
    p.newton_max_iter = 20
    sc.set_params(p)
    sc.set_state(x_rest, v_rest)
    rc, _, _ = sc.step(O.PPN, 1e-4)
    assert rc in (3, 4)
