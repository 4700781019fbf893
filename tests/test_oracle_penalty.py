"""Pins of the oracle's penalty Dirichlet conditions (Sec. 5.1 enforces Dirichlet
constraints with penalty potentials; the reading: a constrained vertex stays a
free degree of freedom with the potential k m_v / (2 dt^2) |x_v - t_v|^2): a
closed-form step, the derivatives of the penalised potential, and the limit of
exact elimination as the stiffness grows."""

import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from ppn_inputs import tiny_scene, twisting_beam_scene


def penalty_params(k):
    p = O.default_params()
    p.dirichlet_penalty = k
    return p


def test_uniform_translation_of_fully_constrained_body_has_closed_form():
    # every vertex held toward t = X + c: a uniform displacement carries no elastic
    # energy, so each vertex solves m/dt^2 (x - xhat) + k m/dt^2 (x - t) = 0 and the
    # first step moves the body by d = (dt^2 g + k c) / (1 + k)
    spec = tiny_scene(cells=(2, 2, 1), seed=4, fixed_face=False)
    spec = dataclasses.replace(spec, fixed=np.arange(spec.n_verts, dtype=np.int32))
    k, c = 300.0, np.array([0.01, -0.02, 0.005])
    sc = O.Scene.from_spec(spec, penalty_params(k))
    sc.set_targets(spec.rest + c)
    rc, x, st = sc.step(O.PPN, 1e-12)
    assert rc == 0
    d = (spec.dt ** 2 * np.array(spec.gravity) + k * c) / (1.0 + k)
    assert np.abs(x - (spec.rest + d)).max() <= 1e-9 * np.abs(d).max()
    assert st["total_projections"] == 0  # a rigid translation keeps every element at rest


@pytest.mark.parametrize("k", [1.0, 50.0])
def test_penalised_gradient_and_hessian_are_derivatives_of_the_potential(k):
    spec = tiny_scene(cells=(2, 1, 1), seed=7)
    sc = O.Scene.from_spec(spec, penalty_params(k))
    rng = np.random.default_rng(8)
    sc.set_targets(spec.rest[spec.fixed] + 0.003 * rng.standard_normal((len(spec.fixed), 3)))
    x = spec.rest + 0.004 * rng.standard_normal(spec.rest.shape)  # constrained vertices move too
    xhat = x + 0.002 * rng.standard_normal(x.shape)
    g = sc.gradient(x, xhat)
    assert np.abs(g[spec.fixed]).max() > 0  # not eliminated
    h = 1e-7
    for _ in range(3):
        v = rng.standard_normal(x.shape)
        dE = (sc.energy(x + h * v, xhat) - sc.energy(x - h * v, xhat)) / (2 * h)
        assert dE == pytest.approx(float((g * v).sum()), rel=1e-6)
    vals = sc.assemble(x)
    rp, col = sc.pattern()
    v = rng.standard_normal(x.shape)
    Hv = np.zeros_like(x)
    for i in range(spec.n_verts):
        for kk in range(rp[i], rp[i + 1]):
            Hv[i] += vals[kk] @ v[col[kk]]
    dg = (sc.gradient(x + h * v, xhat) - sc.gradient(x - h * v, xhat)) / (2 * h)
    assert np.allclose(Hv, dg, rtol=1e-5, atol=1e-6 * np.abs(dg).max())
    # the penalty adds k m / dt^2 to the constrained vertices' diagonal blocks
    sc0 = O.Scene.from_spec(spec, penalty_params(k))
    sc0.set_params(penalty_params(2 * k))
    diff = sc0.assemble(x) - vals
    for i in spec.fixed:
        kk = next(j for j in range(rp[i], rp[i + 1]) if col[j] == i)
        w = diff[kk][0, 0]
        assert np.allclose(diff[kk], w * np.eye(3)) and w > 0
    free = np.setdiff1d(np.arange(spec.n_verts), spec.fixed)
    for i in free:
        assert np.abs(diff[rp[i]:rp[i + 1]]).max() == 0.0


def test_switching_between_elimination_and_penalty_is_refused():
    # the Dirichlet treatment is fixed at creation: an eliminated vertex keeps a zero gradient
    spec = tiny_scene(cells=(1, 1, 1), seed=2)
    sc = O.Scene.from_spec(spec)
    sc.set_params(penalty_params(10.0))
    x = spec.rest + 0.01
    assert np.abs(sc.gradient(x, x)[spec.fixed]).max() == 0.0


def test_penalty_approaches_elimination_as_stiffness_grows():
    spec = twisting_beam_scene(3, 3, 6, h=0.02, E=1e5, nu=0.4, omega=4.0, dt=1 / 30, seed=1)

    def run(params):
        sc = O.Scene.from_spec(spec, params)
        for n in range(2):
            sc.set_targets(spec.targets_at(n))
            rc, x, _ = sc.step(O.PPN, 1e-10)
            assert rc == 0
        return x

    x_elim = run(O.default_params())
    errs, viol = [], []
    for k in (1e2, 1e4, 1e6):
        x = run(penalty_params(k))
        errs.append(np.abs(x - x_elim).max())
        viol.append(np.abs(x[spec.fixed] - spec.targets_at(1)).max())
    # the constraint force is O(1) and the penalty stiffness k m / dt^2: violation and error O(1/k)
    assert errs[1] < 0.03 * errs[0] and errs[2] < 0.03 * errs[1]
    assert viol[1] < 0.03 * viol[0] and viol[2] < 0.03 * viol[1]
    assert errs[2] < 1e-3 * np.abs(x_elim - spec.rest).max()
