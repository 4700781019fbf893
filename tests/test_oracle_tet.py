"""Pins of the oracle's tet element: finite differences, invariances, affine patch tests."""

import numpy as np
import pytest

from oracle import oracle as O
from ppn_inputs import kuhn_grid

E, NU = 1e5, 0.4


def rand_tet(rng):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 0.1
    X += 0.01 * rng.standard_normal((4, 3))
    if np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], 1)) < 0:
        X[[2, 3]] = X[[3, 2]]
    x = X + 0.02 * rng.standard_normal((4, 3))
    return X, x


def rand_rot(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


@pytest.mark.parametrize("seed", range(4))
def test_gradient_and_hessian_match_finite_differences(seed):
    rng = np.random.default_rng(seed)
    mu, lam = O.lame(E, NU)
    X, x = rand_tet(rng)
    psi, g, H = O.tet_eval(X, x, mu, lam)
    h = 1e-7
    fdg = np.zeros(12)
    fdH = np.zeros((12, 12))
    for m in range(12):
        d = np.zeros(12)
        d[m] = h
        pp, gp, _ = O.tet_eval(X, x.reshape(12) + d, mu, lam)
        pm, gm, _ = O.tet_eval(X, x.reshape(12) - d, mu, lam)
        fdg[m] = (pp - pm) / (2 * h)
        fdH[:, m] = (gp - gm) / (2 * h)
    assert np.abs(fdg - g).max() <= 1e-6 * np.abs(g).max()
    assert np.abs(fdH - H).max() <= 1e-6 * np.abs(H).max()
    assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()


@pytest.mark.parametrize("seed", range(4))
def test_translation_and_rotation_invariance(seed):
    rng = np.random.default_rng(10 + seed)
    mu, lam = O.lame(E, NU)
    X, x = rand_tet(rng)
    psi, g, H = O.tet_eval(X, x, mu, lam)
    # internal forces sum to zero and carry no torque
    assert np.abs(g.reshape(4, 3).sum(0)).max() <= 1e-10 * np.abs(g).max()
    torque = np.cross(x, g.reshape(4, 3)).sum(0)
    assert np.abs(torque).max() <= 1e-10 * np.abs(g).max() * np.abs(x).max()
    # translations are in the Hessian's null space
    for k in range(3):
        t = np.zeros((4, 3))
        t[:, k] = 1
        assert np.abs(H @ t.reshape(12)).max() <= 1e-9 * np.abs(H).max()
    # rigid motion of the current state leaves psi unchanged
    R = rand_rot(rng)
    psi2, _, _ = O.tet_eval(X, x @ R.T + rng.standard_normal(3), mu, lam)
    assert abs(psi2 - psi) <= 1e-10 * abs(psi)


def test_rest_and_rigid_states_are_energy_and_force_free():
    rng = np.random.default_rng(3)
    mu, lam = O.lame(E, NU)
    X, _ = rand_tet(rng)
    psi, g, H = O.tet_eval(X, X, mu, lam)
    assert abs(psi) <= 1e-12 and np.abs(g).max() <= 1e-9
    R = rand_rot(rng)
    psi, g, _ = O.tet_eval(X, X @ R.T + 1.0, mu, lam)
    assert abs(psi) <= 1e-9 and np.abs(g).max() <= 1e-8 * E * 1e-2


def test_affine_deformation_energy_is_volume_times_density():
    # x = F X + t reproduces F exactly in a linear tet: psi_e = V psi(F)
    rng = np.random.default_rng(4)
    mu, lam = O.lame(E, NU)
    X, _ = rand_tet(rng)
    F = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
    x = X @ F.T + np.array([0.3, -0.1, 0.2])
    V = np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], 1)) / 6.0
    psi, _, _ = O.tet_eval(X, x, mu, lam)
    assert abs(psi - V * O.snh_psi(F, mu, lam)) <= 1e-10 * abs(psi)


def test_mesh_patch_test_uniform_stress():
    # Under an affine deformation the assembled elastic forces vanish at interior
    # vertices (uniform stress is divergence free) and total energy = volume * psi(F).
    rest, tets = kuhn_grid(4, 4, 4, 0.1, jitter=0.05, seed=2)
    rng = np.random.default_rng(5)
    F = np.eye(3) + 0.1 * rng.standard_normal((3, 3))
    x = rest @ F.T
    sc = O.Scene(rest, tets, np.zeros(0, np.int32), E, NU, 1000.0, 1.0 / 30, gravity=(0, 0, 0))
    psi_e, ge, _ = sc.element_eval(x, want_hessian=False)
    mu, lam = O.lame(E, NU)
    p = rest[tets]
    vol = np.linalg.det(np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]], 2)).sum() / 6
    assert abs(psi_e.sum() - vol * O.snh_psi(F, mu, lam)) <= 1e-10 * abs(psi_e.sum())
    f = np.zeros_like(rest)
    np.add.at(f, sc.tets().reshape(-1), ge.reshape(-1, 3))
    ijk = np.stack(np.unravel_index(np.arange(64), (4, 4, 4), order="F"), 1)
    interior = np.all((ijk > 0) & (ijk < 3), axis=1)
    assert interior.sum() == 8
    assert np.abs(f[interior]).max() <= 1e-9 * np.abs(ge).max()
