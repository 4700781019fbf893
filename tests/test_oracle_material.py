"""Pins of the oracle's Stable Neo-Hookean reading against mathematics it must satisfy.

None of these tests re-types the oracle's formulas: they check finite
differences, invariances and the small-strain limit, which is fixed by
textbook isotropic linear elasticity with Lame parameters of (E, nu).
"""

import numpy as np
import pytest

from oracle import oracle as O

E, NU = 1e5, 0.4


def rand_F(rng, scale=0.3):
    F = np.eye(3) + scale * rng.standard_normal((3, 3))
    return F


def rand_rot(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def test_rest_state_is_stress_free():
    mu, lam = O.lame(E, NU)
    assert O.snh_psi(np.eye(3), mu, lam) == 0.0
    assert np.abs(O.snh_pk1(np.eye(3), mu, lam)).max() == 0.0


@pytest.mark.parametrize("seed", range(5))
def test_pk1_is_gradient_of_energy(seed):
    rng = np.random.default_rng(seed)
    mu, lam = O.lame(E, NU)
    F = rand_F(rng)
    P = O.snh_pk1(F, mu, lam)
    h = 1e-6
    fd = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            d = np.zeros((3, 3))
            d[i, j] = h
            fd[i, j] = (O.snh_psi(F + d, mu, lam) - O.snh_psi(F - d, mu, lam)) / (2 * h)
    assert np.abs(fd - P).max() <= 1e-6 * np.abs(P).max()


@pytest.mark.parametrize("seed", range(5))
def test_tangent_is_gradient_of_pk1(seed):
    rng = np.random.default_rng(100 + seed)
    mu, lam = O.lame(E, NU)
    F = rand_F(rng)
    A = O.snh_dpdf(F, mu, lam)
    h = 1e-6
    fd = np.zeros((9, 9))
    for c in range(9):
        d = np.zeros(9)
        d[c] = h
        fd[:, c] = ((O.snh_pk1(F.reshape(9) + d, mu, lam) - O.snh_pk1(F.reshape(9) - d, mu, lam))
                    .reshape(9) / (2 * h))
    assert np.abs(fd - A).max() <= 1e-6 * np.abs(A).max()
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()


@pytest.mark.parametrize("seed", range(5))
def test_frame_indifference(seed):
    rng = np.random.default_rng(200 + seed)
    mu, lam = O.lame(E, NU)
    F = rand_F(rng)
    R = rand_rot(rng)
    assert abs(O.snh_psi(R @ F, mu, lam) - O.snh_psi(F, mu, lam)) <= 1e-10 * abs(O.snh_psi(F, mu, lam))
    assert np.allclose(O.snh_pk1(R @ F, mu, lam), R @ O.snh_pk1(F, mu, lam), rtol=0, atol=1e-9 * E)
    # a pure rotation stores no energy and carries no stress
    assert abs(O.snh_psi(R, mu, lam)) <= 1e-10 * E
    assert np.abs(O.snh_pk1(R, mu, lam)).max() <= 1e-10 * E


def test_small_strain_tangent_is_isotropic_linear_elasticity():
    # Textbook: C_ijkl = mu (d_ik d_jl + d_il d_jk) + lambda d_ij d_kl with
    # lambda = E nu / ((1 + nu)(1 - 2 nu)), mu = E / (2 (1 + nu)).
    lam_lame = E * NU / ((1 + NU) * (1 - 2 * NU))
    mu_lame = E / (2 * (1 + NU))
    d = np.eye(3)
    Cten = (mu_lame * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d))
            + lam_lame * np.einsum("ij,kl->ijkl", d, d)).reshape(9, 9)
    mu, lam = O.lame(E, NU)
    A = O.snh_dpdf(np.eye(3), mu, lam)
    assert np.allclose(A, Cten, rtol=0, atol=1e-9 * E)


def test_uniaxial_stress_response():
    # Small uniaxial stretch eps along x with lateral strain -nu*eps: sigma_xx = E eps,
    # lateral stresses vanish (to first order).
    mu, lam = O.lame(E, NU)
    eps = 1e-6
    F = np.diag([1 + eps, 1 - NU * eps, 1 - NU * eps])
    P = O.snh_pk1(F, mu, lam)
    assert abs(P[0, 0] - E * eps) <= 1e-4 * E * eps
    assert abs(P[1, 1]) <= 1e-4 * E * eps and abs(P[2, 2]) <= 1e-4 * E * eps


def test_energy_defined_for_inverted_elements():
    mu, lam = O.lame(E, NU)
    F = np.diag([1.0, 1.0, -0.5])
    psi = O.snh_psi(F, mu, lam)
    assert np.isfinite(psi) and psi > 0
