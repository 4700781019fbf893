"""Pins of the oracle's Jacobi eigensolver and eigenvalue clamping.

The clamping semantics are pinned by the paper's own 2x2 example (Sec. 3 and
Sec. 4, stored in tests/golden/toy_matrices.json); the eigensolver is pinned
against LAPACK (numpy.linalg.eigh) and against reconstruction/orthogonality.
"""

import json
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "toy_matrices.json")))


@pytest.mark.parametrize("n", [2, 3, 5, 9, 12])
@pytest.mark.parametrize("seed", range(3))
def test_jacobi_matches_lapack(n, seed):
    rng = np.random.default_rng(seed * 31 + n)
    M = rng.standard_normal((n, n))
    A = M + M.T
    w, Q = O.eigh(A)
    wl = np.linalg.eigvalsh(A)
    assert np.allclose(np.sort(w), wl, rtol=0, atol=1e-12 * np.abs(wl).max())
    assert np.allclose(Q.T @ Q, np.eye(n), atol=1e-13)
    assert np.allclose(Q @ np.diag(w) @ Q.T, A, atol=1e-12 * np.abs(A).max())


def test_two_by_two_closed_form():
    a, b, c = 3.0, 1.5, -2.0
    w, _ = O.eigh(np.array([[a, b], [b, c]]))
    m, r = 0.5 * (a + c), np.hypot(0.5 * (a - c), b)
    assert np.allclose(np.sort(w), [m - r, m + r], atol=1e-14)


def test_toy_matrices_from_the_paper():
    A, B, C = (np.array(GOLD[k], float) for k in "ABC")
    eps = GOLD["eps"]
    assert np.allclose(np.sort(O.eigh(A)[0]), GOLD["eig_A"])
    assert np.allclose(np.sort(O.eigh(A + B)[0]), GOLD["eig_P"])
    assert np.allclose(np.sort(O.eigh(A + B + C)[0]), GOLD["eig_Q"])
    Ahat, dA = O.clamp(A, eps)
    assert np.allclose(Ahat, np.diag([eps, 2.0]), atol=1e-15)
    assert np.allclose(dA, np.diag([eps + 1.0, 0.0]), atol=1e-15)
    # clamping only C suffices to make A + B + C positive definite
    Chat, _ = O.clamp(C, eps)
    assert np.linalg.eigvalsh(A + B + Chat).min() > 0
    # while A + B is SPD without any projection
    assert np.linalg.eigvalsh(A + B).min() > 0
    # B is SPD and is left untouched
    Bhat, dB = O.clamp(B, eps)
    assert np.array_equal(dB, np.zeros((2, 2))) or np.abs(dB).max() <= 1e-15


@pytest.mark.parametrize("seed", range(5))
def test_clamp_properties(seed):
    rng = np.random.default_rng(50 + seed)
    n = 12
    M = rng.standard_normal((n, n))
    H = M + M.T
    eps = 1e-8
    Hh, dH = O.clamp(H, eps)
    wl = np.linalg.eigvalsh(H)
    wh = np.linalg.eigvalsh(Hh)
    # PSD (eigenvalues >= eps up to rounding), positive part kept
    assert wh.min() >= eps - 1e-12
    assert np.allclose(np.sort(wh)[wl < eps].clip(max=None), eps, atol=1e-12)
    assert np.allclose(np.sort(wh)[wl >= eps], wl[wl >= eps], atol=1e-12)
    # rank of the update equals the number of clamped eigenvalues
    assert np.linalg.matrix_rank(dH, tol=1e-10) == int((wl < eps).sum())
    assert np.allclose(dH, dH.T, atol=1e-13)


def test_element_hessian_at_rest_has_six_zero_modes():
    # rigid translations (3) and infinitesimal rotations (3) store no energy at rest
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 0.1
    _, _, H = O.tet_eval(X, X, 1e5, 2e5)
    w = np.linalg.eigvalsh(H)
    assert (np.abs(w) <= 1e-9 * np.abs(w).max()).sum() == 6
    Hh, dH = O.clamp(H, 1e-8)
    assert np.linalg.eigvalsh(Hh).min() >= 1e-8 - 1e-9
