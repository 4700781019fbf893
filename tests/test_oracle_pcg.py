"""Pins of the oracle's block-Jacobi PCG with negative-curvature exit (Sec. 4.1)."""

import json
import os

import numpy as np

from oracle import oracle as O
from ppn_inputs import tiny_scene

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "toy_matrices.json")))


def dense_to_bsr(Ad):
    n = Ad.shape[0] // 3
    rp, col, vals = [0], [], []
    for i in range(n):
        for j in range(n):
            blk = Ad[3 * i:3 * i + 3, 3 * j:3 * j + 3]
            if i == j or np.any(blk != 0):
                col.append(j)
                vals.append(blk)
        rp.append(len(col))
    return np.array(rp), np.array(col, np.int32), np.array(vals)


def random_spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((3 * n, 3 * n)))
    w = np.exp(rng.uniform(0, np.log(cond), 3 * n))
    return (Q * w) @ Q.T


def test_spd_solve_matches_dense_solve():
    A = random_spd(6, 0)
    b = np.random.default_rng(1).standard_normal(18)
    rp, col, vals = dense_to_bsr(A)
    x, info = O.pcg_bsr(rp, col, vals, b, rel_tol=1e-13, max_iter=500)
    assert not info["ind"] and not info["hit_max"]
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-12)
    # relative residual criterion at the paper's tolerance
    x4, info4 = O.pcg_bsr(rp, col, vals, b, rel_tol=1e-4, max_iter=500)
    assert np.linalg.norm(b - A @ x4) <= 1e-4 * np.linalg.norm(b) * (1 + 1e-12)


def test_descent_identity_on_spd_system():
    # dx^T g = -dx^T H dx for H dx = -g (Sec. 3): exact for the exact solve,
    # and dx^T g < 0 for every PCG iterate from zero
    A = random_spd(5, 2)
    g = np.random.default_rng(3).standard_normal(15)
    rp, col, vals = dense_to_bsr(A)
    dx, _ = O.pcg_bsr(rp, col, vals, -g, rel_tol=1e-14, max_iter=500)
    assert abs(dx @ g + dx @ A @ dx) <= 1e-10 * abs(dx @ g)
    dx4, _ = O.pcg_bsr(rp, col, vals, -g, rel_tol=1e-1, max_iter=500)
    assert dx4 @ g < 0


def test_zero_rhs_returns_zero_without_iterations():
    A = random_spd(3, 4)
    rp, col, vals = dense_to_bsr(A)
    x, info = O.pcg_bsr(rp, col, vals, np.zeros(9))
    assert info["iters"] == 0 and not info["ind"] and np.all(x == 0)


def test_indefinite_diagonal_block_reports_ind():
    # the paper's Q = A + B + C = diag(-9, 5) embedded in a 3x3 block
    Q = np.array(GOLD["Q_equals_A_plus_B_plus_C"], float)
    blk = np.eye(3)
    blk[:2, :2] = Q
    x, info = O.pcg_bsr([0, 1], [0], blk[None], np.array([1.0, 1.0, 1.0]))
    assert info["ind"] and info["precond_fail"] and info["iters"] == 0


def test_negative_curvature_direction_stops_cg():
    # SPD diagonal blocks but an indefinite global matrix: [[I, 2I], [2I, I]] has eigenvalue -1
    A = np.block([[np.eye(3), 2 * np.eye(3)], [2 * np.eye(3), np.eye(3)]])
    rp, col, vals = dense_to_bsr(A)
    b = np.array([1.0, 0.5, 0.2, 0.3, -0.7, 0.1])
    x, info = O.pcg_bsr(rp, col, vals, b)
    assert info["ind"] and not info["precond_fail"]
    # the returned iterate is the one before the failing direction; every
    # accepted direction had positive curvature, so it is a descent direction for g = -b
    assert x @ (-b) <= 0


def test_exact_arithmetic_termination_bound():
    A = random_spd(2, 5, cond=10.0)
    rp, col, vals = dense_to_bsr(A)
    b = np.random.default_rng(6).standard_normal(6)
    _, info = O.pcg_bsr(rp, col, vals, b, rel_tol=1e-12, max_iter=100)
    assert info["iters"] <= 6 + 2


def test_assembled_scene_matrix_is_spd_near_rest():
    spec = tiny_scene(cells=(2, 2, 2), seed=1)
    sc = O.Scene.from_spec(spec)
    vals = sc.assemble(spec.rest)
    rp, col = sc.pattern()
    n = spec.n_verts
    Ad = np.zeros((3 * n, 3 * n))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            Ad[3 * i:3 * i + 3, 3 * col[k]:3 * col[k] + 3] = vals[k]
    assert np.linalg.eigvalsh(0.5 * (Ad + Ad.T)).min() > 0
    b = np.random.default_rng(7).standard_normal(3 * n)
    b.reshape(n, 3)[spec.fixed] = 0
    x, info = O.pcg_bsr(rp, col, vals, b, rel_tol=1e-12, max_iter=1000)
    assert not info["ind"]
    assert np.allclose(x, np.linalg.solve(Ad, b), rtol=1e-8, atol=1e-14)
