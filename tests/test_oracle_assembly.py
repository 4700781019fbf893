"""Pins of the oracle's assembled incremental potential, gradient, Hessian, mass and selection.

The assembled gradient and Hessian are checked against finite differences of
the scalar incremental potential; the pattern against the tet adjacency; the
lumped mass against the mesh volume; the selection against a brute-force
evaluation of the heuristic ||S^e g||_inf > delta (Sec. 4).
"""

import numpy as np
import pytest

from oracle import oracle as O
from ppn_inputs import tiny_scene


def dense(sc, vals):
    rp, col = sc.pattern()
    n = sc.n_verts
    Ad = np.zeros((3 * n, 3 * n))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            Ad[3 * i:3 * i + 3, 3 * col[k]:3 * col[k] + 3] = vals[k]
    return Ad


def deformed(spec, seed, amp=0.15):
    rng = np.random.default_rng(seed)
    h = spec.meta["h"]
    x = spec.rest + amp * h * rng.standard_normal(spec.rest.shape)
    x[spec.fixed] = spec.rest[spec.fixed]
    return x


def test_pattern_is_tet_adjacency():
    spec = tiny_scene(cells=(2, 2, 1), seed=0)
    sc = O.Scene.from_spec(spec)
    rp, col = sc.pattern()
    nb = [set([i]) for i in range(spec.n_verts)]
    for t in spec.tets:
        for a in t:
            nb[a].update(int(b) for b in t)
    for i in range(spec.n_verts):
        assert list(col[rp[i]:rp[i + 1]]) == sorted(nb[i])


def test_lumped_mass_sums_to_total_mass():
    spec = tiny_scene(cells=(2, 3, 2), seed=3)
    sc = O.Scene.from_spec(spec)
    p = spec.rest[spec.tets]
    vol = np.abs(np.linalg.det(np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]], 2))).sum() / 6
    assert abs(sc.lumped_mass().sum() - spec.rho * vol) <= 1e-12 * spec.rho * vol


@pytest.mark.parametrize("seed", range(2))
def test_gradient_and_hessian_are_derivatives_of_the_potential(seed):
    spec = tiny_scene(cells=(2, 1, 1), seed=seed)
    sc = O.Scene.from_spec(spec)
    x = deformed(spec, seed)
    rng = np.random.default_rng(seed + 9)
    xhat = x + 0.01 * rng.standard_normal(x.shape)
    g = sc.gradient(x, xhat)
    Hd = dense(sc, sc.assemble(x))
    free = np.ones(spec.n_verts, bool)
    free[spec.fixed] = False
    h = 1e-7
    fdg = np.zeros_like(x)
    fdH = np.zeros((3 * spec.n_verts, 3 * spec.n_verts))
    for v in np.nonzero(free)[0]:
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, k] += h
            xm[v, k] -= h
            fdg[v, k] = (sc.energy(xp, xhat) - sc.energy(xm, xhat)) / (2 * h)
            fdH[:, 3 * v + k] = (sc.gradient(xp, xhat) - sc.gradient(xm, xhat)).reshape(-1) / (2 * h)
    assert np.abs(g[~free]).max() == 0.0
    assert np.abs(fdg - g).max() <= 1e-6 * np.abs(g).max()
    fm = np.repeat(free, 3)
    assert np.abs(fdH[np.ix_(fm, fm)] - Hd[np.ix_(fm, fm)]).max() <= 1e-6 * np.abs(Hd).max()
    # eliminated rows/columns: identity diagonal, zero coupling
    for v in spec.fixed:
        assert np.array_equal(Hd[3 * v:3 * v + 3, 3 * v:3 * v + 3], np.eye(3))
        row = Hd[3 * v:3 * v + 3].copy()
        row[:, 3 * v:3 * v + 3] = 0
        assert np.all(row == 0) and np.all(Hd[:, 3 * v:3 * v + 3][~np.isin(np.arange(3 * spec.n_verts) // 3, [v])] == 0)


def test_projected_assembly_adds_clamped_difference():
    spec = tiny_scene(cells=(2, 1, 1), seed=4)
    sc = O.Scene.from_spec(spec)
    x = deformed(spec, 4, amp=0.6)
    proj = np.zeros(spec.n_tets, np.uint8)
    proj[[0, 3, 5]] = 1
    d0 = dense(sc, sc.assemble(x))
    d1 = dense(sc, sc.assemble(x, proj))
    dH = sc.project(x, np.array([0, 3, 5], np.int32))
    _, _, He = sc.element_eval(x)
    free = np.ones(spec.n_verts, bool)
    free[spec.fixed] = False
    expect = d0.copy()
    tets = sc.tets()
    for k, e in enumerate([0, 3, 5]):
        # dH^e = Hhat^e - H^e, with Hhat^e's spectrum >= eps (independent LAPACK check)
        w = np.linalg.eigvalsh(He[e] + dH[k])
        assert w.min() >= 1e-8 - 1e-9 * np.abs(w).max()
        for a in range(4):
            for b in range(4):
                i, j = tets[e, a], tets[e, b]
                if free[i] and free[j]:
                    expect[3 * i:3 * i + 3, 3 * j:3 * j + 3] += dH[k][3 * a:3 * a + 3, 3 * b:3 * b + 3]
    assert np.allclose(d1, expect, rtol=0, atol=1e-12 * np.abs(d0).max())


def test_selection_matches_brute_force_heuristic():
    spec = tiny_scene(cells=(3, 2, 2), seed=5)
    sc = O.Scene.from_spec(spec)
    tets = sc.tets()
    rng = np.random.default_rng(11)
    g = rng.standard_normal((spec.n_verts, 3))
    g[spec.fixed] = 0
    r = np.array([np.abs(g[t]).max() for t in tets])
    for delta in [np.inf, 2.0, r[7], 0.5, 1e-13]:
        already = (rng.random(spec.n_tets) < 0.3).astype(np.uint8)
        sel, n = sc.select(g, delta, already)
        expect = (~already.astype(bool)) & ((r > delta) | (delta <= 1e-12))
        assert np.array_equal(sel, expect) and n == expect.sum()
    # ties at equality are not selected (strict inequality)
    sel, _ = sc.select(g, r[7])
    assert not sel[7]
