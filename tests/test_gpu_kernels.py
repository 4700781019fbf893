"""GPU parity of each pipeline stage against the FP64 oracle, through the C ABI.

Every test feeds the same seeded inputs to a CUDA stage (through a
``ppn_probe_*`` entry point) and to the oracle, and compares element by
element.  FP64 scenes must match to rounding (relative 1e-10 or tighter); the
mixed-precision path (FP32 Hessians, eigensolves, BSR and PCG) to the bounds
derived from FP32 rounding of O(1e2) operations (relative 2e-5 of the
largest entry).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_21013_gb300")
from oracle import oracle as O  # noqa: E402
from ppn_inputs import tiny_scene, twisting_beam_scene  # noqa: E402

TOL = {P.PREC_FP64: 1e-10, P.PREC_MIXED: 2e-5}
PRECS = [P.PREC_FP64, P.PREC_MIXED]


def scene_pair(spec, prec, mirror=False):
    pg, po = P.ppn_default_params(), O.default_params()
    if mirror:
        pg.projection, po.projection = P.PROJ_MIRROR, O.PROJ_MIRROR
    return P.Scene.from_spec(spec, params=pg, precision=prec), O.Scene.from_spec(spec, po)


def deformed(spec, seed, amp=0.2):
    rng = np.random.default_rng(seed)
    x = spec.rest + amp * spec.meta["h"] * rng.standard_normal(spec.rest.shape)
    x[spec.fixed] = spec.rest[spec.fixed]
    return x


def medium_spec(seed=0):
    # several element/vertex tiles and PCG tiles with ragged tails
    return twisting_beam_scene(7, 6, 13, h=0.02, E=1e5, nu=0.45, omega=5.0, dt=1 / 30, seed=seed)


@pytest.mark.parametrize("prec", PRECS)
def test_element_gradients_hessians_energies(prec):
    spec = medium_spec(1)
    g, o = scene_pair(spec, prec)
    x = deformed(spec, 2, amp=0.4)
    psi, ge, He = g.probe_elements(x)
    psi_o, ge_o, He_o = o.element_eval(x)
    # the CUDA path's orientation normalisation is the oracle's
    assert np.array_equal(g.probe_tets(), o.tets())
    tol = TOL[prec]
    assert np.abs(ge - ge_o).max() <= tol * np.abs(ge_o).max()
    assert np.abs(He - He_o).max() <= tol * np.abs(He_o).max()
    # element energies are FP64 in both precisions (Dm^-1 rounded to the storage type)
    etol = 1e-9 if prec == P.PREC_FP64 else 2e-6
    assert np.abs(psi - psi_o).max() <= etol * np.abs(psi_o).max()


@pytest.mark.parametrize("prec", PRECS)
def test_assembled_gradient_norms_and_energy(prec):
    spec = medium_spec(3)
    g, o = scene_pair(spec, prec)
    x = deformed(spec, 4)
    xhat = x + 0.001 * np.random.default_rng(5).standard_normal(x.shape)
    gg, norms, en = g.probe_gradient(x, xhat)
    go = o.gradient(x, xhat)
    tol = TOL[prec]
    assert np.abs(gg - go).max() <= tol * np.abs(go).max()
    assert np.all(gg[spec.fixed] == 0)
    assert abs(norms[0] - np.linalg.norm(go)) <= tol * np.linalg.norm(go)
    assert abs(norms[1] - np.abs(go).max()) <= tol * np.abs(go).max()
    eo = o.energy(x, xhat)
    assert abs(en - eo) <= (1e-11 if prec == P.PREC_FP64 else 2e-6) * abs(eo)


def test_bsr_pattern_is_identical():
    spec = medium_spec(6)
    g, o = scene_pair(spec, P.PREC_MIXED)
    rp, col = g.probe_pattern()
    rpo, colo = o.pattern()
    assert np.array_equal(rp, rpo) and np.array_equal(col, colo)


@pytest.mark.parametrize("prec", PRECS)
def test_assembly_with_and_without_projection(prec):
    spec = medium_spec(7)
    g, o = scene_pair(spec, prec)
    x = deformed(spec, 8, amp=0.6)
    tol = TOL[prec]
    v = g.probe_assemble(x)
    vo = o.assemble(x)
    assert np.abs(v - vo).max() <= tol * np.abs(vo).max()
    proj = (np.random.default_rng(9).random(spec.n_tets) < 0.3).astype(np.uint8)
    v = g.probe_assemble(x, proj)
    vo = o.assemble(x, proj)
    assert np.abs(v - vo).max() <= 4 * tol * np.abs(vo).max()


def test_selection_is_exact_with_ties():
    spec = medium_spec(10)
    g, o = scene_pair(spec, P.PREC_MIXED)
    rng = np.random.default_rng(11)
    grad = rng.standard_normal((spec.n_verts, 3))
    grad[spec.fixed] = 0
    tets = o.tets()
    r = np.abs(grad[tets]).max(axis=(1, 2))
    for delta, frac in [(np.inf, 0.0), (2.0, 0.2), (float(r[5]), 0.1), (0.7, 0.5), (1e-13, 0.0), (-1.0, 0.0)]:
        already = (rng.random(spec.n_tets) < frac).astype(np.uint8)
        sel, n = g.probe_select(grad, delta, already)
        if delta < 0:  # select-all request (PN)
            assert np.array_equal(sel, ~already.astype(bool))
            continue
        sel_o, n_o = o.select(grad, delta, already)
        assert np.array_equal(sel, sel_o) and n == n_o
    # the exact tie r_e == delta is not selected on either side
    sel, _ = g.probe_select(grad, float(r[5]))
    assert not sel[5]


@pytest.mark.parametrize("form", ["warp", "thread"])
@pytest.mark.parametrize("mirror", [False, True])
@pytest.mark.parametrize("prec", PRECS)
def test_projection_updates(prec, mirror, form, monkeypatch):
    # both forms of the clamping kernel: nine lanes per tet (PPN's selection rounds)
    # and one thread per tet (PN's passes over every element)
    monkeypatch.setenv("PPN_PROJECT_THREAD" if form == "thread" else "PPN_PROJECT_WARP", "1")
    spec = medium_spec(12)
    g, o = scene_pair(spec, prec, mirror)
    x = deformed(spec, 13, amp=1.0)
    sel = np.arange(0, spec.n_tets, 7, dtype=np.int32)
    dH = g.probe_project(x, sel)
    dHo = o.project(x, sel)
    _, _, He = o.element_eval(x)
    scale = np.abs(He[sel]).max(axis=(1, 2))
    err = np.abs(dH - dHo).max(axis=(1, 2)) / scale
    assert err.max() <= (1e-9 if prec == P.PREC_FP64 else 2e-5)
    # PSD after projection (independent LAPACK check)
    w = np.linalg.eigvalsh(He[sel] + dH)
    assert (w.min(axis=1) >= 1e-8 - (1e-9 if prec == P.PREC_FP64 else 2e-5) * scale).all()
    # some element really had negative curvature
    assert (np.linalg.eigvalsh(He[sel]).min(axis=1) < -1e-6 * scale).any()


@pytest.mark.parametrize("prec", PRECS)
def test_pcg_on_spd_and_indefinite_systems(prec):
    spec = medium_spec(14)
    g, o = scene_pair(spec, prec)
    x = spec.rest  # rest state: K + M/dt^2 is SPD
    vals = o.assemble(x)
    rp, col = o.pattern()
    b = np.random.default_rng(16).standard_normal((spec.n_verts, 3))
    b[spec.fixed] = 0
    xg, info = g.probe_pcg(vals, b, rel_tol=1e-4)
    xo, info_o = O.pcg_bsr(rp, col, vals, b.reshape(-1), rel_tol=1e-4, max_iter=5000)
    assert not info["ind"] and not info_o["ind"]
    # same algorithm: the residual criterion holds and the iteration counts agree closely
    A = lambda y: np.einsum("kij,kj->ki", vals, y.reshape(-1, 3)[col]).reshape(-1)
    r = b.reshape(-1) - np.add.reduceat(np.einsum("kij,kj->ki", vals, xg[col]), rp[:-1]).reshape(-1)
    assert np.linalg.norm(r) <= 1e-4 * np.linalg.norm(b) * (1.0 + (1e-6 if prec == P.PREC_FP64 else 5e-2))
    if prec == P.PREC_FP64:
        assert abs(info["iters"] - info_o["iters"]) <= 1
        assert np.abs(xg.reshape(-1) - xo).max() <= 1e-6 * np.abs(xo).max()
    else:
        assert abs(info["iters"] - info_o["iters"]) <= max(3, info_o["iters"] // 10)
    # indefinite: a strongly compressed state has negative-curvature directions
    xi = deformed(spec, 17, amp=3.0)
    vi = o.assemble(xi)
    bi = b.copy()
    xgi, infi = g.probe_pcg(vi, bi, rel_tol=1e-8)
    xoi, infoi = O.pcg_bsr(rp, col, vi, bi.reshape(-1), rel_tol=1e-8, max_iter=5000)
    assert infi["ind"] == infoi["ind"] == True  # noqa: E712
    del A


def test_pcg_zero_rhs_and_nonspd_diagonal():
    spec = medium_spec(18)
    g, o = scene_pair(spec, P.PREC_MIXED)
    vals = o.assemble(spec.rest)
    xg, info = g.probe_pcg(vals, np.zeros((spec.n_verts, 3)))
    assert info["iters"] == 0 and not info["ind"] and np.all(xg == 0)
    rp, col = o.pattern()
    v2 = vals.copy()
    free = np.setdiff1d(np.arange(spec.n_verts), spec.fixed)[0]
    k = rp[free] + np.nonzero(col[rp[free]:rp[free + 1]] == free)[0][0]
    v2[k] = np.diag([-9.0, 5.0, 1.0])  # the paper's Q = A + B + C in a diagonal block
    b = np.ones((spec.n_verts, 3))
    b[spec.fixed] = 0
    xg, info = g.probe_pcg(v2, b)
    assert info["ind"] and info["precond_fail"] and info["iters"] == 0


def test_orientation_normalisation_on_permuted_tets():
    # corners given in random order, so about half the tets arrive negatively oriented:
    # both sides swap corners 2 and 3 of exactly those, and every normalised tet has
    # det[x1-x0, x2-x0, x3-x0] > 0 at rest
    from ppn_inputs.scenes import SceneSpec

    base = medium_spec(24)
    rng = np.random.default_rng(25)
    tets = np.array([t[rng.permutation(4)] for t in base.tets], dtype=np.int32)
    spec = SceneSpec(**{**base.__dict__, "tets": tets})
    g, o = scene_pair(spec, P.PREC_MIXED)
    tg, to = g.probe_tets(), o.tets()
    assert np.array_equal(tg, to)
    X = spec.rest
    D = np.stack([X[tg[:, k]] - X[tg[:, 0]] for k in (1, 2, 3)], axis=2)
    assert (np.linalg.det(D) > 0).all()
    flipped = (tg != tets).any(axis=1)
    assert 0.3 < flipped.mean() < 0.7
    assert np.array_equal(tg[flipped][:, [0, 1, 3, 2]], tets[flipped])
    assert np.array_equal(tg[~flipped], tets[~flipped])


def test_tiny_meshes_and_ragged_sizes():
    for cells in [(1, 1, 1), (2, 1, 1), (3, 2, 1)]:
        spec = tiny_scene(cells=cells, seed=sum(cells))
        g, o = scene_pair(spec, P.PREC_FP64)
        x = deformed(spec, 1, amp=0.3)
        _, ge, He = g.probe_elements(x)
        _, ge_o, He_o = o.element_eval(x)
        assert np.abs(He - He_o).max() <= 1e-10 * np.abs(He_o).max()
        v = g.probe_assemble(x)
        assert np.abs(v - o.assemble(x)).max() <= 1e-10 * np.abs(v).max()


def _probe_layout(spec, vals, b, env, monkeypatch, rel_tol=1e-6):
    for k in ("PPN_PCG_STREAM", "PPN_PCG_SR_GLOBAL", "PPN_PCG_NO_HALO"):
        monkeypatch.delenv(k, raising=False)
    if env:
        monkeypatch.setenv(env, "1")
    sc = P.Scene.from_spec(spec, precision=P.PREC_MIXED)
    x, info = sc.probe_pcg(vals, b, rel_tol=rel_tol)
    layout = P.PCG_LAYOUTS[sc.info()["pcg_layout"]]
    sc.close()
    return x, info, layout


def test_single_reduction_pcg_layouts(monkeypatch):
    # the FP32 kernel with the halo replicated (the default where it fits), with the
    # neighbours' u gathered instead, with the BSR blocks streamed from global memory,
    # and with the vectors in global memory too, performs the same operations in the
    # same order: the same bits
    spec = medium_spec(19)  # 546 rows: 5 CTAs of one tile, the last one ragged
    o = O.Scene.from_spec(spec)
    vals = o.assemble(spec.rest)  # K + M / dt^2 at rest: SPD
    rp, col = o.pattern()
    b = np.random.default_rng(21).standard_normal((spec.n_verts, 3))
    b[spec.fixed] = 0
    runs = {env: _probe_layout(spec, vals, b, env, monkeypatch)
            for env in (None, "PPN_PCG_NO_HALO", "PPN_PCG_STREAM", "PPN_PCG_SR_GLOBAL")}
    assert [r[2] for r in runs.values()] == ["halo", "resident", "streamed", "global"]
    ref = runs[None]
    for x, info, _ in runs.values():
        assert info == ref[1] and np.array_equal(x, ref[0])
    # solved to 1e-6 in FP32: the true residual well within 1e-4
    assert not ref[1]["ind"] and not ref[1]["hit_max"] and ref[1]["iters"] > 20
    r = b.reshape(-1) - np.add.reduceat(np.einsum("kij,kj->ki", vals, ref[0][col]), rp[:-1]).reshape(-1)
    assert np.linalg.norm(r) <= 1e-4 * np.linalg.norm(b)


def test_halo_layout_exits_like_the_resident_one(monkeypatch):
    # negative curvature (an indefinite system) and a failed diagonal block end the
    # halo layout's solve at the same iteration, with the same iterate
    spec = medium_spec(23)
    o = O.Scene.from_spec(spec)
    vi = o.assemble(deformed(spec, 17, amp=3.0))
    b = np.random.default_rng(5).standard_normal((spec.n_verts, 3))
    b[spec.fixed] = 0
    h = _probe_layout(spec, vi, b, None, monkeypatch, rel_tol=1e-8)
    r = _probe_layout(spec, vi, b, "PPN_PCG_NO_HALO", monkeypatch, rel_tol=1e-8)
    assert h[2] == "halo" and r[2] == "resident"
    assert h[1]["ind"] and h[1] == r[1] and np.array_equal(h[0], r[0])
    rp, col = o.pattern()
    v2 = o.assemble(spec.rest)
    free = np.setdiff1d(np.arange(spec.n_verts), spec.fixed)[-1]
    k = rp[free] + np.nonzero(col[rp[free]:rp[free + 1]] == free)[0][0]
    v2[k] = np.diag([-9.0, 5.0, 1.0])
    h = _probe_layout(spec, v2, b, None, monkeypatch)
    assert h[2] == "halo" and h[1]["precond_fail"] and h[1]["ind"] and h[1]["iters"] == 0


def test_tuned_streamed_layouts_give_identical_steps(monkeypatch):
    # 60k vertices: 3 PCG tiles per CTA, too many blocks for the resident layout, so
    # the tuner alternates the two streamed layouts over the first launches; the
    # steps equal those of a run held to the global-memory layout, bit for bit
    spec = twisting_beam_scene(20, 20, 150, h=0.01, E=1e6, nu=0.45, omega=2.0, dt=1.0 / 30.0, seed=3)
    out = []
    for env in (None, "PPN_PCG_SR_GLOBAL"):
        if env:
            monkeypatch.setenv(env, "1")
        sc = P.Scene.from_spec(spec, precision=P.PREC_MIXED)
        xs = []
        for n in range(3):
            sc.set_targets(spec.targets_at(n))
            rc, x, st = sc.step(P.MODE_PPN, 1e-4)
            assert rc == 0
            xs.append((x, st["newton_iters"], st["total_cg_iters"]))
        sc.close()
        out.append(xs)
    for (xa, na, ca), (xb, nb, cb) in zip(*out):
        assert na == nb and ca == cb
        assert np.array_equal(xa, xb)


def _dense(rp, col, vals, n):
    A = np.zeros((3 * n, 3 * n))
    for r in range(n):
        for k in range(rp[r], rp[r + 1]):
            A[3 * r:3 * r + 3, 3 * col[k]:3 * col[k] + 3] = vals[k]
    return A


@pytest.mark.parametrize("prec", PRECS)
def test_pcg_curvature_exit_follows_the_oracle(prec):
    # Indefinite systems of decreasing negative curvature: the Hessian of a compressed
    # state with its spectrum shifted so that the most negative eigenvalue is a fraction
    # f of the original one.  The smaller f, the later CG meets negative curvature.  The
    # FP32 kernel forms the curvature of each direction by the single-reduction
    # recurrence d^T A d = delta - beta gamma / alpha_prev, not by a direct product; it
    # must leave with ind at the oracle's iteration (FP64: exactly up to one iteration;
    # mixed: within 15 %, at least 2), and a shift that makes the system SPD must not
    # report ind.
    spec = medium_spec(14)
    g, o = scene_pair(spec, prec)
    rp, col = o.pattern()
    n = spec.n_verts
    vi = o.assemble(deformed(spec, 17, amp=0.3))
    lmin = np.linalg.eigvalsh(_dense(rp, col, vi, n))[0]
    assert lmin < 0
    diag = np.array([rp[r] + np.nonzero(col[rp[r]:rp[r + 1]] == r)[0][0] for r in range(n)])
    free = np.setdiff1d(np.arange(n), spec.fixed)
    b = np.random.default_rng(16).standard_normal((n, 3))
    b[spec.fixed] = 0
    exits = []
    for f in (0.5, 0.1, 0.02, 0.005, 0.001):
        v2 = vi.copy()
        v2[diag[free]] += (-lmin * (1.0 - f)) * np.eye(3)
        xg, info = g.probe_pcg(v2, b, rel_tol=1e-8)
        xo, info_o = O.pcg_bsr(rp, col, v2, b.reshape(-1), rel_tol=1e-8, max_iter=5000)
        assert info_o["ind"] and info["ind"], f
        assert not info["precond_fail"]
        slack = 1 if prec == P.PREC_FP64 else max(2, int(0.15 * info_o["iters"]))
        assert abs(info["iters"] - info_o["iters"]) <= slack, (f, info, info_o)
        exits.append(info_o["iters"])
    assert exits == sorted(exits) and exits[-1] >= 3 * exits[0]
    # shifted past zero: SPD, no curvature exit on either side
    v2 = vi.copy()
    v2[diag[free]] += (-lmin * 1.05) * np.eye(3)
    xg, info = g.probe_pcg(v2, b, rel_tol=1e-4)
    xo, info_o = O.pcg_bsr(rp, col, v2, b.reshape(-1), rel_tol=1e-4, max_iter=5000)
    assert not info_o["ind"] and not info["ind"] and not info["hit_max"]


def test_l2_priority_of_streamed_blocks_changes_no_bits(monkeypatch):
    # the autotuner's L2 priority of the streamed BSR blocks (evict-first or normal) is a
    # cache hint only: each streamed layout gives the same iterates at both priorities
    spec = medium_spec(28)
    o = O.Scene.from_spec(spec)
    vals = o.assemble(spec.rest)
    b = np.random.default_rng(29).standard_normal((spec.n_verts, 3))
    b[spec.fixed] = 0
    runs = []
    for env in ("PPN_PCG_STREAM", "PPN_PCG_SR_GLOBAL"):
        for keep in (False, True):
            if keep:
                monkeypatch.setenv("PPN_PCG_L2_KEEP", "1")
            else:
                monkeypatch.delenv("PPN_PCG_L2_KEEP", raising=False)
            runs.append(_probe_layout(spec, vals, b, env, monkeypatch))
    monkeypatch.delenv("PPN_PCG_L2_KEEP", raising=False)
    assert [r[2] for r in runs] == ["streamed", "streamed", "global", "global"]
    for x, info, _ in runs:
        assert info == runs[0][1] and np.array_equal(x, runs[0][0])
    # the tuner reports its shape classes through the C ABI
    rec = P.ppn.pcg_tuning()
    assert isinstance(rec, list)
