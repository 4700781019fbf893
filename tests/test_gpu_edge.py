"""Edge cases of the GPU path, each against the oracle's behaviour: degenerate
and out-of-range tets, repeated Dirichlet indices and invalid materials are
rejected by both; the smallest mesh (one free tet in free fall) and a body whose
every vertex is constrained (nothing to solve) step like the oracle."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_21013_gb300")
from oracle import oracle as O  # noqa: E402
from ppn_inputs import tiny_scene  # noqa: E402

TET = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.0, 0.1, 0.0], [0.0, 0.0, 0.1]])


def fp64_params():
    p = P.ppn_default_params()
    p.precision = P.PREC_FP64
    return p


@pytest.mark.parametrize("case", ["coplanar", "index_out_of_range", "repeated_fixed", "nu_half", "dt_zero"])
def test_invalid_scenes_are_rejected_by_both(case):
    rest, tets, fixed, E, nu, rho, dt = TET.copy(), np.array([[0, 1, 2, 3]]), np.zeros(0, np.int32), 1e5, 0.4, 1e3, 0.01
    if case == "coplanar":
        rest[3] = [0.05, 0.05, 0.0]
    elif case == "index_out_of_range":
        tets = np.array([[0, 1, 2, 4]])
    elif case == "repeated_fixed":
        fixed = np.array([1, 1], np.int32)
    elif case == "nu_half":
        nu = 0.5
    elif case == "dt_zero":
        dt = 0.0
    with pytest.raises(P.PPNError) as e:
        P.Scene(rest, tets, fixed, E, nu, rho, dt, fp64_params())
    assert e.value.status == (4 if case == "coplanar" else 1)
    with pytest.raises(ValueError):
        O.Scene(rest, tets, fixed, E, nu, rho, dt)


def test_single_free_tet_falls_like_the_oracle():
    # no constraint and no strain: every vertex follows x_hat (free fall, exact)
    dt = 0.01
    g = P.Scene(TET, [[0, 1, 2, 3]], np.zeros(0, np.int32), 1e5, 0.4, 1e3, dt, fp64_params())
    o = O.Scene(TET, [[0, 1, 2, 3]], np.zeros(0, np.int32), 1e5, 0.4, 1e3, dt)
    for n in range(3):
        rc, x, st = g.step(P.MODE_PPN, 1e-10)
        rco, xo, sto = o.step(O.PPN, 1e-10)
        assert rc == rco == 0
        assert np.abs(x - xo).max() <= 1e-12
    # after 3 steps of implicit Euler from rest: y drops by dt^2 g (1 + 2 + 3)
    assert np.allclose(x[:, 1] - TET[:, 1], -9.81 * dt * dt * 6, rtol=1e-9)


@pytest.mark.parametrize("prec", [P.PREC_FP64, P.PREC_MIXED])
def test_fully_constrained_body_has_nothing_to_solve(prec):
    spec = tiny_scene(cells=(2, 1, 1), seed=5, fixed_face=False)
    fixed = np.arange(spec.n_verts, dtype=np.int32)
    p = P.ppn_default_params()
    p.precision = prec
    g = P.Scene(spec.rest, spec.tets, fixed, spec.E, spec.nu, spec.rho, spec.dt, p)
    o = O.Scene(spec.rest, spec.tets, fixed, spec.E, spec.nu, spec.rho, spec.dt)
    tg = spec.rest + 0.01
    g.set_targets(tg)
    o.set_targets(tg)
    rc, x, st = g.step(P.MODE_PPN, 1e-6)
    rco, xo, sto = o.step(O.PPN, 1e-6)
    assert rc == rco == 0
    assert np.array_equal(xo, tg)
    assert np.abs(x - tg).max() <= 1e-14  # x = X + (t - X) on the GPU: within an ulp of t
    assert st["newton_iters"] == sto["newton_iters"] == 0


def test_step_writes_positions_into_a_caller_buffer():
    # Scene.step(out=...) fills a caller's C-contiguous float64 (n_verts, 3) buffer, here in
    # pinned host memory as the benchmark's end-to-end loop uses it, with the same bits as the
    # default path; a buffer of the wrong shape, type or layout is refused before the call
    torch = pytest.importorskip("torch")
    spec = tiny_scene(cells=(2, 2, 3), seed=7)
    a = P.Scene.from_spec(spec, precision=P.PREC_MIXED)
    b = P.Scene.from_spec(spec, precision=P.PREC_MIXED)
    pinned = torch.empty((spec.n_verts, 3), dtype=torch.float64).pin_memory()
    out = pinned.numpy()
    for n in range(2):
        a.set_targets(spec.targets_at(n))
        b.set_targets(spec.targets_at(n))
        rca, xa, _ = a.step(P.MODE_PPN, 1e-6)
        rcb, xb, _ = b.step(P.MODE_PPN, 1e-6, out=out)
        assert rca == rcb == 0
        assert xb is out
        assert np.array_equal(xa, out)
    for bad in (np.zeros((spec.n_verts, 3), np.float32), np.zeros((spec.n_verts + 1, 3)),
                np.zeros((3, spec.n_verts)).T):
        with pytest.raises(ValueError):
            b.step(P.MODE_PPN, 1e-6, out=bad)
