"""GPU log-barrier contact against analytic obstacles vs the FP64 oracle: drops
onto a plane (every mode) and onto a sphere (indefinite contact elements,
projected by PN and PPN), and stacked boxes in a cylinder under a descending
press plane (moving obstacle).  FP64 mode: relative 1e-5 of the displacement
and +-1 Newton iteration; the mixed mode within its stated bound."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_21013_gb300")
from oracle import oracle as O  # noqa: E402
from ppn_inputs import drop_scene, press_scene  # noqa: E402

MODES = [(P.MODE_NEWTON, O.NEWTON), (P.MODE_PN, O.PN), (P.MODE_PPN, O.PPN), (P.MODE_PDN, O.PDN)]


def run_pair(spec, mode_g, mode_o, steps, tol, prec):
    g = P.Scene.from_spec(spec, precision=prec)
    o = O.Scene.from_spec(spec)
    g.set_obstacles(spec.obstacles_at(-1))  # initial poses
    o.set_obstacles(O.obstacles_from(spec.obstacles_at(-1)))
    out = []
    for n in range(steps):
        obs = spec.obstacles_at(n)
        g.set_obstacles(obs)
        o.set_obstacles(O.obstacles_from(obs))
        rc, x, st = g.step(mode_g, tol)
        rco, xo, sto = o.step(mode_o, tol)
        out.append((rc, x, st, g.iter_stats(), rco, xo, sto))
    return out


@pytest.mark.parametrize("mode_g,mode_o", MODES)
def test_drop_on_plane_fp64_matches_oracle(mode_g, mode_o):
    spec = drop_scene(cells=(3, 3, 3), height=0.002, seed=0)
    for rc, x, st, its, rco, xo, sto in run_pair(spec, mode_g, mode_o, 30, 1e-6, P.PREC_FP64):
        assert rc == rco == 0
        disp = np.abs(xo - spec.rest).max()
        assert np.abs(x - xo).max() <= 1e-5 * disp
        assert abs(st["newton_iters"] - sto["newton_iters"]) <= 1
        assert x[:, 1].min() > 0.0


@pytest.mark.parametrize("mode_g,mode_o", [(P.MODE_PN, O.PN), (P.MODE_PPN, O.PPN)])
def test_drop_on_sphere_projects_contact_elements_like_the_oracle(mode_g, mode_o):
    spec = drop_scene(cells=(3, 3, 3), height=0.002, obstacle="sphere", seed=2)
    for rc, x, st, its, rco, xo, sto in run_pair(spec, mode_g, mode_o, 20, 1e-6, P.PREC_FP64):
        assert rc == rco == 0
        disp = np.abs(xo - spec.rest).max()
        assert np.abs(x - xo).max() <= 1e-5 * disp
        assert abs(st["total_projections"] - sto["total_projections"]) <= spec.n_tets  # tets + contacts


@pytest.mark.parametrize("prec", [P.PREC_FP64, P.PREC_MIXED])
def test_boxes_in_cylinder_under_press_plane(prec):
    spec = press_scene(n=5, boxes=4, press_speed=0.3, dt=1 / 60, seed=1)
    tol = 1e-6 if prec == P.PREC_FP64 else 1e-4
    for n, (rc, x, st, its, rco, xo, sto) in enumerate(run_pair(spec, P.MODE_PPN, O.PPN, 20, tol, prec)):
        assert rc == rco == 0
        disp = np.abs(xo - spec.rest).max()
        assert np.abs(x - xo).max() <= (1e-5 if prec == P.PREC_FP64 else 2e-3) * disp
        assert x[:, 1].min() > 0  # above the ground
        assert (np.hypot(x[:, 0], x[:, 2]) < 0.1).all()  # inside the cylinder
    assert x[:, 1].max() < spec.rest[:, 1].max() - 0.003  # the press compresses the boxes
