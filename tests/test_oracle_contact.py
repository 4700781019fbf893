"""Pins of the oracle's frictionless log-barrier contact against analytic
surfaces (the IPC potentials of the paper's contact scenes, Sec. 5.1): the
barrier and the distances against closed forms and finite differences, the
contact time against the surface equations, and a drop onto the ground."""

import numpy as np
import pytest

from oracle import oracle as O
from ppn_inputs import drop_scene, press_scene

DHAT = 1e-3


def test_barrier_closed_form_and_derivatives():
    b, db, ddb = O.barrier(DHAT, DHAT)
    assert b == db == ddb == 0.0  # C2-continuous at the activation distance
    assert O.barrier(2 * DHAT, DHAT) == (0.0, 0.0, 0.0)
    for d in (1e-6, 1e-4, 5e-4, 9e-4):
        b, db, ddb = O.barrier(d, DHAT)
        assert b == pytest.approx(-(d - DHAT) ** 2 * np.log(d / DHAT), rel=1e-14)
        assert b > 0 and db < 0 and ddb > 0  # repulsive and convex in d
        h = 1e-7 * d
        assert db == pytest.approx((O.barrier(d + h, DHAT)[0] - O.barrier(d - h, DHAT)[0]) / (2 * h), rel=1e-6)
        assert ddb == pytest.approx((O.barrier(d + h, DHAT)[1] - O.barrier(d - h, DHAT)[1]) / (2 * h), rel=1e-6)
    assert O.barrier(1e-12, DHAT)[0] > O.barrier(1e-9, DHAT)[0] > O.barrier(1e-6, DHAT)[0]  # grows without bound
    assert O.barrier(0.0, DHAT)[0] == np.inf


OBSTACLES = [
    O.obstacle(O.OBST_PLANE, (0.1, 0.2, -0.3), np.array([1.0, 2.0, 2.0]) / 3.0),
    O.obstacle(O.OBST_CYLINDER_IN, (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 0.5),
    O.obstacle(O.OBST_SPHERE_OUT, (0.3, -0.1, 0.2), r=0.25),
]


@pytest.mark.parametrize("o", OBSTACLES, ids=["plane", "cylinder_in", "sphere_out"])
def test_distance_gradient_and_hessian_match_finite_differences(o):
    rng = np.random.default_rng(0)
    for _ in range(5):
        x = rng.uniform(-0.35, 0.35, 3)
        if o.type == O.OBST_SPHERE_OUT:
            x = np.array(o.p) + (o.r + 0.1) * x / np.linalg.norm(x)
        d, g, H = O.obstacle_eval(o, x)
        h = 1e-6
        gf = np.array([(O.obstacle_eval(o, x + h * e)[0] - O.obstacle_eval(o, x - h * e)[0]) / (2 * h) for e in np.eye(3)])
        Hf = np.array([(O.obstacle_eval(o, x + h * e)[1] - O.obstacle_eval(o, x - h * e)[1]) / (2 * h) for e in np.eye(3)])
        assert np.allclose(g, gf, atol=1e-8)
        assert np.allclose(H, Hf, atol=1e-6)
        assert np.allclose(H, H.T)
    # closed forms
    x = np.array([0.2, 0.4, 0.1])
    if o.type == O.OBST_PLANE:
        assert O.obstacle_eval(o, x)[0] == pytest.approx(np.dot(o.a, x - np.array(o.p)))
    if o.type == O.OBST_CYLINDER_IN:
        assert O.obstacle_eval(o, x)[0] == pytest.approx(0.5 - np.hypot(0.2, 0.1))
    if o.type == O.OBST_SPHERE_OUT:
        assert O.obstacle_eval(o, x)[0] == pytest.approx(np.linalg.norm(x - np.array(o.p)) - 0.25)


@pytest.mark.parametrize("o", OBSTACLES, ids=["plane", "cylinder_in", "sphere_out"])
def test_contact_time_reaches_the_surface_first(o):
    rng = np.random.default_rng(1)
    hits = 0
    for _ in range(50):
        x = rng.uniform(-0.3, 0.3, 3)
        if o.type == O.OBST_SPHERE_OUT:
            x = np.array(o.p) + (o.r + 0.05) * x / np.linalg.norm(x)
        d0 = O.obstacle_eval(o, x)[0]
        if d0 <= 0:
            continue
        dx = rng.standard_normal(3)
        g = O.obstacle_ccd(o, x, dx)
        if np.isinf(g):
            # never reaches the surface: distance stays positive along the ray
            assert all(O.obstacle_eval(o, x + t * dx)[0] > 0 for t in (0.5, 1, 5, 50))
            continue
        hits += 1
        assert g > 0
        assert abs(O.obstacle_eval(o, x + g * dx)[0]) <= 1e-12 * max(1.0, np.linalg.norm(dx) * g)
        assert all(O.obstacle_eval(o, x + t * g * dx)[0] > 0 for t in (0.1, 0.5, 0.9, 0.999))
    assert hits > 5


def scene_with_obstacles(spec, params=None):
    sc = O.Scene.from_spec(spec, params)
    sc.set_obstacles(O.obstacles_from(spec.obstacles_at(0)))
    return sc


def test_scene_gradient_and_hessian_include_the_barrier():
    spec = drop_scene(cells=(2, 2, 2), height=0.0008, seed=1)  # the lowest vertices start inside dhat
    sc = scene_with_obstacles(spec)
    x = spec.rest.copy()
    xhat = x + 1e-4 * np.random.default_rng(2).standard_normal(x.shape)
    g = sc.gradient(x, xhat)
    h = 1e-8
    rng = np.random.default_rng(3)
    for _ in range(3):
        v = rng.standard_normal(x.shape)
        dE = (sc.energy(x + h * v, xhat) - sc.energy(x - h * v, xhat)) / (2 * h)
        assert dE == pytest.approx(float((g * v).sum()), rel=1e-5)
    # the assembled Hessian is the derivative of the gradient, contact terms included
    vals = sc.assemble(x)
    rp, col = sc.pattern()
    v = rng.standard_normal(x.shape)
    Hv = np.zeros_like(x)
    for i in range(spec.n_verts):
        for k in range(rp[i], rp[i + 1]):
            Hv[i] += vals[k] @ v[col[k]]
    dg = (sc.gradient(x + h * v, xhat) - sc.gradient(x - h * v, xhat)) / (2 * h)
    assert np.allclose(Hv, dg, rtol=1e-4, atol=1e-6 * np.abs(dg).max())
    # some vertices are in contact: the barrier changes the gradient
    sc0 = O.Scene.from_spec(spec)
    assert np.abs(sc0.gradient(x, xhat) - g).max() > 1e-3


@pytest.mark.parametrize("mode", [O.NEWTON, O.PN, O.PPN, O.PDN])
def test_drop_onto_the_ground_stays_feasible_and_comes_to_rest(mode):
    spec = drop_scene(cells=(3, 3, 3), height=0.002, seed=0)
    sc = scene_with_obstacles(spec)
    ymin = []
    for n in range(40):
        rc, x, st = sc.step(mode, 1e-6)
        assert rc == 0
        for it in sc.iter_stats():  # descent, up to the line search's rounding slack
            assert it["dir_deriv"] < 0 and it["energy_new"] <= it["energy"] + 1e-12 * abs(it["energy"])
        ymin.append(x[:, 1].min())
    assert min(ymin) > 0.0  # never penetrates the ground
    assert ymin[0] < spec.rest[:, 1].min()  # it does fall
    _, v = sc.get_state()
    assert np.abs(v).max() < 0.05  # and comes (nearly) to rest on the barrier
    assert ymin[-1] < DHAT


def test_convex_obstacle_contact_is_projected_by_pn_and_ppn():
    # landing on a sphere: the barrier Hessian b' hess(d) is negative along the surface,
    # so contact elements are indefinite and PN clamps them; PPN projects only as needed
    spec = drop_scene(cells=(3, 3, 3), height=0.002, obstacle="sphere", seed=2)
    totals = {}
    for mode in (O.PN, O.PPN):
        sc = scene_with_obstacles(spec)
        tot = 0
        for n in range(25):
            rc, x, st = sc.step(mode, 1e-6)
            assert rc == 0
            tot += st["total_projections"]
            sph = spec.obstacles_at(n)[0]
            assert (np.linalg.norm(x - np.array(sph[1]), axis=1) > sph[3]).all()
        totals[mode] = tot
    assert totals[O.PN] > 25 * spec.n_tets  # tets plus contact elements every iteration
    assert totals[O.PPN] < totals[O.PN]


def test_moving_press_plane_is_held_back_by_the_bodies():
    # the press plane may advance toward the bodies by at most ccd_safety x the smallest
    # vertex distance per step, so the state stays feasible although the requested
    # motion (5 mm per step) is larger than the gap the bodies leave
    spec = press_scene(n=5, boxes=4, press_speed=0.3, dt=1 / 60, seed=1)
    sc = O.Scene.from_spec(spec)
    sc.set_obstacles(O.obstacles_from(spec.obstacles_at(-1)))
    top0 = spec.rest[:, 1].max()
    for n in range(12):
        sc.set_obstacles(O.obstacles_from(spec.obstacles_at(n)))
        rc, x, st = sc.step(O.PPN, 1e-6)
        assert rc == 0
        assert x[:, 1].min() > 0 and (np.hypot(x[:, 0], x[:, 2]) < 0.1).all()
    assert x[:, 1].max() < top0 - 0.003  # compressed by the press
    assert x[:, 1].max() > spec.obstacles_at(11)[2][1][1]  # which lags behind its requested pose
    # a state that an obstacle does not leave feasible is rejected
    bad = O.Scene.from_spec(spec)
    bad.set_obstacles(O.obstacles_from([("plane", (0.0, 0.01, 0.0), (0.0, 1.0, 0.0), 0.0)]))
    rc, _, _ = bad.step(O.PPN, 1e-6)
    assert rc == 1
