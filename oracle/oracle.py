"""ctypes binding of the FP64 CPU oracle (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module.  It loads ``liboracle.so`` (built from the C++ sources beside it) and
marshals numpy arrays; all arithmetic happens in the C++ oracle.
"""

from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build

NEWTON, PN, PPN, PDN = 0, 1, 2, 3
PROJ_CLAMP, PROJ_MIRROR = 0, 1
OBST_PLANE, OBST_CYLINDER_IN, OBST_SPHERE_OUT = 0, 1, 2


class Params(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("eps_delta", C.c_double),
                ("eig_eps", C.c_double), ("pcg_rel_tol", C.c_double), ("armijo_c", C.c_double),
                ("pcg_max_iter", C.c_int), ("newton_max_iter", C.c_int),
                ("ls_max_halvings", C.c_int), ("tol_kind", C.c_int), ("init_guess", C.c_int),
                ("pdn_countdown", C.c_int), ("projection", C.c_int), ("grad_floor", C.c_double),
                ("ls_slack", C.c_double), ("contact_kappa", C.c_double), ("contact_dhat", C.c_double),
                ("ccd_safety", C.c_double), ("dirichlet_penalty", C.c_double), ("tie_band", C.c_double)]


class Obstacle(C.Structure):
    _fields_ = [("type", C.c_int), ("p", C.c_double * 3), ("a", C.c_double * 3), ("r", C.c_double)]


def obstacle(kind, p, a=(0.0, 0.0, 0.0), r=0.0) -> Obstacle:
    o = Obstacle()
    o.type = kind
    o.p[:] = [float(v) for v in p]
    o.a[:] = [float(v) for v in a]
    o.r = float(r)
    return o


class IterStats(C.Structure):
    _fields_ = [("newton_iter", C.c_int), ("pcg_attempts", C.c_int), ("cg_iters", C.c_int),
                ("n_new_projected", C.c_int), ("n_projected_total", C.c_int),
                ("ls_halvings", C.c_int), ("fallback", C.c_int), ("precond_fail", C.c_int),
                ("grad_norm2", C.c_double), ("grad_norminf", C.c_double), ("delta", C.c_double),
                ("gamma", C.c_double), ("energy", C.c_double), ("energy_new", C.c_double),
                ("dir_deriv", C.c_double)]


class Attempt(C.Structure):
    _fields_ = [("newton_iter", C.c_int), ("attempt", C.c_int), ("n_new_projected", C.c_int),
                ("ind", C.c_int), ("cg_iters", C.c_int), ("delta", C.c_double), ("n_ties", C.c_int)]


class StepStats(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("total_projections", C.c_int),
                ("total_cg_iters", C.c_int), ("total_attempts", C.c_int), ("status", C.c_int),
                ("n_ties", C.c_int)]


HOOK = C.CFUNCTYPE(C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p)

_lib = None


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _lp(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _u8(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def lib():
    global _lib
    if _lib is not None:
        return _lib
    L = C.CDLL(_build.build())
    D, I, I64, P = C.c_double, C.c_int, C.c_int64, C.c_void_p
    pd, pi, pl, pu = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_uint8)
    sig = {
        "ora_default_params": (Params, []),
        "ora_num_threads": (I, []),
        "ora_set_num_threads": (None, [I]),
        "ora_last_error": (C.c_char_p, []),
        "ora_lame": (None, [D, D, pd, pd]),
        "ora_snh_psi": (D, [pd, D, D]),
        "ora_snh_pk1": (None, [pd, D, D, pd]),
        "ora_snh_dpdf": (None, [pd, D, D, pd]),
        "ora_tet_eval": (I, [pd, pd, D, D, pd, pd, pd]),
        "ora_eigh": (I, [I, pd, pd, pd]),
        "ora_clamp": (I, [I, pd, D, pd, pd]),
        "ora_project": (I, [I, pd, D, I, pd, pd]),
        "ora_barrier": (I, [D, D, pd, pd, pd]),
        "ora_obstacle_eval": (I, [C.POINTER(Obstacle), pd, pd, pd, pd]),
        "ora_obstacle_ccd": (D, [C.POINTER(Obstacle), pd, pd]),
        "ora_scene_set_obstacles": (None, [P, C.POINTER(Obstacle), I]),
        "ora_pcg_bsr": (I, [I64, pl, pi, pd, pd, D, I, pd, C.POINTER(C.c_int)]),
        "ora_scene_create": (P, [pd, I64, pi, I64, D, D, D, D, pd, pi, I64, C.POINTER(Params)]),
        "ora_scene_destroy": (None, [P]),
        "ora_scene_nnzb": (I64, [P]),
        "ora_scene_pattern": (None, [P, pl, pi]),
        "ora_scene_tets": (None, [P, pi]),
        "ora_scene_lumped_mass": (None, [P, pd]),
        "ora_scene_set_params": (None, [P, C.POINTER(Params)]),
        "ora_scene_set_targets": (I, [P, pd]),
        "ora_scene_get_state": (None, [P, pd, pd]),
        "ora_scene_set_state": (None, [P, pd, pd]),
        "ora_scene_xhat": (None, [P, pd]),
        "ora_scene_set_solve_hook": (None, [P, HOOK, P]),
        "ora_scene_energy": (D, [P, pd, pd]),
        "ora_scene_gradient": (None, [P, pd, pd, pd]),
        "ora_scene_element_eval": (None, [P, pd, pd, pd, pd]),
        "ora_scene_assemble": (None, [P, pd, pu, pd]),
        "ora_scene_select": (I64, [P, pd, D, pu, pu]),
        "ora_scene_project": (None, [P, pd, pi, I64, pd]),
        "ora_scene_step": (I, [P, I, D, pd, C.POINTER(StepStats)]),
        "ora_scene_iter_stats": (I, [P, C.POINTER(IterStats), I]),
        "ora_scene_attempts": (I, [P, C.POINTER(Attempt), I]),
        "ora_scene_attempt_selection": (I64, [P, I, pi, I64]),
        "ora_scene_set_record": (None, [P, I]),
        "ora_scene_iteration_gradient": (I, [P, I, pd]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def default_params() -> Params:
    return lib().ora_default_params()


def num_threads() -> int:
    """Threads of the oracle's parallel loops (OMP_NUM_THREADS)."""
    return int(lib().ora_num_threads())


def set_num_threads(n: int):
    lib().ora_set_num_threads(int(n))


def lame(E, nu):
    mu, lam = C.c_double(), C.c_double()
    lib().ora_lame(E, nu, C.byref(mu), C.byref(lam))
    return mu.value, lam.value


def _f9(F):
    return np.ascontiguousarray(np.asarray(F, dtype=np.float64).reshape(9))


def snh_psi(F, mu, lam):
    return lib().ora_snh_psi(_dp(_f9(F)), mu, lam)


def snh_pk1(F, mu, lam):
    P = np.zeros(9)
    lib().ora_snh_pk1(_dp(_f9(F)), mu, lam, _dp(P))
    return P.reshape(3, 3)


def snh_dpdf(F, mu, lam):
    A = np.zeros(81)
    lib().ora_snh_dpdf(_dp(_f9(F)), mu, lam, _dp(A))
    return A.reshape(9, 9)


def tet_eval(X, x, mu, lam):
    X = np.ascontiguousarray(np.asarray(X, np.float64).reshape(12))
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(12))
    psi = C.c_double()
    g = np.zeros(12)
    H = np.zeros(144)
    rc = lib().ora_tet_eval(_dp(X), _dp(x), mu, lam, C.byref(psi), _dp(g), _dp(H))
    if rc:
        raise ValueError(f"ora_tet_eval failed ({rc})")
    return psi.value, g, H.reshape(12, 12)


def eigh(A):
    A = np.ascontiguousarray(np.asarray(A, np.float64))
    n = A.shape[0]
    w = np.zeros(n)
    Q = np.zeros((n, n))
    lib().ora_eigh(n, _dp(A), _dp(w), _dp(Q))
    return w, Q


def clamp(H, eps=1e-8):
    H = np.ascontiguousarray(np.asarray(H, np.float64))
    n = H.shape[0]
    Hh = np.zeros((n, n))
    dH = np.zeros((n, n))
    lib().ora_clamp(n, _dp(H), eps, _dp(Hh), _dp(dH))
    return Hh, dH


def project(H, eps=1e-8, kind=PROJ_CLAMP):
    """Hhat = Q f(D) Q^T and dH = Hhat - H with f = max(lambda, eps) (clamp) or
    max(|lambda|, eps) (mirror)."""
    H = np.ascontiguousarray(np.asarray(H, np.float64))
    n = H.shape[0]
    Hh = np.zeros((n, n))
    dH = np.zeros((n, n))
    rc = lib().ora_project(n, _dp(H), eps, int(kind), _dp(Hh), _dp(dH))
    if rc:
        raise ValueError(f"ora_project failed ({rc})")
    return Hh, dH


_KINDS = {"plane": OBST_PLANE, "cylinder_in": OBST_CYLINDER_IN, "sphere_out": OBST_SPHERE_OUT}


def obstacles_from(spec_list):
    """ora_obstacle structs from (kind, point, axis_or_normal, radius) tuples."""
    return [obstacle(_KINDS[k], p, a, r) for k, p, a, r in spec_list]


def barrier(d, dhat):
    """(b, b', b'') of the log barrier at distance d."""
    out = [C.c_double(), C.c_double(), C.c_double()]
    lib().ora_barrier(float(d), float(dhat), *[C.byref(o) for o in out])
    return tuple(o.value for o in out)


def obstacle_eval(o, x):
    """(d, grad d, hess d) of an obstacle at point x."""
    x = np.ascontiguousarray(x, np.float64)
    d = C.c_double()
    g = np.zeros(3)
    H = np.zeros((3, 3))
    rc = lib().ora_obstacle_eval(C.byref(o), _dp(x), C.byref(d), _dp(g), _dp(H))
    if rc:
        raise ValueError("obstacle evaluation failed")
    return d.value, g, H


def obstacle_ccd(o, x, dx):
    x = np.ascontiguousarray(x, np.float64)
    dx = np.ascontiguousarray(dx, np.float64)
    return lib().ora_obstacle_ccd(C.byref(o), _dp(x), _dp(dx))


def pcg_bsr(row_ptr, col, vals, b, rel_tol=1e-4, max_iter=1000):
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    vals = np.ascontiguousarray(vals, np.float64).reshape(-1)
    b = np.ascontiguousarray(b, np.float64).reshape(-1)
    x = np.zeros_like(b)
    info = (C.c_int * 4)()
    lib().ora_pcg_bsr(len(row_ptr) - 1, _lp(row_ptr), _ip(col), _dp(vals), _dp(b), rel_tol,
                      max_iter, _dp(x), info)
    return x, {"iters": info[0], "ind": bool(info[1]), "precond_fail": bool(info[2]),
               "hit_max": bool(info[3])}


class Scene:
    """An oracle scene built from a :class:`ppn_inputs.SceneSpec`-like description."""

    def __init__(self, rest, tets, fixed, E, nu, rho, dt, gravity=(0.0, -9.81, 0.0),
                 params: Params | None = None):
        L = lib()
        self.rest = np.ascontiguousarray(rest, np.float64)
        tets = np.ascontiguousarray(tets, np.int32)
        fixed = np.ascontiguousarray(fixed, np.int32)
        self.n_verts = self.rest.shape[0]
        self.n_tets = tets.shape[0]
        self.n_fixed = fixed.shape[0]
        self.fixed = fixed
        g = np.ascontiguousarray(gravity, np.float64)
        p = params if params is not None else default_params()
        self._h = L.ora_scene_create(_dp(self.rest), self.n_verts, _ip(tets), self.n_tets, E, nu,
                                     rho, dt, _dp(g), _ip(fixed), self.n_fixed, C.byref(p))
        if not self._h:
            raise ValueError(L.ora_last_error().decode())
        self.dt = dt
        self._hook = None

    @classmethod
    def from_spec(cls, spec, params: Params | None = None):
        return cls(spec.rest, spec.tets, spec.fixed, spec.E, spec.nu, spec.rho, spec.dt,
                   spec.gravity, params)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ora_scene_destroy(h)
            self._h = None

    # --- structure ---
    @property
    def nnzb(self) -> int:
        return int(lib().ora_scene_nnzb(self._h))

    def pattern(self):
        rp = np.zeros(self.n_verts + 1, np.int64)
        col = np.zeros(self.nnzb, np.int32)
        lib().ora_scene_pattern(self._h, _lp(rp), _ip(col))
        return rp, col

    def tets(self):
        t = np.zeros((self.n_tets, 4), np.int32)
        lib().ora_scene_tets(self._h, _ip(t))
        return t

    def lumped_mass(self):
        m = np.zeros(self.n_verts)
        lib().ora_scene_lumped_mass(self._h, _dp(m))
        return m

    def set_obstacles(self, obstacles):
        arr = (Obstacle * max(1, len(obstacles)))(*obstacles)
        lib().ora_scene_set_obstacles(self._h, arr, len(obstacles))

    def set_params(self, p: Params):
        lib().ora_scene_set_params(self._h, C.byref(p))

    # --- state ---
    def set_targets(self, xyz):
        xyz = np.ascontiguousarray(xyz, np.float64)
        lib().ora_scene_set_targets(self._h, _dp(xyz))

    def get_state(self):
        x = np.zeros((self.n_verts, 3))
        v = np.zeros((self.n_verts, 3))
        lib().ora_scene_get_state(self._h, _dp(x), _dp(v))
        return x, v

    def set_state(self, x, v):
        x = np.ascontiguousarray(x, np.float64)
        v = np.ascontiguousarray(v, np.float64)
        lib().ora_scene_set_state(self._h, _dp(x), _dp(v))

    def xhat(self):
        out = np.zeros((self.n_verts, 3))
        lib().ora_scene_xhat(self._h, _dp(out))
        return out

    def set_solve_hook(self, fn):
        """fn(newton_iter, attempt, n_projected_total) -> -1 | 0 | 1"""
        if fn is None:
            self._hook = None
            lib().ora_scene_set_solve_hook(self._h, HOOK(), None)
            return
        self._hook = HOOK(lambda k, a, n, u: int(fn(k, a, n)))
        lib().ora_scene_set_solve_hook(self._h, self._hook, None)

    # --- evaluation ---
    def energy(self, x, xhat):
        x = np.ascontiguousarray(x, np.float64)
        xhat = np.ascontiguousarray(xhat, np.float64)
        return lib().ora_scene_energy(self._h, _dp(x), _dp(xhat))

    def gradient(self, x, xhat):
        x = np.ascontiguousarray(x, np.float64)
        xhat = np.ascontiguousarray(xhat, np.float64)
        g = np.zeros((self.n_verts, 3))
        lib().ora_scene_gradient(self._h, _dp(x), _dp(xhat), _dp(g))
        return g

    def element_eval(self, x, want_hessian=True):
        x = np.ascontiguousarray(x, np.float64)
        psi = np.zeros(self.n_tets)
        ge = np.zeros((self.n_tets, 12))
        He = np.zeros((self.n_tets, 12, 12)) if want_hessian else None
        lib().ora_scene_element_eval(self._h, _dp(x), _dp(psi), _dp(ge),
                                     _dp(He) if want_hessian else None)
        return psi, ge, He

    def assemble(self, x, proj=None):
        x = np.ascontiguousarray(x, np.float64)
        vals = np.zeros((self.nnzb, 3, 3))
        pr = None if proj is None else np.ascontiguousarray(proj, np.uint8)
        lib().ora_scene_assemble(self._h, _dp(x), _u8(pr) if pr is not None else None, _dp(vals))
        return vals

    def select(self, g, delta, already=None):
        g = np.ascontiguousarray(g, np.float64)
        out = np.zeros(self.n_tets, np.uint8)
        al = None if already is None else np.ascontiguousarray(already, np.uint8)
        n = lib().ora_scene_select(self._h, _dp(g), float(delta), _u8(al) if al is not None else None,
                                   _u8(out))
        return out.astype(bool), int(n)

    def project(self, x, sel):
        x = np.ascontiguousarray(x, np.float64)
        sel = np.ascontiguousarray(sel, np.int32)
        dH = np.zeros((len(sel), 12, 12))
        lib().ora_scene_project(self._h, _dp(x), _ip(sel), len(sel), _dp(dH))
        return dH

    # --- time stepping ---
    def step(self, mode: int, tol: float):
        x = np.zeros((self.n_verts, 3))
        st = StepStats()
        rc = lib().ora_scene_step(self._h, int(mode), float(tol), _dp(x), C.byref(st))
        return rc, x, {k: getattr(st, k) for k, _ in StepStats._fields_}

    def iter_stats(self):
        cap = 256
        buf = (IterStats * cap)()
        n = lib().ora_scene_iter_stats(self._h, buf, cap)
        return [{k: getattr(buf[i], k) for k, _ in IterStats._fields_} for i in range(min(n, cap))]

    def attempts(self):
        cap = 4096
        buf = (Attempt * cap)()
        n = lib().ora_scene_attempts(self._h, buf, cap)
        out = []
        for i in range(min(n, cap)):
            d = {k: getattr(buf[i], k) for k, _ in Attempt._fields_}
            out.append(d)
        return out

    def set_record(self, on: bool):
        lib().ora_scene_set_record(self._h, 1 if on else 0)

    def iteration_gradient(self, k: int):
        """Assembled gradient of Newton iteration k of the last step (recording on)."""
        g = np.zeros((self.n_verts, 3))
        if lib().ora_scene_iteration_gradient(self._h, int(k), _dp(g)) != 0:
            raise IndexError(k)
        return g

    def attempt_selection(self, idx: int):
        """Elements newly selected by the PPN rounds before attempt ``idx`` of the last
        step (ascending; the contact element of vertex v is n_tets + v)."""
        n = lib().ora_scene_attempt_selection(self._h, int(idx), None, 0)
        if n < 0:
            raise IndexError(idx)
        out = np.zeros(n, np.int32)
        lib().ora_scene_attempt_selection(self._h, int(idx), _ip(out), n)
        return out


INF = math.inf
