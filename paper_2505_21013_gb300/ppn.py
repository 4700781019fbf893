"""Thin ctypes binding of ``libppn.so`` (the C ABI declared in ``include/ppn.h``).

Functions keep the C names; this module only marshals numpy arrays and
structs.  Every computation happens in the library's CUDA kernels; there is no
fallback: importing raises if the shared library has not been built.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libppn.so")

PPN_OK = 0
PPN_ERR_NEWTON_MAXITER = 6
PPN_ERR_ADMISSION = 10
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "DEGENERATE_TET", 5: "LINESEARCH",
                6: "NEWTON_MAXITER", 7: "PCG_MAXITER", 8: "NONFINITE", 9: "TIMEOUT", 10: "ADMISSION"}
MODE_NEWTON, MODE_PN, MODE_PPN, MODE_PDN = 0, 1, 2, 3
PROJ_CLAMP, PROJ_MIRROR = 0, 1
PREC_FP64, PREC_MIXED = 0, 1


class ppn_material(C.Structure):
    _fields_ = [("E", C.c_double), ("nu", C.c_double), ("rho", C.c_double)]


class ppn_params(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("eps_delta", C.c_double),
                ("eig_eps", C.c_double), ("pcg_rel_tol", C.c_double), ("armijo_c", C.c_double),
                ("gravity", C.c_double * 3), ("pcg_max_iter", C.c_int), ("newton_max_iter", C.c_int),
                ("ls_max_halvings", C.c_int), ("precision", C.c_int), ("tol_kind", C.c_int),
                ("init_guess", C.c_int), ("pdn_countdown", C.c_int), ("projection", C.c_int),
                ("grad_floor", C.c_double), ("ls_slack", C.c_double), ("contact_kappa", C.c_double),
                ("contact_dhat", C.c_double), ("ccd_safety", C.c_double), ("dirichlet_penalty", C.c_double),
                ("tie_band", C.c_double)]


class ppn_obstacle(C.Structure):
    _fields_ = [("type", C.c_int), ("p", C.c_double * 3), ("a", C.c_double * 3), ("r", C.c_double)]


OBST_KINDS = {"plane": 0, "cylinder_in": 1, "sphere_out": 2}


def obstacles_from(spec_list):
    """ppn_obstacle structs from (kind, point, axis_or_normal, radius) tuples."""
    out = []
    for kind, p, a, r in spec_list:
        o = ppn_obstacle()
        o.type = OBST_KINDS[kind]
        o.p[:] = [float(v) for v in p]
        o.a[:] = [float(v) for v in a]
        o.r = float(r)
        out.append(o)
    return out


class ppn_iter_stats(C.Structure):
    _fields_ = [("newton_iter", C.c_int), ("pcg_attempts", C.c_int), ("cg_iters", C.c_int),
                ("n_new_projected", C.c_int), ("n_projected_total", C.c_int), ("ls_halvings", C.c_int),
                ("fallback", C.c_int), ("precond_fail", C.c_int), ("grad_norm2", C.c_double),
                ("grad_norminf", C.c_double), ("delta", C.c_double), ("gamma", C.c_double),
                ("energy", C.c_double), ("energy_new", C.c_double), ("dir_deriv", C.c_double)]


class ppn_attempt(C.Structure):
    _fields_ = [("newton_iter", C.c_int), ("attempt", C.c_int), ("n_new_projected", C.c_int),
                ("ind", C.c_int), ("cg_iters", C.c_int), ("delta", C.c_double), ("n_ties", C.c_int)]


class ppn_step_stats(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("total_projections", C.c_int), ("total_cg_iters", C.c_int),
                ("total_attempts", C.c_int), ("status", C.c_int), ("final_grad_norm2", C.c_double),
                ("device_ms", C.c_double), ("n_ties", C.c_int)]


class ppn_pcg_tuning(C.Structure):
    _fields_ = [("tiles_per_cta", C.c_int), ("blocks_per_row", C.c_int), ("log2_matrix_mb", C.c_int),
                ("choice", C.c_int), ("launches", C.c_int * 4), ("us_per_iter", C.c_double * 4)]


PCG_TUNING_CHOICES = {0: "streamed, evict-first", 1: "global, evict-first", 2: "streamed, L2 normal",
                      3: "global, L2 normal", -1: "exploring"}


class ppn_server_config(C.Structure):
    _fields_ = [("hbm_fraction", C.c_double), ("max_batch", C.c_int), ("precision", C.c_int)]


class ppn_request_times(C.Structure):
    _fields_ = [("t_submit_ms", C.c_double), ("t_start_ms", C.c_double), ("t_done_ms", C.c_double),
                ("batch_max", C.c_int)]


class ppn_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("rejected_scenes", C.c_int64),
                ("resident_scenes", C.c_int), ("resident_bytes", C.c_double), ("budget_bytes", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("steps_per_s", C.c_double)]


class ppn_scene_info(C.Structure):
    _fields_ = [("n_verts", C.c_int64), ("n_tets", C.c_int64), ("n_fixed", C.c_int64),
                ("nnzb", C.c_int64), ("n_map", C.c_int64), ("device_bytes", C.c_int64),
                ("precision", C.c_int), ("pcg_layout", C.c_int)]


PCG_LAYOUTS = {-1: "none", 0: "resident", 1: "streamed", 2: "global", 3: "halo", 4: "standard", 5: "standard_global"}


class ppn_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double),
                ("bytes", C.c_double)]


_P = C.c_void_p
_pd = C.POINTER(C.c_double)
_pi = C.POINTER(C.c_int32)
_pl = C.POINTER(C.c_int64)
_pu = C.POINTER(C.c_uint8)
_st = C.c_int

SIGNATURES = {
    "ppn_default_params": (ppn_params, []),
    "ppn_status_string": (C.c_char_p, [_st]),
    "ppn_last_error": (C.c_char_p, []),
    "ppn_create_scene": (_st, [_pd, C.c_int64, _pi, C.c_int64, C.POINTER(ppn_material), C.c_double, _pi,
                               C.c_int64, C.POINTER(ppn_params), C.POINTER(_P)]),
    "ppn_destroy_scene": (None, [_P]),
    "ppn_scene_get_info": (_st, [_P, C.POINTER(ppn_scene_info)]),
    "ppn_set_stream": (_st, [_P, _P]),
    "ppn_set_allocator": (_st, [_P, _P, _P]),
    "ppn_set_kinematic_targets": (_st, [_P, _pd]),
    "ppn_set_kinematic_targets_device": (_st, [_P, _P]),
    "ppn_step": (_st, [_P, C.c_int, C.c_double, _pd, C.POINTER(ppn_step_stats)]),
    "ppn_step_batch": (_st, [C.POINTER(_P), C.c_int, C.POINTER(C.c_int), C.c_double,
                             C.POINTER(ppn_step_stats)]),
    "ppn_get_iter_stats": (_st, [_P, C.POINTER(ppn_iter_stats), C.c_int, C.POINTER(C.c_int)]),
    "ppn_get_attempts": (_st, [_P, C.POINTER(ppn_attempt), C.c_int, C.POINTER(C.c_int)]),
    "ppn_set_record_selection": (_st, [_P, C.c_int]),
    "ppn_get_attempt_selection": (_st, [_P, C.c_int, _pi, C.c_int64, _pl]),
    "ppn_probe_tets": (_st, [_P, _pi]),
    "ppn_get_pcg_tuning": (_st, [C.POINTER(ppn_pcg_tuning), C.c_int, C.POINTER(C.c_int)]),
    "ppn_get_iteration_gradient": (_st, [_P, C.c_int, _pd]),
    "ppn_get_state": (_st, [_P, _pd, _pd]),
    "ppn_set_state": (_st, [_P, _pd, _pd]),
    "ppn_get_displacement": (_st, [_P, _pd, _pd]),
    "ppn_set_displacement": (_st, [_P, _pd, _pd]),
    "ppn_set_profiling": (_st, [_P, C.c_int]),
    "ppn_get_kernel_times": (_st, [_P, C.POINTER(ppn_kernel_time), C.c_int, C.POINTER(C.c_int)]),
    "ppn_probe_elements": (_st, [_P, _pd, _pd, _pd, _pd]),
    "ppn_probe_gradient": (_st, [_P, _pd, _pd, _pd, _pd, _pd]),
    "ppn_probe_pattern": (_st, [_P, _pl, _pi]),
    "ppn_probe_assemble": (_st, [_P, _pd, _pu, _pd]),
    "ppn_probe_select": (_st, [_P, _pd, C.c_double, _pu, _pu, _pl, _pl]),
    "ppn_probe_project": (_st, [_P, _pd, _pi, C.c_int64, _pd]),
    "ppn_probe_pcg": (_st, [_P, _pd, _pd, C.c_double, C.c_int, _pd, C.POINTER(C.c_int)]),
    "ppn_probe_bounded_wait": (_st, [C.c_int, C.c_int, C.c_int]),
    "ppn_probe_halo_tables": (_st, [C.c_int, C.POINTER(_pl), C.POINTER(_pi), _pl, C.c_int, _pi, C.c_int64, _pl,
                                    _pi]),
    "ppn_server_default_config": (ppn_server_config, []),
    "ppn_server_create": (_st, [C.POINTER(ppn_server_config), C.POINTER(_P)]),
    "ppn_server_destroy": (None, [_P]),
    "ppn_server_add_scene": (_st, [_P, _pd, C.c_int64, _pi, C.c_int64, C.POINTER(ppn_material), C.c_double, _pi,
                                   C.c_int64, C.POINTER(ppn_params), _pi]),
    "ppn_server_remove_scene": (_st, [_P, C.c_int32]),
    "ppn_server_submit": (_st, [_P, C.c_int32, C.c_int, C.c_double, _pd, _pl]),
    "ppn_server_poll": (_st, [_P, C.c_int64, C.c_int, C.POINTER(C.c_int), _pd, C.POINTER(ppn_step_stats),
                              C.POINTER(ppn_request_times)]),
    "ppn_server_get_stats": (_st, [_P, C.POINTER(ppn_server_stats)]),
    "ppn_set_obstacles": (_st, [_P, C.POINTER(ppn_obstacle), C.c_int]),
    "ppn_pcg_solve_static": (_st, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                   C.c_void_p, C.c_double, C.c_int32, C.POINTER(C.c_int32), C.c_void_p]),
}

_lib = None


def lib():
    """Load libppn.so; raises (no fallback) when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2505_21013_gb300.build.build() "
                          "(nvcc, sm_103a) first; there is no CPU fallback")
    L = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def last_error() -> str:
    """The calling thread's last error message from the library."""
    return lib().ppn_last_error().decode(errors="replace")


class PPNError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().ppn_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({msg})")
        self.status = status


def _check(rc: int, where: str, ok=(PPN_OK,)):
    if rc not in ok:
        raise PPNError(rc, where)
    return rc


def _d(a):
    return a.ctypes.data_as(_pd)


def _arr(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def ppn_default_params() -> ppn_params:
    return lib().ppn_default_params()


def struct_dict(s) -> dict:
    out = {}
    for k, _ in s._fields_:
        v = getattr(s, k)
        if isinstance(v, bytes):
            v = v.decode()
        elif hasattr(v, "_length_"):
            v = list(v)
        out[k] = v
    return out


class Scene:
    """One resident scene (device memory owned by the library)."""

    def __init__(self, rest, tets, fixed, E, nu, rho, dt, params: ppn_params | None = None):
        L = lib()
        self.rest = _arr(rest, np.float64)
        tets = _arr(tets, np.int32)
        self.fixed = _arr(fixed, np.int32)
        self.n_verts = self.rest.shape[0]
        self.n_tets = tets.shape[0]
        self.n_fixed = self.fixed.shape[0]
        mat = ppn_material(E, nu, rho)
        p = params if params is not None else ppn_default_params()
        h = _P()
        _check(L.ppn_create_scene(_d(self.rest), self.n_verts, tets.ctypes.data_as(_pi), self.n_tets,
                                  C.byref(mat), dt, self.fixed.ctypes.data_as(_pi), self.n_fixed,
                                  C.byref(p), C.byref(h)), "ppn_create_scene")
        self._h = h
        self.dt = dt
        self.params = p

    @classmethod
    def from_spec(cls, spec, params: ppn_params | None = None, precision: int | None = None):
        p = params if params is not None else ppn_default_params()
        if precision is not None:
            p.precision = precision
        p.gravity[0], p.gravity[1], p.gravity[2] = spec.gravity
        return cls(spec.rest, spec.tets, spec.fixed, spec.E, spec.nu, spec.rho, spec.dt, p)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().ppn_destroy_scene(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = ppn_scene_info()
        _check(lib().ppn_scene_get_info(self._h, C.byref(i)), "ppn_scene_get_info")
        return struct_dict(i)

    def set_stream(self, stream_ptr: int | None):
        _check(lib().ppn_set_stream(self._h, C.c_void_p(stream_ptr or 0)), "ppn_set_stream")

    def set_targets(self, xyz):
        xyz = _arr(xyz, np.float64)
        _check(lib().ppn_set_kinematic_targets(self._h, _d(xyz)), "ppn_set_kinematic_targets")

    def set_obstacles(self, spec_list):
        """Obstacles as (kind, point, axis_or_normal, radius) tuples (see include/ppn.h)."""
        obs = obstacles_from(spec_list)
        arr = (ppn_obstacle * max(1, len(obs)))(*obs)
        _check(lib().ppn_set_obstacles(self._h, arr, len(obs)), "ppn_set_obstacles")

    def set_targets_device(self, ptr: int):
        _check(lib().ppn_set_kinematic_targets_device(self._h, C.c_void_p(ptr)),
               "ppn_set_kinematic_targets_device")

    def step(self, mode: int, tol: float, want_x: bool = True, raise_on=(PPN_OK, 6, 5), out=None):
        """ppn_step.  The positions go into `out` when given (a C-contiguous float64
        (n_verts, 3) array, for example in pinned host memory), else into a new array
        when want_x."""
        if out is not None:
            if out.dtype != np.float64 or out.shape != (self.n_verts, 3) or not out.flags.c_contiguous:
                raise ValueError("out must be a C-contiguous float64 array of shape (n_verts, 3)")
            want_x = True
        elif want_x:
            out = np.zeros((self.n_verts, 3))
        st = ppn_step_stats()
        rc = lib().ppn_step(self._h, int(mode), float(tol), _d(out) if want_x else None, C.byref(st))
        _check(rc, "ppn_step", ok=raise_on)
        return rc, out, struct_dict(st)

    def iter_stats(self):
        buf = (ppn_iter_stats * 256)()
        n = C.c_int()
        _check(lib().ppn_get_iter_stats(self._h, buf, 256, C.byref(n)), "ppn_get_iter_stats")
        return [struct_dict(buf[i]) for i in range(min(n.value, 256))]

    def attempts(self):
        buf = (ppn_attempt * 4096)()
        n = C.c_int()
        _check(lib().ppn_get_attempts(self._h, buf, 4096, C.byref(n)), "ppn_get_attempts")
        return [struct_dict(buf[i]) for i in range(min(n.value, 4096))]

    def set_record_selection(self, on: bool):
        _check(lib().ppn_set_record_selection(self._h, 1 if on else 0), "ppn_set_record_selection")

    def attempt_selection(self, idx: int):
        """Elements selected before attempt ``idx`` of the last step (recording on):
        ascending tet indices, contact elements as n_tets + v."""
        n = C.c_int64()
        _check(lib().ppn_get_attempt_selection(self._h, int(idx), None, 0, C.byref(n)), "ppn_get_attempt_selection")
        out = np.zeros(n.value, np.int32)
        _check(lib().ppn_get_attempt_selection(self._h, int(idx), out.ctypes.data_as(_pi), out.size, C.byref(n)),
               "ppn_get_attempt_selection")
        return out

    def iteration_gradient(self, k: int):
        """The assembled gradient of Newton iteration k of the last step (recording on)."""
        g = np.zeros((self.n_verts, 3))
        _check(lib().ppn_get_iteration_gradient(self._h, int(k), _d(g)), "ppn_get_iteration_gradient")
        return g

    def get_state(self):
        x = np.zeros((self.n_verts, 3))
        v = np.zeros((self.n_verts, 3))
        _check(lib().ppn_get_state(self._h, _d(x), _d(v)), "ppn_get_state")
        return x, v

    def set_state(self, x, v):
        x = _arr(x, np.float64)
        v = _arr(v, np.float64)
        _check(lib().ppn_set_state(self._h, _d(x), _d(v)), "ppn_set_state")

    def get_displacement(self):
        u = np.zeros((self.n_verts, 3))
        v = np.zeros((self.n_verts, 3))
        _check(lib().ppn_get_displacement(self._h, _d(u), _d(v)), "ppn_get_displacement")
        return u, v

    def set_displacement(self, u, v):
        u = _arr(u, np.float64)
        v = _arr(v, np.float64)
        _check(lib().ppn_set_displacement(self._h, _d(u), _d(v)), "ppn_set_displacement")

    def set_profiling(self, on: bool):
        _check(lib().ppn_set_profiling(self._h, 1 if on else 0), "ppn_set_profiling")

    def kernel_times(self) -> dict:
        buf = (ppn_kernel_time * 32)()
        n = C.c_int()
        _check(lib().ppn_get_kernel_times(self._h, buf, 32, C.byref(n)), "ppn_get_kernel_times")
        return {buf[i].name.decode(): {"launches": buf[i].launches, "total_ms": buf[i].total_ms,
                                       "bytes": buf[i].bytes} for i in range(min(n.value, 32))}

    # ---- stage probes ----
    def probe_elements(self, x):
        x = _arr(x, np.float64)
        psi = np.zeros(self.n_tets)
        ge = np.zeros((self.n_tets, 12))
        He = np.zeros((self.n_tets, 12, 12))
        _check(lib().ppn_probe_elements(self._h, _d(x), _d(psi), _d(ge), _d(He)), "ppn_probe_elements")
        return psi, ge, He

    def probe_gradient(self, x, xhat):
        x = _arr(x, np.float64)
        xhat = _arr(xhat, np.float64)
        g = np.zeros((self.n_verts, 3))
        norms = np.zeros(2)
        en = C.c_double()
        _check(lib().ppn_probe_gradient(self._h, _d(x), _d(xhat), _d(g), _d(norms), C.byref(en)),
               "ppn_probe_gradient")
        return g, norms, en.value

    def probe_pattern(self):
        nnzb = self.info()["nnzb"]
        rp = np.zeros(self.n_verts + 1, np.int64)
        col = np.zeros(nnzb, np.int32)
        _check(lib().ppn_probe_pattern(self._h, rp.ctypes.data_as(_pl), col.ctypes.data_as(_pi)),
               "ppn_probe_pattern")
        return rp, col

    def probe_assemble(self, x, proj=None):
        x = _arr(x, np.float64)
        nnzb = self.info()["nnzb"]
        vals = np.zeros((nnzb, 3, 3))
        pr = None if proj is None else _arr(proj, np.uint8)
        _check(lib().ppn_probe_assemble(self._h, _d(x), pr.ctypes.data_as(_pu) if pr is not None else None,
                                        _d(vals)), "ppn_probe_assemble")
        return vals

    def probe_select(self, g, delta, already=None, with_ties=False):
        g = _arr(g, np.float64)
        out = np.zeros(self.n_tets, np.uint8)
        al = None if already is None else _arr(already, np.uint8)
        n, nt = C.c_int64(), C.c_int64()
        _check(lib().ppn_probe_select(self._h, _d(g), float(delta),
                                      al.ctypes.data_as(_pu) if al is not None else None,
                                      out.ctypes.data_as(_pu), C.byref(n), C.byref(nt)), "ppn_probe_select")
        if with_ties:
            return out.astype(bool), n.value, nt.value
        return out.astype(bool), n.value

    def probe_tets(self):
        """The tets after the orientation normalisation, as the kernels read them."""
        t = np.zeros((self.n_tets, 4), np.int32)
        _check(lib().ppn_probe_tets(self._h, t.ctypes.data_as(_pi)), "ppn_probe_tets")
        return t

    def probe_project(self, x, sel):
        x = _arr(x, np.float64)
        sel = _arr(sel, np.int32)
        dH = np.zeros((len(sel), 12, 12))
        _check(lib().ppn_probe_project(self._h, _d(x), sel.ctypes.data_as(_pi), len(sel), _d(dH)),
               "ppn_probe_project")
        return dH

    def probe_pcg(self, vals, b, rel_tol=1e-4, max_iter=0):
        vals = _arr(vals, np.float64)
        b = _arr(b, np.float64)
        x = np.zeros(self.n_verts * 3)
        info = (C.c_int * 4)()
        _check(lib().ppn_probe_pcg(self._h, _d(vals), _d(b), float(rel_tol), int(max_iter), _d(x), info),
               "ppn_probe_pcg")
        return x.reshape(-1, 3), {"iters": info[0], "ind": bool(info[1]), "precond_fail": bool(info[2]),
                                  "hit_max": bool(info[3])}


def probe_bounded_wait(n_words: int, spin_limit: int, preset: bool) -> int:
    """``ppn_probe_bounded_wait``: the status (PPN_OK, or 9 = PPN_ERR_TIMEOUT when the wait ran out)."""
    return int(lib().ppn_probe_bounded_wait(int(n_words), int(spin_limit), 1 if preset else 0))


def probe_halo_tables(patterns, grid: int):
    """``ppn_probe_halo_tables`` for [(row_ptr, col), ...]: (off [grid + 1, 2], local columns,
    halo references, most halo rows of one CTA)."""
    rps = [np.ascontiguousarray(rp, dtype=np.int64) for rp, _ in patterns]
    cols = [np.ascontiguousarray(c, dtype=np.int32) for _, c in patterns]
    n = len(patterns)
    rp_arr = (_pl * n)(*[a.ctypes.data_as(_pl) for a in rps])
    col_arr = (_pi * n)(*[a.ctypes.data_as(_pi) for a in cols])
    nv = np.array([len(a) - 1 for a in rps], dtype=np.int64)
    need, mh = C.c_int64(0), C.c_int32(0)
    L = lib()
    rc = L.ppn_probe_halo_tables(n, rp_arr, col_arr, nv.ctypes.data_as(_pl), int(grid), None, 0, C.byref(need),
                                 C.byref(mh))
    if rc != PPN_OK and need.value == 0:
        _check(rc, "ppn_probe_halo_tables")
    out = np.zeros(need.value, dtype=np.int32)
    _check(L.ppn_probe_halo_tables(n, rp_arr, col_arr, nv.ctypes.data_as(_pl), int(grid), out.ctypes.data_as(_pi),
                                   out.size, C.byref(need), C.byref(mh)), "ppn_probe_halo_tables")
    no = 2 * (grid + 1)
    off = out[:no].reshape(grid + 1, 2)
    nb = int(off[grid, 0])
    return off, out[no:no + nb], out[no + nb:], int(mh.value)


# ppn_device_alloc_fn / ppn_device_free_fn
DEVICE_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
DEVICE_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_allocator_refs = []  # the installed callbacks, kept alive while scenes may use them


def set_allocator(alloc=None, free=None):
    """Install alloc(bytes) -> device pointer (int, 0 on failure) and free(ptr) as the
    device allocator of scenes, scene groups and servers created afterwards; both None
    restores cudaMalloc / cudaFree.  Owners created earlier keep the allocator they were
    created with, so the callbacks stay referenced here."""
    if (alloc is None) != (free is None):
        raise ValueError("give both alloc and free, or neither")
    if alloc is None:
        _check(lib().ppn_set_allocator(None, None, None), "ppn_set_allocator")
        return
    fa = DEVICE_ALLOC_FN(lambda n, ctx: alloc(int(n)) or None)
    ff = DEVICE_FREE_FN(lambda p, ctx: free(int(p)))
    _allocator_refs.append((fa, ff))
    _check(lib().ppn_set_allocator(C.cast(fa, C.c_void_p), C.cast(ff, C.c_void_p), None), "ppn_set_allocator")


def pcg_tuning():
    """``ppn_get_pcg_tuning``: the linear solver's autotuner records, one dict per shape class."""
    buf = (ppn_pcg_tuning * 64)()
    n = C.c_int()
    _check(lib().ppn_get_pcg_tuning(buf, 64, C.byref(n)), "ppn_get_pcg_tuning")
    out = []
    for i in range(min(n.value, 64)):
        d = struct_dict(buf[i])
        d["kept"] = PCG_TUNING_CHOICES.get(d["choice"], "?")
        out.append(d)
    return out


def ppn_step_batch(scenes, modes, tol):
    n = len(scenes)
    arr = (_P * n)(*[s.handle for s in scenes])
    m = (C.c_int * n)(*[int(x) for x in modes])
    out = (ppn_step_stats * n)()
    rc = lib().ppn_step_batch(arr, n, m, float(tol), out)
    return rc, [struct_dict(out[i]) for i in range(n)]


def pcg_solve_static(row_ptr: int, col: int, val: int, n_rows: int, nnzb: int, b: int, x: int,
                     rel_tol: float = 1e-4, max_iter: int = 0, stream: int = 0) -> dict:
    """``ppn_pcg_solve_static`` on device pointers (see ``include/ppn.h``): int32
    row_ptr/col, component-major FP32 values, 16-byte {x, y, z, pad} FP32 records
    for b and x.  Returns the solver's info; raises PPNError on failure."""
    info = (C.c_int32 * 4)()
    _check(lib().ppn_pcg_solve_static(C.c_void_p(row_ptr), C.c_void_p(col), C.c_void_p(val), int(n_rows),
                                      int(nnzb), C.c_void_p(b), C.c_void_p(x), float(rel_tol), int(max_iter),
                                      info, C.c_void_p(stream or None)), "ppn_pcg_solve_static")
    return {"iters": info[0], "ind": bool(info[1]), "precond_fail": bool(info[2]), "hit_max": bool(info[3])}


class Server:
    """Serving loop over resident scenes (``ppn_server_*`` in include/ppn.h):
    scenes admitted by HBM footprint, one request = one time step, continuous
    batching of the running requests on the device."""

    def __init__(self, hbm_fraction=0.8, max_batch=64, precision=PREC_MIXED):
        cfg = lib().ppn_server_default_config()
        cfg.hbm_fraction = hbm_fraction
        cfg.max_batch = max_batch
        cfg.precision = precision
        h = _P()
        _check(lib().ppn_server_create(C.byref(cfg), C.byref(h)), "ppn_server_create")
        self._h = h
        self.precision = precision
        self.n_verts = {}
        self.n_fixed = {}

    def add_scene(self, spec, params: ppn_params | None = None) -> int:
        p = params if params is not None else ppn_default_params()
        p.precision = self.precision
        p.gravity[0], p.gravity[1], p.gravity[2] = spec.gravity
        rest = _arr(spec.rest, np.float64)
        tets = _arr(spec.tets, np.int32)
        fixed = _arr(spec.fixed, np.int32)
        mat = ppn_material(spec.E, spec.nu, spec.rho)
        sid = C.c_int32()
        _check(lib().ppn_server_add_scene(self._h, _d(rest), rest.shape[0], tets.ctypes.data_as(_pi), tets.shape[0],
                                          C.byref(mat), spec.dt, fixed.ctypes.data_as(_pi), fixed.shape[0],
                                          C.byref(p), C.byref(sid)), "ppn_server_add_scene")
        self.n_verts[sid.value] = rest.shape[0]
        self.n_fixed[sid.value] = fixed.shape[0]
        return sid.value

    def remove_scene(self, sid: int):
        _check(lib().ppn_server_remove_scene(self._h, int(sid)), "ppn_server_remove_scene")
        self.n_verts.pop(sid, None)

    def submit(self, sid: int, mode: int, tol: float, targets=None) -> int:
        t = C.c_int64()
        tg = None if targets is None else _arr(targets, np.float64)
        _check(lib().ppn_server_submit(self._h, int(sid), int(mode), float(tol), _d(tg) if tg is not None else None,
                                       C.byref(t)), "ppn_server_submit")
        return t.value

    def poll(self, ticket: int, sid: int, wait: bool = True):
        """(done, status, positions, stats, times); positions/stats/times are None until done."""
        done = C.c_int()
        x = np.zeros((self.n_verts[sid], 3))
        st = ppn_step_stats()
        tm = ppn_request_times()
        rc = lib().ppn_server_poll(self._h, int(ticket), 1 if wait else 0, C.byref(done), _d(x), C.byref(st),
                                   C.byref(tm))
        if not done.value:
            _check(rc, "ppn_server_poll")
            return False, rc, None, None, None
        return True, rc, x, struct_dict(st), struct_dict(tm)

    def stats(self) -> dict:
        s = ppn_server_stats()
        _check(lib().ppn_server_get_stats(self._h, C.byref(s)), "ppn_server_get_stats")
        return struct_dict(s)

    def close(self):
        if getattr(self, "_h", None):
            lib().ppn_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
