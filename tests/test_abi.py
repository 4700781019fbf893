"""CPU checks of the C-ABI library: it builds, loads and exports every entry
point that include/ppn.h declares (no GPU call is made)."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ppn.h")).read()
    return sorted(set(re.findall(r"PPN_API[^;(]*?\b(ppn_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2505_21013_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for must in ["ppn_create_scene", "ppn_step", "ppn_step_batch", "ppn_get_iter_stats",
                 "ppn_destroy_scene", "ppn_set_kinematic_targets", "ppn_get_state", "ppn_set_state"]:
        assert must in syms


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (ppn_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_binding_loads_and_matches_header(libpath):
    from paper_2505_21013_gb300 import ppn

    L = ppn.lib()
    for s in declared_symbols():
        assert hasattr(L, s)
        assert s in ppn.SIGNATURES, s
    p = ppn.ppn_default_params()
    assert (p.alpha, p.beta, p.eps_delta, p.eig_eps, p.pcg_rel_tol) == (0.5, 2.0, 1e-12, 1e-8, 1e-4)
    assert L.ppn_status_string(0) == b"ok"


def test_invalid_arguments_are_rejected_without_a_gpu(libpath):
    import ctypes as C

    from paper_2505_21013_gb300 import ppn

    L = ppn.lib()
    out = C.c_void_p()
    rc = L.ppn_create_scene(None, 0, None, 0, None, 0.0, None, 0, None, C.byref(out))
    assert rc == 1 and not out.value
    assert L.ppn_last_error()
    # the bounded-wait probe checks its arguments before touching the device
    assert L.ppn_probe_bounded_wait(0, 10, 0) == 1
    assert L.ppn_probe_bounded_wait(8, 0, 0) == 1
    assert L.ppn_probe_bounded_wait(8, (1 << 20) + 1, 1) == 1


def test_allocator_arguments_are_checked_without_a_gpu(libpath):
    import ctypes as C

    from paper_2505_21013_gb300 import ppn

    L = ppn.lib()
    fa = ppn.DEVICE_ALLOC_FN(lambda n, ctx: None)
    ff = ppn.DEVICE_FREE_FN(lambda p, ctx: None)
    # exactly one of the two functions is an error; both or neither is accepted
    assert L.ppn_set_allocator(C.cast(fa, C.c_void_p), None, None) == 1
    assert L.ppn_set_allocator(None, C.cast(ff, C.c_void_p), None) == 1
    assert L.ppn_set_allocator(C.cast(fa, C.c_void_p), C.cast(ff, C.c_void_p), None) == 0
    assert L.ppn_set_allocator(None, None, None) == 0

