"""ppn_pcg_solve_static (PCG from a fixed device arena, no per-call allocation)
against the scene path's PCG on the same FP32 system.

With PPN_PCG_GLOBAL set, a scene solves with the same global-memory
cooperative kernel, so the two entry points must agree bitwise.  Two calls in
a row check that the arena is reset between calls.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_21013_gb300")
from oracle import oracle as O  # noqa: E402
from ppn_inputs import twisting_beam_scene  # noqa: E402


def system(seed):
    spec = twisting_beam_scene(7, 6, 13, h=0.02, E=1e5, nu=0.45, omega=5.0, dt=1 / 30, seed=seed)
    o = O.Scene.from_spec(spec)
    vals = o.assemble(spec.rest).astype(np.float32).astype(np.float64)  # values exactly representable in FP32
    rp, col = o.pattern()
    b = np.random.default_rng(seed).standard_normal((spec.n_verts, 3)).astype(np.float32).astype(np.float64)
    b[spec.fixed] = 0
    return spec, vals, rp, col, b


def device_inputs(vals, rp, col, b):
    dev = torch.device("cuda", 0)
    nnzb = col.size
    comp = np.ascontiguousarray(vals.reshape(nnzb, 9).T, dtype=np.float32)  # [9][nnzb]
    b4 = np.zeros((b.shape[0], 4), np.float32)
    b4[:, :3] = b
    return (torch.tensor(rp.astype(np.int32), device=dev), torch.tensor(col.astype(np.int32), device=dev),
            torch.tensor(comp, device=dev), torch.tensor(b4, device=dev))


@pytest.mark.parametrize("seed", [0, 1])
def test_static_arena_pcg_matches_scene_pcg(seed, monkeypatch):
    monkeypatch.setenv("PPN_PCG_GLOBAL", "1")
    spec, vals, rp, col, b = system(seed)
    sc = P.Scene.from_spec(spec, precision=P.PREC_MIXED)
    x_ref, info_ref = sc.probe_pcg(vals, b, rel_tol=1e-4)
    sc.close()
    d_rp, d_col, d_val, d_b = device_inputs(vals, rp, col, b)
    n = spec.n_verts
    for _ in range(2):
        x = torch.full((n, 4), float("nan"), dtype=torch.float32, device="cuda")
        info = P.ppn.pcg_solve_static(d_rp.data_ptr(), d_col.data_ptr(), d_val.data_ptr(), n, col.size,
                                      d_b.data_ptr(), x.data_ptr(), rel_tol=1e-4)
        torch.cuda.synchronize()
        assert info == info_ref
        xs = x[:, :3].double().cpu().numpy()
        assert np.array_equal(xs, x_ref)


def test_static_arena_rejects_oversize_and_bad_patterns():
    n = 65537
    with pytest.raises(P.PPNError, match="static scratch limit"):
        P.ppn.pcg_solve_static(1, 1, 1, n, n, 1, 1)
    # a row without its diagonal block is caught on the device before the solve
    dev = torch.device("cuda", 0)
    rp = torch.tensor([0, 1, 2], dtype=torch.int32, device=dev)
    col = torch.tensor([1, 0], dtype=torch.int32, device=dev)
    val = torch.ones(18, dtype=torch.float32, device=dev)
    bx = torch.zeros((2, 4), dtype=torch.float32, device=dev)
    with pytest.raises(P.PPNError, match="malformed BSR pattern"):
        P.ppn.pcg_solve_static(rp.data_ptr(), col.data_ptr(), val.data_ptr(), 2, 2, bx.data_ptr(), bx.data_ptr())
    # a row with two diagonal blocks is malformed too (the preconditioner would invert one of them)
    rp2 = torch.tensor([0, 2, 3], dtype=torch.int32, device=dev)
    col2 = torch.tensor([0, 0, 1], dtype=torch.int32, device=dev)
    val2 = torch.ones(27, dtype=torch.float32, device=dev)
    with pytest.raises(P.PPNError, match="malformed BSR pattern"):
        P.ppn.pcg_solve_static(rp2.data_ptr(), col2.data_ptr(), val2.data_ptr(), 2, 3, bx.data_ptr(), bx.data_ptr())
