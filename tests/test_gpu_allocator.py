"""A caller's device allocator (ppn_set_allocator): scenes created while it is installed
take every device buffer from it and give every one back when destroyed, and they step
to the same bits as scenes on cudaMalloc.  A misaligned pointer from the allocator is
handed back and the creation fails cleanly."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2505_21013_gb300")
from paper_2505_21013_gb300 import ppn  # noqa: E402
from ppn_inputs import twisting_beam_scene  # noqa: E402


class TorchBlocks:
    """Device memory from torch's caching allocator, with a ledger of what is out."""

    def __init__(self, offset=0):
        self.out = {}
        self.n_alloc = self.n_free = 0
        self.offset = offset  # a nonzero offset hands out misaligned pointers

    def alloc(self, n):
        base = torch.cuda.caching_allocator_alloc(n + self.offset, device=0)
        self.n_alloc += 1
        self.out[base + self.offset] = base
        return base + self.offset

    def free(self, p):
        torch.cuda.caching_allocator_delete(self.out.pop(p))
        self.n_free += 1


def steps(spec, n, prec):
    sc = P.Scene.from_spec(spec, precision=prec)
    xs = []
    for k in range(n):
        sc.set_targets(spec.targets_at(k))
        rc, x, _ = sc.step(P.MODE_PPN, 1e-4, want_x=True)
        assert rc == 0
        xs.append(x)
    return sc, xs


@pytest.mark.parametrize("prec", [P.PREC_MIXED, P.PREC_FP64])
def test_scenes_on_a_caller_allocator_match_cudamalloc(prec):
    spec = twisting_beam_scene(5, 4, 12, h=0.02, E=1e5, nu=0.45, omega=20.0, dt=1 / 30, seed=3)
    ref_scene, ref = steps(spec, 3, prec)
    del ref_scene
    blocks = TorchBlocks()
    ppn.set_allocator(blocks.alloc, blocks.free)
    try:
        sc, xs = steps(spec, 3, prec)
    finally:
        ppn.set_allocator(None, None)
    assert blocks.n_alloc > 10 and blocks.out  # the scene and its group hold the caller's memory
    for a, b in zip(xs, ref):
        assert np.array_equal(a, b)
    sc.close()  # the scene and the groups it was in give everything back
    assert not blocks.out and blocks.n_free == blocks.n_alloc


def test_misaligned_allocator_memory_is_refused():
    spec = twisting_beam_scene(3, 3, 6, h=0.02, E=1e5, nu=0.45, omega=2.0, dt=1 / 30, seed=0)
    blocks = TorchBlocks(offset=16)
    ppn.set_allocator(blocks.alloc, blocks.free)
    try:
        with pytest.raises(P.PPNError):
            P.Scene.from_spec(spec, precision=P.PREC_MIXED)
    finally:
        ppn.set_allocator(None, None)
    assert blocks.n_alloc >= 1 and blocks.n_free == blocks.n_alloc and not blocks.out
    # the library still works on cudaMalloc afterwards
    _, xs = steps(spec, 1, P.PREC_MIXED)
    assert np.isfinite(xs[0]).all()


def test_server_scenes_on_a_caller_allocator_give_everything_back():
    # the server's scenes and the groups its worker builds for batches take the caller's
    # memory, from the worker thread as well; destroying the server returns all of it
    specs = [twisting_beam_scene(4, 4, 10, h=0.02, E=1e5, nu=0.45, omega=20.0, dt=1 / 30, seed=s) for s in (1, 2)]
    ref = []
    for spec in specs:
        sc, xs = steps(spec, 1, P.PREC_MIXED)
        ref.append(xs[0])
        sc.close()
    blocks = TorchBlocks()
    ppn.set_allocator(blocks.alloc, blocks.free)
    try:
        srv = P.Server(precision=P.PREC_MIXED, max_batch=2)
        ids = [srv.add_scene(spec) for spec in specs]
        tickets = [srv.submit(sid, P.MODE_PPN, 1e-4, spec.targets_at(0)) for sid, spec in zip(ids, specs)]
        for sid, t, x_ref in zip(ids, tickets, ref):
            done, rc, x, _, _ = srv.poll(t, sid)
            assert done and rc == 0
            disp = np.abs(x_ref - specs[ids.index(sid)].rest).max()
            assert np.abs(x - x_ref).max() <= 1e-6 * disp  # (the serving tests' bound for a scene in a mix)
        srv.close()
    finally:
        ppn.set_allocator(None, None)
    assert blocks.n_alloc > 0 and not blocks.out and blocks.n_free == blocks.n_alloc
