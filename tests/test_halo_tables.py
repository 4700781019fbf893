"""Host-side tables of the PCG's halo layout (``ppn_probe_halo_tables``, no GPU
needed), checked against their definition: CTA b of G owns launch tiles
[b T / G, (b + 1) T / G) of 128 rows; each of its blocks' local column names
the block's column (an own row by its position in the CTA, any other row by
its place in the CTA's halo list); the halo list holds exactly the other
CTAs' rows that the CTA's blocks refer to, ascending.  The patterns are the
oracle's BSR patterns of the benchmark beam, of a mix of request-stream scenes
whose CTAs hold tiles of two scenes, and of small scenes at the extreme grids."""

import numpy as np
import pytest

P = pytest.importorskip("paper_2505_21013_gb300")
from oracle import oracle as O  # noqa: E402
from ppn_inputs import cube_scene, serving_scenes, twisting_beam_scene  # noqa: E402

TILE, ROW_BITS = 128, 26


def pattern(spec):
    rp, col = O.Scene.from_spec(spec).pattern()
    return np.asarray(rp, np.int64), np.asarray(col, np.int32)


def expected_max_halo_and_check(pats, grid):
    """Checks the library's tables against the definition; returns the most halo rows."""
    off, lcol, ref, mh = P.ppn.probe_halo_tables(pats, grid)
    ntile = [(len(rp) - 1 + TILE - 1) // TILE for rp, _ in pats]
    toff = np.concatenate([[0], np.cumsum(ntile)]).astype(np.int64)
    T = int(toff[-1])
    # every block of the launch, slot after slot, rows and blocks ascending: the kernel's
    # order, in which each CTA's blocks are one contiguous run
    k = np.concatenate([np.full(len(c), s) for s, (_, c) in enumerate(pats)]).astype(np.int64)
    j = np.concatenate([c for _, c in pats]).astype(np.int64)
    row = np.concatenate([np.repeat(np.arange(len(rp) - 1), np.diff(rp)) for rp, _ in pats])
    owner = lambda t: ((t + 1) * grid + T - 1) // T - 1  # CTA of launch tile t
    b = owner(toff[k] + row // TILE)
    assert np.all(np.diff(b) >= 0)
    t0 = (np.arange(grid + 1) * T) // grid
    starts = np.searchsorted(b, np.arange(grid + 1))
    assert np.array_equal(off[:, 0], starts) and off[grid, 0] == len(lcol) == len(j)
    ct = toff[k] + j // TILE  # launch tile of each block's column
    own = (ct >= t0[b]) & (ct < t0[b + 1])
    assert np.array_equal(lcol[own], (ct - t0[b])[own] * TILE + j[own] % TILE)
    n_items = (t0[b + 1] - t0[b]) * TILE
    h = lcol - n_items
    assert np.all(h[~own] >= 0) and np.all(lcol[own] < n_items[own])
    key = (k << ROW_BITS) | j
    assert np.array_equal(ref[off[b[~own], 1] + h[~own]], key[~own])
    most = 0
    for c in range(grid):
        hl = ref[off[c, 1]:off[c + 1, 1]]
        mine = np.unique(key[(b == c) & ~own])
        assert np.array_equal(hl, mine)  # exactly the referenced rows of other CTAs, ascending
        most = max(most, len(hl))
    assert mh == most
    return mh


def test_beam_tables_at_the_benchmark_grid():
    spec = twisting_beam_scene(20, 20, 80, h=0.01, E=1e6, nu=0.45, omega=2.0, dt=1.0 / 30.0, seed=0)
    mh = expected_max_halo_and_check([pattern(spec)], 152)
    # 250 tiles over 152 CTAs: two-tile CTAs see about one 20x20 layer on either side
    assert 400 < mh < 700


def test_request_stream_mix_with_ctas_spanning_scenes():
    pool = serving_scenes(200, seed=1)
    pats = [pattern(pool[i]) for i in (108, 118, 125, 144, 191)]
    assert expected_max_halo_and_check(pats, 152) > 0  # 192 tiles: 40 CTAs hold two


@pytest.mark.parametrize("grid", [1, 2, 3, 4, 5])
def test_small_scenes_at_every_grid(grid):
    # 343 + 160 rows: 3 + 2 tiles, the last of each ragged; two CTAs split the cube
    pats = [pattern(cube_scene(7, seed=2)), pattern(twisting_beam_scene(4, 4, 10, h=0.02, seed=3))]
    mh = expected_max_halo_and_check(pats, grid)
    assert (mh == 0) == (grid == 1)


def test_invalid_arguments():
    pat = pattern(cube_scene(4, seed=1))  # 125 rows: one tile
    with pytest.raises(P.PPNError):
        P.ppn.probe_halo_tables([pat], 0)
    with pytest.raises(P.PPNError):
        P.ppn.probe_halo_tables([pat], 2)  # more CTAs than tiles
    with pytest.raises(P.PPNError):
        P.ppn.probe_halo_tables([pat] * 9, 1)  # more scenes than one launch of the layout takes
