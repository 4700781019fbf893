"""Structured tetrahedral meshes (Kuhn / Freudenthal 6-tet split of a voxel grid).

Every hexahedral cell of an ``nx x ny x nz`` vertex grid is split into the six
tets that follow the monotone lattice paths from its corner (0,0,0) to its
corner (1,1,1).  All cells use the same main diagonal, so neighbouring cells
share their face triangulations and the mesh is conforming.  Vertex ``(i,j,k)``
has index ``i + nx*(j + ny*k)`` (x fastest).

Rest positions may be jittered uniformly by up to ``jitter`` times the edge
length per coordinate, drawn from ``numpy.random.default_rng(seed)``; tets are
oriented on the unjittered grid so that every tet has a positive signed volume
(a jitter below ~10 % of the edge cannot flip one).
"""

from __future__ import annotations

import itertools

import numpy as np


def grid_index(i, j, k, nx: int, ny: int):
    """Vertex index of lattice point (i, j, k) in an nx x ny x nz grid."""
    return i + nx * (j + ny * k)


def kuhn_grid(nx: int, ny: int, nz: int, h: float, origin=(0.0, 0.0, 0.0),
              jitter: float = 0.0, seed: int = 0):
    """Return ``(rest, tets)`` for an ``nx x ny x nz`` vertex grid of spacing ``h``.

    ``rest`` is ``(nx*ny*nz, 3)`` float64, ``tets`` is ``(6*(nx-1)*(ny-1)*(nz-1), 4)``
    int32 with positive orientation (det[x1-x0, x2-x0, x3-x0] > 0).
    """
    if min(nx, ny, nz) < 2:
        raise ValueError("a Kuhn grid needs at least 2 vertices per axis")
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    # x fastest: flatten in (k, j, i) order
    lattice = np.stack([ii.transpose(2, 1, 0).ravel(),
                        jj.transpose(2, 1, 0).ravel(),
                        kk.transpose(2, 1, 0).ravel()], axis=1).astype(np.float64)
    grid = np.asarray(origin, dtype=np.float64)[None, :] + h * lattice

    ci, cj, ck = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), np.arange(nz - 1), indexing="ij")
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()

    def corner(b):
        return grid_index(ci + b[0], cj + b[1], ck + b[2], nx, ny)

    tets = []
    for perm in itertools.permutations(range(3)):
        b = [0, 0, 0]
        path = [corner(tuple(b))]
        for ax in perm:
            b[ax] = 1
            path.append(corner(tuple(b)))
        tets.append(np.stack(path, axis=1))
    # interleave so that the 6 tets of one cell are adjacent in memory
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int64)

    # orient on the unjittered grid
    p = grid[tets]
    d = np.linalg.det(np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]], axis=2))
    neg = d < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()

    rest = grid.copy()
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        rest += rng.uniform(-jitter * h, jitter * h, size=rest.shape)
    return rest, tets.astype(np.int32)
