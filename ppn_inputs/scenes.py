"""Seeded synthetic scenes shaped like the paper's workloads.

A scene is a tet mesh plus material, time step, gravity, the indices of the
Dirichlet (fixed or kinematically driven) vertices and a function giving those
vertices' target positions at the end of every time step.  Parameter ranges
follow the paper's scene table (E 1e4-1e10 Pa, nu 0.3-0.49, rho 1000 kg/m^3,
dt 1/30-1/300 s); the meshes are Kuhn grids because the paper's meshes are not
available.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from .meshes import grid_index, kuhn_grid

GRAVITY = (0.0, -9.81, 0.0)


@dataclass
class SceneSpec:
    name: str
    rest: np.ndarray              # (n_v, 3) float64
    tets: np.ndarray              # (n_t, 4) int32
    fixed: np.ndarray             # (n_fixed,) int32, sorted, unique
    E: float
    nu: float
    rho: float
    dt: float
    gravity: tuple = GRAVITY
    # targets(n) -> (n_fixed, 3) float64 positions of ``fixed`` at the end of step n
    targets: Optional[Callable[[int], np.ndarray]] = None
    meta: dict = field(default_factory=dict)
    # obstacles(n) -> analytic surfaces at the end of step n, each a tuple
    # (kind, point, axis_or_normal, radius) with kind "plane" | "cylinder_in" | "sphere_out"
    obstacles: Optional[Callable[[int], list]] = None

    @property
    def n_verts(self) -> int:
        return int(self.rest.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    def targets_at(self, n: int) -> np.ndarray:
        if self.targets is None:
            return self.rest[self.fixed].copy()
        return np.ascontiguousarray(self.targets(n), dtype=np.float64)

    def obstacles_at(self, n: int) -> list:
        return [] if self.obstacles is None else list(self.obstacles(n))


def _face(nx, ny, nz, axis, index):
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    sel = (ii, jj, kk)[axis] == index
    return np.sort(grid_index(ii[sel], jj[sel], kk[sel], nx, ny)).astype(np.int32)


def cube_scene(n: int = 5, size: float = 1.0, E: float = 1e5, nu: float = 0.4,
               rho: float = 1000.0, dt: float = 1.0 / 60.0, jitter: float = 0.01,
               seed: int = 0, name: Optional[str] = None) -> SceneSpec:
    """``n^3``-vertex cube of edge ``size`` resting on its fixed y=0 face, under gravity."""
    h = size / (n - 1)
    rest, tets = kuhn_grid(n, n, n, h, jitter=jitter, seed=seed)
    fixed = _face(n, n, n, axis=1, index=0)
    return SceneSpec(name or f"cube{n}", rest, tets, fixed, E, nu, rho, dt,
                     meta={"kind": "cube", "dims": (n, n, n), "h": h, "seed": seed})


def twisting_beam_scene(nx: int = 20, ny: int = 20, nz: int = 80, h: float = 0.01,
                        E: float = 1e6, nu: float = 0.45, rho: float = 1000.0,
                        dt: float = 1.0 / 30.0, omega: float = 2.0, jitter: float = 0.01,
                        seed: int = 0, name: Optional[str] = None) -> SceneSpec:
    """Beam along z: the z=0 end is clamped, the z=max end turns about the beam axis at ``omega`` rad/s."""
    rest, tets = kuhn_grid(nx, ny, nz, h, jitter=jitter, seed=seed)
    clamp = _face(nx, ny, nz, axis=2, index=0)
    driven = _face(nx, ny, nz, axis=2, index=nz - 1)
    fixed = np.concatenate([clamp, driven]).astype(np.int32)
    order = np.argsort(fixed)
    fixed = fixed[order]
    is_driven = np.concatenate([np.zeros(len(clamp), bool), np.ones(len(driven), bool)])[order]
    cx = 0.5 * (nx - 1) * h
    cy = 0.5 * (ny - 1) * h
    base = rest[fixed].copy()

    def targets(n: int) -> np.ndarray:
        ang = omega * dt * (n + 1)
        c, s = np.cos(ang), np.sin(ang)
        out = base.copy()
        px = base[is_driven, 0] - cx
        py = base[is_driven, 1] - cy
        out[is_driven, 0] = cx + c * px - s * py
        out[is_driven, 1] = cy + s * px + c * py
        return out

    return SceneSpec(name or f"beam{nx}x{ny}x{nz}", rest, tets, fixed, E, nu, rho, dt,
                     targets=targets,
                     meta={"kind": "beam", "dims": (nx, ny, nz), "h": h, "omega": omega,
                           "seed": seed})


def tiny_scene(cells=(1, 1, 1), h: float = 0.1, E: float = 1e4, nu: float = 0.4,
               rho: float = 1000.0, dt: float = 1.0 / 30.0, jitter: float = 0.02,
               seed: int = 0, fixed_face: bool = True) -> SceneSpec:
    """A few-tet grid for brute-force checks (``cells`` hexahedra, 6 tets each)."""
    nx, ny, nz = (c + 1 for c in cells)
    rest, tets = kuhn_grid(nx, ny, nz, h, jitter=jitter, seed=seed)
    fixed = _face(nx, ny, nz, axis=1, index=0) if fixed_face else np.zeros(0, np.int32)
    return SceneSpec(f"tiny{cells}", rest, tets, fixed, E, nu, rho, dt,
                     meta={"kind": "tiny", "dims": (nx, ny, nz), "h": h, "seed": seed})


def _grid_dims_for_tets(T: float, beam: bool):
    if beam:
        c = max(1, int(round((T / 24.0) ** (1.0 / 3.0))))
        return c + 1, c + 1, 4 * c + 1
    c = max(1, int(round((T / 6.0) ** (1.0 / 3.0))))
    return c + 1, c + 1, c + 1


def _random_scene(rng, idx: int, tmin: float, tmax: float, seed: int) -> SceneSpec:
    T = float(np.exp(rng.uniform(np.log(tmin), np.log(tmax))))
    beam = bool(rng.integers(0, 2))
    nx, ny, nz = _grid_dims_for_tets(T, beam)
    E = float(np.exp(rng.uniform(np.log(1e4), np.log(1e7))))
    nu = float(rng.uniform(0.3, 0.48))
    dt = float(rng.choice([1.0 / 30.0, 1.0 / 60.0, 1.0 / 120.0]))
    if beam:
        h = 0.8 / (nz - 1)
        spec = twisting_beam_scene(nx, ny, nz, h=h, E=E, nu=nu, dt=dt, omega=1.0,
                                   seed=seed * 1000 + idx, name=f"beam_{idx}")
    else:
        spec = cube_scene(nx, size=0.5, E=E, nu=nu, dt=dt, seed=seed * 1000 + idx,
                          name=f"cube_{idx}")
    spec.meta["target_tets"] = T
    return spec


def random_batch_scenes(n: int = 64, tmin: float = 1e3, tmax: float = 5e4,
                        seed: int = 0) -> list:
    """``n`` independent cube/beam scenes with log-uniform tet counts and materials."""
    rng = np.random.default_rng(seed)
    return [_random_scene(rng, i, tmin, tmax, seed) for i in range(n)]


def serving_scenes(n: int = 200, tmin: float = 2e3, tmax: float = 2e5, seed: int = 1) -> list:
    """Resident scenes for the request-stream workload (tet counts log-uniform)."""
    rng = np.random.default_rng(seed)
    return [_random_scene(rng, i, tmin, tmax, seed) for i in range(n)]


def poisson_arrivals(rate_hz: float, n: int, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson stream."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))


def drop_scene(cells=(3, 3, 3), size: float = 0.1, height: float = 0.002, E: float = 1e5,
               nu: float = 0.4, rho: float = 1000.0, dt: float = 1.0 / 60.0, obstacle: str = "plane",
               seed: int = 0, name: Optional[str] = None) -> SceneSpec:
    """A free cube (no Dirichlet vertices) whose lowest face starts ``height`` above
    the ground plane y = 0 and falls under gravity onto it.  ``obstacle`` = "sphere"
    adds a sphere below the cube's centre that the cube lands on instead (its
    contact Hessians are indefinite)."""
    nx, ny, nz = (c + 1 for c in cells)
    h = size / max(cells)
    rest, tets = kuhn_grid(nx, ny, nz, h, jitter=0.01, seed=seed)
    rest[:, 1] += height
    centre = rest.mean(axis=0)
    obst = [("plane", (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 0.0)]
    if obstacle == "sphere":
        r = 0.5 * size
        obst = [("sphere_out", (centre[0], -r + 0.5 * height, centre[2]), (0.0, 0.0, 0.0), r)] + obst
    return SceneSpec(name or f"drop{nx}x{ny}x{nz}", rest, tets, np.zeros(0, np.int32), E, nu, rho, dt,
                     obstacles=lambda n: obst, meta={"kind": "drop", "h": h, "seed": seed})


def press_scene(n: int = 40, boxes: int = 4, edge: float = 0.06, radius: float = 0.1, E: float = 1e5,
                nu: float = 0.4, rho: float = 1000.0, dt: float = 1.0 / 60.0, press_speed: float = 0.05,
                gap: float = 0.002, seed: int = 0, name: Optional[str] = None) -> SceneSpec:
    """Boxes of n^3 vertices (edge ``edge``) side by side on a square grid with
    ``gap`` between them, standing on the ground plane y = 0 inside a vertical
    cylinder of ``radius`` (axis y through the grid's centre), under a press plane
    that starts ``gap`` above them and descends at ``press_speed``.  (Boxes do not
    touch each other: contact is with the analytic obstacles only.  The press's
    rotation about the vertical axis does not act on frictionless contact.)
    ``obstacles_at(-1)`` is the initial pose."""
    h = edge / (n - 1)
    k = int(np.ceil(np.sqrt(boxes)))
    width = k * edge + (k - 1) * gap
    if np.hypot(width / 2, width / 2) >= radius - gap:
        raise ValueError("the boxes do not fit inside the cylinder")
    parts_x, parts_t = [], []
    off = 0
    for b in range(boxes):
        i, j = b % k, b // k
        x, t = kuhn_grid(n, n, n, h, jitter=0.005, seed=seed + b)
        x[:, 0] += -width / 2 + i * (edge + gap)
        x[:, 2] += -width / 2 + j * (edge + gap)
        x[:, 1] += gap
        parts_x.append(x)
        parts_t.append(t + off)
        off += x.shape[0]
    rest = np.concatenate(parts_x)
    tets = np.concatenate(parts_t).astype(np.int32)
    top = float(rest[:, 1].max()) + gap

    def obstacles(step):
        y = top - press_speed * dt * (step + 1)
        return [("plane", (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 0.0),
                ("cylinder_in", (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), radius),
                ("plane", (0.0, y, 0.0), (0.0, -1.0, 0.0), 0.0)]

    return SceneSpec(name or f"press{boxes}x{n}", rest, tets, np.zeros(0, np.int32), E, nu, rho, dt,
                     obstacles=obstacles, meta={"kind": "press", "h": h, "seed": seed})
