"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This package holds mesh and scene generators only: vertex grids, tet
connectivity, material draws and boundary kinematics.  It contains none of the
solver's arithmetic (no energy, no derivative, no projection, no solve), so
both the CUDA path and the FP64 oracle may consume its outputs without sharing
any code of the method.
"""

from .meshes import kuhn_grid, grid_index
from .scenes import (
    SceneSpec,
    cube_scene,
    twisting_beam_scene,
    random_batch_scenes,
    serving_scenes,
    poisson_arrivals,
    tiny_scene,
    drop_scene,
    press_scene,
)

__all__ = [
    "kuhn_grid",
    "grid_index",
    "SceneSpec",
    "cube_scene",
    "twisting_beam_scene",
    "random_batch_scenes",
    "serving_scenes",
    "poisson_arrivals",
    "tiny_scene",
    "drop_scene",
    "press_scene",
]
