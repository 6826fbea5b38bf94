"""Seeded synthetic inputs shared by the oracle and the GPU path.

This package only *generates* inputs: mesh coordinates and connectivity,
element partitions, initial states and noise.  It contains none of the
discretisation's arithmetic (no basis functions, metrics, fluxes or solvers),
so that the oracle and the CUDA library stay independent of one another while
being fed identical data.
"""

from .mesh import QuadMesh, structured_quads, uniform_nodes, geometric_nodes, tanh_nodes
from .states import (
    gaussian_scalar,
    isentropic_vortex,
    uniform_noise,
    freestream,
)
from .configs import CONFIGS, make_config

__all__ = [
    "QuadMesh",
    "structured_quads",
    "uniform_nodes",
    "geometric_nodes",
    "tanh_nodes",
    "gaussian_scalar",
    "isentropic_vortex",
    "uniform_noise",
    "freestream",
    "CONFIGS",
    "make_config",
]
