"""Seeded synthetic inputs for the NEAREST regularized-stokeslet method.

This package is the one piece shared by the CPU oracle and the CUDA path.
It produces *inputs only*: body-frame point clouds (force points, quadrature
points with their area weights), prescribed deformation velocities, and the
initial rigid-body state of each body.  It contains none of the method's
arithmetic (no stokeslet, no nearest-neighbour search, no assembly, no solve).

Random draws use SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), one seed per workload.
"""

from .geometry import (  # noqa: F401
    SplitMix64,
    Body,
    Problem,
    cube_sphere_vertices,
    cube_sphere_cells,
    tube_shape,
    sphere_config,
    sphere_cells_config,
    swimmer_config,
    swimmers_config,
    sperm_channel_config,
    node_config,
    node_batch,
    vogel_disc,
    rod_line,
    workload,
    pack_shapes,
    initial_state,
    WORKLOADS,
)
from .mlp_inputs import mlp_init, mlp_batch, mlp_perturb  # noqa: F401,E402
