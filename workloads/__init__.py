"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This package holds no arithmetic of the solver: it only produces node sets
(interior nodes first, then Dirichlet boundary nodes), evaluation points, the
manufactured exact solutions and the right-hand side data derived from them.
Both sides of every parity check draw their inputs from here.
"""
from .nodes import (  # noqa: F401
    NodeSet,
    cube_grid,
    cube_faces_halton,
    sphere_fibonacci_ball,
    cube_faces_random,
    pump_like,
    batch_instances,
    stop_instances,
    paper_nodes,
    test_points,
    scrambled_halton,
    fibonacci_sphere,
    preset,
    PRESETS,
)
from .problem import (  # noqa: F401
    plane_wave,
    plane_wave_rhs,
    gaussian,
    gaussian_source,
    gaussian_rhs,
    instance_rhs,
    instance_field,
)
