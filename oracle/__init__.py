"""FP64 CPU oracle for the staggered-mesh MHD step.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only the test suite, the package smoke check
and the CPU-baseline leg of the benchmark may import it; the library itself
never does, and it shares no code with the CUDA sources.
"""
from .stagger import (  # noqa: F401
    Grid, Params, up, dn, ddup, dddn, rhs, rhs_parts, rk3_step, step, courant_dt,
    courant_fields, courant_limits,
    diagnostics, step_adjoint, quench, max3, smooth3, ALPHA, BETA,
    mirror_extend, fill_wall_ghosts, rhs_walls, courant_walls, step_walls, diagnostics_walls,
    WALL_PARITY, Z_FACE,
    face_densities, fill_rigid_ghosts, rhs_rigid, courant_rigid, step_rigid, diagnostics_rigid,
    fill_open_ghosts, rhs_open, courant_open, step_open, diagnostics_open, potential_horizontal,
)
