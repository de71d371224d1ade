"""Seeded synthetic workloads for the LBRS solver and its oracle.

Every input of the tests and the benchmark comes from here: primitive fields
(rho, u, [v,] p), boundary conditions, the lattice speed lambda, the number of
steps.  The generators draw with numpy's PCG64 and hold no arithmetic of the
lattice Boltzmann relaxation scheme itself; both the CUDA path and the CPU
oracle convert the primitive fields to conserved variables on their own.
"""
from .generators import (  # noqa: F401
    CONFIG_NAMES,
    GAMMA,
    Workload1D,
    Workload2D,
    TubeBatch,
    adjoint_pulses,
    batched_tubes,
    burgers_2d,
    burgers_steady_exact,
    bouchut_speed,
    explosion,
    forward_facing_step,
    from_config,
    load_config,
    normal_shock_state,
    shock_diffraction,
    lambda_1d_riemann,
    lambda_2d_quadrants,
    oblique_shock_reflection,
    paper_riemann_case4,
    quadrant_riemann,
    sod,
    steady_contact,
    steady_shock,
    uniform_2d,
)
