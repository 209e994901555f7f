"""Seeded synthetic inputs for parametrized Lyapunov sweeps.

This package holds only problem generators (the application models of the
paper's §3 and the parameter sweeps of its experiments). It contains none of
the solution method's arithmetic, so both the CPU oracle and the GPU library's
tests and benchmark can draw their inputs from it.
"""
from .generators import (  # noqa: F401
    Problem,
    mass_spring_chain,
    two_row_masses,
    two_row_system,
    multi_agent,
    haar_orthogonal,
    generic_dense,
    config_rngs,
    workload_small_fp64,
    workload_precision,
    workload_serving_seeds,
    workload_serving_requests,
    workload_differentiation,
    workload_multi_agent,
    order_nearest_neighbour,
    chain_stiffness,
    rayleigh_chain,
    workload_rayleigh,
    ex3_laplacian,
    agent_network,
    ex3_problem,
    ex3_grid,
    stable_mask,
    workload_ex3,
    EX3_POSITIONS,
)
