"""Seeded synthetic LP inputs shared by the tests, the bench and the oracle runs.

This package only draws random numbers and lays out sparse matrices; it holds
none of the factorisation, solve or regularisation arithmetic.
"""
from .lp import (  # noqa: F401
    LP,
    random_lp,
    grid_multicommodity,
    block_angular,
    batched_random,
    batched_sizes,
    batched_instance,
    staircase,
    feasible_rhs,
    theta_loguniform,
    theta_schedule,
    rhs_normal,
    random_perm,
    by_name,
)
