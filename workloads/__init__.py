"""Seeded synthetic inputs for the all-at-once heat problems.

This package only draws random numbers and evaluates the input functions
(sine series, Gaussian random fields, the wind and wall data of the
convection-diffusion example).  It holds none of the method's
arithmetic, so both the CPU oracle and the GPU path may use it.
"""
from .heat import (  # noqa: F401
    HeatCase,
    grid_points,
    heat_case_1d,
    heat_case_2d,
    eps_sqrt_tau,
    batch_cases,
    grf_log_coefficient,
    circulating_wind_case,
)
