"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds no arithmetic of the multiscale method itself: it draws
log-normal permeability fields, places wells and states the workload
parameters (grid, coarsening, fluid, time step, solver options).  Both the
CPU oracle and the GPU binding receive the same arrays from here.
"""
from .fields import gaussian_field, lognormal_permeability  # noqa: F401
from .configs import (Workload, WORKLOADS, make_inputs, line_columns,  # noqa: F401
                      ensemble_members)
