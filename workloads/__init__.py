"""Seeded synthetic inputs shared by the oracle-side tests and the GPU-side tests/bench.

This package holds input generators and workload descriptions only: no step of the
solver's arithmetic lives here (see ``generators`` for what each input is).
"""
from .generators import (  # noqa: F401
    WORKLOADS,
    Workload,
    batch_problems,
    layered_wavenumber,
    layered_wavenumber_elements,
    random_complex,
    point_source_rhs,
    plane_wave_2d,
    problem_inputs,
)
