"""Seeded synthetic workloads for the PT-TEBD time step.

This package holds only problem parameters and seeded random draws. It contains
none of the method's arithmetic: no Liouvillians, no propagators, no influence
functionals, no contractions. Both the FP64 oracle (``oracle/``) and the GPU path
(``paper_2201_05529_gb300``) build their own inputs from these descriptions.
"""
from .configs import (  # noqa: F401
    ChainSpec, BathSpec, DriveSpec, Workload, workload, WORKLOAD_NAMES, BASE_SEED,
)
