"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package only draws random numbers and lays out input arrays: permeability
fields, well source fields, subdomain edge lists and patch sizes.  It holds none
of the method's arithmetic (no transmissibilities, no interface spaces, no
solves), so that the oracle and the GPU path can both read the same inputs
without sharing any computation.
"""
from .fields import gaussian_field, layered_field, lognormal_K
from .wells import corner_wells, five_spot_wells
from .configs import Workload, workload, WORKLOADS

__all__ = [
    "gaussian_field", "layered_field", "lognormal_K",
    "corner_wells", "five_spot_wells",
    "Workload", "workload", "WORKLOADS",
]
