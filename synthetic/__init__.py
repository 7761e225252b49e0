"""Seeded synthetic inputs for the color-gradient LBM (sphere-pack rock images).

This module only draws random geometry and initial fluid layouts. It holds none
of the lattice Boltzmann arithmetic, so both the CUDA path and the CPU oracle
can take their inputs from it without sharing any of the method's code.

Array convention everywhere: a 3-D voxel array has shape (nz, ny, nx) in C
order, so x varies fastest and the flat voxel index is x + nx*(y + ny*z).
"""
from .spherepack import (  # noqa: F401
    SpherePack,
    sphere_pack,
    add_walls,
    uniform_affinity,
    random_affinity,
    phi0_iid,
    phi0_blob,
    phi0_reservoir,
    Workload,
    workload_parity32,
    workload_steady256,
    workload_precision1024,
    workload_batched_job,
    serving_job,
    crop,
)
