"""Seeded synthetic workloads for the particle time step.

This package only *generates inputs*: meshes, per-element particle counts and
initial scalar slabs, and the configuration values of each workload.  It holds
none of the method's arithmetic, so both the CUDA library and the CPU oracle
consume exactly the same inputs without sharing any computation.
"""
from .channel import channel_mesh, scalar_slab, TAG_WALL, TAG_PERIODIC, TAG_INFLOW, TAG_OUTFLOW, TAG_NOSLIP
from .configs import CONFIGS, OBSTACLES, workload
from .obstacles import counts_by_area, obstacle_mesh

__all__ = ["channel_mesh", "scalar_slab", "CONFIGS", "OBSTACLES", "workload", "obstacle_mesh", "counts_by_area",
           "TAG_WALL", "TAG_PERIODIC", "TAG_INFLOW", "TAG_OUTFLOW", "TAG_NOSLIP"]
