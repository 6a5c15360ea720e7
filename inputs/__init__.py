"""Seeded synthetic workloads for the particle time step.

This package only *generates inputs*: meshes, per-element particle counts and
initial scalar slabs, and the configuration values of each workload.  It holds
none of the method's arithmetic, so both the CUDA library and the CPU oracle
consume exactly the same inputs without sharing any computation.
"""
from .channel import channel_mesh, scalar_slab, TAG_WALL, TAG_PERIODIC, TAG_INFLOW, TAG_OUTFLOW
from .configs import CONFIGS, workload

__all__ = ["channel_mesh", "scalar_slab", "CONFIGS", "workload",
           "TAG_WALL", "TAG_PERIODIC", "TAG_INFLOW", "TAG_OUTFLOW"]
