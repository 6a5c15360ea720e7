"""GB300-native particle time step of the joint velocity-frequency-scalar PDF
method (Bakosi 2008) behind a C-ABI library of hand-written sm_103a kernels.

The Python layer only marshals arguments; `capi.lib()` loads libpdfgb.so
(building it with nvcc if needed) and raises if that is impossible.
"""
from . import capi
from .capi import PdfError, lib
from .api import (Mesh, Mlp, Particles, pdf_mlp_batch, pdf_mlp_features, model_params, pdf_elem_coeff, pdf_estimate_stats,
                  pdf_estimate_stats_noalloc, pdf_kernel_launches,
                  pdf_last_error, pdf_mesh_create, pdf_particles_init, pdf_particles_load, pdf_particles_save, pdf_profile_enable, pdf_profile_only,
                  pdf_profile_query, pdf_profile_reset, pdf_relax_rhs, pdf_relax_solve, pdf_relax_solve_particles,
                  pdf_relax_set_solver, pdf_rng_gauss,
                  pdf_pressure_project, pdf_pressure_field, pdf_pressure_set_solver, pdf_redistribute,
                  pdf_step, pdf_step_host, pdf_step_host_stats)

__all__ = ["capi", "PdfError", "lib", "Mesh", "Mlp", "pdf_mlp_batch", "pdf_mlp_features", "Particles", "model_params", "pdf_mesh_create",
           "pdf_particles_init", "pdf_particles_save", "pdf_particles_load", "pdf_step", "pdf_estimate_stats", "pdf_estimate_stats_noalloc", "pdf_elem_coeff", "pdf_rng_gauss",
           "pdf_last_error", "pdf_profile_enable", "pdf_profile_only", "pdf_profile_reset", "pdf_profile_query",
           "pdf_kernel_launches", "pdf_relax_solve", "pdf_relax_solve_particles", "pdf_relax_rhs", "pdf_relax_set_solver",
           "pdf_pressure_project", "pdf_pressure_field", "pdf_pressure_set_solver", "pdf_redistribute",
           "pdf_step_host", "pdf_step_host_stats"]
