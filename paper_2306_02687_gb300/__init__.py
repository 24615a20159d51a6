"""GB300 (sm_103a) hyper-reduced FE^2 online path.

Implements, from Lange, Huetter, Kiefer, "A Monolithic Hyper ROM FE^2 Method
with Clustered Training at Finite Deformations" (arXiv 2306.02687), the
batched evaluation of the ROM/ECM-reduced RVE at every macro integration
point of a monolithic Newton iteration, its static condensation into the
homogenized stress and consistent tangent, the macro element assembly and the
implicit adjoint, as CUDA kernels behind the C ABI of include/rverom.h.

Python entry points (thin marshalling over librverom.so, see api.py):
  rve_rom_create, rve_rom_set_moduli, rve_rom_autotune, rve_rom_select_kernel,
                  rve_rom_kernel_info, rve_rom_eval_batch, rve_rom_adjoint,
  macro_mesh_create, macro_gradient, macro_assemble, macro_residual_norms,
                  macro_solve (global Newton correction on the device),
                  macro_gradient_range, macro_assemble_range (one element shard)
  parallel: element sharding and the all-reduce of the assembled system
  rve_rom_eval_batch_j2, rve_rom_mmax (history-dependent J2 law at the ECM points)
  rve_rom_biot_cauchy (Biot / Cauchy outputs), surrogate_linear_eval,
                  paths_kmeans (clustered training)
  rverom_df_log, rverom_peak_probe (diagnostics)
"""
from .api import (FP64, MIXED, RomHandle, MeshHandle, load_rom_file, rve_rom_create,  # noqa: F401
                  rve_rom_set_moduli, rve_rom_autotune, rve_rom_select_kernel,
                  rve_rom_kernel_info, rve_rom_eval_batch, rve_rom_adjoint, rve_rom_adjoint_static,
                  macro_mesh_create,
                  macro_gradient, macro_assemble, macro_residual_norms, macro_solve, rve_rom_mmax,
                  macro_gradient_range, macro_assemble_range,
                  rve_rom_eval_batch_j2, rve_rom_biot_cauchy,
                  surrogate_linear_eval, paths_kmeans, rverom_df_log, rverom_peak_probe)
from .autograd import RveStress, rve_stress  # noqa: F401
