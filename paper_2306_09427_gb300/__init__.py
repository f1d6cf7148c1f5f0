"""Batched fiber-network RVE solver for GB300 (sm_103a).

Python binding of the C ABI declared in ``include/rve.h``: argument
marshalling only, every step of the solve runs in the CUDA kernels of
``librve.so``.  Importing this package fails loudly when the library has
not been built: there is no CPU fallback.
"""
from ._lib import (RVE_DAMP_KINETIC, RVE_DAMP_VISCOUS, RVE_KERNEL_AUTO, RVE_KERNEL_NODE, RVE_KERNEL_TWO_PHASE, RVE_EADMIT, RVE_ECUDA, RVE_EINVAL, RVE_ENOMEM, RVE_OK, RVE_PREC_BATCHED_F64,
                   RVE_PREC_MIXED, RVE_PREC_PLAIN_F64, RVE_STATUS_CONVERGED, RVE_STATUS_EMPTY,
                   RVE_STATUS_MAX_ITER, RVE_STATUS_NONFINITE, RVE_STATUS_RUNNING, RveBatch, RveError, RveServer, lib, lib_path,
                   rve_batch_create, rve_batch_destroy, rve_batch_get_info, rve_batch_get_sizes,
                   rve_get_positions, rve_set_positions, rve_last_error, rve_options_default, rve_reset_state,
                   rve_set_options, rve_solve, rve_solve_host, rve_solve_plain_noalloc, rve_solve_subset,
                   rve_tangent, RVE_NOALLOC_MAX_ACTIVE_FIBERS, RVE_NOALLOC_MAX_FREE_NODES,
                   rve_server_create, rve_server_destroy, rve_server_drain, rve_server_get_stats,
                   rve_server_poll, rve_server_step, rve_server_submit, rve_server_set_wave_iters,
                   rve_server_add_rves, rve_server_remove_rves, rve_autotune, rve_batch_get_bins,
                   rve_set_kernel_timing, rve_last_kernel_ms, rve_tangent_mandel, rve_orientation, rve_energy)

__all__ = [n for n in dir() if n.startswith(("rve_", "RVE_", "Rve"))] + ["lib", "lib_path"]
