"""GB300-native anharmonic lattice-dynamics hot path (arXiv:2009.01967).

The computation lives in libkald.so (CUDA, sm_103a), whose C ABI is
include/kald.h; this package is its thin Python binding.  Build the library
with `paper_2009_01967_gb300.build.build()` (or `__graft_entry__.build()`).
"""

from ._abi import (Context, KaldError, Options, EXPORTS, LIB_PATH, load_library,  # noqa: F401
                   kald_phonons, kald_linewidths, kald_kappa_rta, kald_kappa_qhgk,
                   kald_kappa_rta_noalloc, kald_kernel_launches, kald_linewidths_qrange,
                   kald_linewidths_qlist,
                   kald_phonons_batch, kald_phase_space, kald_diffusivity,
                   kald_scattering_matrix, kald_kappa_bte, kald_interpolate_gamma,
                   kald_fd_force_constants)

__all__ = ["Context", "KaldError", "Options", "EXPORTS", "LIB_PATH", "load_library",
           "kald_phonons", "kald_linewidths", "kald_kappa_rta", "kald_kappa_qhgk",
           "kald_kappa_rta_noalloc", "kald_kernel_launches", "kald_linewidths_qrange",
           "kald_linewidths_qlist",
           "kald_phonons_batch", "kald_phase_space", "kald_diffusivity",
           "kald_scattering_matrix", "kald_kappa_bte", "kald_interpolate_gamma",
           "kald_fd_force_constants"]
