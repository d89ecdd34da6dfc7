"""GB300-native CD-CCSD analytic gradients (arXiv 2512.21909 hot path).

The computation lives in libcdcc.so (CUDA, sm_103a) behind the C ABI of
include/cdcc.h; `cdcc` is its ctypes binding.
"""
from . import cdcc  # noqa: F401
from .cdcc import (cd_ccsd_init, ccsd_solve, lambda_solve, build_density,  # noqa
                   contract_dL, gradient, cdcc_get_gamma, cdcc_get_amplitudes,
                   cdcc_phase_times, cdcc_kernel_launches, cdcc_last_error,
                   cd_ccsd_free, cdcc_default_options, cdcc_packed_size,
                   init_from_system, CdccError)
