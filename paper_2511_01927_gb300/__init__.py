"""GB300-native contour-integral generalized eigensolver (arXiv 2511.01927 hot path).

Python binding of the C ABI in include/gcie.h: the functions here carry the C names and only
marshal arguments (numpy / torch buffers to pointers, option structs); every step of the solve
runs in libgcie.so's CUDA kernels.  There is no CPU fallback: importing works without the
library, but the first call raises if libgcie.so is missing or cannot be loaded.
"""
from ._binding import (  # noqa: F401
    GcieError, STATUS, lib, library_path, csr_struct, default_opts,
    gcie_create, gcie_destroy, gcie_pencil_create, gcie_pencil_destroy, gcie_solve, gcie_solve_pencil, gcie_solve_batch,
    gcie_kde_contours, gcie_plan_contours, gcie_count_miss, gcie_resplit, gcie_trapezoid_nodes, gcie_shifted_spmm_f32, gcie_shifted_spmm_f64, gcie_shifted_solve, gcie_moments,
    gcie_m_orthonormalize, gcie_rayleigh_ritz, gcie_jacobi_eig, gcie_jacobi_eig_noalloc, gcie_get_stats, gcie_reset_stats, gcie_set_profile,
    gcie_gemm_tf32x3, gcie_gemm_bf16, gcie_density_net_create, gcie_density_net_destroy, gcie_density_predict,
    gcie_hist_quantiles, DENSITY_NWEIGHTS, DENSITY_BINS, gcie_fp64_rates,
    EXPORTED_SYMBOLS,
)
