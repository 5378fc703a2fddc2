"""GB300 Golub-Kahan partial SVD and numerical rank (arXiv 2104.10785).

The compute path is libgk.so (CUDA, sm_103a) behind the C ABI in include/gk.h;
this package holds the kernels' sources (csrc/), the build step and the ctypes
binding.
"""
from .gk import (  # noqa: F401
    CSR,
    GKError,
    gk_block_fsvd,
    gk_block_numrank,
    gk_block_numrank_workspace,
    gk_fsvd,
    gk_matvec,
    gk_mlp_forward,
    gk_mlp_grad,
    gk_mlp_train,
    gk_matvec_static,
    gk_numrank,
    gk_numrank_batched,
    gk_numrank_workspace,
    gk_psvd,
    gk_psvd_batched,
    gk_psvd_workspace,
    gk_residuals,
    gk_rsgd_batched,
    gk_sketch_batched,
    host_empty,
    host_free,
    last_cuda_error,
    launch_count,
    lib,
    library_path,
    status_string,
    version,
    wait_selftest,
)
