"""Block subsampled randomized Hadamard transform (block SRHT) on one GB300.

Python face of libbsrht (C ABI in include/bsrht.h). The sketch B = Omega A of
a tall matrix A (Sec. 2, eq. 2.3-2.4), the randomized SVD (Algorithm 1) and
the randomized Nystrom approximation (Algorithm 2) all run in the library's
sm_103a CUDA kernels; torch only supplies device memory and streams.
"""

from ._binding import (  # noqa: F401
    BF16, F16, F32, F64, VARIANT_AUTO, VARIANT_CUDACORE, VARIANT_TENSOR, VARIANT_GAUSSIAN, PREC_AUTO, PREC_F64,
    BsrhtError, LIB_PATH, Server,
    bsrht_kernel_launches, bsrht_selftest_pool_allocator, bsrht_sketch_autotune, bsrht_sketch_autotune_reset, bsrht_nystrom, bsrht_nystrom_rbf, bsrht_nystrom_rbf_workspace, bsrht_profile_enable, bsrht_profile_stages, bsrht_nystrom_workspace, bsrht_release_pool, bsrht_rsvd, bsrht_rsvd_workspace, bsrht_srsvd, bsrht_srsvd_workspace,
    bsrht_sketch, bsrht_sketch_workspace, lib, sketch_out_dtype, strerror, version,
)

__version__ = "0.1.0"
