"""GB300-native partial-fraction matrix exponential: exp(tA)V ~ e^c R_n(tA - cI)V.

Thin Python binding of ``libexpm.so`` (C interface in ``include/expm.h``).
Every function here only marshals arguments: all arithmetic of the method runs in
the CUDA kernels behind the C interface.  There is no CPU fallback -- importing
the package raises if the native library has not been built.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; complex data must be
complex128 (interleaved re/im).  Device tensors are used in place and the call
is asynchronous on ``stream`` (default: torch's current stream); host buffers
are staged by the library and the call is synchronous.
"""

from ._native import (  # noqa: F401
    EXPM_FP64,
    EXPM_MIXED_F32X2,
    EXPM_MIXED_FP32,
    EXPM_MIXED_TF32X3,
    EXPM_MIXED_BF16X3,
    EXPM_FLAG_SKIP_FINAL_RESIDUAL,
    BatchGraph,
    ExpmError,
    Plan,
    Queue,
    Server,
    expm_apply_batched,
    expm_apply_dense,
    expm_apply_dense_full,
    expm_apply_dense_reduced,
    expm_apply_laplacian2d,
    expm_apply_tridiag,
    expm_apply_tridiag_noalloc,
    expm_profile_enable,
    expm_profile_read,
    expm_coeffs,
    expm_opts,
    expm_info,
    lib,
    library_path,
)
