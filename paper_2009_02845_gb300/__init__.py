"""GB300 sketched ANLS (SANLS/DSANLS hot path, arXiv 2009.02845) -- Python binding.

A thin ctypes layer over the C ABI of ``libdsanls.so`` (declared in
``include/dsanls.h``).  It only marshals arguments: every step of the method
runs in the library's CUDA kernels.  PyTorch supplies device memory (output
tensors of the stateless primitives, device-resident inputs) and streams
(the current torch stream is handed to the library).

The library must have been built (``paper_2009_02845_gb300.build.build()``);
importing the binding without it raises ImportError -- there is no CPU path.
"""
from ._lib import (  # noqa: F401
    DSANLS, Batch, MLP, DSANLSError, GAUSSIAN, SUBSAMPLE, IDENTITY, RADEMACHER, COUNT, SRHT, PGD, RCD, FP32, BF16, FP8,
    ORDER_PAPER, ORDER_REASSOCIATED,
    STREAM_SKETCH_U, STREAM_SKETCH_V, STREAM_INIT_U, STREAM_INIT_V,
    lib, lib_path, kernel_launches, PHASES, gram_noalloc, debug_fail_alloc_after, debug_tc_wait, philox_field, gaussian_field, rademacher_field, count_field,
    srht_field, uniform_field,
    subsample_indices,
    EXPORTED_SYMBOLS,
)
