"""GB300 (sm_103a) library for the Piacsek-Williams advection scheme.

The compute path is libpw.so (CUDA kernels behind the C ABI in include/pw.h);
this package is its Python binding (pw.py) plus the seeded input generator
(inputs.py).  Build the library with build.build().
"""
from .pw import (DTYPES, PW, Batch, Grid, PwError, lib, LIB_PATH, SIGNATURES,  # noqa: F401
                 PW_OK, PW_ERR_ARG, PW_ERR_ALIGN, PW_ERR_CUDA, PW_ERR_OOM, PW_ERR_DEVICE_TIMEOUT,
                 PW_ERR_UNSUPPORTED, PW_ADJ_ACCUMULATE, PW_ADJ_PERIODIC, PW_ADJ_ADD_LAMBDA,
                 INJECT_ALLOC, INJECT_TENSOR_MAP, inject_failures)
