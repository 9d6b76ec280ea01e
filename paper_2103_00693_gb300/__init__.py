"""GB300 (sm_103a) solver for the full-sampling 2D hidden linear function
problem of arXiv 2103.00693: stage 1 (GF(2) factorisation, the CLA module of
§2) and stage 2 (Gray-code enumeration and on-device reduction of all 2^r
solutions) as hand-written CUDA kernels behind a C ABI (include/hlf.h).
"""

from .hlf import (  # noqa: F401
    MAX_N,
    MAX_W,
    REDUCE_WORDS,
    SIGNATURES,
    STATUS,
    Factorization,
    HlfError,
    ReduceResult,
    hlf_destroy,
    hlf_device_count,
    hlf_enumerate_reduce,
    hlf_enumerate_reduce_chunks,
    hlf_enumerate_store,
    hlf_factor,
    hlf_get_factor,
    hlf_get_rank,
    hlf_get_shape,
    hlf_get_status,
    hlf_sample,
    hlf_status_string,
    lib_path,
    load,
    pack_rows,
    unpack_rows,
    words,
)
