"""Batch-dynamic SpGEMM on one GB300 GPU (sm_103a).

C = A B over (+,.) on double or (min,+) on int32 is kept up to date under
batches of entry insertions, deletions and value changes by recomputing only
the rows of C the batch can change (van der Grinten et al., Section 5,
general updates).  All computation is in the CUDA library built from
``csrc/`` (C ABI: ``include/dspg.h``); ``dspg.py`` is the Python binding.
"""

from .dspg import (  # noqa: F401
    EXPORTED,
    STAGES,
    MIN_PLUS_I32,
    OP_DELETE,
    OP_INSERT,
    OP_SET,
    PLUS_TIMES_F64,
    CsrArrays,
    DspgError,
    DynamicSpGEMM,
    EST_PARAMS,
    Estimator,
    Group,
    SIZE_BOUND,
    SIZE_EXACT,
    SIZE_LEARNED,
    TUNING_FIELDS,
    fault_inject,
    kernel_launches,
    library_path,
    multiply_rows_noalloc,
    tuning_candidates,
    load,
)
