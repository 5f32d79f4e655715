"""Seeded synthetic inputs for batch-dynamic SpGEMM.

This package holds only random-input construction (matrices and update
batches). It contains none of the method's arithmetic: no products, no
merges, no affected-row logic. Both the CPU oracle tests and the CUDA path
tests draw their inputs from here, so that the two sides see identical data.
"""

from .gen import (  # noqa: F401
    CSR,
    Batch,
    PLUS_TIMES_F64,
    MIN_PLUS_I32,
    OP_INSERT,
    OP_DELETE,
    OP_SET,
    er_matrix,
    stencil7,
    rmat_symmetric,
    bernoulli_sparse,
    er_batch,
    stencil_batch,
    stencil_insert_batch,
    rmat_edge_batch,
    random_batch,
    random_csr,
    concat_batches,
    EdgeStream,
    mlp_init_params,
)
