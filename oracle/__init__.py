"""CPU oracle for batch-dynamic SpGEMM -- TEST INFRASTRUCTURE ONLY.

A plain, slow C restatement (single-threaded unless ``set_threads`` asks
for the all-cores timing of its row loops) (``dspg_oracle.c``) of what the
library computes, wrapped with ctypes. Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it;
the library itself never does, and the oracle imports nothing from the
library. See ``dspg_oracle.c`` for the paper passages each routine follows.

Pinned by ``tests/test_oracle_pins.py`` against dense brute force, numpy's
dense matmul, Floyd-Warshall and Dijkstra (scipy), a Python dictionary model
of sequential updates, the paper's identities (Eq. 1 and the locality of
general updates) and hand-worked fixtures in ``tests/golden/``.

``mlp.py`` is the oracle of the learned row-size estimator (plain numpy,
float64), pinned by ``tests/test_oracle_mlp.py``.
"""

from .oracle import (  # noqa: F401
    OMat,
    OracleError,
    affected_rows,
    build_oracle,
    oracle_lib,
    row_dynamic,
    set_threads,
)
from . import mlp  # noqa: F401,E402
