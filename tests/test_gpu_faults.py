"""Failure handling on the host side, without faulting the GPU: injected
allocation and check failures (dspg_fault_inject) return a clean status and
leave the handle as it was; the per-batch JSON trace (DSPG_TRACE) records
each batch's statistics."""

import json
import os

import numpy as np
import pytest

from oracle import OMat
from parity import assert_matches, oracle_product
from workloads import PLUS_TIMES_F64, er_matrix, random_batch

pytestmark = pytest.mark.gpu


def _state_matches(g, Ao, what):
    C_o, S_o = oracle_product(Ao, Ao)
    assert_matches(g.read_C(), C_o, S_o, what=what)
    Ag, Aw = g.read_A(), Ao.to_csr()
    assert np.array_equal(Ag.rowptr, Aw.rowptr) and np.array_equal(Ag.col, Aw.col) and np.array_equal(Ag.val, Aw.val)


def test_allocation_failures_during_build(dspg):
    A = er_matrix(2000, 6, seed=5)
    Ao = OMat.from_csr(A)
    failed = 0
    try:
        for n in range(1, 8):
            dspg.fault_inject(f"alloc@{n}")
            with pytest.raises(dspg.DspgError) as e:
                dspg.DynamicSpGEMM(A)
            assert e.value.status == 2 and "injected" in str(e.value)
            failed += 1
    finally:
        dspg.fault_inject(None)
    assert failed == 7
    g = dspg.DynamicSpGEMM(A)
    _state_matches(g, Ao, "build after the injected failures")
    g.close()


def test_failures_before_a_batch_changes_anything(dspg):
    n = 3000
    A = er_matrix(n, 6, seed=6)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    small = [random_batch(n, n, 500, 10 + k, PLUS_TIMES_F64, A=A) for k in range(3)]
    for b in small[:2]:  # the 1024-entry launch size: eager, then captured
        g.apply_batch(b)
        Ao.apply(b)
    big = random_batch(n, n, 40000, 20, PLUS_TIMES_F64, A=A)  # its buffers must grow
    try:
        dspg.fault_inject("alloc@1")
        with pytest.raises(dspg.DspgError) as e:
            g.apply_batch(big)
        assert e.value.status == 2
        _state_matches(g, Ao, "after an allocation failure")
        dspg.fault_inject("validate@1")
        with pytest.raises(dspg.DspgError) as e:
            g.apply_batch(small[2])
        assert e.value.status == 1
        _state_matches(g, Ao, "after a check failure")
    finally:
        dspg.fault_inject(None)
    # the same batches go through afterwards (the captured pipeline of the
    # small size replays with any buffers that moved)
    for b in (small[2], big):
        g.apply_batch(b)
        Ao.apply(b)
        _state_matches(g, Ao, "after the failures")
    g.close()


def test_batch_trace_jsonl(dspg, tmp_path):
    n = 2000
    A = er_matrix(n, 6, seed=7)
    g = dspg.DynamicSpGEMM(A)
    path = tmp_path / "trace.jsonl"
    os.environ["DSPG_TRACE"] = str(path)
    try:
        stats = [g.apply_batch(random_batch(n, n, 300, 30, PLUS_TIMES_F64, A=A))]
        g.set_profiling(True)
        stats.append(g.apply_batch(random_batch(n, n, 300, 31, PLUS_TIMES_F64, A=A)))
        g.set_profiling(False)
    finally:
        del os.environ["DSPG_TRACE"]
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(lines) == 2
    for rec, st in zip(lines, stats):
        assert rec["path"] == "rows"
        for k in ("n_updates", "affected_rows", "products", "nnz_written", "a_entries"):
            assert rec[k] == st[k], k
    assert "stage_ms" not in lines[0] and set(lines[1]["stage_ms"]) == set(dspg.STAGES)
    g.close()
