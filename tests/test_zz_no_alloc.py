"""The entry point that allocates nothing (dspg_multiply_rows_noalloc).

It serves callers that cannot let a library allocate device memory, because
their memory belongs to another allocator or because cudaMalloc/cudaFree
(which synchronise the device) do not fit their latency budget.  It keeps
its working memory in a fixed device array inside the library, so these
tests check that two calls in a row (the second one reusing whatever the
first left in that array) both agree with the handle-based path
(dspg_read_rows_C after dspg_build) within the library's tolerance.

This file is named to be collected last, and it passes both on its own in a
fresh process and after the other tests.
"""

import numpy as np
import pytest

from oracle import OMat
from workloads import MIN_PLUS_I32, PLUS_TIMES_F64, random_csr, CSR

pytestmark = pytest.mark.gpu


def _to_device(M):
    import torch
    return CSR(M.nrows, M.ncols, torch.from_numpy(M.rowptr).cuda(), torch.from_numpy(M.col).cuda(),
               torch.from_numpy(M.val).cuda())


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_noalloc_matches_handle_path_on_two_calls(dspg, sr):
    import torch
    A = random_csr(2500, 1800, 14, 101, sr, empty_frac=0.15)
    B = random_csr(1800, 3000, 12, 102, sr, empty_frac=0.15)
    g = dspg.DynamicSpGEMM(A, B)
    Ad, Bd = _to_device(A), _to_device(B)
    Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
    rng = np.random.default_rng(103)
    for call in range(2):
        rows = rng.choice(A.nrows, size=700, replace=True).astype(np.int32)  # any order, repeats allowed
        want_rp, want_col, want_val = g.read_rows_C(rows)
        rp, col, val = dspg.multiply_rows_noalloc(Ad, Bd, torch.from_numpy(rows).cuda(), sr)
        rp, col, val = rp.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
        assert np.array_equal(rp, want_rp), f"call {call}: row lengths"
        assert np.array_equal(col, want_col), f"call {call}: columns"
        if sr == MIN_PLUS_I32:
            assert np.array_equal(val, want_val), f"call {call}: (min,+) values"
        else:
            # both sides are within 1e-12 * sum|ab| of the exact value
            _, _, sabs = Ao.multiply_rows(Bo, rows, absval=True)
            assert np.all(np.abs(val - want_val) <= 2e-12 * sabs), f"call {call}: (+,.) values"


def test_noalloc_rejects_too_wide_b(dspg):
    import torch
    A = random_csr(10, 10, 3, 1, PLUS_TIMES_F64)
    B = random_csr(10, 70000, 3, 2, PLUS_TIMES_F64)
    with pytest.raises(dspg.DspgError) as e:
        dspg.multiply_rows_noalloc(_to_device(A), _to_device(B), torch.arange(10, dtype=torch.int32).cuda())
    assert e.value.status == 1
    assert "65536" in str(e.value)


def test_noalloc_bad_row_index_is_reported(dspg):
    """A row index outside A's rows is skipped by the kernel and reported by
    the call as DSPG_ERR_INVALID with the index message."""
    import torch
    A = random_csr(50, 40, 5, 11, PLUS_TIMES_F64)
    B = random_csr(40, 60, 5, 12, PLUS_TIMES_F64)
    Ad, Bd = _to_device(A), _to_device(B)
    for bad in (-1, A.nrows):
        rows = torch.tensor([0, 3, bad, 7], dtype=torch.int32).cuda()
        with pytest.raises(dspg.DspgError) as e:
            dspg.multiply_rows_noalloc(Ad, Bd, rows)
        assert e.value.status == 1 and "out of range" in str(e.value)
    # the array is usable again right after the failed calls
    rp, col, val = dspg.multiply_rows_noalloc(Ad, Bd, torch.tensor([0, 3, 7], dtype=torch.int32).cuda())
    orp, ocol, _ = OMat.from_csr(A).multiply_rows(OMat.from_csr(B), np.array([0, 3, 7], np.int32))
    assert np.array_equal(rp.cpu().numpy(), orp) and np.array_equal(col.cpu().numpy(), ocol)


def test_noalloc_capacity_and_size_query(dspg):
    """The size query (col = NULL) writes rowptr and the result size only;
    a fill call with one entry less room than the result returns
    DSPG_ERR_INVALID and reports the size it needs; the exact room works."""
    import torch
    A = random_csr(300, 200, 8, 21, MIN_PLUS_I32)
    B = random_csr(200, 500, 8, 22, MIN_PLUS_I32)
    Ad, Bd = _to_device(A), _to_device(B)
    rows_np = np.arange(0, 300, 3, dtype=np.int32)
    rows = torch.from_numpy(rows_np).cuda()
    qrp, nnz = dspg.multiply_rows_noalloc(Ad, Bd, rows, query_only=True)
    orp, ocol, oval = OMat.from_csr(A).multiply_rows(OMat.from_csr(B), rows_np)
    assert nnz == int(orp[-1]) > 0
    assert np.array_equal(qrp.cpu().numpy(), orp)
    with pytest.raises(dspg.DspgError) as e:
        dspg.multiply_rows_noalloc(Ad, Bd, rows, capacity=nnz - 1)
    assert e.value.status == 1 and "capacity" in str(e.value) and e.value.needed == nnz
    rp, col, val = dspg.multiply_rows_noalloc(Ad, Bd, rows, capacity=nnz)
    assert np.array_equal(rp.cpu().numpy(), orp) and np.array_equal(col.cpu().numpy(), ocol)
    assert np.array_equal(val.cpu().numpy(), oval)
