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
