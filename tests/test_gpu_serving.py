"""The serving loop (continuous batching over one handle) against the oracle.

Every request's result (its affected rows of C right after it commits) must
be the same whether it ran inside a wave of merged requests or alone in
arrival order, and both must be the oracle's rows at that version: patterns
and (min,+) values bit-exact, (+,.) values within 1e-12 * sum|ab|.
"""

import numpy as np
import pytest

import oracle
from oracle import OMat
from parity import assert_rows_match
from workloads import MIN_PLUS_I32, PLUS_TIMES_F64, er_matrix, random_batch, rmat_symmetric

pytestmark = pytest.mark.gpu

G500 = (0.57, 0.19, 0.19, 0.05)


def _requests(A, count, seed):
    """Small mixed batches (1..5 entries, half on present entries), all
    queued at once, so that waves form and some footprints collide."""
    from paper_2202_08808_gb300.serving import Request
    rng = np.random.default_rng(seed)
    return [Request(k, 0.0, random_batch(A.nrows, A.ncols, int(rng.integers(1, 6)), seed=seed * 1000 + k,
                                         kind=A.semiring, A=A, dup_frac=0.0)) for k in range(count)]


def _alone_and_oracle(dspg, A, reqs, results):
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    by_id = {r.rid: r for r in results}
    for req in reqs:
        g.apply_batch(req.batch)
        rows = g.last_affected()
        rp, col, val = g.read_rows_C(rows)
        R_o = oracle.row_dynamic(Ao, Co, req.batch)
        assert np.array_equal(rows, R_o), f"request {req.rid}: alone R differs from the oracle"
        mix = by_id[req.rid]
        assert np.array_equal(mix.rows, rows), f"request {req.rid}: R in the mix differs from alone"
        o_rp, o_col, o_val = Ao.multiply_rows(Ao, rows)
        o_abs = Ao.multiply_rows(Ao, rows, absval=True)[2] if Ao.sr == PLUS_TIMES_F64 else None
        assert_rows_match(rp, col, val, o_rp, o_col, o_val, o_abs, what=f"request {req.rid} alone")
        assert_rows_match(mix.rowptr, mix.col, mix.val, o_rp, o_col, o_val, o_abs, what=f"request {req.rid} mix")


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_each_result_is_the_same_alone_and_in_the_mix(dspg, sr):
    from paper_2202_08808_gb300.serving import Server
    A = er_matrix(4096, 4, seed=121, kind=sr)
    reqs = _requests(A, 80, 122)
    srv = Server(dspg.DynamicSpGEMM(A), max_wave=16)
    results = srv.serve(reqs)
    assert len(results) == len(reqs)
    assert srv.waves < len(reqs), "no two requests were merged"
    assert srv.conflicts > 0, "no footprint conflict was exercised"
    assert max(r.wave_size for r in results) > 1
    _alone_and_oracle(dspg, A, reqs, results)


def test_memory_admission_stops_a_wave(dspg):
    """With no free memory to spare, every wave holds one request (the first
    request of a wave is always admitted, so the stream still drains)."""
    from paper_2202_08808_gb300.serving import Server
    A = er_matrix(1024, 4, seed=131, kind=PLUS_TIMES_F64)
    reqs = _requests(A, 12, 132)
    srv = Server(dspg.DynamicSpGEMM(A), max_wave=8, hbm_reserve=0, hbm_free=lambda: 1)
    results = srv.serve(reqs)
    assert srv.waves == len(reqs) and srv.memory_stops > 0
    _alone_and_oracle(dspg, A, reqs, results)


def test_footprint_rejects_out_of_range_entries(dspg):
    import torch
    from workloads import Batch
    A, _ = rmat_symmetric(8, 8, G500, seed=141, kind=PLUS_TIMES_F64)
    g = dspg.DynamicSpGEMM(A)
    f = torch.zeros((A.nrows + 31) // 32, dtype=torch.int32, device="cuda")
    bad = Batch(np.array([3, A.nrows], np.int32), np.array([1, 2], np.int32), np.zeros(2), np.zeros(2, np.uint8))
    with pytest.raises(dspg.DspgError):
        g.footprint(bad, f)


def test_overtaking_keeps_every_result(dspg):
    """With overtake on, a request may run before earlier ones it does not
    conflict with; every result must still be the one it has alone in
    arrival order."""
    from paper_2202_08808_gb300.serving import Server
    A = er_matrix(4096, 4, seed=181, kind=MIN_PLUS_I32)
    reqs = _requests(A, 60, 182)
    srv = Server(dspg.DynamicSpGEMM(A), max_wave=8, overtake=True)
    results = srv.serve(reqs)
    assert len(results) == len(reqs) and srv.conflicts > 0
    order = [r.rid for r in sorted(results, key=lambda r: (r.wave, r.rid))]
    assert order != sorted(order), "no request overtook an earlier one"
    _alone_and_oracle(dspg, A, reqs, results)


def test_footprint_is_the_rows_a_batch_can_reach(dspg):
    """For C = A A the footprint of a batch is its rows, its columns and every
    row i with A(i,k) != 0 for a row k of the batch (on A's current pattern):
    compared bit for bit with a brute-force set; the admission test against a
    wave bitmap agrees with set intersection."""
    import torch
    A = er_matrix(2048, 5, seed=191, kind=PLUS_TIMES_F64)
    g = dspg.DynamicSpGEMM(A)
    words = (A.nrows + 31) // 32
    rows_of = A.row_ids()
    cols = A.col.astype(np.int64)

    def brute(b):
        s = set(b.row.tolist()) | set(b.col.tolist())
        for k in set(b.row.tolist()):
            s |= set(rows_of[cols == k].tolist())
        return s

    def bits(f):
        w = f.cpu().numpy().view(np.uint32)
        return set(np.nonzero(np.unpackbits(w.view(np.uint8), bitorder="little"))[0].tolist())

    b1 = random_batch(A.nrows, A.ncols, 7, seed=192, kind=PLUS_TIMES_F64, A=A, dup_frac=0.0)
    b2 = random_batch(A.nrows, A.ncols, 7, seed=193, kind=PLUS_TIMES_F64, A=A, dup_frac=0.0)
    f1 = torch.zeros(words, dtype=torch.int32, device="cuda")
    f2 = torch.zeros(words, dtype=torch.int32, device="cuda")
    u = torch.zeros(words, dtype=torch.int32, device="cuda")
    n1, adm1 = g.footprint(b1, f1, u)
    assert bits(f1) == brute(b1) and n1 == len(brute(b1)) and adm1
    assert bits(u) == brute(b1)
    n2, adm2 = g.footprint(b2, f2, u)
    assert bits(f2) == brute(b2)
    assert adm2 == (not (brute(b1) & brute(b2)))
    n3, adm3 = g.footprint(b1, f1)  # no wave bitmap: no admission
    assert adm3 is None and n3 == n1


def test_pipelined_waves_overlap_on_the_device(dspg):
    """Pipelined serving: the next wave's pipeline runs while the previous
    wave's rows are read on another stream (their CUDA event intervals
    intersect), and every result is still the one it has alone."""
    from paper_2202_08808_gb300.serving import Server
    A = er_matrix(1 << 16, 6, seed=201, kind=PLUS_TIMES_F64)
    reqs = _requests(A, 48, 202)
    srv = Server(dspg.DynamicSpGEMM(A), max_wave=6)
    assert srv.pipelined
    results = srv.serve(reqs)
    assert len(results) == len(reqs) and srv.waves > 2
    assert srv.overlaps() > 0, "no wave's read ran beside the next wave's apply"
    _alone_and_oracle(dspg, A, reqs, results)


@pytest.mark.parametrize("overtake", [False, True])
def test_footprint_batch_equals_calls_in_a_row(dspg, overtake):
    """One dspg_footprint_batch call admits exactly what the same batches
    given one by one to dspg_footprint admit, and leaves the same wave bitmap
    (first conflict ends the run, or with overtake is passed over)."""
    import torch
    A = er_matrix(4096, 4, seed=211, kind=PLUS_TIMES_F64)
    g = dspg.DynamicSpGEMM(A)
    words = (A.nrows + 31) // 32
    bs = [random_batch(A.nrows, A.ncols, 3, seed=212 + k, kind=PLUS_TIMES_F64, A=A, dup_frac=0.0) for k in range(20)]
    f = torch.zeros((len(bs), words), dtype=torch.int32, device="cuda")
    u = torch.zeros(words, dtype=torch.int32, device="cuda")
    adm, rows = g.footprint_batch(bs, f, u, or_anyway=overtake)
    u1 = torch.zeros(words, dtype=torch.int32, device="cuda")
    f1 = torch.zeros(words, dtype=torch.int32, device="cuda")
    want, stopped = [], False
    for k, b in enumerate(bs):
        if stopped:
            want.append(False)
            continue
        n, ok = g.footprint(b, f1, u1, or_anyway=overtake)
        assert torch.equal(f1, f[k]) and n == rows[k]
        want.append(ok)
        if not ok and not overtake:
            stopped = True
    assert adm == want and any(adm) and not all(adm)
    assert torch.equal(u, u1)


def test_async_apply_equals_apply_and_guards_the_handle(dspg):
    """dspg_apply_batch_async + dspg_apply_batch_wait give what
    dspg_apply_batch gives; in between, other calls are refused
    (DSPG_ERR_STATE) except reads."""
    A = er_matrix(4096, 8, seed=221, kind=MIN_PLUS_I32)
    g1, g2 = dspg.DynamicSpGEMM(A), dspg.DynamicSpGEMM(A)
    for t in range(3):  # eager, captured, replayed
        b = random_batch(A.nrows, A.ncols, 300, seed=222 + t, kind=MIN_PLUS_I32, A=A)
        s1 = g1.apply_batch(b)
        g2.apply_batch_async(b)
        with pytest.raises(dspg.DspgError) as e:
            g2.apply_batch(b)
        assert e.value.status == 5
        g2.read_rows_C(np.array([0, 1], np.int32))  # reads are allowed meanwhile
        s2 = g2.apply_batch_wait()
        assert s1 == s2
        assert np.array_equal(g1.last_affected(), g2.last_affected())
    c1, c2 = g1.read_C(), g2.read_C()
    assert np.array_equal(c1.rowptr, c2.rowptr) and np.array_equal(c1.col, c2.col) and np.array_equal(c1.val, c2.val)
    with pytest.raises(dspg.DspgError):
        g2.apply_batch_wait()  # nothing in flight
