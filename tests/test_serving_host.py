"""The serving loop's scheduling, on the CPU, against a stand-in handle.

The stand-in's footprint of a request is the set of rows its entries name
(the library's footprint also holds the rows those entries connect; only
the set matters to the scheduler), its affected rows after a wave are the
rows of the wave's batch, and it records every batch it is given.  These
tests pin the admission rules the module states: arrival order, a wave
ends at the first conflict (or, with overtake, a request joins only if it
meets no footprint examined before it), the wave's slots and entries, the
memory budget, and each request's result rows are the wave's affected rows
inside its own footprint."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2202_08808_gb300.serving import Request, Server, UpdateBatch  # noqa: E402


class StandIn:
    sr = 0

    def __init__(self, n):
        self.n = n
        self.applied = []  # row arrays of the batches applied, in order
        self.footprints = 0

    def info(self):
        return {"n": self.n, "k": self.n, "m": self.n, "nnz_a": 0, "nnz_c": 8 * self.n}

    def footprint(self, batch, f, u=None, or_anyway=False):
        self.footprints += 1
        rows = np.unique(np.asarray(batch.row)).astype(np.int64)
        fa = f.numpy().view(np.uint32)
        fa[:] = 0
        np.bitwise_or.at(fa, rows >> 5, (np.ones_like(rows) << (rows & 31)).astype(np.uint32))
        ua = u.numpy().view(np.uint32)
        disjoint = not np.any(fa & ua)
        if disjoint or or_anyway:
            ua |= fa
        return int(rows.size), disjoint

    def apply_batch(self, b):
        self.applied.append(np.asarray(b.row).copy())

    def last_affected(self):
        return np.unique(self.applied[-1]).astype(np.int32)

    def read_rows_C(self, rows):
        return np.zeros(rows.size + 1, np.int64), np.zeros(0, np.int32), np.zeros(0)


def req(rid, rows, arrival=0.0):
    rows = np.asarray(rows, np.int32)
    k = rows.size
    return Request(rid, arrival, UpdateBatch(rows, rows.copy(), np.ones(k), np.zeros(k, np.uint8)))


def waves_of(results):
    out = {}
    for r in results:
        out.setdefault(r.wave, []).append(r.rid)
    return [sorted(v) for _, v in sorted(out.items())]


def serve(reqs, n=256, **kw):
    g = StandIn(n)
    kw.setdefault("hbm_free", lambda: 1 << 40)
    kw.setdefault("hbm_reserve", 0)
    srv = Server(g, bitmap_device="cpu", **kw)
    return g, srv, srv.serve(reqs, clock=lambda: 0.0)


def test_disjoint_requests_share_one_wave_in_arrival_order():
    g, srv, res = serve([req(i, [40 * i, 40 * i + 1]) for i in range(5)], max_wave=8)
    assert waves_of(res) == [[0, 1, 2, 3, 4]]
    assert np.array_equal(g.applied[0], np.array([0, 1, 40, 41, 80, 81, 120, 121, 160, 161]))
    for r in res:
        assert np.array_equal(r.rows, [40 * r.rid, 40 * r.rid + 1])


def test_first_conflict_ends_the_wave():
    g, srv, res = serve([req(0, [1]), req(1, [1, 50]), req(2, [100])], max_wave=8)
    assert waves_of(res) == [[0], [1, 2]]
    assert srv.conflicts == 1


def test_overtake_passes_over_conflicts_but_keeps_their_order():
    # r2 commutes with r1 (disjoint) and overtakes it
    _, srv, res = serve([req(0, [1]), req(1, [1, 50]), req(2, [100])], max_wave=8, overtake=True)
    assert waves_of(res) == [[0, 2], [1]]
    # r2 meets the passed-over r1, so it may not overtake it
    _, _, res = serve([req(0, [1]), req(1, [1, 50]), req(2, [50])], max_wave=8, overtake=True)
    assert waves_of(res) == [[0], [1], [2]]


def test_wave_slots_and_entries():
    _, _, res = serve([req(i, [10 * i]) for i in range(6)], max_wave=4)
    assert waves_of(res) == [[0, 1, 2, 3], [4, 5]]
    _, _, res = serve([req(i, [10 * i, 10 * i + 1]) for i in range(6)], max_wave=8, max_wave_entries=5)
    assert waves_of(res) == [[0, 1], [2, 3], [4, 5]]


def test_memory_budget_closes_the_wave():
    # room for one request's buffers only: every wave still takes its first request
    _, srv, res = serve([req(i, [10 * i]) for i in range(3)], max_wave=8, hbm_free=lambda: 100)
    assert waves_of(res) == [[0], [1], [2]]
    assert srv.memory_stops == 2


def test_results_are_the_wave_rows_inside_each_footprint():
    _, _, res = serve([req(0, [3, 4]), req(1, [70]), req(2, [200, 5])], max_wave=8)
    assert waves_of(res) == [[0, 1, 2]]
    got = {r.rid: list(r.rows) for r in res}
    assert got == {0: [3, 4], 1: [70], 2: [5, 200]}


def test_plain_queue_takes_no_footprints():
    g, _, res = serve([req(0, [1]), req(1, [1]), req(2, [2])], max_wave=1)
    assert waves_of(res) == [[0], [1], [2]]
    assert g.footprints == 0
