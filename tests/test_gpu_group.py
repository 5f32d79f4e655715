"""Row-bin tuning, the autotuner and groups of instances, against the oracle.

- Every candidate tuning (thresholds that move rows between the thread-merge,
  hash and dense bins) must give the same C: patterns and (min,+) values
  bit-exact, (+,.) values within 1e-12 * sum|ab|.
- The autotuner applies its calibration batches for real; the state after it
  must equal the oracle's after the same batches.
- A group applies one batch per member as branches of one CUDA graph; every
  member must end exactly where it would alone, on the eager first apply, the
  capturing second apply and the replays after it; a member's invalid batch
  fails that member only.
"""

import numpy as np
import pytest

import oracle
from oracle import OMat
from parity import assert_matches, oracle_product
from workloads import MIN_PLUS_I32, PLUS_TIMES_F64, Batch, random_batch, rmat_edge_batch, rmat_symmetric

pytestmark = pytest.mark.gpu

G500 = (0.57, 0.19, 0.19, 0.05)


def _check(g, A_or, what):
    C_o, S_o = oracle_product(A_or, A_or)
    assert_matches(g.read_C(), C_o, S_o, what=what)


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_every_candidate_tuning_gives_the_same_C(dspg, sr):
    """R-MAT scale 12: product bounds from 1 to the column count, so the
    candidates move rows across every bin boundary."""
    A, held = rmat_symmetric(12, 8, G500, seed=21, kind=sr, holdout=3000)
    b = rmat_edge_batch(A, held, 600, seed=22)
    Ao = OMat.from_csr(A)
    C0, S0 = oracle_product(Ao, Ao)
    Co = Ao.multiply(Ao)
    R = oracle.row_dynamic(Ao, Co, b)
    C1, S1 = oracle_product(Ao, Ao)
    for k, cand in enumerate(dspg.tuning_candidates()):
        g = dspg.DynamicSpGEMM(A)
        g.set_tuning(cand)
        assert g.get_tuning() == cand
        g.recompute_all()
        assert_matches(g.read_C(), C0, S0, what=f"candidate {k} static")
        g.apply_batch(b)
        assert np.array_equal(g.last_affected(), R)
        assert_matches(g.read_C(), C1, S1, what=f"candidate {k} after batch")
        g.close()


def test_set_tuning_rejects_out_of_range(dspg):
    A, _ = rmat_symmetric(8, 8, G500, seed=3, kind=PLUS_TIMES_F64)
    g = dspg.DynamicSpGEMM(A)
    bad = dict(dspg.tuning_candidates()[0], lanes_min=12)
    with pytest.raises(dspg.DspgError) as e:
        g.set_tuning(bad)
    assert e.value.status == 1
    assert g.get_tuning() == dspg.tuning_candidates()[0]


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_autotune_applies_its_batches_and_keeps_C_exact(dspg, sr):
    A, held = rmat_symmetric(12, 8, G500, seed=31, kind=sr, holdout=6000)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    batches = [rmat_edge_batch(A, held, 500, seed=40 + k) for k in range(4)]
    best, ms = g.autotune(batches)
    assert best in dspg.tuning_candidates()
    assert len(ms) == len(dspg.tuning_candidates()) and all(t > 0 for t in ms)
    assert g.get_tuning() == best
    for b in batches:
        oracle.row_dynamic(Ao, Co, b)
    _check(g, Ao, "after autotune")
    # and the tuned handle keeps matching on the next batch
    b = random_batch(A.nrows, A.ncols, 800, seed=49, kind=sr, A=A)
    g.apply_batch(b)
    R = oracle.row_dynamic(Ao, Co, b)
    assert np.array_equal(g.last_affected(), R)
    _check(g, Ao, "tuned, next batch")


def _instances(count, seed):
    """Uneven instances: R-MAT scales 8..11, alternating semirings."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(count):
        sr = PLUS_TIMES_F64 if t % 2 == 0 else MIN_PLUS_I32
        scale = int(rng.integers(8, 12))
        A, held = rmat_symmetric(scale, 8, G500, seed=seed * 100 + t, kind=sr, holdout=100)
        size = int(10 ** rng.uniform(1, 2.5))
        out.append((A, held, size))
    return out


def test_group_matches_each_member_alone(dspg):
    insts = _instances(12, 7)
    gs = [dspg.DynamicSpGEMM(A) for A, _, _ in insts]
    Aos = [OMat.from_csr(A) for A, _, _ in insts]
    Cos = [Ao.multiply(Ao) for Ao in Aos]
    grp = dspg.Group(gs)
    for rep in range(4):  # eager, capture, replay, replay
        bs = [rmat_edge_batch(A, held, size, seed=1000 * rep + t) if t != 5 else None
              for t, (A, held, size) in enumerate(insts)]
        k0 = dspg.kernel_launches()
        stats, status = grp.apply(bs)
        assert dspg.kernel_launches() > k0
        assert status == [0] * len(gs)
        for t, (g, Ao, Co) in enumerate(zip(gs, Aos, Cos)):
            if bs[t] is None:
                assert stats[t]["n_updates"] == 0 and stats[t]["affected_rows"] == 0
                continue
            R = oracle.row_dynamic(Ao, Co, bs[t])
            assert stats[t]["affected_rows"] == R.shape[0], f"rep {rep} member {t}"
            assert np.array_equal(g.last_affected(), R), f"rep {rep} member {t}: R"
            C_o = Co.to_csr()
            S_o = Ao.multiply(Ao, absval=True).to_csr() if Ao.sr == PLUS_TIMES_F64 else None
            assert_matches(g.read_C(), C_o, S_o, what=f"rep {rep} member {t}")
    grp.close()


def test_group_invalid_member_fails_alone(dspg):
    insts = _instances(4, 9)
    gs = [dspg.DynamicSpGEMM(A) for A, _, _ in insts]
    Aos = [OMat.from_csr(A) for A, _, _ in insts]
    Cos = [Ao.multiply(Ao) for Ao in Aos]
    before = [g.read_C() for g in gs]
    grp = dspg.Group(gs)
    bs = [rmat_edge_batch(A, held, size, seed=77 + t) for t, (A, held, size) in enumerate(insts)]
    bad = bs[2]
    row = bad.row.copy()
    row[len(row) // 2] = insts[2][0].nrows + 5  # out of range
    bs[2] = Batch(row, bad.col, bad.val, bad.op)
    stats, status = grp.apply(bs, raise_on_error=False)
    assert status[2] == 1 and [s for t, s in enumerate(status) if t != 2] == [0, 0, 0]
    after = gs[2].read_C()
    assert np.array_equal(after.rowptr, before[2].rowptr) and np.array_equal(after.col, before[2].col)
    assert np.array_equal(after.val, before[2].val)
    for t in (0, 1, 3):
        oracle.row_dynamic(Aos[t], Cos[t], bs[t])
        _check(gs[t], Aos[t], f"member {t}")
    with pytest.raises(dspg.DspgError):
        grp.apply(bs)
    grp.close()


def test_group_rejects_repeated_member(dspg):
    A, _ = rmat_symmetric(7, 8, G500, seed=1, kind=PLUS_TIMES_F64)
    g = dspg.DynamicSpGEMM(A)
    with pytest.raises(dspg.DspgError):
        dspg.Group([g, g])


def test_reserved_group_replays_any_sizes(dspg):
    """Members reserved for batches up to 3000 entries: after the eager and
    the capturing apply, the group replays one captured pipeline for fresh
    uneven sizes every step (empty batches included), and every member
    matches the oracle."""
    insts = _instances(6, 17)
    # room in the arenas: a buffer that moves retires the captured pipeline
    gs = [dspg.DynamicSpGEMM(A, arena_headroom=3.0) for A, _, _ in insts]
    for g in gs:
        g.reserve(3000)
    Aos = [OMat.from_csr(A) for A, _, _ in insts]
    Cos = [Ao.multiply(Ao) for Ao in Aos]
    grp = dspg.Group(gs)
    rng = np.random.default_rng(18)
    for rep in range(6):
        bs = []
        for t, (A, held, _) in enumerate(insts):
            size = int(rng.integers(0, 1500))
            bs.append(rmat_edge_batch(Aos[t].to_csr(), held, size, seed=400 * rep + t) if size else None)
        r0 = [g.run_counts() for g in gs]
        stats, status = grp.apply(bs)
        assert status == [0] * len(gs)
        r1 = [g.run_counts() for g in gs]
        if rep >= 2:
            assert all(b["replayed"] - a["replayed"] == 1 for a, b in zip(r0, r1)), f"rep {rep}: not replayed"
        for t, (g, Ao, Co) in enumerate(zip(gs, Aos, Cos)):
            if bs[t] is None:
                assert stats[t]["affected_rows"] == 0
                continue
            R = oracle.row_dynamic(Ao, Co, bs[t])
            assert np.array_equal(g.last_affected(), R), f"rep {rep} member {t}: R"
            _check(g, Ao, f"rep {rep} member {t}")
    grp.close()
