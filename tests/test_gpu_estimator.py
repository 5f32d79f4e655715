"""The learned row-size estimator on the GPU against its oracle (oracle/mlp.py),
and the three ways of sizing the recompute's tables against the SpGEMM
oracle.

- Features of rows of C and the exact-size targets match the oracle's.
- Gradients of the GPU network (float32 accumulation, bfloat16 weights)
  match the oracle's back-propagation (float64) at the same inputs; one SGD
  step moves the weights as the oracle's step does.
- Training on sizes the library produced lowers the loss.
- Exact sizing, learned sizing with a trained network, and learned sizing
  with a network that predicts far too small (every table overflows and is
  recomputed after an exact count) all give the oracle's C: patterns and
  (min,+) values bit-exact, (+,.) values within 1e-12 * sum|ab|.
"""

import numpy as np
import pytest

import oracle
from oracle import OMat, mlp
from parity import assert_matches, oracle_product
from workloads import MIN_PLUS_I32, PLUS_TIMES_F64, mlp_init_params, random_batch, rmat_edge_batch, rmat_symmetric

pytestmark = pytest.mark.gpu

G500 = (0.57, 0.19, 0.19, 0.05)


def test_row_features_and_targets_match_the_oracle(dspg):
    A, _ = rmat_symmetric(12, 8, G500, seed=51, kind=PLUS_TIMES_F64)
    g = dspg.DynamicSpGEMM(A)
    X, y = g.row_features()
    Xo = mlp.row_features(A, A)
    assert np.allclose(X.cpu().numpy(), Xo, rtol=2e-6, atol=2e-6)
    Ao = OMat.from_csr(A)
    lens = np.diff(Ao.multiply(Ao).to_csr().rowptr)
    assert np.allclose(y.cpu().numpy(), np.log2(1.0 + lens), rtol=2e-6, atol=2e-6)
    rows = np.array([5, 0, 4095, 17, 17], dtype=np.int32)
    Xr, yr = g.row_features(rows)
    assert np.array_equal(Xr.cpu().numpy(), X.cpu().numpy()[rows])
    assert np.array_equal(yr.cpu().numpy(), y.cpu().numpy()[rows])


def _training_set(seed, n=3000):
    rng = np.random.default_rng(seed)
    X = mlp.features(rng.integers(0, 60, n), rng.integers(0, 20000, n), rng.integers(0, 900, n))
    y = np.log2(1.0 + np.minimum(rng.integers(0, 20000, n), 2 ** X[:, 1]))
    return X.astype(np.float32), y.astype(np.float32)


def test_gradient_matches_oracle_backprop(dspg):
    X, y = _training_set(61)
    p = mlp_init_params(62).astype(np.float32)
    est = dspg.Estimator(p)
    loss_g, grad_g = est.grad(X, y)
    loss_o, grad_o = mlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), y.astype(np.float64))
    assert abs(loss_g - loss_o) <= 1e-5 * loss_o
    scale = np.abs(grad_o).max()
    err = np.abs(grad_g - grad_o)
    assert np.all(err <= 1e-3 * np.abs(grad_o) + 1e-4 * scale), f"max err {err.max()} (scale {scale})"
    assert np.array_equal(est.params(), p)  # grad() does not update


def test_sgd_step_matches_oracle(dspg):
    X, y = _training_set(63, n=1024)
    p = mlp_init_params(64).astype(np.float32)
    est = dspg.Estimator(p)
    lr = 1e-3
    est.train(X, y, batch=1024, steps=1, lr=lr)
    _, grad_o = mlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), y.astype(np.float64))
    want = mlp.sgd_step(p, grad_o, lr)
    got = est.params().astype(np.float64)
    moved = np.abs(want - p)
    assert np.all(np.abs(got - want) <= 1e-3 * moved + 1e-7 * np.abs(want) + 1e-9)


def _trained_estimator(dspg, seeds=(71, 72), scale=12):
    import torch
    Xs, ys = [], []
    for sd in seeds:
        A, _ = rmat_symmetric(scale, 8, G500, seed=sd, kind=PLUS_TIMES_F64)
        g = dspg.DynamicSpGEMM(A)
        X, y = g.row_features()
        Xs.append(X)
        ys.append(y)
        g.close()
    X, y = torch.cat(Xs), torch.cat(ys)
    perm = torch.randperm(X.shape[0], generator=torch.Generator().manual_seed(0)).cuda()
    X, y = X[perm].contiguous(), y[perm].contiguous()
    est = dspg.Estimator(mlp_init_params(73).astype(np.float32))
    loss0, _ = est.grad(X, y)
    loss1 = est.train(X, y, batch=2048, steps=1500, lr=5e-4)
    return est, loss0, loss1


def test_training_lowers_the_loss(dspg):
    est, loss0, loss1 = _trained_estimator(dspg)
    assert loss1 < 0.05 * loss0, (loss0, loss1)


def _run_sizing(dspg, sr, setup, seed):
    A, held = rmat_symmetric(12, 8, G500, seed=seed, kind=sr, holdout=4000)
    g = dspg.DynamicSpGEMM(A)
    setup(g)
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    stats = []
    for k in range(3):
        b = rmat_edge_batch(A, held, 400, seed=seed + 10 + k) if k != 1 else \
            random_batch(A.nrows, A.ncols, 600, seed=seed + 20, kind=sr, A=A)
        st = g.apply_batch(b)
        R = oracle.row_dynamic(Ao, Co, b)
        assert np.array_equal(g.last_affected(), R)
        C_o, S_o = oracle_product(Ao, Ao)
        assert_matches(g.read_C(), C_o, S_o, what=f"batch {k}")
        stats.append(st)
    return stats


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_exact_sizing_gives_the_same_C(dspg, sr):
    stats = _run_sizing(dspg, sr, lambda g: g.set_sizing(dspg.SIZE_EXACT), 81)
    assert all(s["est_rows"] == 0 for s in stats)


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_learned_sizing_gives_the_same_C(dspg, sr):
    est, _, _ = _trained_estimator(dspg)
    stats = _run_sizing(dspg, sr, lambda g: g.set_sizing(dspg.SIZE_LEARNED, est, est_min=0, margin=0.25), 91)
    assert sum(s["est_rows"] for s in stats) > 0


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_every_overflow_falls_back_to_an_exact_count(dspg, sr):
    """A network that predicts 0 for every row: each estimated table is cut
    to max len(B_k), so rows overflow, are counted exactly and recomputed."""
    est = dspg.Estimator(np.zeros(dspg.EST_PARAMS, dtype=np.float32))
    stats = _run_sizing(dspg, sr, lambda g: g.set_sizing(dspg.SIZE_LEARNED, est, est_min=0, margin=0.0), 101)
    assert sum(s["est_overflows"] for s in stats) > 0
    assert all(s["est_overflows"] <= s["est_rows"] for s in stats)


def test_learned_sizing_inside_a_group(dspg):
    est = dspg.Estimator(np.zeros(dspg.EST_PARAMS, dtype=np.float32))
    insts = [rmat_symmetric(sc, 8, G500, seed=111 + sc, kind=sr, holdout=200)
             for sc, sr in ((10, PLUS_TIMES_F64), (11, MIN_PLUS_I32), (9, PLUS_TIMES_F64))]
    gs = [dspg.DynamicSpGEMM(A) for A, _ in insts]
    for g in gs:
        g.set_sizing(dspg.SIZE_LEARNED, est, est_min=0, margin=0.0)
    Aos = [OMat.from_csr(A) for A, _ in insts]
    Cos = [Ao.multiply(Ao) for Ao in Aos]
    grp = dspg.Group(gs)
    for rep in range(3):
        bs = [rmat_edge_batch(A, held, 80, seed=300 * rep + t) for t, (A, held) in enumerate(insts)]
        stats, status = grp.apply(bs)
        assert status == [0, 0, 0]
        for t in range(3):
            oracle.row_dynamic(Aos[t], Cos[t], bs[t])
            C_o, S_o = oracle_product(Aos[t], Aos[t])
            assert_matches(gs[t].read_C(), C_o, S_o, what=f"rep {rep} member {t}")


def test_learned_sizing_gain_over_the_bound(dspg):
    """What the trained network buys over sizing without it, measured in
    memory the recompute reserves (not time): on the same R-MAT stream, the
    learned tables of the rows it sizes, plus the second tables of the rows
    whose prediction was too small, take fewer accumulator slots than tables
    sized by the product bound (the method without the network); and unlike
    exact sizing it needs no count-only pass over every product first.  C'
    is the oracle's in all three."""
    est, _, _ = _trained_estimator(dspg)
    A, held = rmat_symmetric(13, 8, G500, seed=131, kind=PLUS_TIMES_F64, holdout=8000)
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    batches = [rmat_edge_batch(A, held, 1000, seed=132 + k) for k in range(3)]
    slots, ovf, rows_est = {}, 0, 0
    for mode in ("bound", "exact", "learned"):
        g = dspg.DynamicSpGEMM(A)
        if mode == "exact":
            g.set_sizing(dspg.SIZE_EXACT)
        elif mode == "learned":
            g.set_sizing(dspg.SIZE_LEARNED, est, est_min=0, margin=0.25)
        Am, Cm = Ao.copy(), Co.copy()
        total = 0
        for k, b in enumerate(batches):
            st = g.apply_batch(b)
            oracle.row_dynamic(Am, Cm, b)
            C_o, S_o = oracle_product(Am, Am)
            assert_matches(g.read_C(), C_o, S_o, what=f"{mode} batch {k}")
            total += st["table_slots"]
            if mode == "learned":
                ovf += st["est_overflows"]
                rows_est += st["est_rows"]
        slots[mode] = total
        g.close()
    print("table slots", slots, "estimated rows", rows_est, "overflows", ovf)
    assert rows_est > 0 and ovf <= 0.05 * rows_est
    assert slots["exact"] <= slots["learned"] < 0.8 * slots["bound"], slots
