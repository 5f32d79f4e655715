"""Pins of the estimator oracle (oracle/mlp.py) against facts outside it:
bfloat16 rounding values fixed by the format, a network worked by hand, the
composed-matrix closed form of the network where no ReLU is active, central
finite differences of the loss, and brute-force features on a small matrix.
"""

import numpy as np
import pytest

from oracle import mlp
from workloads import mlp_init_params, random_csr


def test_bf16_rounding_values_of_the_format():
    u = 2.0 ** -7  # spacing of bfloat16 numbers in [1, 2)
    cases = {
        1.0: 1.0,
        1.0 + u / 2: 1.0,                       # tie, rounds to the even mantissa (...0)
        1.0 + 1.5 * u: 1.0 + 2 * u,             # tie, rounds to the even mantissa (...10)
        1.0 + u / 2 + 2.0 ** -20: 1.0 + u,      # just above the tie rounds up
        1.0 + u / 2 - 2.0 ** -20: 1.0,          # just below rounds down
        -1.5: -1.5,
        0.1: 0.10009765625,                     # 0x3DCCCCCD -> 0x3DCD
        0.0: 0.0,
    }
    got = mlp.bf16_round(np.array(list(cases.keys())))
    assert np.array_equal(got, np.array(list(cases.values())))


def _single_path_params():
    W1 = np.zeros((64, 4)); W1[0, 0] = 1.0
    b1 = np.zeros(64)
    W2 = np.zeros((64, 64)); W2[0, 0] = 2.0
    b2 = np.zeros(64)
    W3 = np.zeros((1, 64)); W3[0, 0] = 3.0
    b3 = np.array([1.0])
    return mlp.pack([W1, b1, W2, b2, W3, b3])


def test_network_worked_by_hand():
    """One active path x0 -> h1_0 -> h2_0 -> o: o = 3 * (2 * (1 * x0)) + 1.
    With x0 = 1 and y = 5: o = 7, L = (7 - 5)^2 = 4, and by the chain rule
    dL/dW3[0,0] = 2 (o - y) h2_0 = 8, dL/dW2[0,0] = 2 (o - y) W3 h1_0 = 12,
    dL/dW1[0,0] = 2 (o - y) W3 W2 x0 = 24, dL/db3 = 2 (o - y) = 4."""
    p = _single_path_params()
    X = np.array([[1.0, 0.7, 0.2, 0.9]])
    L, g = mlp.loss_and_grad(p, X, np.array([5.0]))
    assert L == 4.0
    gW1, gb1, gW2, gb2, gW3, gb3 = mlp.unpack(g)
    assert gW3[0, 0] == 8.0 and gW2[0, 0] == 12.0 and gW1[0, 0] == 24.0 and gb3[0] == 4.0
    assert gW1[0, 1] == 2 * 2 * 3 * 2 * 0.7  # the other inputs of unit 0 get x_j times the same factor
    assert np.count_nonzero(gW2) == 1 and np.count_nonzero(gW3) == 1
    o, _ = mlp.forward(p, X)
    assert o[0] == 7.0


def test_linear_regime_matches_composed_matrices():
    """With non-negative weights, biases and inputs no ReLU clips, so the
    network is the affine map o = (W3 W2 W1) x + W3 W2 b1 + W3 b2 + b3,
    computed here by composing the matrices in the mathematical order
    (a transposed operand in the layer-by-layer oracle would differ)."""
    rng = np.random.default_rng(3)
    W1 = rng.uniform(0, 1, (64, 4)); b1 = rng.uniform(0, 1, 64)
    W2 = rng.uniform(0, 1, (64, 64)); b2 = rng.uniform(0, 1, 64)
    W3 = rng.uniform(-1, 1, (1, 64)); b3 = rng.uniform(-1, 1, 1)
    p = mlp.pack([W1, b1, W2, b2, W3, b3])
    X = rng.uniform(0, 3, (9, 4))
    M = W3 @ W2 @ W1
    c = W3 @ W2 @ b1 + W3 @ b2 + b3
    want = np.array([(M @ x + c)[0] for x in X])
    o, _ = mlp.forward(p, X, rounded=False)
    assert np.allclose(o, want, rtol=1e-12, atol=1e-9)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    p = mlp_init_params(11) + rng.normal(0, 0.05, mlp.N_PARAMS)
    X = rng.uniform(0, 10, (13, 4))
    y = rng.uniform(0, 12, 13)
    L, g = mlp.loss_and_grad(p, X, y, rounded=False)
    h = 1e-6
    idx = rng.choice(mlp.N_PARAMS, size=60, replace=False)
    idx = np.concatenate([idx, [mlp.N_PARAMS - 1, 0, 255, 256]])  # b3, W1[0,0], W1[63,3], b1[0]
    for k in idx:
        e = np.zeros(mlp.N_PARAMS); e[k] = h
        fd = (mlp.loss(p + e, X, y, rounded=False) - mlp.loss(p - e, X, y, rounded=False)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_rounded_gradient_is_the_gradient_at_the_rounded_weights():
    rng = np.random.default_rng(6)
    p = mlp_init_params(12)
    X = rng.uniform(0, 8, (20, 4))
    y = rng.uniform(0, 10, 20)
    L1, g1 = mlp.loss_and_grad(p, X, y, rounded=True)
    L2, g2 = mlp.loss_and_grad(mlp.bf16_round(p), X, y, rounded=False)
    assert L1 == L2 and np.array_equal(g1, g2)
    # rounding changes the weights by at most half a bfloat16 spacing (2^-8 relative)
    r = mlp.bf16_round(p)
    nz = p != 0
    assert np.all(np.abs(r[nz] - p[nz]) <= 2.0 ** -8 * np.abs(p[nz]))


def test_sgd_learns_a_feature_of_the_input():
    """The target log2(1 + sum) is the second input itself; SGD from the
    initial weights must bring the loss down by 100x."""
    rng = np.random.default_rng(7)
    X = mlp.features(rng.integers(1, 50, 256), rng.integers(1, 5000, 256), rng.integers(1, 100, 256))
    y = X[:, 1].copy()
    p = mlp_init_params(13)
    L0 = mlp.loss(p, X, y)
    for _ in range(400):
        _, g = mlp.loss_and_grad(p, X, y)
        p = mlp.sgd_step(p, g, 5e-4)
    assert mlp.loss(p, X, y) < L0 / 100


def test_features_by_brute_force():
    A = random_csr(40, 30, 9, seed=8)
    B = random_csr(30, 50, 12, seed=9)
    X = mlp.row_features(A, B)
    blen = np.diff(B.rowptr)
    for i in range(A.nrows):
        cols = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        lens = [int(blen[k]) for k in cols]
        raw = [len(cols), sum(lens), max(lens) if lens else 0, (sum(lens) / len(cols)) if len(cols) else 0.0]
        assert np.allclose(X[i], np.log2(1.0 + np.array(raw, dtype=float)), rtol=0, atol=1e-15)
    # a worked row: A row reading B rows of lengths 3 and 5 -> log2(1 + [2, 8, 5, 4])
    f = mlp.features(np.array([2]), np.array([8]), np.array([5]))
    assert np.allclose(f[0], [np.log2(3), np.log2(9), np.log2(6), np.log2(5)], atol=1e-15)
    assert np.array_equal(mlp.features(np.array([0]), np.array([0]), np.array([0]))[0], np.zeros(4))


def test_param_count_and_layout():
    assert mlp.N_PARAMS == 64 * 4 + 64 + 64 * 64 + 64 + 64 + 1 == 4545
    p = np.arange(mlp.N_PARAMS, dtype=float)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p)
    assert W1[0, 1] == 1 and b1[0] == 256 and W2[0, 1] == 321 and b2[0] == 4416 and W3[0, 0] == 4480 and b3[0] == 4544
    assert np.array_equal(mlp.pack(mlp.unpack(p)), p)


def test_predict_nnz_worked_value():
    """The estimate is 2^o - 1 (the inverse of the target y = log2(1 + nnz)).
    The one-path network of test_network_worked_by_hand gives o = 6 x0 + 1;
    with x0 = 1 that is o = 7, an estimate of 2^7 - 1 = 127 entries, and
    with x0 = 0 (an empty A row) o = 1 and the estimate is 1.  A network
    whose output is the target itself recovers nnz exactly: log2(1 + 127) = 7."""
    p = _single_path_params()
    X = np.array([[1.0, 0.7, 0.2, 0.9], [0.0, 3.0, 1.0, 2.0]])
    est = mlp.predict_nnz(p, X)
    assert est.tolist() == [127.0, 1.0]
    assert np.log2(1.0 + est[0]) == 7.0
