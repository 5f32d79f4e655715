"""Oracle of the learned row-size estimator (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` use this module; the library never does.

The paper sizes nothing by learning: it recomputes each affected row with
Gustavson's algorithm (Section 6.1).  The estimator predicts, for a row i of
C = A B, the number of non-zeros nnz(C_i) from four features of the row
(the length of A_i and the sum, maximum and mean of the lengths of the B
rows it reads), so that the row can be given a hash table near its true
size instead of its product bound.  The prediction only picks a table: a
row whose table turns out too small is recomputed after an exact count, so
C never depends on it.

This module states the network in plain numpy float64, one operation per
line, so each step can be checked by eye:

    features  x = log2(1 + [len(A_i), sum_k len(B_k), max_k len(B_k), mean_k len(B_k)])
    layer 1   h1 = relu(W1 x + b1)           W1: 64 x 4
    layer 2   h2 = relu(W2 h1 + b2)          W2: 64 x 64
    output    o  = W3 h2 + b3                W3: 1 x 64
    target    y  = log2(1 + nnz(C_i))
    loss      L  = mean over rows of (o - y)^2

Weights are used rounded to bfloat16 (round to nearest, ties to even, from
their float32 value); arithmetic is float64 here (float32 accumulation on
the GPU).  Gradients are taken with respect to the rounded weights and
applied to the float32 master copy by plain SGD (p <- p - lr * g).  The
parameters are one flat vector in the order W1 (row-major), b1, W2
(row-major), b2, W3, b3: 4545 numbers.
"""

from __future__ import annotations

import numpy as np

N_IN = 4
N_HID = 64
SHAPES = [(N_HID, N_IN), (N_HID,), (N_HID, N_HID), (N_HID,), (1, N_HID), (1,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)


def bf16_round(a) -> np.ndarray:
    """float32 value of a, rounded to bfloat16 (8 exponent bits, 7 stored
    mantissa bits) to nearest with ties to even; returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    keep_lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + keep_lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p: np.ndarray):
    out, at = [], 0
    for shape in SHAPES:
        k = int(np.prod(shape))
        out.append(np.asarray(p[at:at + k], dtype=np.float64).reshape(shape))
        at += k
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(x, dtype=np.float64).reshape(-1) for x in parts])


def features(alen: np.ndarray, bsum: np.ndarray, bmax: np.ndarray) -> np.ndarray:
    """The four inputs of each row from len(A_i) and the sum and maximum of
    the B-row lengths it reads (mean = sum / len(A_i), 0 for an empty row)."""
    alen = np.asarray(alen, dtype=np.float64)
    bsum = np.asarray(bsum, dtype=np.float64)
    bmax = np.asarray(bmax, dtype=np.float64)
    mean = np.where(alen > 0, bsum / np.maximum(alen, 1), 0.0)
    return np.log2(1.0 + np.stack([alen, bsum, bmax, mean], axis=1))


def row_features(A, B) -> np.ndarray:
    """features() of every row of A (CSR) against B's row lengths."""
    blen = np.diff(np.asarray(B.rowptr)).astype(np.int64)
    n = A.nrows
    alen = np.diff(np.asarray(A.rowptr)).astype(np.int64)
    rows = np.repeat(np.arange(n), alen)
    lens = blen[np.asarray(A.col)]
    bsum = np.bincount(rows, weights=lens, minlength=n)
    bmax = np.zeros(n)
    np.maximum.at(bmax, rows, lens)
    return features(alen, bsum, bmax)


def forward(p: np.ndarray, X: np.ndarray, rounded: bool = True):
    """Outputs o (one per row) and the activations the gradient needs."""
    W1, b1, W2, b2, W3, b3 = unpack(bf16_round(p) if rounded else p)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    o = h2 @ W3[0] + b3[0]
    return o, (X, z1, h1, z2, h2)


def loss(p: np.ndarray, X: np.ndarray, y: np.ndarray, rounded: bool = True) -> float:
    o, _ = forward(p, X, rounded)
    return float(np.mean((o - y) ** 2))


def loss_and_grad(p: np.ndarray, X: np.ndarray, y: np.ndarray, rounded: bool = True):
    """L and dL/dw at the (rounded) weights, by the chain rule layer by
    layer (back-propagation)."""
    W1, b1, W2, b2, W3, b3 = unpack(bf16_round(p) if rounded else p)
    o, (X, z1, h1, z2, h2) = forward(p, X, rounded)
    n = X.shape[0]
    d_o = 2.0 * (o - y) / n                      # dL/do, one per row
    g_W3 = (d_o @ h2)[None, :]                   # dL/dW3 = sum_r d_o[r] h2[r]
    g_b3 = np.array([d_o.sum()])
    d_h2 = np.outer(d_o, W3[0])                  # dL/dh2
    d_z2 = d_h2 * (z2 > 0)                       # through relu
    g_W2 = d_z2.T @ h1
    g_b2 = d_z2.sum(axis=0)
    d_h1 = d_z2 @ W2
    d_z1 = d_h1 * (z1 > 0)
    g_W1 = d_z1.T @ X
    g_b1 = d_z1.sum(axis=0)
    return float(np.mean((o - y) ** 2)), pack([g_W1, g_b1, g_W2, g_b2, g_W3, g_b3])


def sgd_step(p: np.ndarray, g: np.ndarray, lr: float) -> np.ndarray:
    """One SGD step on the float32 master weights."""
    return (np.asarray(p, np.float32) - np.float32(lr) * np.asarray(g, np.float32)).astype(np.float64)


def predict_nnz(p: np.ndarray, X: np.ndarray) -> np.ndarray:
    """The estimate 2^o - 1 of nnz(C_i) (before any clamping)."""
    o, _ = forward(p, X)
    return np.exp2(o) - 1.0
