"""Reference of the learned damping network (TEST INFRASTRUCTURE ONLY).

omega = 2 sigmoid(W3 relu(W2 relu(W1 f + b1) + b2) + b3) per row, f = 4 row
features.  Plain numpy in float64 on the given (already bf16-rounded) weights;
the CUDA library computes the same map with bf16 weights and float32
accumulation.  The parameter vector is laid out as
[W1 (32x4, row-major), b1 (32), W2 (32x32), b2 (32), W3 (32), b3 (1)].

Also: the row features the library computes on each hierarchy level, from the
level's CSR and l1 norms (plain loops over rows):
  f0 = a_ii / l1_i
  f1 = ln(l1_i) - mean over the stored columns j of row i of ln(l1_j)
  f2 = nnz_i / 27
  f3 = level / 4
"""
from __future__ import annotations

import numpy as np

H = 32
NPARAM = 32 * 4 + 32 + 32 * 32 + 32 + 32 + 1  # 1249


def unpack(theta):
    t = np.asarray(theta, dtype=np.float64)
    assert t.shape == (NPARAM,)
    o = 0
    W1 = t[o:o + 128].reshape(32, 4); o += 128
    b1 = t[o:o + 32]; o += 32
    W2 = t[o:o + 1024].reshape(32, 32); o += 1024
    b2 = t[o:o + 32]; o += 32
    W3 = t[o:o + 32]; o += 32
    b3 = t[o]
    return W1, b1, W2, b2, W3, b3


def forward(theta, feats):
    """omega for every row of feats (n x 4)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    f = np.asarray(feats, dtype=np.float64)
    h1 = np.maximum(f @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    o = h2 @ W3 + b3
    return 2.0 / (1.0 + np.exp(-o))


def backward(theta, feats, domega):
    """d(sum_i domega_i omega_i)/d theta."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    f = np.asarray(feats, dtype=np.float64)
    a1 = f @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    o = h2 @ W3 + b3
    s = 1.0 / (1.0 + np.exp(-o))
    dout = np.asarray(domega, dtype=np.float64) * 2.0 * s * (1.0 - s)
    dW3 = h2.T @ dout
    db3 = dout.sum()
    dh2 = np.outer(dout, W3) * (a2 > 0)
    dW2 = dh2.T @ h1
    db2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (a1 > 0)
    dW1 = dh1.T @ f
    db1 = dh1.sum(axis=0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3, [db3]])


def features(rp, ci, v, l1, level):
    n = len(rp) - 1
    out = np.zeros((n, 4))
    ll = np.log(l1)
    for i in range(n):
        cols = ci[rp[i]:rp[i + 1]]
        vals = v[rp[i]:rp[i + 1]]
        d = vals[cols == i][0]
        out[i, 0] = d / l1[i]
        out[i, 1] = ll[i] - ll[cols].mean()
        out[i, 2] = (rp[i + 1] - rp[i]) / 27.0
        out[i, 3] = level / 4.0
    return out
