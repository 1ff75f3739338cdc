"""Exact products with the exponential kernel.  Test infrastructure.

Matrix: ``a_ij = sum_k c_k exp(-|t_i - t_j| / l_k)`` with sorted points t.
Its off-diagonal blocks have exact rank K (HODLR) and its HSS block rows
rank 2K, which makes it an exact-rank fixture.  ``apply`` computes ``A X`` in
O(n K r) by two first-order recurrences per k:

    f_i = e^{-(t_i - t_{i-1})/l} f_{i-1} + x_i   (sum over j <= i)
    b_i = e^{-(t_{i+1} - t_i)/l} b_{i+1} + x_i   (sum over j >= i)
    y_i = sum_k c_k (f_i + b_i - x_i)

Every factor lies in (0, 1], so the recurrences are stable.
"""

import numpy as np


def entries(t, ck, lk, rows, cols):
    """Entry-by-entry evaluation of A(rows, cols)."""
    t = np.asarray(t, dtype=np.float64)
    d = np.abs(t[np.asarray(rows)][:, None] - t[np.asarray(cols)][None, :])
    out = np.zeros(d.shape)
    for c_, l_ in zip(ck, lk):
        out += c_ * np.exp(-d / l_)
    return out


def apply(t, ck, lk, X):
    t = np.asarray(t, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    n, r = X.shape
    Y = np.zeros((n, r))
    if n == 0:
        return Y
    dt = np.diff(t)
    for c_, l_ in zip(ck, lk):
        e = np.exp(-dt / l_)
        f = np.empty((n, r))
        b = np.empty((n, r))
        f[0] = X[0]
        for i in range(1, n):
            f[i] = e[i - 1] * f[i - 1] + X[i]
        b[n - 1] = X[n - 1]
        for i in range(n - 2, -1, -1):
            b[i] = e[i] * b[i + 1] + X[i]
        Y += c_ * (f + b - X)
    return Y
