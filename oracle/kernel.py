"""Dense NumPy formulations of the Biot-Savart kernel and its Jacobian.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

These are the paper's matrix forms, written independently of the C loops in
``bs_direct.c`` so that the two can pin each other:

* ``velocity_K``: f = K gamma (Sec. 2, Eq. 4-6).  kappa_ij = e3 x (x_i - x_j)
  / (|x_i - x_j|^2 + delta); K = diag(K^ul, K^br) with K^ul_ij = kappa_ij1,
  K^br_ij = kappa_ij2; gamma = [Gamma; Gamma] / (2 pi).
* ``jacobian``: the full N_d x N_d matrix d f / d x, assembled from the
  analytic 2x2 pair blocks (diagonal block D_i, off-diagonal -gamma_j A_ij).
* ``dfdGamma``: the N_d x N matrix d f / d Gamma.
"""
from __future__ import annotations

import numpy as np


def _diffs(x):
    n = x.size // 2
    chi, psi = x[:n], x[n:]
    a = chi[:, None] - chi[None, :]
    b = psi[:, None] - psi[None, :]
    return a, b


def velocity_K(x, Gamma, delta):
    """f = K gamma (Eq. 6).  The diagonal kappa_ii is zero (the j != i term)."""
    a, b = _diffs(np.asarray(x, dtype=np.float64))
    s = a * a + b * b + delta
    self_pair = (a == 0.0) & (b == 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        k1 = np.where(self_pair, 0.0, -b / s)   # first component of e3 x r
        k2 = np.where(self_pair, 0.0, a / s)    # second component
    n = a.shape[0]
    K = np.zeros((2 * n, 2 * n))
    K[:n, :n] = k1
    K[n:, n:] = k2
    gamma = np.concatenate([Gamma, Gamma]) / (2.0 * np.pi)
    return K @ gamma


def pair_blocks(a, b, delta):
    """A(r) entries for arrays a, b (r = (a, b)): derivative of (-b, a)/s."""
    s = a * a + b * b + delta
    A00 = 2.0 * a * b / s**2
    A01 = -1.0 / s + 2.0 * b * b / s**2
    A10 = 1.0 / s - 2.0 * a * a / s**2
    A11 = -2.0 * a * b / s**2
    return A00, A01, A10, A11


def jacobian(x, Gamma, delta):
    """Dense d f / d x (N_d x N_d) in the [chi; psi] layout."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size // 2
    a, b = _diffs(x)
    self_pair = (a == 0.0) & (b == 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        blocks = pair_blocks(a, b, delta)
    g = np.asarray(Gamma, dtype=np.float64) / (2.0 * np.pi)
    J = np.zeros((2 * n, 2 * n))
    quads = [(slice(0, n), slice(0, n)), (slice(0, n), slice(n, 2 * n)),
             (slice(n, 2 * n), slice(0, n)), (slice(n, 2 * n), slice(n, 2 * n))]
    for A, (rs, cs) in zip(blocks, quads):
        A = np.where(self_pair, 0.0, A)
        off = -A * g[None, :]                   # d f_i / d x_j, j != i
        diag = (A * g[None, :]).sum(axis=1)     # D_i = sum_j gamma_j A_ij
        blk = off.copy()
        np.fill_diagonal(blk, diag)
        J[rs, cs] = blk
    return J


def dfdGamma(x, Gamma, delta):
    """Dense d f / d Gamma (N_d x N): column k holds kappa_ik / (2 pi)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size // 2
    a, b = _diffs(x)
    s = a * a + b * b + delta
    self_pair = (a == 0.0) & (b == 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        k1 = np.where(self_pair, 0.0, -b / s)
        k2 = np.where(self_pair, 0.0, a / s)
    return np.concatenate([k1, k2], axis=0) / (2.0 * np.pi)
