"""Quantities of interest and invariants (Sec. 6.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import numpy as np


def hamiltonian(x, Gamma):
    """H = 1/(4 pi) sum_j sum_{i != j} Gamma_j Gamma_i log |x_j - x_i| (Sec. 6.1)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size // 2
    a = x[:n, None] - x[None, :n]
    b = x[n:, None] - x[None, n:]
    r = np.sqrt(a * a + b * b)
    np.fill_diagonal(r, 1.0)          # log 1 = 0 removes the i == j term
    G = np.asarray(Gamma)
    return float((G[:, None] * G[None, :] * np.log(r)).sum() / (4.0 * np.pi))


def ae_h(h_rom, h_fom):
    """AE_H = |(H_III - H_I) / H_I| (Eq. AE_Hamiltonian)."""
    return abs((h_rom - h_fom) / h_fom)


def mae_d(x_fom, x_rom, x0):
    """MAE_D = 1/(l N) sum_i |x_i,I - x_i,III|, l = |x_N^0 - x_1^0| (Eq. MAE_trajectory)."""
    n = x0.size // 2
    l = np.hypot(x0[n - 1] - x0[0], x0[2 * n - 1] - x0[n])
    d = np.hypot(x_fom[:n] - x_rom[:n], x_fom[n:] - x_rom[n:])
    return float(d.sum() / (l * n))


def linear_impulse(x, Gamma):
    n = x.size // 2
    return np.array([np.dot(Gamma, x[:n]), np.dot(Gamma, x[n:])])


def angular_impulse(x, Gamma):
    n = x.size // 2
    return float(np.dot(Gamma, x[:n] ** 2 + x[n:] ** 2))
