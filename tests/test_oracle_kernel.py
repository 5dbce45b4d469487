"""Pins of the oracle's Biot-Savart sums and Jacobians (CPU only).

Each check ties the oracle to something other than itself: hand-evaluated
values (golden file), exact rational arithmetic, the paper's second matrix
formulation (Eq. 4-6), conserved invariants of the pair kernel, central finite
differences and the adjoint identity.
"""
from fractions import Fraction
import os

import numpy as np
import pytest

from oracle import direct, kernel
from paper_2103_01983_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "three_body.txt")


def _golden():
    rows = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        rows[key] = np.array([float(Fraction(v)) for v in vals])
    return rows


@pytest.mark.parametrize("delta,tag", [(0.0, "delta0"), (0.5, "delta05")])
def test_three_body_hand_values(delta, tag):
    g = _golden()
    x = np.concatenate([g["chi"], g["psi"]])
    Gamma = 2.0 * np.pi * g["gamma_over_2pi"]
    f, D = direct.velocity(x, Gamma, delta, with_selfjac=True)
    np.testing.assert_allclose(f[:3], g[f"{tag}_f_chi"], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(f[3:], g[f"{tag}_f_psi"], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(kernel.velocity_K(x, Gamma, delta), f, rtol=1e-14, atol=1e-14)
    if tag == "delta0":
        for k, row in enumerate(["D00", "D01", "D10"]):
            np.testing.assert_allclose(D[k], g[f"delta0_{row}"], rtol=1e-14, atol=1e-14)


def _exact_velocity(chi, psi, gam, delta):
    """Eq. 2 in exact rationals (gam = Gamma/(2 pi) given as Fractions)."""
    n = len(chi)
    out = []
    for i in range(n):
        u = Fraction(0)
        v = Fraction(0)
        for j in range(n):
            if j == i:
                continue
            a, b = chi[i] - chi[j], psi[i] - psi[j]
            s = a * a + b * b + delta
            u += gam[j] * (-b) / s
            v += gam[j] * a / s
        out.append((u, v))
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_exact_rational_small_n(seed):
    rng = np.random.default_rng(seed)
    n = 6
    chi = [Fraction(int(k), 64) for k in rng.integers(-64, 64, n)]
    psi = [Fraction(int(k), 64) for k in rng.integers(-64, 64, n)]
    gam = [Fraction(int(k), 16) for k in rng.integers(-32, 32, n)]
    delta = Fraction(1, 20)
    exact = _exact_velocity(chi, psi, gam, delta)
    x = np.array([float(c) for c in chi] + [float(p) for p in psi])
    Gamma = 2.0 * np.pi * np.array([float(g) for g in gam])
    f = direct.velocity(x, Gamma, float(delta))
    ref = np.array([float(u) for u, _ in exact] + [float(v) for _, v in exact])
    np.testing.assert_allclose(f, ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("delta", [0.05, 0.0])
def test_loop_matches_matrix_form(delta):
    x, G = W.disk(200, seed=4)
    f = direct.velocity(x, G, delta)
    fk = kernel.velocity_K(x, G, delta)
    assert np.linalg.norm(f - fk) <= 1e-13 * np.linalg.norm(f)


@pytest.mark.parametrize("delta", [0.05, 0.02])
def test_pair_antisymmetry_invariants(delta):
    """sum_i Gamma_i f_i = 0 and sum_i Gamma_i x_i . f_i = 0 (pairwise cancellation)."""
    x, G = W.two_cluster(512, seed=5)
    f = direct.velocity(x, G, delta)
    n = G.size
    scale = np.abs(G).sum() * np.abs(f).max()
    assert abs(np.dot(G, f[:n])) <= 1e-13 * scale
    assert abs(np.dot(G, f[n:])) <= 1e-13 * scale
    ang = np.dot(G, x[:n] * f[:n] + x[n:] * f[n:])
    assert abs(ang) <= 1e-13 * scale * np.abs(x).max()


def test_two_vortex_angular_velocity():
    """Two vortices at distance d co-rotate at omega = (G1+G2)/(2 pi (d^2+delta))."""
    d, delta, g1, g2 = 0.7, 0.05, 1.3, 0.4
    x, G = W.two_vortex(d, g1, g2)
    f = direct.velocity(x, G, delta)
    omega = (g1 + g2) / (2.0 * np.pi * (d * d + delta))
    rel = np.array([f[1] - f[0], f[3] - f[2]])     # d/dt (x_2 - x_1)
    # relative vector (d, 0) rotates counter-clockwise: velocity (0, omega d)
    np.testing.assert_allclose(rel, [0.0, omega * d], rtol=1e-14, atol=1e-15)


def _fd_jacobian(fun, x, h):
    cols = []
    for k in range(x.size):
        e = np.zeros_like(x)
        e[k] = h
        cols.append((fun(x + e) - fun(x - e)) / (2.0 * h))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("delta", [0.05, 0.3])
def test_jacobian_central_differences(delta):
    x, G = W.disk(8, seed=6)
    J = kernel.jacobian(x, G, delta)
    Jfd = _fd_jacobian(lambda y: direct.velocity(y, G, delta), x, 1e-6)
    assert np.abs(J - Jfd).max() <= 1e-6 * np.abs(J).max()
    Gfd = _fd_jacobian(lambda g: direct.velocity(x, g, delta), G, 1e-6)
    np.testing.assert_allclose(kernel.dfdGamma(x, G, delta), Gfd, atol=1e-8)
    # the self block the C loop returns is the diagonal block of J, trace-free
    _, D = direct.velocity(x, G, delta, with_selfjac=True)
    n = G.size
    np.testing.assert_allclose(D[0], np.diag(J[:n, :n]), atol=1e-12)
    np.testing.assert_allclose(D[1], np.diag(J[:n, n:]), atol=1e-12)
    np.testing.assert_allclose(D[2], np.diag(J[n:, :n]), atol=1e-12)
    np.testing.assert_allclose(-D[0], np.diag(J[n:, n:]), atol=1e-12)


def test_jvp_vjp_match_dense_and_adjoint():
    x, G = W.disk(96, seed=7)
    delta = 0.05
    J = kernel.jacobian(x, G, delta)
    v, w = W.random_vectors(x.size, 2, seed=8)
    jv = direct.jvp(x, G, delta, v)
    gx, gG = direct.vjp(x, G, delta, w)
    np.testing.assert_allclose(jv, J @ v, rtol=0, atol=1e-11 * np.abs(J @ v).max())
    np.testing.assert_allclose(gx, J.T @ w, rtol=0, atol=1e-11 * np.abs(gx).max())
    np.testing.assert_allclose(gG, kernel.dfdGamma(x, G, delta).T @ w, atol=1e-12)
    # adjoint identity between two differently ordered loops
    assert abs(np.dot(w, jv) - np.dot(gx, v)) <= 1e-12 * np.abs(w).sum() * np.abs(jv).max()
    phi = W.random_vectors(x.size, 3, seed=9).T
    np.testing.assert_allclose(direct.jphi(x, G, delta, phi), J @ phi,
                               atol=1e-11 * np.abs(J @ phi).max())


def test_targets_apart_from_sources():
    """Grid targets (Sec. 6.1 velocity field): same sum with distinct targets."""
    x, G = W.disk(50, seed=10)
    t = np.concatenate([np.linspace(-1, 1, 7), np.linspace(-0.5, 0.5, 7)])
    f = direct.velocity(x, G, 0.05, targets=t)
    n = G.size
    ref = np.zeros(14)
    for i in range(7):
        a = t[i] - x[:n]
        b = t[7 + i] - x[n:]
        s = a * a + b * b + 0.05
        ref[i] = np.sum(G / (2 * np.pi) * (-b) / s)
        ref[7 + i] = np.sum(G / (2 * np.pi) * a / s)
    np.testing.assert_allclose(f, ref, rtol=1e-13, atol=1e-15)
