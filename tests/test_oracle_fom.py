"""Pins of the oracle's implicit trapezoid FOM (CPU only)."""
import numpy as np
import pytest

from oracle import direct, fom, qoi
from paper_2103_01983_gb300 import workloads as W


@pytest.mark.parametrize("mode", ["dense", "blockdiag", "jfnk"])
def test_two_vortex_trapezoid_rotation(mode):
    """The trapezoid rule maps the relative vector by a Cayley transform:
    |r| is kept and the angle advances by exactly 2 atan(omega dt / 2)."""
    d, delta, g1, g2, dt = 0.8, 0.05, 1.0, 1.0, 0.1
    x, G = W.two_vortex(d, g1, g2)
    omega = (g1 + g2) / (2 * np.pi * (d * d + delta))
    traj, _ = fom.rollout(x, G, delta, dt, 10, mode=mode, tol=1e-14)
    r = np.stack([traj[:, 1] - traj[:, 0], traj[:, 3] - traj[:, 2]], axis=1)
    ang = np.unwrap(np.arctan2(r[:, 1], r[:, 0]))
    np.testing.assert_allclose(np.diff(ang), 2 * np.arctan(omega * dt / 2), rtol=1e-11)
    np.testing.assert_allclose(np.hypot(r[:, 0], r[:, 1]), d, rtol=1e-12)
    # Gamma-weighted centroid is fixed
    c = (g1 * traj[:, [0, 2]] + g2 * traj[:, [1, 3]]) / (g1 + g2)
    np.testing.assert_allclose(c, 0.0, atol=1e-13)


def test_modes_agree_and_impulse_conserved():
    x, G = W.disk(128, seed=11)
    delta, dt = 0.05, 0.01
    out = {}
    for mode in ["dense", "blockdiag", "jfnk"]:
        traj, it = fom.rollout(x, G, delta, dt, 5, mode=mode, tol=1e-13)
        out[mode] = traj
        P = np.array([qoi.linear_impulse(s, G) for s in traj])
        # sum_i Gamma_i r_i = P(x^n) - P(x^{n-1}) because sum_i Gamma_i f_i = 0,
        # so the drift per step is bounded by |Gamma|_2 * ||r||_2 <= |Gamma|_2 tol |x|
        bound = np.linalg.norm(G) * 1e-13 * np.linalg.norm(traj, axis=1).max() * 5 + 1e-14
        np.testing.assert_allclose(P, np.broadcast_to(P[0], P.shape), rtol=0, atol=bound)
    np.testing.assert_allclose(out["blockdiag"], out["dense"], atol=1e-11)
    np.testing.assert_allclose(out["jfnk"], out["dense"], atol=1e-11)


def test_residual_zero_at_solution():
    x, G = W.disk(64, seed=12)
    delta, dt = 0.05, 0.01
    f0 = direct.velocity(x, G, delta)
    x1, f1, k, rn = fom.step(x, f0, G, delta, dt, mode="dense", tol=1e-14)
    r = x1 - x - 0.5 * dt * (direct.velocity(x1, G, delta) + f0)
    assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(x1)
    np.testing.assert_allclose(f1, direct.velocity(x1, G, delta), rtol=0, atol=0)


def test_hamiltonian_two_vortex():
    """H = Gamma1 Gamma2 log(d) / (2 pi) for two bodies (both ordered pairs)."""
    x, G = W.two_vortex(2.5, 1.5, -0.7)
    assert qoi.hamiltonian(x, G) == pytest.approx(1.5 * -0.7 * np.log(2.5) / (2 * np.pi), rel=1e-14)


def test_adjoint_of_linear_impulse_is_closed_form():
    """P(T) = sum Gamma x(T) is conserved, so d/dx0 (P_chi + P_psi) = Gamma
    for both components and d/dGamma (with Gamma also in L) = chi0 + psi0."""
    x0, G = W.disk(24, seed=13)
    n = G.size
    lam_T = np.concatenate([G, G])
    gx, gG, traj = fom.adjoint_rollout(x0, G, 0.05, 0.01, 8, lam_T)
    np.testing.assert_allclose(gx, np.concatenate([G, G]), atol=1e-10)
    gG_total = gG + traj[-1][:n] + traj[-1][n:]          # explicit d L / d Gamma
    np.testing.assert_allclose(gG_total, x0[:n] + x0[n:], atol=1e-10)


def test_adjoint_matches_finite_differences():
    x0, G = W.disk(16, seed=14)
    lam_T = W.random_vectors(x0.size, 1, seed=15)[0]
    gx, gG, _ = fom.adjoint_rollout(x0, G, 0.05, 0.01, 6, lam_T)
    dirs = W.random_vectors(x0.size + G.size, 4, seed=16)
    h = 1e-5
    for d in dirs:
        dx, dg = d[:x0.size], d[x0.size:]
        Lp = lam_T @ fom.rollout(x0 + h * dx, G + h * dg, 0.05, 0.01, 6, mode="dense", tol=1e-14)[0][-1]
        Lm = lam_T @ fom.rollout(x0 - h * dx, G - h * dg, 0.05, 0.01, 6, mode="dense", tol=1e-14)[0][-1]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - (gx @ dx + gG @ dg)) <= 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("mode", ["dense", "blockdiag", "jfnk"])
def test_inflow_without_circulation_is_uniform_motion(mode):
    """Gamma = 0 leaves only the superimposed inflow (Sec. 6.3): every body
    moves by dt u per step, exactly."""
    x, _, u = W.mushroom(-100.0, 100.0, n=16)
    G = np.zeros(16)
    traj, it = fom.rollout(x, G, 0.15, 0.005, 6, mode=mode, tol=1e-14, u_inf=u)
    k = np.arange(7)[:, None]
    np.testing.assert_allclose(traj, x + k * 0.005 * u, rtol=0, atol=1e-12)


def test_uniform_inflow_is_a_galilean_shift():
    """Pair sums depend on differences only, so a uniform inflow U moves the
    whole no-inflow trajectory by n dt U (Newton tolerance)."""
    x, G = W.disk(48, seed=5)
    delta, dt, steps = 0.05, 0.01, 8
    U = np.concatenate([np.full(48, 0.7), np.full(48, -1.3)])
    ref, _ = fom.rollout(x, G, delta, dt, steps, mode="dense", tol=1e-14)
    got, _ = fom.rollout(x, G, delta, dt, steps, mode="dense", tol=1e-14, u_inf=U)
    k = np.arange(steps + 1)[:, None]
    np.testing.assert_allclose(got, ref + k * dt * U, rtol=0, atol=1e-11)


def test_mushroom_workload_matches_the_paper():
    """Sec. 6.3: end bodies at (-37.43, -10) and (37.43, -10), spacing 0.15,
    the inflow peak 5 * 1.125 + 0.5 at the middle and 5 sqrt(1.125^2 - 1) + 0.5
    at the ends."""
    x, G, u = W.mushroom(-220.0, 110.0)
    n = 500
    assert (x[0], x[n - 1], x[n], x[2 * n - 1]) == (-37.43, 37.43, -10.0, -10.0)
    assert np.diff(x[:n]) == pytest.approx(0.15, abs=2e-4)
    assert (G[0], G[-1], G[1]) == (-220.0, 110.0, 0.01)
    assert np.all(u[:n] == 0.0)
    assert u[n] == pytest.approx(5 * np.sqrt(1.125 ** 2 - 1) + 0.5, rel=1e-15)
    assert u[n:].max() == pytest.approx(5 * 1.125 + 0.5, rel=1e-5)
    train, query = W.mushroom_params(0)
    assert train.shape == (4, 2) and query.shape == (36, 2)
    assert np.all((train[:, 0] >= -220) & (train[:, 0] <= -110) & (train[:, 1] >= 110) & (train[:, 1] <= 220))


def test_mae_d_and_ae_h_closed_forms():
    """MAE_D (Eq. MAE_trajectory): every body displaced by the same vector d
    gives |d| / l with l = |x_N^0 - x_1^0|; AE_H (Eq. AE_Hamiltonian) is the
    relative gap of the Hamiltonians; a rigid translation leaves H unchanged."""
    x0 = np.array([0.0, 3.0, 1.0, 0.0, 4.0, 2.0])          # bodies (0,0), (3,4), (1,2): l = |(1,2)| = sqrt 5
    G = np.array([1.0, -2.0, 0.5])
    d = np.array([0.3, -0.4])                              # |d| = 0.5
    shifted = x0 + np.repeat(d, 3)
    assert qoi.mae_d(x0, shifted, x0) == pytest.approx(0.5 / np.sqrt(5.0), rel=1e-15)
    assert qoi.hamiltonian(shifted, G) == pytest.approx(qoi.hamiltonian(x0, G), rel=1e-14)
    assert qoi.ae_h(1.1, 1.0) == pytest.approx(0.1, rel=1e-14)
    # three-body H by hand: pairs (1,2) r = 5, (1,3) r = sqrt 5, (2,3) r = sqrt 8
    h = (1.0 * -2.0 * np.log(5.0) + 1.0 * 0.5 * np.log(np.sqrt(5.0)) + -2.0 * 0.5 * np.log(np.sqrt(8.0))) / (2 * np.pi)
    assert qoi.hamiltonian(x0, G) == pytest.approx(h, rel=1e-14)


def test_impulses_closed_forms():
    """Linear impulse P = sum Gamma_i x_i and angular impulse I = sum Gamma_i
    |x_i|^2 on a hand-sized case."""
    x = np.array([1.0, -2.0, 0.5, 3.0])                    # bodies (1, 0.5), (-2, 3)
    G = np.array([2.0, -1.0])
    np.testing.assert_array_equal(qoi.linear_impulse(x, G), [2.0 * 1.0 - 1.0 * -2.0, 2.0 * 0.5 - 1.0 * 3.0])
    assert qoi.angular_impulse(x, G) == 2.0 * (1.0 + 0.25) - 1.0 * (4.0 + 9.0)
