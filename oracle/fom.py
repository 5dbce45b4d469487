"""Full-order model: implicit trapezoid rule solved by Newton (Sec. 2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Time-discrete residual (Eq. linKstep with the trapezoid coefficients
k=1, alpha0=1, alpha1=-1, beta0=beta1=1/2):

    r(xi) = xi - x^{n-1} - dt/2 (f(xi) + f(x^{n-1})).

Newton on r(xi) = 0 from xi = x^{n-1}, at most ``max_iter`` (100, Sec. 6)
iterations, each solving (I - dt/2 J) delta = -r with J one of
  * "dense":     the full d f / d x (``kernel.jacobian``),
  * "blockdiag": only the per-body 2x2 self blocks D_i -- the paper's inexact
                 kernel Jacobian (Sec. 2, last paragraph),
  * "jfnk":      the full J applied matrix-free (``direct.jvp``) inside GMRES,
                 right-preconditioned by the block-diagonal matrix.
The Jacobian is refreshed every ``p_it`` Newton iterations (1 = every one).
Convergence: ||r||_2 <= tol * max(1, ||xi||_2), tested right after f(xi) is
evaluated, so the returned f is f at the returned state.

Superimposed inflow (Sec. 6.3, and the inflow sweeps Sec. 5.2 mentions): a
constant velocity u_i per body is added to the right-hand side,
dx_i/dt = f_i(x) + u_i.  The trapezoid rule then averages u with itself, so
the residual gains -dt u; u does not depend on x, so no Jacobian changes.
``f`` stays the pair sum of Eq. 2 alone.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import direct, kernel


def residual(xi, x_prev, f_xi, f_prev, dt, u_inf=None):
    r = xi - x_prev - 0.5 * dt * (f_xi + f_prev)
    if u_inf is not None:
        r = r - dt * np.asarray(u_inf, dtype=np.float64)
    return r


def _blockdiag_solve(D, rhs, dt):
    """Solve (I - dt/2 D_i) y_i = rhs_i for every body (2x2 each)."""
    n = D.shape[1]
    d00, d01, d10 = D
    d11 = -d00
    m00 = 1.0 - 0.5 * dt * d00
    m01 = -0.5 * dt * d01
    m10 = -0.5 * dt * d10
    m11 = 1.0 - 0.5 * dt * d11
    det = m00 * m11 - m01 * m10
    r0, r1 = rhs[:n], rhs[n:]
    return np.concatenate([(m11 * r0 - m01 * r1) / det, (m00 * r1 - m10 * r0) / det])


def step(x_prev, f_prev, Gamma, delta, dt, mode="dense", tol=1e-12, max_iter=100,
         p_it=1, gmres_tol=1e-10, gmres_restart=30, u_inf=None):
    """One implicit trapezoid step.  Returns (x^n, f(x^n), iterations, ||r||)."""
    x_prev = np.asarray(x_prev, dtype=np.float64)
    n = x_prev.size // 2
    xi = x_prev.copy()
    lin = None
    for k in range(max_iter + 1):
        need_D = mode in ("blockdiag", "jfnk") and (k % p_it == 0 or lin is None)
        if need_D:
            f, D = direct.velocity(xi, Gamma, delta, with_selfjac=True)
        else:
            f = direct.velocity(xi, Gamma, delta)
        r = residual(xi, x_prev, f, f_prev, dt, u_inf)
        rn = float(np.linalg.norm(r))
        if rn <= tol * max(1.0, float(np.linalg.norm(xi))) or k == max_iter:
            return xi, f, k, rn
        if mode == "dense":
            if k % p_it == 0 or lin is None:
                lin = np.eye(2 * n) - 0.5 * dt * kernel.jacobian(xi, Gamma, delta)
            d = np.linalg.solve(lin, -r)
        elif mode == "blockdiag":
            if need_D:
                lin = D
            d = _blockdiag_solve(lin, -r, dt)
        elif mode == "jfnk":
            if need_D:
                lin = D
            xk = xi.copy()
            A = spla.LinearOperator(
                (2 * n, 2 * n), dtype=np.float64,
                matvec=lambda v: v - 0.5 * dt * direct.jvp(xk, Gamma, delta, v))
            Dk = lin
            Mp = spla.LinearOperator(
                (2 * n, 2 * n), dtype=np.float64,
                matvec=lambda v: _blockdiag_solve(Dk, v, dt))
            d, info = spla.gmres(A, -r, M=Mp, rtol=gmres_tol, atol=0.0,
                                 restart=gmres_restart, maxiter=50)
        else:
            raise ValueError(mode)
        xi = xi + d
    raise AssertionError("unreachable")


def rollout(x0, Gamma, delta, dt, steps, mode="dense", tol=1e-12, **kw):
    """Trajectory x^0..x^steps (rows) plus per-step iteration counts."""
    x = np.asarray(x0, dtype=np.float64).copy()
    f = direct.velocity(x, Gamma, delta)
    traj = [x.copy()]
    iters = []
    for _ in range(steps):
        x, f, k, _ = step(x, f, Gamma, delta, dt, mode=mode, tol=tol, **kw)
        traj.append(x.copy())
        iters.append(k)
    return np.array(traj), np.array(iters)


def adjoint_rollout(x0, Gamma, delta, dt, steps, lam_T, tol=1e-13):
    """Gradient of L = lam_T . x^steps with respect to x^0 and Gamma by the
    adjoint of each trapezoid step (implicit function theorem on Eq.
    linKstep), with dense Jacobians:
        mu = (I - dt/2 J(x^n))^{-T} lam,  lam <- mu + dt/2 J(x^{n-1})^T mu,
        gGamma += dt/2 (F(x^n) + F(x^{n-1}))^T mu,  F = d f / d Gamma."""
    traj, _ = rollout(x0, Gamma, delta, dt, steps, mode="dense", tol=tol)
    n2 = traj.shape[1]
    h = 0.5 * dt
    lam = np.array(lam_T, dtype=np.float64)
    gG = np.zeros(len(Gamma))
    for k in range(steps, 0, -1):
        xn, xp = traj[k], traj[k - 1]
        mu = np.linalg.solve((np.eye(n2) - h * kernel.jacobian(xn, Gamma, delta)).T, lam)
        gG += h * (kernel.dfdGamma(xn, Gamma, delta).T @ mu + kernel.dfdGamma(xp, Gamma, delta).T @ mu)
        lam = mu + h * kernel.jacobian(xp, Gamma, delta).T @ mu
    return lam, gG, traj
