"""Differentiation on the GPU: the velocity's hand-written adjoint behind
torch autograd, and the checkpointed adjoint of implicit rollouts.

Pins: the oracle's adjoint (dense, FP64), central finite differences of GPU
rollouts (FP64 kernels, h = 1e-4), and the closed-form gradient of the
conserved linear impulse (which checks that every adjoint term cancels)."""
import numpy as np
import pytest
import torch

from oracle import direct, fom
from paper_2103_01983_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2103_01983_gb300 import autograd, ptrom
    return ptrom, autograd


def _dev(a, grad=False):
    t = torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    return t.requires_grad_(grad)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32c", 1e-5)])
def test_velocity_autograd_matches_oracle_vjp(mods, prec, tol):
    ptrom, ag = mods
    x, G = W.two_cluster(600, seed=70)
    w = W.random_vectors(x.size, 1, seed=71)[0]
    xt, Gt = _dev(x, True), _dev(G, True)
    f = ag.velocity(xt, Gt, 0.02, prec=prec)
    (f * _dev(w)).sum().backward()
    gx, gG = direct.vjp(x, G, 0.02, w)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(xt.grad.cpu().numpy(), gx) <= tol
    assert rel(Gt.grad.cpu().numpy(), gG) <= tol


def test_velocity_gradcheck_fp64(mods):
    ptrom, ag = mods
    x, G = W.disk(7, seed=72)
    xt, Gt = _dev(x, True), _dev(G, True)
    assert torch.autograd.gradcheck(lambda a, b: ag.velocity(a, b, 0.05, prec="fp64"), (xt, Gt),
                                    eps=1e-6, atol=1e-7, rtol=1e-5)


def _params(ptrom, prec):
    if prec == "fp64":
        return ptrom.fom_params(0.005, 0.02, "jfnk", tol=1e-13, prec="fp64", gmres_rtol=1e-12,
                                gmres_max_iter=400)
    return ptrom.fom_params(0.005, 0.02, "jfnk", prec="fp32c", gmres_rtol=1e-8, gmres_max_iter=400)


def test_rollout_gradient_matches_oracle_adjoint(mods):
    """N=1024 two clusters, 30 steps, checkpoint every 10: GPU adjoint
    (FP64 kernels) against the oracle's dense adjoint."""
    ptrom, ag = mods
    x0, G = W.two_cluster(1024, seed=73)
    lam_T = W.random_vectors(x0.size, 1, seed=74)[0]
    gx_ref, gG_ref, traj = fom.adjoint_rollout(x0, G, 0.02, 0.005, 30, lam_T)
    xt, Gt = _dev(x0, True), _dev(G, True)
    xT = ag.rollout(xt, Gt, _params(ptrom, "fp64"), 30, every=10)
    np.testing.assert_allclose(xT.detach().cpu().numpy(), traj[-1], atol=1e-10)
    (xT * _dev(lam_T)).sum().backward()
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(xt.grad.cpu().numpy(), gx_ref) <= 1e-8
    assert rel(Gt.grad.cpu().numpy(), gG_ref) <= 1e-8


def test_rollout_gradient_matches_central_differences(mods):
    """Central differences (h = 1e-4, FP64 kernels) of a random linear
    functional of x(T), N = 512 two clusters, 20 steps with a checkpoint every
    10, along 64 random directions in (x0, Gamma)."""
    ptrom, ag = mods
    x0, G = W.two_cluster(512, seed=75)
    lam_T = _dev(W.random_vectors(x0.size, 1, seed=76)[0])
    p = _params(ptrom, "fp64")
    xt, Gt = _dev(x0, True), _dev(G, True)
    (ag.rollout(xt, Gt, p, 20, every=10) * lam_T).sum().backward()
    h = 1e-4
    dirs = W.random_vectors(x0.size + G.size, 64, seed=77)

    def L(dx, dg, hh):
        with torch.no_grad():
            return (ag.rollout(_dev(x0) + hh * dx, _dev(G) + hh * dg, p, 20) * lam_T).sum().item()

    worst = 0.0
    for d in dirs:
        dx, dg = _dev(d[:x0.size]), _dev(d[x0.size:])
        fd = (L(dx, dg, h) - L(dx, dg, -h)) / (2 * h)
        fd2 = (L(dx, dg, h / 2) - L(dx, dg, -h / 2)) / h
        an = float((xt.grad * dx).sum() + (Gt.grad * dg).sum())
        # the central difference's O(h^2) truncation error, estimated from the
        # same difference at h/2 (it shrinks 4-fold); Richardson's combination
        # (4 fd(h/2) - fd(h)) / 3 removes it and must match the adjoint closely
        trunc = abs(fd - fd2) * 4.0 / 3.0
        assert abs(fd - an) <= trunc * 1.5 + 1e-8 * max(1.0, abs(fd)), (fd, fd2, an)
        rich = (4.0 * fd2 - fd) / 3.0
        assert abs(rich - an) <= 1e-7 * max(1.0, abs(an)), (rich, an)
        worst = max(worst, abs(fd - an) / max(1.0, abs(fd)))
    print(f"64 directions: largest |central difference - adjoint| {worst:.1e} (relative)")


@pytest.mark.parametrize("n,steps,every,prec,tol", [(1024, 40, 10, "fp64", 1e-9),
                                                    (16384, 20, 10, "fp32c", 1e-5),
                                                    (65536, 100, 10, "fp32c", 1e-5)])
def test_linear_impulse_gradient_closed_form(mods, n, steps, every, prec, tol):
    """L = sum Gamma_i (chi_i(T) + psi_i(T)) is conserved: dL/dx0 = Gamma on
    both components and the total dL/dGamma = chi0 + psi0.  The largest case
    is the full-size differentiation workload: N = 65536, the gradient of the
    final linear impulse after 100 steps with a checkpoint every 10."""
    ptrom, ag = mods
    x0, G = W.two_cluster(n, seed=78)
    xt, Gt = _dev(x0, True), _dev(G, True)
    xT = ag.rollout(xt, Gt, _params(ptrom, prec), steps, every=every)
    L = (Gt * (xT[:n] + xT[n:])).sum()
    L.backward()
    gx, gG = xt.grad.cpu().numpy(), Gt.grad.cpu().numpy()
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(gx, np.concatenate([G, G])) <= tol
    assert rel(gG, x0[:n] + x0[n:]) <= tol
