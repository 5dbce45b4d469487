"""Batched FOM over instances of uneven N (one launch per Newton iteration)."""
import numpy as np
import pytest
import torch

from oracle import direct, fom
from paper_2103_01983_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2103_01983_gb300 import ptrom
    return ptrom


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _instances(sizes, seed=80):
    out = []
    rng = np.random.default_rng(seed)
    for k, n in enumerate(sizes):
        sep, ratio = rng.uniform(0.8, 1.2), rng.uniform(0.5, 2.0)
        out.append(W.two_cluster(n, seed=k, sep=sep, ratio=ratio))
    return out


@pytest.mark.parametrize("prec,tol", [("fp32c", 1e-5), ("fp64", 1e-12)])
def test_batched_velocity_matches_oracle(P, prec, tol):
    inst = _instances([64, 1000, 3000, 130, 2048, 514])
    xs = [_dev(x) for x, _ in inst]
    Gs = [_dev(G) for _, G in inst]
    fs, Ds = P.bs_velocity_batched(xs, Gs, [0.02] * len(inst), selfjac=True, prec=prec)
    for (x, G), f, D in zip(inst, fs, Ds):
        fo, Do = direct.velocity(x, G, 0.02, with_selfjac=True)
        assert np.linalg.norm(f.cpu().numpy() - fo) / np.linalg.norm(fo) <= tol
        assert np.linalg.norm(D.cpu().numpy().reshape(3, -1) - Do) / np.linalg.norm(Do) <= tol


def test_batched_fom_step_matches_single_and_oracle(P):
    inst = _instances([128, 600, 1500, 3000])
    p = P.fom_params(0.005, 0.02, "blockdiag", prec="fp64", tol=1e-13)
    xs = [_dev(x) for x, _ in inst]
    Gs = [_dev(G) for _, G in inst]
    fs = [P.bs_velocity(x, G, 0.02, prec="fp64") for x, G in zip(xs, Gs)]
    works = [P.fom_workspace(p, G.numel()) for G in Gs]
    for _ in range(3):
        stats = P.fom_step_batched(p, Gs, xs, fs, works)
    assert all(s["newton_iters"] > 0 for s in stats)
    for (x0, G), xb, fb in zip(inst, xs, fs):
        ref, _ = fom.rollout(x0, G, 0.02, 0.005, 3, mode="blockdiag", tol=1e-13)
        np.testing.assert_allclose(xb.cpu().numpy(), ref[-1], atol=1e-11)
        np.testing.assert_allclose(fb.cpu().numpy(), direct.velocity(ref[-1], G, 0.02), atol=1e-9)
