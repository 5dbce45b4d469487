"""The online PTROM kernel at its size limits, against the oracle's online stage.

A GNAT-style model (every source body its own cluster, Sec. 4.1) on the
two-cluster workload, N = 2048, delta = 0.02, dt = 0.005: the largest basis
(M = 128: the two components of the monomials chi^a psi^b of degree <= 10,
orthonormalised), the largest residual basis (M_r = 256: that basis plus
seeded random fields, orthonormalised), the most sampled bodies (n_s = 512,
half from each cluster, each against the 2047 others).

* FP32 least squares: this size fits one CTA's shared memory, and one
  Gauss-Newton update and a 10-step trajectory match the oracle (1e-4 and
  1e-3 relative: FP32 pair sums against FP64).
* FP64 least squares: [A C | A r] alone would take 264 KB, so the model is
  refused with PTROM_EINVAL; with M_r = 160 it fits and matches the oracle."""
import numpy as np
import pytest
import torch

from _ptrom_cases import model_arrays
from oracle import rom
from paper_2103_01983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N, DELTA, DT = 2048, 0.02, 0.005


def _orth(Q):
    return np.linalg.qr(Q)[0]


def _case(Mr):
    x0, G = W.two_cluster(N, seed=0)
    chi, psi = x0[:N], x0[N:]
    c, s = (chi - chi.mean()) / chi.std(), (psi - psi.mean()) / psi.std()
    mono = [c ** a * s ** b for d in range(11) for a in range(d + 1) for b in [d - a]]
    fields = [np.r_[m, 0 * m] for m in mono] + [np.r_[0 * m, m] for m in mono]
    Phi = _orth(np.array(fields).T)[:, :128]
    extra = W.random_vectors(2 * N, 256, seed=90).T
    Phi_r = _orth(np.concatenate([Phi, extra], axis=1))[:, :Mr]
    rng = np.random.default_rng(91)
    half = N // 2
    sampled = np.sort(np.concatenate([rng.choice(half, 256, replace=False), half + rng.choice(half, 256, replace=False)]))
    A = rom.gappy_operator(Phi_r, sampled, N)
    lists = [[j for j in range(N) if j != t] for t in sampled]
    cl = rom.Clusters([[j] for j in range(N)], G.copy(), Phi.copy(), x0.copy(), lists, sampled)
    return dict(cl=cl, Phi=Phi, x0=x0, G=G, A=A)


def _model(P, case, qr, **kw):
    arr = model_arrays(case)
    return P.PtromModel(arr["phi_s"], arr["x0_s"], arr["phi_c"], arr["x0_c"], arr["gamma_c"], arr["A"],
                        arr["off"], arr["idx"], DT, DELTA, qr_prec=qr, **kw)


@pytest.mark.parametrize("Mr,qr", [(256, "fp32c"), (160, "fp64")])
def test_limits_match_oracle(Mr, qr):
    from paper_2103_01983_gb300 import ptrom as P
    case = _case(Mr)
    cl, Phi, x0, A = case["cl"], case["Phi"], case["x0"], case["A"]
    M = Phi.shape[1]
    ref1, _ = rom.ptrom_online(cl, Phi, x0, A, DELTA, DT, 1, tol=1e-4, max_gn=1)
    m1 = _model(P, case, qr, tol=1e-4, max_gn=1)
    assert (m1.M, m1.M_r, m1.n_s) == (128, Mr, 512)
    xh = torch.zeros(M, dtype=torch.float64, device="cuda")
    P.ptrom_step([m1], [m1.new_state()], 1, xhat=[xh])
    err = np.linalg.norm(xh.cpu().numpy() - ref1[1]) / np.linalg.norm(ref1[1])
    assert err <= 1e-4, err
    steps = 10
    ref, _ = rom.ptrom_online(cl, Phi, x0, A, DELTA, DT, steps, tol=1e-4)
    m = _model(P, case, qr, tol=1e-4)
    hist = torch.zeros(steps, M, dtype=torch.float64, device="cuda")
    s = P.ptrom_step([m], [m.new_state()], steps, hist=[hist])
    assert s["noconv"] == 0
    rel = np.linalg.norm(hist.cpu().numpy() - ref[1:], axis=1) / np.linalg.norm(ref[1:], axis=1)
    assert rel.max() <= 1e-3, rel.max()


def test_fp64_least_squares_too_large_is_refused():
    from paper_2103_01983_gb300 import ptrom as P
    case = _case(256)
    with pytest.raises(P.PtromError) as err:
        _model(P, case, "fp64")
    assert err.value.status == -1 and "shared memory" in str(err.value)
