"""The paper's single-vortex reproductive experiment (Sec. 6.4) on the GPU path.

Table 1's N = 100 case (dt = 0.01, Gamma_center = 500, t in [0, 20]: 2000
steps, delta = 0) with Table 2's narrow-width PTROM of Bases Case 1 (tol
1e-1, M = 13, M_r = 2M, n_s = M_r, neighbour clusters with p_c = 0).  The
paper reports N_c = 68 for this case and sub-0.1 % time-averaged QoI errors.
"""
import numpy as np
import pytest
import torch

from paper_2103_01983_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _hamiltonian(x, G, n):
    X, Y = x[:n], x[n:]
    d2 = (X[:, None] - X[None, :]) ** 2 + (Y[:, None] - Y[None, :]) ** 2
    iu = np.triu_indices(n, 1)
    return -np.sum(G[iu[0]] * G[iu[1]] * np.log(d2[iu])) / (4 * np.pi)


def test_single_vortex_n100_bases_case1():
    from paper_2103_01983_gb300 import ptrom as P
    n, M = 100, 13
    x0, G, dt, steps = W.single_vortex(n)
    fp = P.fom_params(dt, 0.0, "dense", tol=1e-12, prec="fp64")
    xd = torch.tensor(x0, device="cuda")
    Gd = torch.tensor(G, device="cuda")
    model, info = P.ptrom_build(xd[None], Gd[None], M, 2 * M, 2 * M, steps, fp, criterion="nb", p_c=0.0,
                                tol=1e-1, qr_prec="fp64")
    assert abs(info["N_c"] - 68) <= 7, info["N_c"]
    x = xd.clone()
    f = P.bs_velocity(x, Gd, 0.0, prec="fp64")
    work = P.fom_workspace(fp, n)
    fom = []
    for _ in range(steps):
        P.fom_step(fp, Gd, x, f, work=work)
        fom.append(x.cpu().numpy())
    fom = np.array(fom)
    st = model.new_state()
    hist = torch.zeros(steps, M, dtype=torch.float64, device="cuda")
    s = P.ptrom_step([model], [st], steps, hist=[hist])
    assert s["noconv"] == 0
    rec = np.array([model.reconstruct(hist[k]).cpu().numpy() for k in range(steps)])
    l = float(np.hypot(x0[n - 1] - x0[0], x0[2 * n - 1] - x0[n]))
    mae = np.mean(np.hypot(rec[:, :n] - fom[:, :n], rec[:, n:] - fom[:, n:]), axis=1) / l
    aeh = [abs(_hamiltonian(rec[k], G, n) - _hamiltonian(fom[k], G, n)) / abs(_hamiltonian(fom[k], G, n))
           for k in range(0, steps, 100)]
    assert mae.mean() <= 1e-3 and np.mean(aeh) <= 1e-3, (mae.mean(), np.mean(aeh))
