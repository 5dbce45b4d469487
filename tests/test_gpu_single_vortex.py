"""The paper's single-vortex reproductive experiment (Sec. 6.4) on the GPU path.

Table 1's N = 100 case (dt = 0.01, Gamma_center = 500, t in [0, 20]: 2000
steps, delta = 0) with Table 2's narrow-width PTROM of Bases Case 1 (tol
1e-1, M = 13, M_r = 2M, n_s = M_r, neighbour clusters with p_c = 0).  The
paper reports N_c = 68 for this case and sub-0.1 % time-averaged QoI errors.
"""
import numpy as np
import pytest
import torch

from oracle import qoi
from paper_2103_01983_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _hamiltonian(x, G, n):
    return qoi.hamiltonian(x, G)


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


@pytest.mark.parametrize("n,M,pc,paper_nc", [(2000, 26, 0.0, 134), (5000, 26, 1.0, 143)])
def test_single_vortex_larger_cases(n, M, pc, paper_nc):
    """Table 1's N = 2000 and N = 5000 conditions with the bases-case-4 PTROM
    (tol 1e-4, M_r = 2M, n_s = M_r) of Table 2 (narrow width, p_c = 0) and
    Table 3 (moderate width, p_c = 1): N_c near the paper's (134 and 143) and
    time-averaged QoI errors below 0.1 % (the paper's result for every case;
    here the looser bases case 1 reaches 0.2-1.3 % at N >= 2000).  The FOM is
    FP64 JFNK; its trajectory is the PTROM's training snapshots."""
    from paper_2103_01983_gb300 import ptrom as P
    x0, G, dt, steps = W.single_vortex(n)
    fp = P.fom_params(dt, 0.0, "jfnk", tol=1e-12, prec="fp64", gmres_rtol=1e-10, gmres_max_iter=400)
    xd = torch.tensor(x0, device="cuda")
    Gd = torch.tensor(G, device="cuda")
    x = xd.clone()
    f = P.bs_velocity(x, Gd, 0.0, prec="fp64")
    work = P.fom_workspace(fp, n)
    fom = torch.empty(steps, 2 * n, dtype=torch.float64, device="cuda")
    for k in range(steps):
        P.fom_step(fp, Gd, x, f, work=work)
        fom[k] = x
    model, info = P.ptrom_build(xd[None], Gd[None], M, 2 * M, 2 * M, steps, fp, criterion="nb", p_c=pc,
                                tol=1e-4, qr_prec="fp64", snapshots=fom)
    print(f"N={n}: N_c {info['N_c']} (paper {paper_nc})")
    assert abs(info["N_c"] - paper_nc) <= 0.25 * paper_nc, info["N_c"]
    st = model.new_state()
    hist = torch.zeros(steps, M, dtype=torch.float64, device="cuda")
    s = P.ptrom_step([model], [st], steps, hist=[hist])
    assert s["noconv"] == 0
    fom_h = fom.cpu().numpy()
    rec = np.array([model.reconstruct(hist[k]).cpu().numpy() for k in range(steps)])
    l = float(np.hypot(x0[n - 1] - x0[0], x0[2 * n - 1] - x0[n]))
    mae = np.mean(np.hypot(rec[:, :n] - fom_h[:, :n], rec[:, n:] - fom_h[:, n:]), axis=1) / l
    aeh = [abs(_hamiltonian(rec[k], G, n) - _hamiltonian(fom_h[k], G, n)) / abs(_hamiltonian(fom_h[k], G, n))
           for k in range(99, steps, 200)]
    print(f"N={n}: MAE_D {mae.mean():.2e}, AE_H {np.mean(aeh):.2e}")
    assert mae.mean() <= 1e-3 and np.mean(aeh) <= 1e-3, (mae.mean(), np.mean(aeh))
