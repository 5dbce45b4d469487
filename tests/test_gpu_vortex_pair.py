"""The paper's vortex-pair parametric experiment (Sec. 6.2) on the GPU path.

N = 500 bodies on the diagonal, end circulations mu = (Gamma_1, Gamma_N) in
[0.25, 1] x 255, the others 0.01, delta = 0.2121, dt = 0.01, 500 steps.  The
PTROM is trained at 4 Latin-hypercube parameters (FOM snapshots, POD M = 85,
residual POD M_r = 110, 60 sampled bodies, neighbour clusters p_c = 1) and
queried at parameters it was not trained on.  The paper reports time-averaged
errors of 0.0136 % (MAE_D) and 6.09e-4 % (AE_H) averaged over its 6 x 6 query
grid, and states sub-0.1 % errors; here every query is held to the 0.1 %
bound, the cluster count to the paper's order (N_c = 233 there), and every
Gauss-Newton step must converge.
"""
import numpy as np
import pytest
import torch

from oracle import qoi
from _ptrom_cases import oracle_online_on_library_model
from paper_2103_01983_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _hamiltonian(x, G, n):
    return qoi.hamiltonian(x, G)


def test_vortex_pair_parametric_queries():
    from paper_2103_01983_gb300 import ptrom as P
    V = W.VORTEX_PAIR
    n, delta, dt, steps = V["n"], V["delta"], V["dt"], V["steps"]
    train, query = W.vortex_pair_params(0)
    fp = P.fom_params(dt, delta, "jfnk", tol=1e-12, prec="fp64", gmres_rtol=1e-10, gmres_max_iter=400)
    xs, gs = zip(*[W.vortex_pair(a, b) for a, b in train])
    dev = "cuda"
    model, info = P.ptrom_build(torch.tensor(np.stack(xs), device=dev), torch.tensor(np.stack(gs), device=dev),
                                85, 110, 60, steps, fp, criterion="nb", p_c=1.0, tol=1e-4, qr_prec="fp64")
    assert 100 <= info["N_c"] <= 400, info["N_c"]
    l = float(np.hypot(2 * V["half_width"], 2 * V["half_width"]))
    for g1, gN in query[[0, 14, 21, 35]]:  # two grid corners and two interior points
        x0, G = W.vortex_pair(g1, gN)
        x = torch.tensor(x0, device=dev)
        Gd = torch.tensor(G, device=dev)
        f = P.bs_velocity(x, Gd, delta, prec="fp64")
        work = P.fom_workspace(fp, n, dev)
        fom = []
        for _ in range(steps):
            P.fom_step(fp, Gd, x, f, work=work)
            fom.append(x.cpu().numpy())
        fom = np.array(fom)
        model.set_param_full(torch.tensor(x0, device=dev), Gd)
        st = model.new_state(dev)
        hist = torch.zeros(steps, model.M, dtype=torch.float64, device=dev)
        s = P.ptrom_step([model], [st], steps, hist=[hist])
        assert s["noconv"] == 0
        rec = np.array([model.reconstruct(hist[k]).cpu().numpy() for k in range(steps)])
        mae = np.mean(np.hypot(rec[:, :n] - fom[:, :n], rec[:, n:] - fom[:, n:]), axis=1) / l
        if g1 == query[0][0] and gN == query[0][1]:
            # the oracle's online stage on this very model: the CUDA PTROM's
            # reduced trajectory, reconstructed, against the oracle's
            q = model.query()
            red = oracle_online_on_library_model(model, q["phi"], x0, delta, dt, steps)
            rec_o = x0 + red[1:] @ q["phi"].T
            d = np.mean(np.hypot(rec[:, :n] - rec_o[:, :n], rec[:, n:] - rec_o[:, n:]), axis=1) / l
            print("CUDA vs oracle PTROM, time-averaged MAE_D:", d.mean())
            assert d.mean() <= 1e-4, d.mean()
        ks = range(0, steps, 25)
        aeh = [abs(_hamiltonian(rec[k], G, n) - _hamiltonian(fom[k], G, n)) / abs(_hamiltonian(fom[k], G, n))
               for k in ks]
        assert mae.mean() <= 1e-3 and np.mean(aeh) <= 1e-3, (g1, gN, mae.mean(), np.mean(aeh))
