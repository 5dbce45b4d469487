"""The benchmark's PTROM model, built by the library (reproductive, the
two-cluster workload at N = 16384, delta = 0.02, dt = 0.005, 200 JFNK FOM
steps; POD rank 20, residual rank 40, 40 sampled bodies, Barnes-Hut theta =
0.25 and 0.5, FP64 least squares), with its online stage (Alg. 4 over Alg. 5)
run by the CUDA kernel and by the oracle on the same model pieces (basis,
sampled bodies, clusters with their surrogates, A).

Tolerance: the reduced trajectories over 100 steps agree to 1e-3 relative per
step (FP32 pair sums and gathers against FP64; both stop Gauss-Newton at
eps <= 1e-4), and the reconstructed states to MAE_D 1e-5 of the domain length."""
import numpy as np
import pytest
import torch

from _ptrom_cases import oracle_online_on_library_model
from oracle import qoi, rom
from paper_2103_01983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N, DELTA, DT, TRAIN, STEPS = 16384, 0.02, 0.005, 200, 100


@pytest.mark.parametrize("theta", [0.25, 0.5])
def test_bench_ptrom_model_online_matches_oracle(theta):
    from paper_2103_01983_gb300 import ptrom as P
    x0, G = W.two_cluster(N, seed=0)
    x0d = torch.tensor(x0, device="cuda")
    Gd = torch.tensor(G, device="cuda")
    fp = P.fom_params(DT, DELTA, "jfnk", tol=1e-8, prec="fp32c")
    model, info = P.ptrom_build(x0d[None], Gd[None], 20, 40, 40, TRAIN, fp, criterion="bh", theta=theta, tol=1e-4,
                                qr_prec="fp64")
    M = model.M
    hist = torch.zeros(STEPS, M, dtype=torch.float64, device="cuda")
    P.ptrom_step([model], [model.new_state()], STEPS, hist=[hist])
    gpu = hist.cpu().numpy()
    Phi = model.query()["phi"]
    ref = oracle_online_on_library_model(model, Phi, x0, DELTA, DT, STEPS)[1:]
    rel = np.linalg.norm(gpu - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() <= 1e-3, (rel.max(), info["N_c"])
    mae = max(qoi.mae_d(rom.reconstruct(a, Phi, x0), rom.reconstruct(b, Phi, x0), x0) for a, b in zip(gpu, ref))
    assert mae <= 1e-5, mae
