"""Parity of the CUDA online PTROM step (Alg. 4 over Alg. 5) with the oracle.

Models are built once by the FP64 oracle and loaded into the library, so both
sides run the same model:
  * "disk_gnat":  the small FP64 case (disk, N=256, delta=0.05, dt=0.01,
    100 steps), POD rank 8, 32 sampled bodies, M_r=16, no clustering (GNAT);
  * "disk_bh":    the same with Barnes-Hut clustering, theta = 0.5;
  * "pair_gnat":  two same-sign Gaussian clusters, N=512, delta=0.02,
    dt=0.005, 100 steps, M=20, 40 sampled bodies, M_r=40, no clustering.
Tolerances: one Gauss-Newton update to 1e-5 relative (FP32 pair sums and
products against FP64); whole trajectories at the level of the paper's QoI:
MAE_D and AE_H differences below 1e-4 (0.01 %, ten times inside the paper's
0.1 % QoI bound).  Both sides stop Gauss-Newton at eps <= 1e-4, so each step
may end on iterates that differ by up to ~1e-4 of the last update."""
import numpy as np
import pytest
import torch

from oracle import qoi, rom
from _ptrom_cases import build_case, model_arrays
from paper_2103_01983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

_CASES = {}


def _case(name):
    if name not in _CASES:
        if name == "mushroom_bh":
            # the mushroom-cloud workload (Sec. 6.3) at 200 bodies: opposite
            # end vortices and the semicircular superimposed inflow
            x0, G, u = W.mushroom(-200.0, 150.0, n=200)
            _CASES[name] = build_case(x0, G, 0.15, 0.005, 100, M=16, n_s=40, M_r=32, criterion="nb",
                                      p_c=1.0, u_inf=u)
        elif name.startswith("disk"):
            x0, G = W.disk(256, seed=0)
            th = 0.0 if name == "disk_gnat" else 0.5
            _CASES[name] = build_case(x0, G, 0.05, 0.01, 100, M=8, n_s=32, M_r=16, theta=th)
        else:
            x0, G = W.two_cluster(512, seed=0)
            _CASES[name] = build_case(x0, G, 0.02, 0.005, 100, M=20, n_s=40, M_r=40, theta=0.0,
                                      fom_mode="jfnk")
    return _CASES[name]


def _model(P, case, **kw):
    arr = model_arrays(case)
    return P.PtromModel(arr["phi_s"], arr["x0_s"], arr["phi_c"], arr["x0_c"], arr["gamma_c"], arr["A"],
                        arr["off"], arr["idx"], case["dt"], case["delta"], u_s=arr["u_s"], **kw)


@pytest.fixture(scope="module")
def P():
    from paper_2103_01983_gb300 import ptrom
    return ptrom


@pytest.fixture(scope="module", params=["disk_gnat", "disk_bh", "pair_gnat", "mushroom_bh"])
def case(request):
    return _case(request.param)


@pytest.mark.parametrize("qr", ["fp64", "fp32c"])
def test_one_gauss_newton_update(P, case, qr):
    M = case["Phi"].shape[1]
    ref, _ = rom.ptrom_online(case["cl"], case["Phi"], case["x0"], case["A"], case["delta"], case["dt"],
                              1, tol=1e-4, max_gn=1, u_inf=case.get("u"))
    m = _model(P, case, tol=1e-4, max_gn=1, qr_prec=qr)
    st = m.new_state()
    xh = torch.zeros(M, dtype=torch.float64, device="cuda")
    s = P.ptrom_step([m], [st], 1, xhat=[xh])
    assert s["gn_iters"] == 1 and s["steps"] == 1
    err = np.linalg.norm(xh.cpu().numpy() - ref[1]) / np.linalg.norm(ref[1])
    assert err <= 1e-5, err


def _qoi_gap(case, xa, xb):
    """MAE_D (Eq. MAE_trajectory) between two reduced trajectories, and the
    Hamiltonian gap relative to the reference's largest |H| (the mixed-sign
    disk's H crosses zero, where AE_H of Eq. AE_Hamiltonian is undefined)."""
    Phi, x0, G = case["Phi"], case["x0"], case["G"]
    mae, dh, hs = [], [], []
    for za, zb in zip(xa, xb):
        pa, pb = rom.reconstruct(za, Phi, x0), rom.reconstruct(zb, Phi, x0)
        mae.append(qoi.mae_d(pa, pb, x0))
        ha, hb = qoi.hamiltonian(pa, G), qoi.hamiltonian(pb, G)
        dh.append(abs(ha - hb))
        hs.append(abs(hb))
    return max(mae), max(dh) / max(hs)


@pytest.mark.parametrize("qr", ["fp64", "fp32c"])
def test_trajectory_matches_oracle_qoi(P, case, qr):
    M = case["Phi"].shape[1]
    ref, it_ref = rom.ptrom_online(case["cl"], case["Phi"], case["x0"], case["A"], case["delta"],
                                   case["dt"], 100, tol=1e-4, u_inf=case.get("u"))
    m = _model(P, case, tol=1e-4, qr_prec=qr)
    st = m.new_state()
    hist = torch.zeros(100, M, dtype=torch.float64, device="cuda")
    s = P.ptrom_step([m], [st], 100, hist=[hist])
    gpu = np.vstack([np.zeros(M), hist.cpu().numpy()])
    mae, aeh = _qoi_gap(case, gpu, ref)
    assert mae <= 1e-4 and aeh <= 1e-4, (mae, aeh)
    assert s["noconv"] == 0
    assert abs(s["gn_iters"] - it_ref.sum()) <= 0.1 * it_ref.sum()


def test_gnat_tracks_the_fom():
    """Without clustering the reduced model follows the FP64 FOM trajectory it
    was trained on (same-sign two-cluster case, basis spans the trajectory)."""
    from paper_2103_01983_gb300 import ptrom as P
    case = _case("pair_gnat")
    M = case["Phi"].shape[1]
    m = _model(P, case, tol=1e-4)
    st = m.new_state()
    hist = torch.zeros(100, M, dtype=torch.float64, device="cuda")
    P.ptrom_step([m], [st], 100, hist=[hist])
    x0, G, tr = case["x0"], case["G"], case["traj"]
    rec = np.array([rom.reconstruct(z, case["Phi"], x0) for z in hist.cpu().numpy()])
    disp = np.abs(tr - x0).max()
    assert np.abs(rec - tr[1:]).max() <= 1e-5 * disp
    aeh = max(abs(qoi.hamiltonian(a, G) - qoi.hamiltonian(b, G)) / abs(qoi.hamiltonian(b, G))
              for a, b in zip(rec, tr[1:]))
    assert aeh <= 1e-3   # the paper's 0.1 % QoI bound


def test_batched_instances_and_split_calls(P):
    case = _case("disk_bh")
    """8 instances in one launch equal one instance; 100 steps in one call
    equal 4 calls of 25 steps (state carried in the state buffer)."""
    M = case["Phi"].shape[1]
    m = _model(P, case)
    sts = [m.new_state() for _ in range(8)]
    outs = [torch.zeros(M, dtype=torch.float64, device="cuda") for _ in range(8)]
    P.ptrom_step([m] * 8, sts, 100, xhat=outs)
    st1 = m.new_state()
    one = torch.zeros(M, dtype=torch.float64, device="cuda")
    for _ in range(4):
        P.ptrom_step([m], [st1], 25, xhat=[one])
    ref = outs[0].cpu().numpy()
    for o in outs[1:]:
        np.testing.assert_array_equal(o.cpu().numpy(), ref)
    np.testing.assert_allclose(one.cpu().numpy(), ref, rtol=0, atol=0)


def test_exactness_without_clustering(P):
    """Basis spans the trajectory, every body sampled, no clustering: the GPU
    PTROM reproduces the FOM (to FP32 pair-sum accuracy)."""
    from oracle import fom
    n, steps, dt, delta = 20, 50, 0.01, 0.05
    x0, G = W.disk(n, seed=7)
    traj, _ = fom.rollout(x0, G, delta, dt, steps, mode="dense", tol=1e-14)
    S = traj[1:].T
    M = 2 * n                                   # the basis spans the state space
    Phi, sig = rom.pod(S, M)
    cl, _ = rom.cluster_tables(Phi, sig, x0, G, np.arange(n), criterion="bh", theta=0.0)
    _, snaps = rom.lspg_tier2(cl, Phi, x0, delta, dt, steps, tol=1e-10)
    U, s, _ = np.linalg.svd(snaps, full_matrices=False)
    Mr = min(int(np.sum(s > 1e-8 * s[0])), 2 * n)
    A = rom.gappy_operator(U[:, :Mr], np.arange(n), n)
    case = dict(cl=cl, Phi=Phi, x0=x0, A=A, dt=dt, delta=delta)
    m = _model(P, case, tol=1e-6)
    st = m.new_state()
    hist = torch.zeros(steps, M, dtype=torch.float64, device="cuda")
    P.ptrom_step([m], [st], steps, hist=[hist])
    rec = np.array([rom.reconstruct(z, Phi, x0) for z in hist.cpu().numpy()])
    err = np.abs(rec - traj[1:]).max() / np.abs(traj[1:] - x0).max()
    assert err <= 1e-4, err


def test_one_launch_of_different_models(P):
    """Instances of different models (sizes M = 8 / 16, n_s = 32 / 40,
    different cluster counts, one with a superimposed inflow) share one
    launch: every instance ends exactly where it ends when launched alone."""
    ca, cb = _case("disk_bh"), _case("mushroom_bh")
    ma, mb = _model(P, ca), _model(P, cb)
    models = [ma, mb, ma, mb]
    sts = [m.new_state() for m in models]
    outs = [torch.zeros(m.M, dtype=torch.float64, device="cuda") for m in (ma, mb, ma, mb)]
    s = P.ptrom_step(models, sts, 30, xhat=outs)
    assert s["steps"] == 4 * 30
    for m, o in ((ma, outs[0]), (mb, outs[1])):
        st = m.new_state()
        alone = torch.zeros(m.M, dtype=torch.float64, device="cuda")
        P.ptrom_step([m], [st], 30, xhat=[alone])
        np.testing.assert_array_equal(o.cpu().numpy(), alone.cpu().numpy())
    np.testing.assert_array_equal(outs[0].cpu().numpy(), outs[2].cpu().numpy())
    np.testing.assert_array_equal(outs[1].cpu().numpy(), outs[3].cpu().numpy())
