"""Oracle-built PTROM models for the tests and the benchmark's CPU leg.

Runs the paper's offline stages with the FP64 oracle (Stage 1 FOM snapshots,
Stage 2 POD + ClusterPOD, Stage 3 Tier-II LSPG residual snapshots, Stage 4
greedy sampling) and returns the arrays the library's model takes."""
import numpy as np

from oracle import fom, rom


def build_case(x0, G, delta, dt, steps, M, n_s, M_r, criterion="bh", theta=0.5, p_c=1.0,
               tol=1e-4, fom_mode="dense", u_inf=None):
    N = G.size
    traj, _ = fom.rollout(x0, G, delta, dt, steps, mode=fom_mode, tol=1e-12, u_inf=u_inf)
    S = traj[1:].T                                              # R1: the states x^1..x^Nt
    Phi, sig = rom.pod(S, M)
    cl_all, _ = rom.cluster_tables(Phi, sig, x0, G, np.arange(N), criterion=criterion,
                                   theta=theta, p_c=p_c)
    _, snaps = rom.lspg_tier2(cl_all, Phi, x0, delta, dt, steps, tol=tol, u_inf=u_inf)
    Phi_r, _ = rom.pod(snaps, M_r)
    sampled = rom.greedy_sample(Phi_r, n_s, N)
    A = rom.gappy_operator(Phi_r, sampled, N)
    cl, _ = rom.cluster_tables(Phi, sig, x0, G, sampled, criterion=criterion, theta=theta, p_c=p_c)
    return dict(traj=traj, Phi=Phi, sig=sig, cl=cl, A=A, sampled=sampled, x0=x0, G=G,
                delta=delta, dt=dt, u=u_inf)


def model_arrays(case):
    """Arrays in the layouts of include/ptrom.h for the library's model."""
    cl, Phi, x0 = case["cl"], case["Phi"], case["x0"]
    Phi_t, x0_t = rom.target_rows(Phi, x0, cl.targets)
    off = np.zeros(len(cl.lists) + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(li) for li in cl.lists])
    idx = np.concatenate([np.asarray(li, dtype=np.int32) for li in cl.lists]) if off[-1] else np.zeros(0, np.int32)
    u = case.get("u")
    u_s = None if u is None else rom.target_rows(np.asarray(u)[:, None], x0, cl.targets)[0][:, 0]
    return dict(phi_s=Phi_t, x0_s=x0_t, phi_c=cl.Phit, x0_c=cl.x0t, gamma_c=cl.Gt, A=case["A"],
                off=off, idx=idx, u_s=u_s)


def oracle_online_on_library_model(model, Phi, x0, delta, dt, steps, tol=1e-4, max_gn=100, u_inf=None):
    """The oracle's online Gauss-Newton (Alg. 4 over Alg. 5 HyperPair) run on
    the library model's own offline pieces (basis, sampled bodies, clusters
    with their current surrogates, A), so that the online stage alone is
    compared; returns the reduced trajectory (steps + 1, M)."""
    q = model.query()
    c = model.query_clusters()
    cl = rom.Clusters(c["members"], c["gamma_c"], c["phi_c"], c["x0_c"], c["lists"],
                      np.asarray(q["sampled"]))
    red, _ = rom.ptrom_online(cl, Phi, x0, q["A"], delta, dt, steps, tol=tol, max_gn=max_gn, u_inf=u_inf)
    return red
