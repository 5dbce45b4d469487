"""Where the parametric PTROM's error comes from, computed by the oracle alone.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``): a study script, run by hand,
whose printed numbers are quoted in the design notes; it imports only the
oracle and the seeded input generators.

The parametric two-cluster workload (Sec. 5.1-5.2 training and reload on a
parametric family): bodies of ``workloads.two_cluster`` with common random
numbers, separation in [0.8, 1.2] and circulation ratio in [0.5, 2.0];
8 Latin-hypercube training parameters (seed 1) and 4 held-out ones (seed 2);
delta = 0.02, dt = 0.005, ``--steps`` implicit steps; POD rank k, M_r = 2k,
n_s sampled bodies, Barnes-Hut theta.  For every held-out parameter it
reports the time-averaged MAE_D and AE_H (Sec. 6.1) against the oracle FOM of

  best   the best point of the trial manifold, x^0 + Phi Phi^T (x - x^0)
         (the basis alone);
  lspg   LSPG over all bodies without clustering (the projected dynamics);
  tier2  LSPG over all bodies with the clustered sources (Stage 3's model);
  gnat   the hyper-reduced model without clustering (sampling alone);
  ptrom  the full PTROM: sampled bodies against their clusters (Alg. 4/5).

Usage:  python -m oracle.parametric_study --n 512 --steps 1000 --k 20
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import time

import numpy as np

DT, DELTA = 0.005, 0.02


def _gen(n, sep, ratio):
    from paper_2103_01983_gb300 import workloads as W
    return W.two_cluster(n, seed=0, sep=float(sep), ratio=float(ratio))


def _fom(args):
    from oracle import fom
    n, sep, ratio, steps = args
    x0, G = _gen(n, sep, ratio)
    traj, _ = fom.rollout(x0, G, DELTA, DT, steps, mode="blockdiag", tol=1e-12)
    return traj


def _tier2(args):
    """Residual snapshots of one training parameter (Stage 3)."""
    from oracle import rom
    cl, Phi, x0, steps = args
    _, snaps = rom.lspg_tier2(cl, Phi, x0, DELTA, DT, steps)
    return snaps


def _qoi(traj_rom, traj_fom, x0, G, every):
    from oracle import qoi
    ks = range(every, traj_fom.shape[0], every)
    mae = np.mean([qoi.mae_d(traj_fom[k], traj_rom[k], x0) for k in ks])
    aeh = np.mean([qoi.ae_h(qoi.hamiltonian(traj_rom[k], G), qoi.hamiltonian(traj_fom[k], G)) for k in ks])
    return float(mae), float(aeh)


def _held_out(args):
    """The five approximations of one held-out parameter and their QoI errors."""
    from oracle import rom
    n, sep, ratio, steps, Phi, sigma, xt0, Gt0, sampled, A, theta, every = args
    x0, G = _gen(n, sep, ratio)
    ref = _fom((n, sep, ratio, steps))
    out = {"sep": float(sep), "ratio": float(ratio)}
    best = x0 + (ref - x0) @ Phi @ Phi.T
    out["best"] = _qoi(best, ref, x0, G, every)
    allb = np.arange(n)
    for name, th, targets in (("lspg", 0.0, allb), ("tier2", theta, allb), ("gnat", 0.0, sampled),
                              ("ptrom", theta, sampled)):
        cl, _ = rom.cluster_tables(Phi, sigma, xt0, Gt0, targets, criterion="bh", theta=th)
        cl = rom.reload_parameters(cl, Phi, x0, G)
        if targets is allb:
            red, _ = rom.lspg_tier2(cl, Phi, x0, DELTA, DT, steps)
        else:
            red, _ = rom.ptrom_online(cl, Phi, x0, A, DELTA, DT, steps)
        rec = np.array([rom.reconstruct(z, Phi, x0) for z in red])
        out[name] = _qoi(rec, ref, x0, G, every)
    return out


def main():
    from oracle import rom
    from paper_2103_01983_gb300 import workloads as W
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--k", type=int, default=20)
    ap.add_argument("--ns", type=int, default=0, help="sampled bodies (default 2k)")
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--every", type=int, default=25, help="QoI sampling interval in steps")
    ap.add_argument("--procs", type=int, default=8)
    a = ap.parse_args()
    k, Mr, ns = a.k, 2 * a.k, a.ns or 2 * a.k
    train, held = W.param_lhs(8, seed=1), W.param_lhs(4, seed=2)
    t0 = time.time()
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.procs) as pool:
        trajs = pool.map(_fom, [(a.n, s, r, a.steps) for s, r in train])
        S = np.concatenate([t[1:] for t in trajs]).T                   # states x^1..x^Nt of every parameter
        Phi, sigma = rom.pod(S, k)
        xt0, Gt0 = _gen(a.n, *train[0])
        cl, _ = rom.cluster_tables(Phi, sigma, xt0, Gt0, np.arange(a.n), criterion="bh", theta=a.theta)
        jobs = []
        for s, r in train:
            x0, G = _gen(a.n, s, r)
            jobs.append((rom.reload_parameters(cl, Phi, x0, G), Phi, x0, a.steps))
        snaps = np.concatenate(pool.map(_tier2, jobs), axis=1)
        U, sv, _ = np.linalg.svd(snaps, full_matrices=False)
        Phi_r = U[:, :Mr]
        sampled = rom.greedy_sample(Phi_r, ns, a.n)
        A = rom.gappy_operator(Phi_r, sampled, a.n)
        rows = pool.map(_held_out, [(a.n, s, r, a.steps, Phi, sigma, xt0, Gt0, sampled, A, a.theta, a.every)
                                    for s, r in held])
    print(json.dumps({"n": a.n, "steps": a.steps, "k": k, "M_r": Mr, "n_s": ns, "theta": a.theta,
                      "seconds": round(time.time() - t0, 1), "held_out": rows}))


if __name__ == "__main__":
    main()
