"""The online PTROM step (Alg. 4 over Alg. 5) with more clusters than shared
memory holds, against the oracle's online stage on the same model.

With N_c above roughly 18 000 the clusters' current positions x^QT no longer
fit in one instance's shared memory beside the rest of its working set; the
kernel then keeps them in the instance's state buffer and reads Gamma~ in
place.  The models here are GNAT-style (every source body its own cluster,
Sec. 4.1): the two-cluster workload (Sec. 6.2 geometry) at N = 20 000 and
70 000, each sampled body interacting with

  * "all":  every other body (N_c = N, lists read from global memory as
            32-bit indices; at N = 70 000 they exceed 16 bits), or
  * "own":  the other bodies of its own Gaussian cluster, few enough sampled
            bodies that the lists fit in shared memory as 16-bit indices
            beside the global x^QT.

The trial basis is analytic rather than trained (no FOM run at these sizes):
per Gaussian cluster, the translations, the rigid rotation and an
r^2-weighted swirl about its centre, orthonormalised (M = 8); the residual
basis adds per-cluster dilation, two strains and an r^2-weighted dilation
(M_r = 16); the sampled bodies are a seeded draw of n_s / 2 from each cluster
(n_s = 32 for "all", 8 for "own").  Both
sides run the same model, so the test isolates the online stage.

Tolerances: FP32 pair sums over up to 7e4 sources per sampled body (about
2e3 terms per lane) against FP64: one Gauss-Newton update to 1e-4 relative;
20-step trajectories to MAE_D (Sec. 6.1) below 1e-4 and reduced coordinates
to 1e-3 relative (both sides stop Gauss-Newton at eps <= 1e-4)."""
import numpy as np
import pytest
import torch

from _ptrom_cases import model_arrays
from oracle import qoi, rom
from paper_2103_01983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DELTA, DT, STEPS = 0.02, 0.005, 20


def _fields(x0, n):
    """Per-cluster displacement fields at the bodies, columns of (2n, .)."""
    chi, psi = x0[:n], x0[n:]
    half = n // 2
    trial, extra = [], []
    for sel in (np.arange(n) < half, np.arange(n) >= half):
        cx, cy = chi[sel].mean(), psi[sel].mean()
        a, b = np.where(sel, chi - cx, 0.0), np.where(sel, psi - cy, 0.0)
        one = sel.astype(float)
        r2 = a * a + b * b
        trial += [np.concatenate([one, 0 * one]), np.concatenate([0 * one, one]),
                  np.concatenate([-b, a]), np.concatenate([-b * r2, a * r2])]
        extra += [np.concatenate([a, b]), np.concatenate([a, -b]), np.concatenate([b, a]),
                  np.concatenate([a * r2, b * r2])]
    return np.array(trial).T, np.array(extra).T


def _orth(Q):
    q, _ = np.linalg.qr(Q)
    return q


def _case(n, lists_kind):
    x0, G = W.two_cluster(n, seed=0)
    trial, extra = _fields(x0, n)
    Phi = _orth(trial)                                            # (2n, 8)
    Phi_r = _orth(np.concatenate([trial, extra], axis=1))          # (2n, 16)
    n_s = 32 if lists_kind == "all" else 8
    half = n // 2
    rng = np.random.default_rng(7)                                # n_s / 2 bodies from each cluster
    sampled = np.sort(np.concatenate([rng.choice(half, n_s // 2, replace=False),
                                      half + rng.choice(half, n_s // 2, replace=False)]))
    A = rom.gappy_operator(Phi_r, sampled, n)
    lists = []
    for s in sampled:
        pool = np.arange(n) if lists_kind == "all" else (np.arange(half) if s < half else np.arange(half, n))
        lists.append(pool[pool != s].tolist())
    cl = rom.Clusters([[j] for j in range(n)], G.copy(), Phi.copy(), x0.copy(), lists, sampled)
    ref1, _ = rom.ptrom_online(cl, Phi, x0, A, DELTA, DT, 1, tol=1e-4, max_gn=1)
    ref, it_ref = rom.ptrom_online(cl, Phi, x0, A, DELTA, DT, STEPS, tol=1e-4)
    return dict(cl=cl, Phi=Phi, x0=x0, G=G, A=A, n=n, ref1=ref1, ref=ref, it_ref=it_ref)


_CASES = {}


@pytest.fixture(scope="module", params=[(20000, "all"), (20000, "own"), (70000, "all")],
            ids=["n20000_all", "n20000_own", "n70000_all"])
def case(request):
    if request.param not in _CASES:
        _CASES[request.param] = _case(*request.param)
    return _CASES[request.param]


def _model(case, **kw):
    from paper_2103_01983_gb300 import ptrom as P
    arr = model_arrays(case)
    return P.PtromModel(arr["phi_s"], arr["x0_s"], arr["phi_c"], arr["x0_c"], arr["gamma_c"], arr["A"],
                        arr["off"], arr["idx"], DT, DELTA, **kw)


def test_state_holds_the_cluster_positions(case):
    """The instance state grows by the 2 N_c FP32 positions (256-byte aligned)."""
    from paper_2103_01983_gb300 import ptrom as P
    m = _model(case)
    base = ((m.M + 2 * m.n_s + 8) * 8 + 255) // 256 * 256
    assert P.lib.ptrom_state_bytes(m.handle) == base + (8 * m.N_c + 255) // 256 * 256
    assert m.N_c == case["n"]


@pytest.mark.parametrize("qr", ["fp64", "fp32c"])
def test_one_update_and_trajectory(case, qr):
    from paper_2103_01983_gb300 import ptrom as P
    Phi, x0, ref1, ref, it_ref = case["Phi"], case["x0"], case["ref1"], case["ref"], case["it_ref"]
    M = Phi.shape[1]
    m1 = _model(case, tol=1e-4, max_gn=1, qr_prec=qr)
    xh = torch.zeros(M, dtype=torch.float64, device="cuda")
    s = P.ptrom_step([m1], [m1.new_state()], 1, xhat=[xh])
    assert s["gn_iters"] == 1
    err = np.linalg.norm(xh.cpu().numpy() - ref1[1]) / np.linalg.norm(ref1[1])
    assert err <= 1e-4, err

    m = _model(case, tol=1e-4, qr_prec=qr)
    hist = torch.zeros(STEPS, M, dtype=torch.float64, device="cuda")
    s = P.ptrom_step([m], [m.new_state()], STEPS, hist=[hist])
    gpu = hist.cpu().numpy()
    assert s["noconv"] == 0 and s["steps"] == STEPS
    rel = np.linalg.norm(gpu - ref[1:], axis=1) / np.linalg.norm(ref[1:], axis=1)
    assert rel.max() <= 1e-3, rel.max()
    mae = max(qoi.mae_d(rom.reconstruct(a, Phi, x0), rom.reconstruct(b, Phi, x0), x0)
              for a, b in zip(gpu, ref[1:]))
    assert mae <= 1e-4, mae
    assert abs(s["gn_iters"] - it_ref.sum()) <= 0.1 * it_ref.sum() + 1


def test_batch_of_large_models(case):
    """Several instances of one large-N_c model in one launch: each instance
    keeps its own x^QT in its own state buffer, so equal instances agree
    bit for bit and a differently parameterised one differs."""
    from paper_2103_01983_gb300 import ptrom as P
    M = case["Phi"].shape[1]
    m = _model(case, tol=1e-4)
    xs = [torch.zeros(M, dtype=torch.float64, device="cuda") for _ in range(3)]
    P.ptrom_step([m, m, m], [m.new_state() for _ in range(3)], 5, xhat=xs)
    a, b, c = (t.cpu().numpy() for t in xs)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    assert np.all(np.isfinite(a)) and np.linalg.norm(a) > 0
