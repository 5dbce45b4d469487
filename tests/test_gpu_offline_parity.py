"""Offline training stages of the library against the oracle, element by
element (GPU):

* Stage 2 clusters (Alg. 2/3, UniqueSearch) of the sampled bodies: each
  body's set of clusters, as member sets, exactly; every cluster's Gamma~,
  POD surrogate Phi~ and reference position x^0_QT (Def. 1) to 1e-12.
* Stage 3 Tier-II LSPG: the library's reduced trajectory of every training
  parameter against ``rom.lspg_tier2`` run on the oracle's own clusters from
  the library's basis (the library's pair sums are FP32).
* Stage 4 on the library's residual basis Phi_r: the sampled bodies equal
  ``rom.greedy_sample`` bit for bit; A equals ``rom.gappy_operator`` to
  round-off and A P Phi_r = I.
The oracle gets the library's POD basis (itself pinned to the oracle's POD in
test_gpu_ptrom_build.py) so each stage is compared on equal inputs.
"""
import numpy as np
import pytest
import torch

from oracle import rom
from paper_2103_01983_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2103_01983_gb300 import ptrom
    return ptrom


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _wpts(q):
    """W = Phi sigma summed mode by mode in order, as the library does."""
    Wp = np.zeros(q["phi"].shape[0])
    for m in range(q["phi"].shape[1]):
        Wp = Wp + q["phi"][:, m] * q["sigma"][m]
    return Wp


def _build(P, criterion, param, n=512, M=12, Mr=24, ns=24, steps=40):
    x0, G = W.two_cluster(n, seed=11)
    x1, G1 = W.two_cluster(n, seed=11, sep=1.1, ratio=0.8)
    fp = P.fom_params(0.005, 0.02, "jfnk", prec="fp64", tol=1e-12)
    model, info = P.ptrom_build(_dev(np.stack([x0, x1])), _dev(np.stack([G, G1])), M, Mr, ns, steps, fp,
                                criterion=criterion, theta=param, p_c=param, tol=1e-6, max_gn=20)
    return model, info, (x0, G), (x1, G1), steps


@pytest.fixture(scope="module", params=[("bh", 0.5), ("nb", 1.0)], ids=["bh0.5", "nb1"])
def built(P, request):
    criterion, param = request.param
    model, info, p0, p1, steps = _build(P, criterion, param)
    q = model.query()
    q.update(model.query_training())
    q["clusters"] = model.query_clusters()
    return {"criterion": criterion, "param": param, "model": model, "info": info, "q": q,
            "params": [p0, p1], "steps": steps}


def _kw(b):
    return {"theta": b["param"]} if b["criterion"] == "bh" else {"p_c": b["param"]}


def test_sampled_clusters_match_oracle_exactly(built):
    q = built["q"]
    x0, G = built["params"][0]
    cl, _ = rom.cluster_tables(q["phi"], q["sigma"], x0, G, q["sampled"], criterion=built["criterion"],
                               W=_wpts(q), **_kw(built))
    lib = q["clusters"]
    assert len(lib["members"]) == len(cl.members) == built["info"]["N_c"]
    key_lib = [tuple(sorted(m)) for m in lib["members"]]
    key_or = [tuple(sorted(m)) for m in cl.members]
    for s in range(len(q["sampled"])):
        assert {key_lib[c] for c in lib["lists"][s]} == {key_or[c] for c in cl.lists[s]}, s
        assert len(lib["lists"][s]) == len(cl.lists[s])
    Nc = len(key_or)
    pos = {k: c for c, k in enumerate(key_or)}
    for c, k in enumerate(key_lib):
        o = pos[k]
        np.testing.assert_allclose(lib["gamma_c"][c], cl.Gt[o], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(lib["phi_c"][c], cl.Phit[o], rtol=0, atol=1e-12)
        np.testing.assert_allclose(lib["phi_c"][Nc + c], cl.Phit[Nc + o], rtol=0, atol=1e-12)
        np.testing.assert_allclose([lib["x0_c"][c], lib["x0_c"][Nc + c]], [cl.x0t[o], cl.x0t[Nc + o]],
                                   rtol=0, atol=1e-12)


def test_tier2_trajectories_match_oracle(built):
    """Tier II (Stage 3) for both training parameters, the second on clusters
    reloaded from the stored memberships (Sec. 5.2).  Tolerance: 1e-6 of the
    reduced trajectory's size, for the library's FP32 pair sums and FP32 basis
    rows against the oracle's FP64 (measured on GB300: 2e-8 .. 6e-8), with
    both Gauss-Newton loops stopping at 1e-6."""
    q = built["q"]
    (x0, G), (x1, G1) = built["params"]
    cl, _ = rom.cluster_tables(q["phi"], q["sigma"], x0, G, np.arange(G.size), criterion=built["criterion"],
                               W=_wpts(q), **_kw(built))
    assert len(cl.members) == built["info"]["N_c_all"]
    for k, (xa, Ga) in enumerate(((x0, G), (x1, G1))):
        clk = cl if k == 0 else rom.reload_parameters(cl, q["phi"], xa, Ga)
        red, _ = rom.lspg_tier2(clk, q["phi"], xa, 0.02, 0.005, built["steps"], tol=1e-6, max_gn=20)
        got = q["tier2"][k]
        err = np.linalg.norm(got - red) / np.linalg.norm(red)
        print(f"param {k}: Tier-II reduced trajectory rel-L2 {err:.2e}")
        assert err <= 1e-6, err


def test_sampling_and_gappy_operator_on_the_library_basis(built):
    q = built["q"]
    N = q["phi"].shape[0] // 2
    Phi_r = q["phi_r"]
    ns = len(q["sampled"])
    np.testing.assert_array_equal(q["sampled"], rom.greedy_sample(Phi_r, ns, N))
    A_or = rom.gappy_operator(Phi_r, q["sampled"], N)
    np.testing.assert_allclose(q["A"], A_or, rtol=0, atol=1e-10 * np.abs(A_or).max())
    dofs = np.concatenate([q["sampled"], N + q["sampled"]])
    np.testing.assert_allclose(q["A"] @ Phi_r[dofs], np.eye(Phi_r.shape[1]), atol=1e-10)
    # the residual basis is orthonormal and spans the library's residual snapshots' leading modes
    np.testing.assert_allclose(Phi_r.T @ Phi_r, np.eye(Phi_r.shape[1]), atol=1e-10)
