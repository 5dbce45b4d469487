"""Pins of the oracle's PTROM pieces (CPU only): POD, quadtree, ClusterPOD,
HyperPair, greedy sampling, gappy operator, and PTROM exactness."""
import numpy as np
import pytest

from oracle import direct, fom, rom
from paper_2103_01983_gb300 import workloads as W


def test_pod_properties():
    """Orthonormal columns, descending values, the Gram matrix's leading
    eigenpairs, and the projection error equals the discarded energy
    (Eckart-Young), on a matrix with a known spectrum."""
    rng = np.random.default_rng(1)
    Q1, _ = np.linalg.qr(rng.standard_normal((60, 12)))
    Q2, _ = np.linalg.qr(rng.standard_normal((20, 12)))
    true = 2.0 ** -np.arange(12)
    S = Q1 @ np.diag(true) @ Q2.T
    Phi, sig = rom.pod(S, 6)
    np.testing.assert_allclose(Phi.T @ Phi, np.eye(6), atol=1e-12)
    np.testing.assert_allclose(sig, true[:6], rtol=1e-12)
    np.testing.assert_allclose(Phi @ Phi.T, Q1[:, :6] @ Q1[:, :6].T, atol=1e-12)
    # Phi spans the leading eigenvectors of S S^T
    np.testing.assert_allclose((S @ S.T) @ Phi, Phi * sig**2, atol=1e-12)
    err = np.linalg.norm(S - Phi @ (Phi.T @ S)) ** 2
    np.testing.assert_allclose(err, np.sum(true[6:] ** 2), rtol=1e-10)
    # sign convention: largest-magnitude entry of each column is positive
    assert np.all(Phi[np.argmax(np.abs(Phi), axis=0), np.arange(6)] > 0)


def test_quadtree_structure():
    rng = np.random.default_rng(2)
    P = rng.uniform(-1, 1, (300, 2))
    t = rom.QuadTree(P)
    leaves = [nd for nd in t.nodes if nd.is_leaf]
    counts = np.zeros(300, int)
    for nd in leaves:
        assert len(nd.members) == 1
        counts[nd.members] += 1
    assert np.all(counts == 1)
    for nd in t.nodes:
        for m in nd.members:
            x, y = P[m]
            assert nd.box[0] <= x <= nd.box[1] and nd.box[2] <= y <= nd.box[3]
        if nd.children:
            assert sorted(sum((c.members for c in nd.children), [])) == sorted(nd.members)
            for c in nd.children:
                assert c.width == pytest.approx(nd.width / 2)


def _setup(n=120, M=4, seed=3):
    x0, G = W.disk(n, seed=seed)
    traj, _ = fom.rollout(x0, G, 0.05, 0.01, 12, mode="dense", tol=1e-13)
    Phi, sig = rom.pod(traj[1:].T, M)
    return x0, G, Phi, sig


@pytest.mark.parametrize("criterion,param", [("bh", 0.5), ("bh", 1.0), ("nb", 1.0), ("nb", 0.0)])
def test_clusters_partition_every_target(criterion, param):
    """For each target, its clusters' members are all other bodies, once each;
    each cluster's Gamma~ is the brute-force member sum; x0_QT + Phi~ xhat is
    the |Gamma|-weighted centroid of the members' reduced positions."""
    x0, G, Phi, sig = _setup()
    N = G.size
    kw = {"theta": param} if criterion == "bh" else {"p_c": param}
    cl, tree = rom.cluster_tables(Phi, sig, x0, G, np.arange(N), criterion=criterion, **kw)
    for i, li in enumerate(cl.lists):
        mem = sorted(sum((cl.members[c] for c in li), []))
        assert mem == [j for j in range(N) if j != i]
    for c, m in enumerate(cl.members):
        assert cl.Gt[c] == pytest.approx(G[m].sum(), abs=1e-15)
    xhat = np.random.default_rng(4).standard_normal(Phi.shape[1])
    xq = cl.x0t + cl.Phit @ xhat
    x = x0 + Phi @ xhat
    Nc = len(cl.members)
    for c, m in enumerate(cl.members):
        w = np.abs(G[m])
        np.testing.assert_allclose(xq[c], np.dot(w, x[m]) / w.sum(), atol=1e-13)
        np.testing.assert_allclose(xq[Nc + c], np.dot(w, x[N + np.array(m)]) / w.sum(), atol=1e-13)
    if criterion == "bh":
        # every pruned node satisfies the opening criterion for its target, and
        # none of its ancestors did (the traversal stops at the first)
        W_ = Phi @ sig
        pts = np.stack([W_[:N], W_[N:]], axis=1)
        parent = {c.id: nd.id for nd in tree.nodes for c in nd.children}
        for i, pr in enumerate(cl.pruned):
            for nid in pr:
                nd = tree.nodes[nid]
                w = np.abs(G[nd.members])
                cen = (w[:, None] * pts[nd.members]).sum(0) / w.sum()
                assert i not in nd.members
                assert nd.width / np.linalg.norm(cen - pts[i]) <= param + 1e-12
                a = parent.get(nid)
                while a is not None:
                    an = tree.nodes[a]
                    wa = np.abs(G[an.members])
                    ca = (wa[:, None] * pts[an.members]).sum(0) / wa.sum()
                    d = np.linalg.norm(ca - pts[i])
                    assert i in an.members or d == 0 or an.width / d > param
                    a = parent.get(a)
        assert np.mean([len(li) for li in cl.lists]) < N - 1   # something was clustered


def test_hyperpair_without_clustering_is_the_fom_velocity():
    """theta = 0 never prunes: HyperPair equals Eq. 2 at x = x0 + Phi xhat."""
    x0, G, Phi, sig = _setup()
    N = G.size
    cl, _ = rom.cluster_tables(Phi, sig, x0, G, np.arange(N), criterion="bh", theta=0.0)
    assert all(len(li) == N - 1 for li in cl.lists)
    xhat = np.random.default_rng(5).standard_normal(Phi.shape[1]) * 0.1
    Phi_t, x0_t = rom.target_rows(Phi, x0, cl.targets)
    f, D = rom.hyperpair(xhat, cl, Phi_t, x0_t, 0.05)
    x = x0 + Phi @ xhat
    fo, Do = direct.velocity(x, G, 0.05, with_selfjac=True)
    np.testing.assert_allclose(f, fo, atol=1e-13)
    np.testing.assert_allclose(D, Do, atol=1e-12)


def test_greedy_sampling_small_case():
    rng = np.random.default_rng(6)
    N, Mr = 30, 4
    Phi_r, _ = np.linalg.qr(rng.standard_normal((2 * N, Mr)))
    s = rom.greedy_sample(Phi_r, 6, N)
    assert len(s) == 6 and len(set(s)) == 6
    np.testing.assert_array_equal(s, rom.greedy_sample(Phi_r, 6, N))
    # n_c = min(4, 12) = 4, n_it = 4: iteration 1 takes n_a1 = 2 bodies by the
    # energy of the first basis column alone
    e1 = Phi_r[:N, 0] ** 2 + Phi_r[N:, 0] ** 2
    assert list(s[:2]) == list(np.argsort(-e1, kind="stable")[:2])
    A = rom.gappy_operator(Phi_r, s, N)
    dofs = np.concatenate([s, N + s])
    np.testing.assert_allclose(A @ Phi_r[dofs], np.eye(Mr), atol=1e-12)


def test_gappy_operator_with_more_residual_modes_than_sampled_dofs():
    """M_r > n_d (the mushroom cloud of Sec. 6.3: M_r = 185, n_d = 150): the
    least squares of Eq. approx_resi is under-determined and [P Phi_r]^+ is
    the minimum-norm solution operator.  It is a right inverse of P Phi_r,
    its rows lie in the row space of P Phi_r, and sampling is still n_s
    distinct bodies chosen from the first n_c = n_d modes."""
    rng = np.random.default_rng(8)
    N, Mr, ns = 40, 14, 5
    Phi_r, _ = np.linalg.qr(rng.standard_normal((2 * N, Mr)))
    s = rom.greedy_sample(Phi_r, ns, N)
    assert len(set(s)) == ns
    dofs = np.concatenate([s, N + s])
    PPr = Phi_r[dofs]                              # n_d x M_r = 10 x 14
    A = rom.gappy_operator(Phi_r, s, N)
    assert A.shape == (Mr, 2 * ns)
    np.testing.assert_allclose(PPr @ A, np.eye(2 * ns), atol=1e-12)
    # minimum norm: A's columns are combinations of P Phi_r's rows
    coef = np.linalg.lstsq(PPr.T, A, rcond=None)[0]
    np.testing.assert_allclose(PPr.T @ coef, A, atol=1e-12)
    # any other right inverse has a larger Frobenius norm
    Z = (np.eye(Mr) - np.linalg.pinv(PPr) @ PPr) @ rng.standard_normal((Mr, 2 * ns))
    assert np.linalg.norm(A + Z) > np.linalg.norm(A)


def test_ptrom_reproduces_fom_when_basis_spans_trajectory():
    """A basis spanning the state space (as many independent snapshots as
    dofs), every body sampled, no clustering: the PTROM trajectory is the FOM
    trajectory (Gauss-Newton tolerance)."""
    n, steps, dt, delta = 20, 50, 0.01, 0.05
    x0, G = W.disk(n, seed=7)
    traj, _ = fom.rollout(x0, G, delta, dt, steps, mode="dense", tol=1e-14)
    S = traj[1:].T
    M = 2 * n                                 # all left singular vectors: Phi spans R^(2n)
    Phi, sig = rom.pod(S, M)
    cl, _ = rom.cluster_tables(Phi, sig, x0, G, np.arange(n), criterion="bh", theta=0.0)
    red2, snaps = rom.lspg_tier2(cl, Phi, x0, delta, dt, steps, tol=1e-12)
    U, s, _ = np.linalg.svd(snaps, full_matrices=False)
    Mr = int(np.sum(s > 1e-10 * s[0]))
    Phi_r = U[:, :Mr]
    A = rom.gappy_operator(Phi_r, np.arange(n), n)
    red3, iters = rom.ptrom_online(cl, Phi, x0, A, delta, dt, steps, tol=1e-12)
    rec = np.array([rom.reconstruct(z, Phi, x0) for z in red3])
    assert np.abs(rec - traj).max() <= 1e-9
    rec2 = np.array([rom.reconstruct(z, Phi, x0) for z in red2])
    assert np.abs(rec2 - traj).max() <= 1e-9


def test_ptrom_reproduces_fom_with_inflow_when_basis_spans_trajectory():
    """As above with a non-uniform superimposed inflow (Sec. 6.3): the inflow
    enters Tier II, the residual snapshots and the online residual alike, so
    the PTROM still reproduces the FOM trajectory."""
    n, steps, dt, delta = 20, 50, 0.01, 0.05
    x0, G = W.disk(n, seed=7)
    u = np.concatenate([np.zeros(n), 0.5 + np.linspace(-1.0, 1.0, n) ** 2])
    traj, _ = fom.rollout(x0, G, delta, dt, steps, mode="dense", tol=1e-14, u_inf=u)
    Phi, sig = rom.pod(traj[1:].T, 2 * n)
    cl, _ = rom.cluster_tables(Phi, sig, x0, G, np.arange(n), criterion="bh", theta=0.0)
    red2, snaps = rom.lspg_tier2(cl, Phi, x0, delta, dt, steps, tol=1e-12, u_inf=u)
    U, s, _ = np.linalg.svd(snaps, full_matrices=False)
    Phi_r = U[:, :int(np.sum(s > 1e-10 * s[0]))]
    A = rom.gappy_operator(Phi_r, np.arange(n), n)
    red3, _ = rom.ptrom_online(cl, Phi, x0, A, delta, dt, steps, tol=1e-12, u_inf=u)
    for red in (red2, red3):
        rec = np.array([rom.reconstruct(z, Phi, x0) for z in red])
        assert np.abs(rec - traj).max() <= 1e-9
    # without the inflow term the same model drifts away from the trajectory
    red0, _ = rom.ptrom_online(cl, Phi, x0, A, delta, dt, steps, tol=1e-12)
    rec0 = np.array([rom.reconstruct(z, Phi, x0) for z in red0])
    assert np.abs(rec0 - traj).max() > 1e-2


def _phi_r(N, cols):
    """(2N, len(cols)) matrix from {dof: value} dicts; dof k < N is chi_k,
    dof N + k is psi_k."""
    P = np.zeros((2 * N, len(cols)))
    for m, col in enumerate(cols):
        for d, v in col.items():
            P[d, m] = v
    return P


def _greedy_variant(Phi_r, n_samples, N, variant):
    """greedy_sample with one planted mistake, to show the pins below catch it."""
    M_r = Phi_r.shape[1]
    chosen, n_a, n_b = [], n_samples, 0
    n_c = min(M_r, 2 * n_samples)
    n_it = min(n_c, n_a)
    for i in range(1, n_it + 1):
        n_ci = n_c // n_it + (1 if i <= n_c % n_it else 0)
        n_ai = n_a // n_it + (1 if i <= n_a % n_it else 0)
        R = Phi_r[:, n_b:n_b + n_ci]
        if i > 1 and variant != "no_reconstruction":
            dofs = np.concatenate([chosen, N + np.asarray(chosen)]).astype(int)
            if variant == "all_rows":
                dofs = np.arange(2 * N)
            cols = slice(n_b - 1, n_b) if variant == "last_block_column" else slice(0, n_b)
            coef = np.linalg.lstsq(Phi_r[dofs, cols], R[dofs], rcond=None)[0]
            R = R + Phi_r[:, cols] @ coef if variant == "sign" else R - Phi_r[:, cols] @ coef
        err = (R[:N] ** 2).sum(axis=1) + (R[N:] ** 2).sum(axis=1)
        for _ in range(n_ai):
            e = err.copy()
            e[chosen] = -np.inf
            chosen.append(int(np.argmax(e)))
        n_b += n_ci
    return chosen


def test_greedy_sampling_picks_follow_the_gappy_residual_by_hand():
    """Alg. 1 on N = 6 bodies, M_r = 3, n_s = 3 (n_c = 3, n_it = 3, one
    column and one body per iteration).  Columns (chi_k = dof k, psi_k = dof
    6 + k):
      c0: chi3 = -1, psi0 = 1, psi4 = 2
      c1: chi5 = 2, psi0 = -2, psi4 = -2
      c2: chi0 = 1, chi3 = 1, psi4 = 1
    i = 1: R = c0, body energies 1 (0), 1 (3), 4 (4)          -> body 4.
    i = 2: on body 4's dofs c0 = (0, 2), c1 = (0, -2): coefficient -1, so
           R = c1 + c0 = (chi3 -1, chi5 2, psi0 -1): energies 1, 1, 4 -> body 5.
    i = 3: on bodies 4, 5 the rows of [c0 c1] are (0,0), (0,2), (2,-2), (0,0)
           against c2's (0, 0, 1, 0): coefficients (1/2, 0), so
           R = c2 - c0/2 = (chi0 1, chi3 3/2, psi0 -1/2): energies
           5/4 (0), 9/4 (3)                                    -> body 3.
    Each planted mistake changes a pick: no reconstruction or a flipped sign
    at i = 2 (body 0), reconstruction over all dofs or from the last block
    column only at i = 3 (body 0)."""
    N = 6
    Phi_r = _phi_r(N, [{3: -1, 6: 1, 10: 2}, {5: 2, 6: -2, 10: -2}, {0: 1, 3: 1, 10: 1}])
    assert list(rom.greedy_sample(Phi_r, 3, N)) == [4, 5, 3]
    assert _greedy_variant(Phi_r, 3, N, "ok") == [4, 5, 3]
    assert _greedy_variant(Phi_r, 3, N, "no_reconstruction")[1] == 0
    assert _greedy_variant(Phi_r, 3, N, "sign")[1] == 0
    assert _greedy_variant(Phi_r, 3, N, "all_rows")[2] == 0
    assert _greedy_variant(Phi_r, 3, N, "last_block_column")[2] == 0


def test_greedy_sampling_rank_deficient_reconstruction_is_minimum_norm():
    """Alg. 1 with a rank-deficient gappy least squares at i = 2: N = 5,
    M_r = 4, n_s = 2 (n_c = 4, n_it = 2: two columns and one body per
    iteration).  Columns:
      c0: chi0 = 2, chi1 = 1;  c1: chi0 = 1, psi2 = 1
      c2: chi0 = 5, chi3 = 1, psi4 = 1/2;  c3: psi3 = 1/5
    i = 1: R = [c0 c1], energies 5 (0), 1 (1), 1 (2)          -> body 0.
    i = 2: on body 0's dofs [c0 c1] = [[2, 1], [0, 0]] has rank 1; for c2
           (5, 0) every c with 2 c_0 + c_1 = 5 fits exactly, the minimum-norm
           one is (2, 1); c3 is 0 there (coefficients 0).  R = [c2 - 2 c0 - c1, c3]:
           chi1 -2, psi2 -1, chi3 1, psi4 1/2, psi3 1/5: energies 4 (1),
           1 (2), 1.04 (3), 1/4 (4)                            -> body 1.
    Skipping the reconstruction when the system is singular would pick body 3
    (c2's chi3 and c3's psi3), and the basic solution (0, 5) body 2."""
    N = 5
    Phi_r = _phi_r(N, [{0: 2, 1: 1}, {0: 1, 7: 1}, {0: 5, 3: 1, 9: 0.5}, {8: 0.2}])
    assert list(rom.greedy_sample(Phi_r, 2, N)) == [0, 1]
    assert _greedy_variant(Phi_r, 2, N, "no_reconstruction") == [0, 3]
    R = Phi_r[:, 2:] - Phi_r[:, :2] @ np.array([[0.0, 0.0], [5.0, 0.0]])
    e = (R[:N] ** 2).sum(axis=1) + (R[N:] ** 2).sum(axis=1)
    e[0] = -np.inf
    assert int(np.argmax(e)) == 2


def test_ptrom_reproduces_fom_with_a_rank_deficient_basis():
    """n = 20 bodies over 8 steps: the basis spans {x^0 .. x^8} (rank 9 of
    2n = 40), so the affine trial manifold x^0 + Phi xhat holds the whole
    trajectory but not R^(2n).  Every body sampled, no clustering: Tier-II
    LSPG and the online PTROM reproduce the FOM trajectory to the Newton
    tolerance, and a basis of the 4 leading modes (the states' singular values
    fall from 10 to 4e-13; the fifth is 2e-6) does not."""
    n, steps, dt, delta = 20, 8, 0.01, 0.05
    x0, G = W.disk(n, seed=9)
    traj, _ = fom.rollout(x0, G, delta, dt, steps, mode="dense", tol=1e-14)
    S = traj.T                                  # [x^0 .. x^8]
    M = np.linalg.matrix_rank(S)
    assert M == steps + 1 < 2 * n
    Phi, sig = rom.pod(S, M)
    cl, _ = rom.cluster_tables(Phi, sig, x0, G, np.arange(n), criterion="bh", theta=0.0)
    red2, snaps = rom.lspg_tier2(cl, Phi, x0, delta, dt, steps, tol=1e-12)
    U, s, _ = np.linalg.svd(snaps, full_matrices=False)
    Phi_r = U[:, :int(np.sum(s > 1e-10 * s[0]))]
    A = rom.gappy_operator(Phi_r, np.arange(n), n)
    red3, _ = rom.ptrom_online(cl, Phi, x0, A, delta, dt, steps, tol=1e-12)
    for red in (red2, red3):
        rec = np.array([rom.reconstruct(z, Phi, x0) for z in red])
        assert np.abs(rec - traj).max() <= 1e-9
    Phi_s, sig_s = rom.pod(S, 4)
    cl_s, _ = rom.cluster_tables(Phi_s, sig_s, x0, G, np.arange(n), criterion="bh", theta=0.0)
    red_s, _ = rom.lspg_tier2(cl_s, Phi_s, x0, delta, dt, steps, tol=1e-12)
    rec_s = np.array([rom.reconstruct(z, Phi_s, x0) for z in red_s])
    assert np.abs(rec_s - traj).max() > 1e-7


def test_tier2_clustered_residual_by_hand():
    """Tier II with one pruned node (Barnes-Hut theta = 0.6).  The weighted POD
    space is made the positions themselves (Phi = I, sigma = x^0), so the
    quadtree is over the four bodies: the target at (-10, 0) and a group at
    (5, 0), (5.2, 0.1), (5, -0.2) whose node (width 7.6, centroid ~15.1 away,
    ratio 0.50 <= 0.6) is pruned for it.  The target's velocity is then one
    surrogate, Gamma~ = 0.5 + 1 + 1.5 = 3 at the |Gamma|-weighted centroid
    ((0.5*5 + 1*5.2 + 1.5*5)/3, (0.5*0 + 1*0.1 + 1.5*(-0.2))/3)
    = (5.0666.., -0.0666..), and Tier II's first residual at xhat = 0 is
    -dt f there."""
    x0 = np.array([-10.0, 5.0, 5.2, 5.0, 0.0, 0.0, 0.1, -0.2])
    G = np.array([2.0, 0.5, 1.0, 1.5])
    n, delta, dt = 4, 0.05, 0.01
    Phi, sig = np.eye(2 * n), x0.copy()
    cl, tree = rom.cluster_tables(Phi, sig, x0, G, np.arange(n), criterion="bh", theta=0.6)
    assert len(cl.lists[0]) == 1 and sorted(cl.members[cl.lists[0][0]]) == [1, 2, 3]
    cx, cy = (0.5 * 5 + 1 * 5.2 + 1.5 * 5) / 3, (0.5 * 0 + 1 * 0.1 + 1.5 * -0.2) / 3
    a, b = -10.0 - cx, 0.0 - cy
    q = 3.0 / (2 * np.pi) / (a * a + b * b + delta)
    f0 = np.array([-q * b, q * a])                  # e3 x (a, b) = (-b, a)
    Phi_t, x0_t = rom.target_rows(Phi, x0, cl.targets)
    f, _ = rom.hyperpair(np.zeros(2 * n), cl, Phi_t, x0_t, delta)
    np.testing.assert_allclose([f[0], f[n]], f0, rtol=1e-14)
    _, snaps = rom.lspg_tier2(cl, Phi, x0, delta, dt, 1, tol=1e-12)
    np.testing.assert_allclose([snaps[0, 0], snaps[n, 0]], -dt * f0, rtol=1e-13)
    # without the pruning the target sees the three bodies separately
    fo = direct.velocity(x0, G, delta)
    assert abs(fo[0] - f0[0]) > 1e-6 * abs(f0[0])
