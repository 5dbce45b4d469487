"""Parity of the CUDA all-pairs kernels with the FP64 oracle (GPU).

Tolerance: relative L2 error <= 1e-5 for the FP32-compensated path (the
velocity-field bound, applied to every pair product), <= 1e-12 for the FP64
path.  Sizes span several 64-target tiles and 32-source chunks with ragged
tails, source splits 1..16 with both combines, delta = 0
(masked self pairs), distinct targets, and full-size spot checks.
"""
import numpy as np
import pytest
import torch

from oracle import direct
from paper_2103_01983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp32c": 1e-5, "fp64": 1e-12}


@pytest.fixture(scope="module")
def P():
    from paper_2103_01983_gb300 import ptrom
    yield ptrom
    ptrom.set_source_split(0)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _jittered_grid(n, seed):
    """n bodies on a jittered square lattice: minimum spacing >= half the
    lattice pitch, so FP32 position rounding stays ~2^-24 relative to every
    pair distance even at delta = 0."""
    rng = np.random.default_rng(seed)
    m = int(np.ceil(np.sqrt(n)))
    k = np.arange(n)
    h = 2.0 / m
    chi = -1 + h * (k % m) + 0.25 * h * rng.uniform(-1, 1, n)
    psi = -1 + h * (k // m) + 0.25 * h * rng.uniform(-1, 1, n)
    G = rng.standard_normal(n)
    return np.concatenate([chi, psi]), G


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
@pytest.mark.parametrize("n,delta,gen", [(1000, 0.05, "disk"), (777, 0.0, "grid"),
                                          (2050, 0.02, "two_cluster")])
def test_velocity_and_selfjac(P, prec, n, delta, gen):
    if gen == "disk":
        x, G = W.disk(n, seed=21)
    elif gen == "grid":
        x, G = _jittered_grid(n, seed=21)
    else:
        x, G = W.two_cluster(n, seed=22)
    fo, Do = direct.velocity(x, G, delta, with_selfjac=True)
    f = P.bs_velocity(_dev(x), _dev(G), delta, prec=prec).cpu().numpy()
    assert _rel(f, fo) <= TOL[prec]
    f2, D = P.bs_velocity(_dev(x), _dev(G), delta, selfjac=True, prec=prec)
    assert _rel(f2.cpu().numpy(), fo) <= TOL[prec]
    assert _rel(D.cpu().numpy(), Do) <= TOL[prec]


@pytest.mark.parametrize("mode,split", [(1, 1), (1, 2), (1, 3), (1, 5), (1, 8),
                                        (2, 2), (2, 3), (2, 7), (2, 11), (2, 16), (0, 0)])
def test_every_source_split_and_combine(P, mode, split):
    """Cluster (mode 1) and global (mode 2) combines of the source split, and
    the automatic choice; N = 1530 leaves a ragged last target block and a
    ragged last chunk, and S = 16 gives some CTAs no chunk at all."""
    x, G = W.two_cluster(1530, seed=23)
    fo, Do = direct.velocity(x, G, 0.02, with_selfjac=True)
    P.set_split_mode(mode)
    P.set_source_split(split)
    try:
        f, D = P.bs_velocity(_dev(x), _dev(G), 0.02, selfjac=True)
        v = W.random_vectors(x.size, 1, seed=24)[0]
        jv = P.bs_jvp(_dev(x), _dev(G), 0.02, _dev(v))
        gx, gG = P.bs_vjp(_dev(x), _dev(G), 0.02, _dev(v))
        jv2 = P.bs_jvp(_dev(x), _dev(G), 0.02, _dev(v))
    finally:
        P.set_source_split(0)
        P.set_split_mode(0)
    assert torch.equal(jv, jv2)  # the fixed-order combine is deterministic
    assert _rel(f.cpu().numpy(), fo) <= 1e-5
    assert _rel(D.cpu().numpy(), Do) <= 1e-5
    assert _rel(jv.cpu().numpy(), direct.jvp(x, G, 0.02, v)) <= 1e-5
    gxo, gGo = direct.vjp(x, G, 0.02, v)
    assert _rel(gx.cpu().numpy(), gxo) <= 1e-5
    assert _rel(gG.cpu().numpy(), gGo) <= 1e-5


@pytest.mark.parametrize("ny", [29, 893])
def test_distinct_targets_grid(P, ny):
    """Grid targets; 37 x 893 = 33041 targets take the 4-set velocity kernel
    (ragged last 256-target block)."""
    x, G = W.disk(900, seed=25)
    gx, gy = np.meshgrid(np.linspace(-1.2, 1.2, 37), np.linspace(-1.1, 1.1, ny))
    t = np.concatenate([gx.ravel(), gy.ravel()])
    fo = direct.velocity(x, G, 0.05, targets=t)
    f = P.bs_velocity(_dev(x), _dev(G), 0.05, xt=_dev(t)).cpu().numpy()
    assert _rel(f, fo) <= 1e-5


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
@pytest.mark.parametrize("n,delta", [(1000, 0.05), (333, 0.0), (2051, 0.02)])
def test_jvp_vjp(P, prec, n, delta):
    if delta == 0.0:
        x, G = _jittered_grid(n, seed=26)
    else:
        x, G = W.two_cluster(n + (n % 2), seed=26)
    v, w = W.random_vectors(x.size, 2, seed=27)
    jv = P.bs_jvp(_dev(x), _dev(G), delta, _dev(v), prec=prec).cpu().numpy()
    assert _rel(jv, direct.jvp(x, G, delta, v)) <= TOL[prec]
    gxo, gGo = direct.vjp(x, G, delta, w)
    gx, gG = P.bs_vjp(_dev(x), _dev(G), delta, _dev(w), prec=prec)
    assert _rel(gx.cpu().numpy(), gxo) <= TOL[prec]
    assert _rel(gG.cpu().numpy(), gGo) <= TOL[prec]
    gx2, none = P.bs_vjp(_dev(x), _dev(G), delta, _dev(w), want_gamma=False, prec=prec)
    assert none is None and _rel(gx2.cpu().numpy(), gxo) <= TOL[prec]
    none, gG2 = P.bs_vjp(_dev(x), _dev(G), delta, _dev(w), want_x=False, prec=prec)
    assert none is None and _rel(gG2.cpu().numpy(), gGo) <= TOL[prec]


def test_adjoint_identity_fp32c(P):
    x, G = W.two_cluster(4096, seed=28)
    v, w = W.random_vectors(x.size, 2, seed=29)
    jv = P.bs_jvp(_dev(x), _dev(G), 0.02, _dev(v)).cpu().numpy()
    gx, _ = P.bs_vjp(_dev(x), _dev(G), 0.02, _dev(w), want_gamma=False)
    lhs, rhs = np.dot(w, jv), np.dot(gx.cpu().numpy(), v)
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(w) * np.linalg.norm(jv)


def test_degenerate_sizes(P):
    # one body: only the skipped self pair -> zero velocity and zero block
    x = np.array([0.3, -0.2])
    f, D = P.bs_velocity(_dev(x), _dev(np.array([1.0])), 0.05, selfjac=True)
    assert np.all(f.cpu().numpy() == 0) and np.all(D.cpu().numpy() == 0)
    # two bodies at delta = 0: closed form
    x, G = W.two_vortex(0.5, 1.0, 2.0)
    f = P.bs_velocity(_dev(x), _dev(G), 0.0).cpu().numpy()
    np.testing.assert_allclose(f, direct.velocity(x, G, 0.0), rtol=1e-6, atol=1e-7)
    # coincident pair at delta = 0 is skipped, not NaN
    x = np.array([0.1, 0.1, 0.4, 0.2, 0.2, 0.0])
    G = np.array([1.0, -1.0, 0.5])
    f = P.bs_velocity(_dev(x), _dev(G), 0.0).cpu().numpy()
    assert np.all(np.isfinite(f))
    # body 3 feels two exactly cancelling terms: FP32 leaves ~1e-8 there
    np.testing.assert_allclose(f, direct.velocity(x, G, 0.0), rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("n", [16384, 65536])
def test_full_size_sampled_rows(P, n):
    """Full-size two-cluster workloads: every output checked on 256 sampled
    bodies against the oracle (row-sampled sums), same launch as the bench."""
    x, G = W.two_cluster(n, seed=0)
    delta = 0.02
    rows = np.random.default_rng(30).choice(n, 256, replace=False)
    idx = np.r_[rows, n + rows]
    v, w = W.random_vectors(x.size, 2, seed=31)
    f, D = P.bs_velocity(_dev(x), _dev(G), delta, selfjac=True)
    fo, Do = direct.velocity(x, G, delta, targets=x[idx], with_selfjac=True)
    assert _rel(f.cpu().numpy()[idx], fo) <= 1e-5
    assert _rel(D.cpu().numpy()[:, rows], Do) <= 1e-5
    f1 = P.bs_velocity(_dev(x), _dev(G), delta).cpu().numpy()  # velocity alone (4 target sets at N >= 32768)
    assert _rel(f1[idx], fo) <= 1e-5
    jv = P.bs_jvp(_dev(x), _dev(G), delta, _dev(v)).cpu().numpy()
    assert _rel(jv[idx], direct.jvp(x, G, delta, v, rows=rows)) <= 1e-5
    gx, gG = P.bs_vjp(_dev(x), _dev(G), delta, _dev(w))
    gxo, gGo = direct.vjp(x, G, delta, w, rows=rows)
    assert _rel(gx.cpu().numpy()[idx], gxo) <= 1e-5
    assert _rel(gG.cpu().numpy()[rows], gGo) <= 1e-5


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
@pytest.mark.parametrize("n,M,delta", [(1000, 20, 0.05), (777, 7, 0.0), (2050, 33, 0.02)])
def test_jphi(P, prec, n, M, delta):
    if delta == 0.0:
        x, G = _jittered_grid(n, seed=60)
    else:
        x, G = W.two_cluster(n + (n % 2), seed=61)
    phi = W.random_vectors(x.size, M, seed=62).T          # (2n, M)
    ref = direct.jphi(x, G, delta, phi)
    out = P.bs_jphi(_dev(x), _dev(G), delta, _dev(phi), prec=prec).cpu().numpy()
    assert _rel(out, ref) <= TOL[prec]
    # every column equals the J v product of that column
    jv = P.bs_jvp(_dev(x), _dev(G), delta, _dev(phi[:, 3]), prec=prec).cpu().numpy()
    assert _rel(out[:, 3], jv) <= 2 * TOL[prec]


def test_jphi_full_size_sampled_rows(P):
    n, M = 16384, 20
    x, G = W.two_cluster(n, seed=0)
    phi = W.random_vectors(2 * n, M, seed=63).T
    out = P.bs_jphi(_dev(x), _dev(G), 0.02, _dev(phi)).cpu().numpy()
    rows = np.random.default_rng(64).choice(n, 128, replace=False)
    idx = np.r_[rows, n + rows]
    ref = np.stack([direct.jvp(x, G, 0.02, phi[:, m], rows=rows) for m in range(M)], axis=1)
    assert _rel(out[idx], ref) <= 1e-5


@pytest.mark.parametrize("split", [1, 3, 7])
def test_jphi_source_splits_are_deterministic(P, split):
    """J Phi with its sources split over 1, 3 or 7 CTAs per target block: the
    splits' partials are added in a fixed order, so two launches agree bit
    for bit, and every split agrees with the oracle (M = 25 leaves a ragged
    last 12-column slice)."""
    n, M = 2050, 25
    x, G = W.two_cluster(n, seed=65)
    phi = W.random_vectors(x.size, M, seed=66).T
    ref = direct.jphi(x, G, 0.02, phi)
    P.set_source_split(split)
    try:
        a = P.bs_jphi(_dev(x), _dev(G), 0.02, _dev(phi))
        b = P.bs_jphi(_dev(x), _dev(G), 0.02, _dev(phi))
    finally:
        P.set_source_split(0)
    assert torch.equal(a, b)
    assert _rel(a.cpu().numpy(), ref) <= 1e-5


@pytest.mark.parametrize("n", [16384, 65536])
def test_full_size_sampled_rows_tuned_split(P, n):
    """The bench's launch configuration: the split autotuned for the shape
    first (ptrom_tune_pairs, as bench.py does before its warm-up), then every
    all-pairs output on 256 sampled bodies against the oracle."""
    x, G = W.two_cluster(n, seed=0)
    delta = 0.02
    rows = np.random.default_rng(32).choice(n, 256, replace=False)
    idx = np.r_[rows, n + rows]
    v, w = W.random_vectors(x.size, 2, seed=33)
    P.autotune_reset()
    try:
        P.tune_pairs(n, delta)
        f, D = P.bs_velocity(_dev(x), _dev(G), delta, selfjac=True)
        fo, Do = direct.velocity(x, G, delta, targets=x[idx], with_selfjac=True)
        assert _rel(f.cpu().numpy()[idx], fo) <= 1e-5
        assert _rel(D.cpu().numpy()[:, rows], Do) <= 1e-5
        assert _rel(P.bs_velocity(_dev(x), _dev(G), delta).cpu().numpy()[idx], fo) <= 1e-5
        jv = P.bs_jvp(_dev(x), _dev(G), delta, _dev(v)).cpu().numpy()
        assert _rel(jv[idx], direct.jvp(x, G, delta, v, rows=rows)) <= 1e-5
        gx, gG = P.bs_vjp(_dev(x), _dev(G), delta, _dev(w))
        gxo, gGo = direct.vjp(x, G, delta, w, rows=rows)
        assert _rel(gx.cpu().numpy()[idx], gxo) <= 1e-5
        assert _rel(gG.cpu().numpy()[rows], gGo) <= 1e-5
    finally:
        P.autotune_reset()


def test_autotuned_split_keeps_results(P):
    """After ptrom_tune_pairs (explicit) and with tuning on first use, every
    all-pairs kernel still matches the oracle at the tuned shapes."""
    n = 3002
    x, G = W.two_cluster(n, seed=67)
    v = W.random_vectors(x.size, 1, seed=68)[0]
    P.autotune_reset()
    try:
        P.tune_pairs(n, 0.02)
        f, D = P.bs_velocity(_dev(x), _dev(G), 0.02, selfjac=True)
        jv = P.bs_jvp(_dev(x), _dev(G), 0.02, _dev(v))
        fo, Do = direct.velocity(x, G, 0.02, with_selfjac=True)
        assert _rel(f.cpu().numpy(), fo) <= 1e-5 and _rel(D.cpu().numpy(), Do) <= 1e-5
        assert _rel(jv.cpu().numpy(), direct.jvp(x, G, 0.02, v)) <= 1e-5
        P.set_autotune(True)
        x2, G2 = W.two_cluster(2500, seed=69)
        f2 = P.bs_velocity(_dev(x2), _dev(G2), 0.02)      # tuned on first use
        f3 = P.bs_velocity(_dev(x2), _dev(G2), 0.02)      # cached split
        assert torch.equal(f2, f3)
        assert _rel(f3.cpu().numpy(), direct.velocity(x2, G2, 0.02)) <= 1e-5
    finally:
        P.set_autotune(False)
        P.autotune_reset()
