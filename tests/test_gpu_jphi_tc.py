"""J Phi on the tensor cores (bs_jphi, prec "tf32x3" and "f16x3") against the
FP64 oracle.

The kernel writes (J Phi)_i = S_i Phi_i - sum_j K_ij Phi_j (K_ij the 2x2 pair
block of Sec. 2's kernel Jacobian, S_i = sum_j K_ij) and runs the contraction
on tcgen05 MMAs with TF32 (or power-of-two-scaled FP16) hi/lo splits.  Tolerance: 1e-5 relative (L2 over
the whole output), the same bar as the FP32 pipes; the 3-term split keeps each
product to ~2^-20 and no hi*hi accumulator in tensor memory takes more than 64
MMA steps before it is folded into a compensated total, so the expected error
is ~1e-6 (checked against the SIMT kernel too).

Cases: 128-target blocks with a ragged last block and a ragged last 16-source
tile, one to four 64-column slices with a ragged last slice (N = 16 .. 64 per
MMA), two bodies and one column, delta = 0 (coincidence masking) on a jittered
lattice with exactly coincident bodies, source splits 1 .. 7 (partials added
in split order: bit-identical run to run; splits of one tile), a smooth basis
(where S_i Phi_i and the contraction partly cancel), the full-size case
N = 65536, M = 60 on sampled rows, and the bounded-wait failure path."""
import numpy as np
import pytest
import torch

from oracle import direct
from paper_2103_01983_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    from paper_2103_01983_gb300 import ptrom
    yield ptrom
    ptrom.set_source_split(0)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _lattice(n, seed):
    rng = np.random.default_rng(seed)
    m = int(np.ceil(np.sqrt(n)))
    k = np.arange(n)
    h = 2.0 / m
    chi = -1 + h * (k % m) + 0.25 * h * rng.uniform(-1, 1, n)
    psi = -1 + h * (k // m) + 0.25 * h * rng.uniform(-1, 1, n)
    return np.concatenate([chi, psi]), rng.standard_normal(n)


PRECS = ["tf32x3", "f16x3"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,M,delta", [(1000, 20, 0.05), (777, 7, 0.0), (2050, 33, 0.02), (130, 64, 0.02),
                                       (3001, 100, 0.02), (4096, 128, 0.02)])
def test_jphi_tf32x3_matches_oracle(P, prec, n, M, delta):
    if delta == 0.0:
        x, G = _lattice(n, seed=70)
    else:
        x, G = W.two_cluster(n + (n % 2), seed=71)
    phi = W.random_vectors(x.size, M, seed=72).T
    ref = direct.jphi(x, G, delta, phi)
    out = P.bs_jphi(_dev(x), _dev(G), delta, _dev(phi), prec=prec).cpu().numpy()
    assert np.all(np.isfinite(out))
    err = _rel(out, ref)
    assert err <= TOL, err
    simt = P.bs_jphi(_dev(x), _dev(G), delta, _dev(phi), prec="fp32c").cpu().numpy()
    assert _rel(out, simt) <= TOL


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("split", [1, 3, 7])
def test_jphi_tf32x3_splits_deterministic(P, split, prec):
    n, M = 6000, 25
    x, G = W.two_cluster(n, seed=73)
    phi = W.random_vectors(x.size, M, seed=74).T
    ref = direct.jphi(x, G, 0.02, phi)
    P.set_source_split(split)
    try:
        a = P.bs_jphi(_dev(x), _dev(G), 0.02, _dev(phi), prec=prec)
        b = P.bs_jphi(_dev(x), _dev(G), 0.02, _dev(phi), prec=prec)
    finally:
        P.set_source_split(0)
    assert torch.equal(a, b)
    assert _rel(a.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("prec", PRECS)
def test_jphi_tf32x3_smooth_basis(P, prec):
    """Columns that vary smoothly over the bodies (rigid motions and strains
    of each Gaussian cluster, orthonormalised): Phi_i - Phi_j is small for
    near pairs, so the two terms of S_i Phi_i - sum_j K_ij Phi_j partly
    cancel."""
    n = 4096
    x, G = W.two_cluster(n, seed=75)
    chi, psi = x[:n], x[n:]
    cols = []
    for sel in (np.arange(n) < n // 2, np.arange(n) >= n // 2):
        a = np.where(sel, chi - chi[sel].mean(), 0.0)
        b = np.where(sel, psi - psi[sel].mean(), 0.0)
        one = sel.astype(float)
        cols += [np.r_[one, 0 * one], np.r_[0 * one, one], np.r_[-b, a], np.r_[a, b], np.r_[a, -b], np.r_[b, a],
                 np.r_[-b * (a * a + b * b), a * (a * a + b * b)]]
    phi, _ = np.linalg.qr(np.array(cols).T)
    ref = direct.jphi(x, G, 0.02, phi)
    out = P.bs_jphi(_dev(x), _dev(G), 0.02, _dev(phi), prec=prec).cpu().numpy()
    assert _rel(out, ref) <= TOL


@pytest.mark.parametrize("prec", PRECS)
def test_jphi_tf32x3_full_size_sampled_rows(P, prec):
    """N = 65536, M = 60 (the size the benchmark times): 128 sampled bodies'
    rows of every column against the oracle's J v of that column."""
    n, M = 65536, 60
    x, G = W.two_cluster(n, seed=0)
    phi = W.random_vectors(2 * n, M, seed=76).T
    out = P.bs_jphi(_dev(x), _dev(G), 0.02, _dev(phi), prec=prec).cpu().numpy()
    rows = np.random.default_rng(77).choice(n, 128, replace=False)
    idx = np.r_[rows, n + rows]
    ref = np.stack([direct.jvp(x, G, 0.02, phi[:, m], rows=rows) for m in range(M)], axis=1)
    assert _rel(out[idx], ref) <= TOL


def test_jphi_tf32x3_rejected_elsewhere(P):
    """The tensor-core precision is J Phi's alone: the other pair sums refuse it."""
    n = 64
    x, G = W.two_cluster(n, seed=78)
    with pytest.raises(P.PtromError):
        P.bs_velocity(_dev(x), _dev(G), 0.02, prec="tf32x3")
    with pytest.raises(P.PtromError):
        P.bs_jvp(_dev(x), _dev(G), 0.02, _dev(np.ones(2 * n)), prec="tf32x3")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,M,split", [(2, 1, 0), (130, 256, 0), (130, 61, 7)])
def test_jphi_tf32x3_edge_shapes(P, n, M, split, prec):
    """Two bodies and one column (one partly empty tile and target block);
    four 64-column slices (N = 256 columns); more splits than a split's
    share of tiles (9 tiles over 7 splits)."""
    x, G = W.two_cluster(n, seed=79)
    phi = W.random_vectors(x.size, M, seed=80).T
    ref = direct.jphi(x, G, 0.02, phi)
    P.set_source_split(split)
    try:
        out = P.bs_jphi(_dev(x), _dev(G), 0.02, _dev(phi), prec=prec).cpu().numpy()
    finally:
        P.set_source_split(0)
    assert _rel(out, ref) <= TOL


def test_jphi_tf32x3_coincident_bodies_delta0(P):
    """delta = 0 with exactly coincident bodies: those pairs are skipped, as
    in every pair sum of the library and the oracle."""
    n = 700
    x, G = _lattice(n, seed=81)
    x[10], x[n + 10] = x[20], x[n + 20]      # body 10 on body 20
    x[300], x[n + 300] = x[301], x[n + 301]  # body 300 on body 301
    phi = W.random_vectors(x.size, 9, seed=82).T
    ref = direct.jphi(x, G, 0.0, phi)
    out = P.bs_jphi(_dev(x), _dev(G), 0.0, _dev(phi), prec="tf32x3").cpu().numpy()
    assert np.all(np.isfinite(out))
    assert _rel(out, ref) <= TOL


def test_jphi_tf32x3_wait_bound_and_recovery(P):
    """Failure path without a fault: the test hook withholds the tile copies,
    every CTA's pipeline waits run out at their bound, the call returns
    PTROM_ETIMEOUT, and the next call on the same context is correct."""
    n, M = 1000, 20
    x, G = W.two_cluster(n, seed=83)
    phi = W.random_vectors(x.size, M, seed=84).T
    P.test_withhold_jphi_tc(True)
    with pytest.raises(P.PtromError) as err:
        P.bs_jphi(_dev(x), _dev(G), 0.02, _dev(phi), prec="tf32x3")
    assert err.value.status == -5  # PTROM_ETIMEOUT
    ref = direct.jphi(x, G, 0.02, phi)
    out = P.bs_jphi(_dev(x), _dev(G), 0.02, _dev(phi), prec="tf32x3").cpu().numpy()
    assert _rel(out, ref) <= TOL


def test_jphi_f16x3_wide_dynamic_range(P):
    """FP16 operands are scaled by powers of two into range: circulations
    spanning 1e-6 .. 1 and basis columns spanning 1e-8 .. 1e3 keep the same
    1e-5 bar (the scales come from the largest |gamma| / delta and the
    largest entry of each column)."""
    n, M = 3000, 12
    x, _ = W.two_cluster(n, seed=85)
    rng = np.random.default_rng(86)
    G = rng.standard_normal(n) * 10.0 ** rng.uniform(-6, 0, n)
    phi = W.random_vectors(x.size, M, seed=87).T * (10.0 ** np.linspace(-8, 3, M))[None, :]
    ref = direct.jphi(x, G, 0.01, phi)
    out = P.bs_jphi(_dev(x), _dev(G), 0.01, _dev(phi), prec="f16x3").cpu().numpy()
    assert np.all(np.isfinite(out))
    for m in range(M):   # every column on its own scale
        assert _rel(out[:, m], ref[:, m]) <= TOL, m
