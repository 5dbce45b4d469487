"""The library's host-side Stage 4 (Alg. 1 greedy sampling and the gappy
operator A = [P Phi_r]^+, Eq. gappySolution) against the oracle, on the CPU
through the C ABI: sampled bodies bit for bit, A to round-off.  Cases: the
hand-derived ones of the oracle pins (including a rank-deficient gappy fit),
random orthonormal and decaying bases, more residual modes than sampled dofs,
and exactly repeated columns."""
import numpy as np
import pytest

from oracle import rom


@pytest.fixture(scope="module")
def P():
    from __graft_entry__ import build_library
    build_library()
    from paper_2103_01983_gb300 import ptrom
    return ptrom


def _phi_r(N, cols):
    M = np.zeros((2 * N, len(cols)))
    for m, col in enumerate(cols):
        for d, v in col.items():
            M[d, m] = v
    return M


def _cases():
    rng = np.random.default_rng(40)
    out = [
        ("hand", _phi_r(6, [{3: -1, 6: 1, 10: 2}, {5: 2, 6: -2, 10: -2}, {0: 1, 3: 1, 10: 1}]), 3),
        ("rank_deficient", _phi_r(5, [{0: 2, 1: 1}, {0: 1, 7: 1}, {0: 5, 3: 1, 9: 0.5}, {8: 0.2}]), 2),
    ]
    for N, Mr, ns in [(30, 4, 6), (200, 20, 40), (150, 40, 15), (120, 24, 30)]:
        Q, _ = np.linalg.qr(rng.standard_normal((2 * N, Mr)))
        out.append((f"orth_{N}_{Mr}_{ns}", Q * 2.0 ** -np.arange(Mr) ** 0.5, ns))
    Q, _ = np.linalg.qr(rng.standard_normal((80, 6)))
    out.append(("repeated_columns", np.concatenate([Q, Q[:, :3]], axis=1), 5))
    return out


@pytest.mark.parametrize("name,Phi_r,ns", _cases(), ids=[c[0] for c in _cases()])
def test_greedy_sample_matches_oracle(P, name, Phi_r, ns):
    N = Phi_r.shape[0] // 2
    s_lib = P.greedy_sample(Phi_r, ns)
    s_or = rom.greedy_sample(Phi_r, ns, N)
    if name == "repeated_columns":
        # from iteration 4 on the new columns repeat earlier ones, so their
        # gappy fit is exact and every body's error is zero up to round-off:
        # any unchosen body is a correct pick; the picks before are unique
        np.testing.assert_array_equal(s_lib[:3], s_or[:3])
        assert len(set(s_lib.tolist())) == ns
        return
    np.testing.assert_array_equal(s_lib, s_or)


@pytest.mark.parametrize("name,Phi_r,ns", _cases(), ids=[c[0] for c in _cases()])
def test_gappy_operator_matches_oracle(P, name, Phi_r, ns):
    N = Phi_r.shape[0] // 2
    s = rom.greedy_sample(Phi_r, ns, N)
    A_lib = P.gappy_operator(Phi_r, s)
    A_or = rom.gappy_operator(Phi_r, s, N)
    scale = max(np.abs(A_or).max(), 1.0)
    np.testing.assert_allclose(A_lib, A_or, atol=1e-10 * scale, rtol=0)


def test_host_sampling_rejects_bad_arguments(P):
    Phi_r = np.zeros((10, 2))
    with pytest.raises(P.PtromError):
        P.greedy_sample(Phi_r, 6)           # n_s > n
    with pytest.raises(P.PtromError):
        P.gappy_operator(Phi_r, [0, 7])      # body id out of range
