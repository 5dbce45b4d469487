"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws numbers (NumPy PCG64 via ``default_rng``) in a fixed
order and arranges them in the paper's state layout (Sec. 2, Eq. 3:
x = [chi_1..chi_N, psi_1..psi_N]).  It contains none of the method's
arithmetic (no velocity, Jacobian, solver or reduction code), so the CUDA path
and the oracle can both consume it without sharing any implementation.

Workloads (all synthetic; the paper's experiments are synthetic too):

* ``disk``      -- N bodies uniform in the unit disk, Gamma ~ N(0,1) shifted so
                   that sum(Gamma) = 1 (the small FP64 FOM + PTROM case,
                   N=256, delta=0.05, dt=0.01).
* ``two_cluster`` -- two Gaussian vortex clusters (std 0.1) whose centres are a
                   distance ``sep`` apart on the chi axis; cluster A carries total
                   circulation 1, cluster B total circulation ``ratio``
                   (N=16384 / 65536 scale-up and differentiation cases).
* ``param_lhs`` -- Latin-hypercube samples of (sep, ratio) in
                   [0.8,1.2] x [0.5,2.0] for the parametric PTROM case.
* ``batch_sizes`` -- log-uniform N in [4096, 131072] for the batched case.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "disk",
    "two_cluster",
    "param_lhs",
    "batch_instances",
    "random_vectors",
    "two_vortex",
]


def disk(n: int = 256, seed: int = 0):
    """Bodies uniform in the unit disk; Gamma ~ N(0,1) shifted to sum to 1.

    Draw order: theta ~ U(0, 2 pi) [n], u ~ U(0,1) [n] (radius = sqrt(u)),
    g ~ N(0,1) [n].  Returns (x [2n] in the layout [chi..., psi...], Gamma [n]).
    """
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.0, 2.0 * np.pi, n)
    rho = np.sqrt(rng.uniform(0.0, 1.0, n))
    g = rng.standard_normal(n)
    g = g - g.mean() + 1.0 / n
    x = np.concatenate([rho * np.cos(theta), rho * np.sin(theta)])
    return x.astype(np.float64), g.astype(np.float64)


def _cluster_offsets(n: int, seed: int):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 2))


def two_cluster(n: int = 16384, seed: int = 0, sep: float = 1.0,
                ratio: float = 1.0, std: float = 0.1):
    """Two Gaussian clusters of n/2 bodies each.

    Body k < n/2 belongs to cluster A centred at (-sep/2, 0), the rest to
    cluster B centred at (+sep/2, 0).  Offsets are std * z with one draw
    z ~ N(0,1)^(n x 2) (seed fixed), so the same seed gives the same body
    identities for every (sep, ratio): common random numbers across
    parameters.  Cluster A carries total circulation 1 and cluster B total
    circulation ``ratio``, spread evenly over its bodies.
    """
    if n % 2:
        raise ValueError("two_cluster needs an even n")
    z = _cluster_offsets(n, seed)
    h = n // 2
    cx = np.where(np.arange(n) < h, -0.5 * sep, 0.5 * sep)
    chi = cx + std * z[:, 0]
    psi = std * z[:, 1]
    g = np.where(np.arange(n) < h, 1.0 / h, ratio / h)
    return np.concatenate([chi, psi]).astype(np.float64), g.astype(np.float64)


def param_lhs(count: int, seed: int, sep_range=(0.8, 1.2), ratio_range=(0.5, 2.0)):
    """Latin-hypercube samples of (sep, ratio): one point per stratum per axis.

    Draw order: permutation for axis 0, permutation for axis 1, then the
    in-stratum uniforms [count x 2].
    """
    rng = np.random.default_rng(seed)
    p0 = rng.permutation(count)
    p1 = rng.permutation(count)
    u = rng.uniform(0.0, 1.0, (count, 2))
    a = (p0 + u[:, 0]) / count
    b = (p1 + u[:, 1]) / count
    sep = sep_range[0] + a * (sep_range[1] - sep_range[0])
    ratio = ratio_range[0] + b * (ratio_range[1] - ratio_range[0])
    return np.stack([sep, ratio], axis=1)


def batch_instances(count: int = 64, seed: int = 3, n_lo: int = 4096,
                    n_hi: int = 131072, even: bool = True):
    """Per-instance (N, sep, ratio) for the batched case.

    Draw order: log N ~ U(ln n_lo, ln n_hi) [count], sep ~ U(0.8,1.2) [count],
    ratio ~ U(0.5, 2.0) [count].  N is rounded to the nearest integer (and to
    the nearest even integer when ``even``, since the two-cluster layout splits
    bodies in halves).
    """
    rng = np.random.default_rng(seed)
    logn = rng.uniform(np.log(n_lo), np.log(n_hi), count)
    sep = rng.uniform(0.8, 1.2, count)
    ratio = rng.uniform(0.5, 2.0, count)
    n = np.rint(np.exp(logn)).astype(np.int64)
    if even:
        n = 2 * np.rint(n / 2.0).astype(np.int64)
    return n, sep, ratio


def random_vectors(n_d: int, count: int, seed: int):
    """``count`` standard-normal vectors of length n_d, shape [count, n_d]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((count, n_d))


def two_vortex(d: float = 1.0, g1: float = 1.0, g2: float = 1.0):
    """Two point vortices on the chi axis, a distance d apart, centred at 0."""
    x = np.array([-0.5 * d, 0.5 * d, 0.0, 0.0], dtype=np.float64)
    return x, np.array([g1, g2], dtype=np.float64)


# --------------------------------------------------------------- the paper's
# vortex-pair experiment (Sec. 6.2): N bodies evenly spaced on the diagonal
# from (-52.93, -52.93) to (52.93, 52.93); the two end bodies carry the
# parameter circulations mu = (Gamma_1, Gamma_N) in [0.25, 1] x Gamma_max
# (Gamma_max = 255), every other body 0.01; delta = 0.2121 (the initial axis
# spacing), dt = 0.01, t in [0, 5].
VORTEX_PAIR = {"n": 500, "half_width": 52.93, "gamma_max": 255.0, "gamma_weak": 0.01, "delta": 0.2121,
               "dt": 0.01, "steps": 500, "lo": 0.25}


def vortex_pair(g1: float, gN: float, n: int = VORTEX_PAIR["n"]):
    """State [chi..., psi...] and circulations of the vortex-pair experiment."""
    s = np.linspace(-VORTEX_PAIR["half_width"], VORTEX_PAIR["half_width"], n)
    x = np.concatenate([s, s])
    G = np.full(n, VORTEX_PAIR["gamma_weak"])
    G[0], G[-1] = g1, gN
    return x, G


def vortex_pair_params(seed: int = 0):
    """Training mu (4 Latin-hypercube points) and the 6 x 6 query grid over
    [lo, 1] x Gamma_max in both circulations (Sec. 6.2)."""
    lo, gmax = VORTEX_PAIR["lo"], VORTEX_PAIR["gamma_max"]
    train = lo * gmax + param_lhs(4, seed, (0.0, 1.0), (0.0, 1.0)) * (1.0 - lo) * gmax
    g = np.linspace(lo * gmax, gmax, 6)
    query = np.array([(a, b) for a in g for b in g])
    return train, query


# --------------------------------------------------------------- the paper's
# mushroom-cloud experiment (Sec. 6.3): N bodies evenly spaced on the line
# psi = -10 from chi = -37.43 to 37.43 (spacing 0.15); end circulations
# mu = (Gamma_1, Gamma_N) in [-1, -0.5] x [0.5, 1] x Gamma_max (Gamma_max =
# 220, opposite senses), every other body 0.01; delta = 0.15 (the initial
# spacing, taken as the additive constant as for the vortex pair), dt =
# 0.005, t in [0, 5].  Every body also carries a constant inflow velocity
# (0, 5 sqrt(1.125^2 - s_i^2) + 0.5), s_i = linspace(-1, 1, N)_i: a
# semicircular profile over the body index.
MUSHROOM = {"n": 500, "half_width": 37.43, "psi0": -10.0, "gamma_max": 220.0, "gamma_weak": 0.01,
            "delta": 0.15, "dt": 0.005, "steps": 1000, "lo": 0.5}


def mushroom(g1: float, gN: float, n: int = MUSHROOM["n"]):
    """State [chi..., psi...], circulations and inflow [u_chi..., u_psi...]
    of the mushroom-cloud experiment."""
    s = np.linspace(-MUSHROOM["half_width"], MUSHROOM["half_width"], n)
    x = np.concatenate([s, np.full(n, MUSHROOM["psi0"])])
    G = np.full(n, MUSHROOM["gamma_weak"])
    G[0], G[-1] = g1, gN
    c = np.linspace(-1.0, 1.0, n)
    u = np.concatenate([np.zeros(n), 5.0 * np.sqrt(1.125 ** 2 - c * c) + 0.5])
    return x, G, u


def mushroom_params(seed: int = 0):
    """Training mu (4 Latin-hypercube points) and the 6 x 6 query grid over
    [-1, -lo] x [lo, 1] x Gamma_max (Sec. 6.3)."""
    lo, gmax = MUSHROOM["lo"], MUSHROOM["gamma_max"]
    unit = param_lhs(4, seed, (0.0, 1.0), (0.0, 1.0))
    train = np.stack([-gmax + unit[:, 0] * (1.0 - lo) * gmax, lo * gmax + unit[:, 1] * (1.0 - lo) * gmax], axis=1)
    ga, gb = np.linspace(-gmax, -lo * gmax, 6), np.linspace(lo * gmax, gmax, 6)
    query = np.array([(a, b) for a in ga for b in gb])
    return train, query


# --------------------------------------------------------------- the paper's
# single-vortex reproductive experiment (Sec. 6.4, Table 1): N bodies on the
# line linspace(-N, N, N) in both coordinates, delta = 0, every body 0.01
# except the centre body (index N // 2), which carries Gamma_center; dt and
# the time range per N, 2000 steps in every case.
SINGLE_VORTEX = {  # N: (dt, Gamma_center, t_final)
    100: (0.01, 500.0, 20.0), 500: (2.5e-3, 1e4, 5.0), 1000: (2.5e-4, 1e5, 0.5), 2000: (1.25e-4, 2e5, 0.25),
    3000: (1e-4, 3e5, 0.2), 4000: (7.5e-5, 4e5, 0.15), 5000: (5e-5, 6.75e5, 0.1)}


def single_vortex(n: int):
    """State [chi..., psi...], circulations, dt and step count of Table 1's case n."""
    dt, gc, tf = SINGLE_VORTEX[n]
    s = np.linspace(-float(n), float(n), n)
    G = np.full(n, 0.01)
    G[n // 2] = gc
    return np.concatenate([s, s]), G, dt, int(round(tf / dt))
