"""Projection-tree reduced-order model, written plainly from the paper.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Pieces, in the paper's order and notation:

* ``pod``               -- Sec. 3.1: Phi = leading M left singular vectors of
                           the snapshot matrix (thin SVD).
* ``QuadTree``          -- Barnes-Hut quadtree (Sec. 4) over 2-D points, one
                           body per leaf.
* ``cluster_tables``    -- Alg. 2 WeightedMean (node surrogates, Def. 1),
                           Alg. 2 FindClusters/Traverse with Alg. 3 checkPrune
                           (Barnes-Hut or neighbour criterion, Def. 2), and
                           UniqueSearch, all in the weighted POD space W = Phi s.
* ``hyperpair``         -- Alg. 5: velocity, inexact Jacobian blocks and
                           residual at a set of targets against their clusters.
* ``lspg_tier2``        -- Stage 3: LSPG (Eq. GNLinearLeastSquares/GNUpdate)
                           over all targets with clustered sources, collecting
                           the residual at every Gauss-Newton iterate.
* ``greedy_sample``     -- Alg. 1 (greedy sampling of bodies).
* ``gappy_operator``    -- A = [P Phi_r]^+ (Eq. gappySolution).
* ``ptrom_online``      -- Alg. 4 (Gauss-Newton over HyperPair at the sampled
                           bodies).

Readings where the paper is silent or garbled (each used by the CUDA path too):
  R1 snapshots are the states themselves, S = [x^1 .. x^Nt] (Sec. 3.1 as
     printed), not offsets from x^0: the leading POD mode is then close to the
     mean configuration, so the weighted POD space W = Phi sigma is close to
     the bodies' positions and its quadtree groups physically neighbouring
     bodies.  (With offsets W holds only displacement patterns and the
     clustering loses most of its accuracy.)
  R2 singular-vector sign: each column's largest-magnitude entry is positive.
  R3 tree: square root cell (bounding box padded to its longest side), midpoint
     split into four, leaf = one body, depth cap 40 (then a leaf may hold more).
  R4 weighted means use |Gamma| (identical to Def. 1 when a node's
     circulations share a sign; avoids dividing by ~0 for mixed signs);
     Gamma~ of a node is the signed sum.
  R5 Barnes-Hut test: distance in W space from the target's point to the
     node's |Gamma|-weighted centroid; a node containing the target is never
     pruned; d = 0 never prunes; "<= theta" prunes.
  R6 neighbour test: the interval overlap of Alg. 3 with its strict
     inequalities, H = target leaf box grown by p_c * (leaf width).
  R7 an unpruned leaf contributes its bodies one by one, never the target
     itself (j != i of Eq. 1); a pruned node holding one body is that body.
  R8 x^QT = x^0_QT + Phi~ xhat and x^GP = x^0 + Phi xhat with the total xhat
     (Alg. 5's "Delta xhat" notation is read as the current coordinates).
  R9 Gauss-Newton runs while eps > tol (Alg. 4 prints "<"), at most 100
     iterations; the update is applied before eps is tested (Alg. 4 order).
     eps is the gradient of the objective being minimised relative to its
     value at the step's first iterate: ||C^T r|| for LSPG (Tier II, as
     printed) and ||(A C)^T (A r)|| for the hyper-reduced problem (Tier III).
     Alg. 4 prints the unweighted ||Phi^T J^T r||, which does not vanish at
     the minimiser of ||A r|| when M_r > M, so that test could never be met.
  R10 A = [P Phi_r]^+ multiplies both C and D (Alg. 4 as printed).
  R11 f~^0 is HyperPair's velocity at xhat = 0; the velocity carried to the
      next step is the last one HyperPair computed in the step (Alg. 5 stores
      it at every call).
  R12 residual snapshots: every Gauss-Newton iterate's residual (first
      included), every step, every training parameter.
  R13 Alg. 1: n_c = min(M_r, n_d), n_a = n - |N|, n_it = min(n_c, n_a),
      n_ci = floor(n_c/n_it) + [i <= n_c mod n_it],
      n_ai = floor(n_a/n_it) + [i <= n_a mod n_it]; bodies are chosen on
      every iteration (i = 1 included); ties go to the lowest body index.
  R14 the inexact residual Jacobian of Alg. 5 keeps the per-target 2x2
      blocks d f~_i / d x~_i only: J = I - dt/2 blockdiag(D~).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * np.pi


# ------------------------------------------------------------------ POD
def pod(S, M):
    """Leading M left singular vectors and values of S (N_d x K), Sec. 3.1:
    S = U Sigma V^T, Phi = [U^1 .. U^M] (thin SVD, the paper's definition)."""
    U, sigma, _ = np.linalg.svd(S, full_matrices=False)
    U, sigma = U[:, :M], sigma[:M]
    if np.any(sigma == 0.0):
        raise ValueError("POD rank M exceeds the rank of the snapshots")
    # R2: sign convention
    idx = np.argmax(np.abs(U), axis=0)
    sgn = np.sign(U[idx, np.arange(U.shape[1])])
    sgn[sgn == 0] = 1.0
    return U * sgn, sigma


# ------------------------------------------------------------------ quadtree
@dataclass
class Node:
    id: int
    box: tuple            # (xmin, xmax, ymin, ymax)
    members: list
    depth: int
    children: list = field(default_factory=list)

    @property
    def width(self):
        return max(self.box[1] - self.box[0], self.box[3] - self.box[2])

    @property
    def is_leaf(self):
        return not self.children


class QuadTree:
    """Barnes-Hut quadtree over points P (N x 2), Sec. 4 with reading R3."""

    def __init__(self, P, max_depth=40):
        self.P = np.asarray(P, dtype=np.float64)
        lo = self.P.min(axis=0)
        side = float((self.P.max(axis=0) - lo).max())
        if side == 0.0:
            side = 1.0
        self.nodes = []
        self.leaf_of = np.full(len(self.P), -1, dtype=np.int64)
        self.max_depth = max_depth
        self.root = self._build(list(range(len(self.P))), (lo[0], lo[0] + side, lo[1], lo[1] + side), 0)

    def _build(self, members, box, depth):
        node = Node(len(self.nodes), box, members, depth)
        self.nodes.append(node)
        if len(members) <= 1 or depth >= self.max_depth:
            for m in members:
                self.leaf_of[m] = node.id
            return node
        xm = 0.5 * (box[0] + box[1])
        ym = 0.5 * (box[2] + box[3])
        quads = [[], [], [], []]
        for m in members:
            q = (1 if self.P[m, 0] >= xm else 0) + (2 if self.P[m, 1] >= ym else 0)
            quads[q].append(m)
        boxes = [(box[0], xm, box[2], ym), (xm, box[1], box[2], ym),
                 (box[0], xm, ym, box[3]), (xm, box[1], ym, box[3])]
        for q in range(4):
            if quads[q]:
                node.children.append(self._build(quads[q], boxes[q], depth + 1))
        return node


# ------------------------------------------------------------------ clustering
@dataclass
class Clusters:
    """Unique source clusters and, per target, the list of cluster indices."""
    members: list            # per cluster: list of body ids
    Gt: np.ndarray           # Gamma~ per cluster (signed sum)
    Phit: np.ndarray         # (2 Nc, M): rows [chi rows of all clusters; psi rows]
    x0t: np.ndarray          # (2 Nc,): x^0_QT in the [chi; psi] layout
    lists: list              # per target (in `targets` order): cluster indices
    targets: np.ndarray
    pruned: list = field(default_factory=list)   # per target: ids of the pruned tree nodes


def _weighted_mean(members, Gamma, rows):
    w = np.abs(Gamma[members])
    if w.sum() == 0.0:
        w = np.ones_like(w)
    return (w[:, None] * rows[members]).sum(axis=0) / w.sum()


def cluster_tables(Phi, sigma, x0, Gamma, targets, criterion="bh", theta=0.5, p_c=1.0,
                   max_depth=40, W=None):
    """Alg. 2 (WeightedMean, FindClusters/Traverse, UniqueSearch) with Alg. 3.

    The tree lives in the weighted POD space W = Phi sigma (Sec. 4.1.1):
    body i is the point (W_i, W_{i+N}).  W may be passed in precomputed (the
    neighbour test compares box edges that coincide in exact arithmetic, so
    its outcome can depend on how W was rounded)."""
    N = Gamma.size
    M = Phi.shape[1]
    if W is None:
        W = Phi @ sigma
    pts = np.stack([W[:N], W[N:]], axis=1)
    tree = QuadTree(pts, max_depth=max_depth)
    # WeightedMean: |Gamma|-weighted centroid of each node in W (R4)
    cen = np.array([_weighted_mean(nd.members, Gamma, pts) for nd in tree.nodes])
    keys, index, lists, pruned = [], {}, [], []
    for i in targets:
        own_leaf = tree.nodes[tree.leaf_of[i]]
        out, pr = [], []
        stack = [tree.root]
        while stack:
            nd = stack.pop()
            contains = i in nd.members
            if not contains and _prune(nd, cen[nd.id], pts[i], own_leaf, criterion, theta, p_c):
                out.append(tuple(sorted(nd.members)))
                pr.append(nd.id)
                continue
            if nd.is_leaf:
                out.extend((m,) for m in nd.members if m != i)   # R7
            else:
                stack.extend(reversed(nd.children))
        # UniqueSearch: a cluster is identified by its member set
        li = []
        for key in out:
            if key not in index:
                index[key] = len(keys)
                keys.append(key)
            li.append(index[key])
        lists.append(li)
        pruned.append(pr)
    Nc = len(keys)
    members = [list(k) for k in keys]
    Gt = np.array([Gamma[m].sum() for m in members])
    rows_chi, rows_psi = Phi[:N], Phi[N:]
    xchi, xpsi = x0[:N], x0[N:]
    Phit = np.zeros((2 * Nc, M))
    x0t = np.zeros(2 * Nc)
    for c, m in enumerate(members):
        if len(m) == 1:
            Phit[c], Phit[Nc + c] = rows_chi[m[0]], rows_psi[m[0]]
            x0t[c], x0t[Nc + c] = xchi[m[0]], xpsi[m[0]]
        else:
            Phit[c] = _weighted_mean(m, Gamma, rows_chi)
            Phit[Nc + c] = _weighted_mean(m, Gamma, rows_psi)
            x0t[c] = _weighted_mean(m, Gamma, xchi[:, None])[0]
            x0t[Nc + c] = _weighted_mean(m, Gamma, xpsi[:, None])[0]
    return Clusters(members, Gt, Phit, x0t, lists, np.asarray(targets), pruned), tree


def _prune(nd, centroid, s_i, own_leaf, criterion, theta, p_c):
    """Alg. 3 checkPrune (readings R5, R6)."""
    if criterion == "bh":
        d = float(np.linalg.norm(centroid - s_i))
        return d > 0.0 and nd.width / d <= theta
    w_t = own_leaf.width
    h = (own_leaf.box[0] - p_c * w_t, own_leaf.box[1] + p_c * w_t,
         own_leaf.box[2] - p_c * w_t, own_leaf.box[3] + p_c * w_t)
    b = nd.box
    overlap_x = h[1] > b[0] and h[0] < b[1]
    overlap_y = h[3] > b[2] and h[2] < b[3]
    return not (overlap_x and overlap_y)


def reload_parameters(cl: Clusters, Phi, x0, Gamma):
    """Cluster quantities for a new parameter (Gamma, x^0) from the stored
    memberships, no retraining (Sec. 5.2)."""
    N = Gamma.size
    Nc = len(cl.members)
    Gt = np.array([Gamma[m].sum() for m in cl.members])
    Phit = np.zeros_like(cl.Phit)
    x0t = np.zeros(2 * Nc)
    for c, m in enumerate(cl.members):
        if len(m) == 1:
            Phit[c], Phit[Nc + c] = Phi[m[0]], Phi[N + m[0]]
            x0t[c], x0t[Nc + c] = x0[m[0]], x0[N + m[0]]
        else:
            Phit[c] = _weighted_mean(m, Gamma, Phi[:N])
            Phit[Nc + c] = _weighted_mean(m, Gamma, Phi[N:])
            x0t[c] = _weighted_mean(m, Gamma, x0[:N, None])[0]
            x0t[Nc + c] = _weighted_mean(m, Gamma, x0[N:, None])[0]
    return Clusters(cl.members, Gt, Phit, x0t, cl.lists, cl.targets, cl.pruned)


# ------------------------------------------------------------------ Alg. 5
def hyperpair(xhat, cl: Clusters, Phi_t, x0_t, delta):
    """Velocity f~ (2 nt) and inexact blocks D~ (3, nt) at the targets.

    Phi_t (2 nt, M) and x0_t (2 nt) are the targets' rows of Phi and x^0 in
    the [chi; psi] layout.  x^GP = x0_t + Phi_t xhat, x^QT = x^0_QT + Phi~ xhat."""
    nt = len(cl.lists)
    Nc = len(cl.members)
    xg = x0_t + Phi_t @ xhat
    xq = cl.x0t + cl.Phit @ xhat
    f = np.zeros(2 * nt)
    D = np.zeros((3, nt))
    for i, li in enumerate(cl.lists):
        if not li:
            continue
        li = np.asarray(li)
        a = xg[i] - xq[li]
        b = xg[nt + i] - xq[Nc + li]
        g = cl.Gt[li] / TWO_PI
        keep = ~((a == 0.0) & (b == 0.0))
        a, b, g = a[keep], b[keep], g[keep]
        s = a * a + b * b + delta
        f[i] = np.sum(g * (-b) / s)
        f[nt + i] = np.sum(g * a / s)
        D[0, i] = np.sum(g * 2.0 * a * b / s**2)
        D[1, i] = np.sum(g * (-1.0 / s + 2.0 * b * b / s**2))
        D[2, i] = np.sum(g * (1.0 / s - 2.0 * a * a / s**2))
    return f, D


def jacobian_rows(D, Phi_t, dt):
    """C = (I - dt/2 blockdiag(D~)) Phi_t  (R14)."""
    nt = D.shape[1]
    top, bot = Phi_t[:nt], Phi_t[nt:]
    h = 0.5 * dt
    C_top = top - h * (D[0][:, None] * top + D[1][:, None] * bot)
    C_bot = bot - h * (D[2][:, None] * top - D[0][:, None] * bot)
    return np.concatenate([C_top, C_bot])


def target_rows(Phi, x0, targets):
    N = x0.size // 2
    idx = np.concatenate([targets, N + np.asarray(targets)])
    return Phi[idx], x0[idx]


# ------------------------------------------------------------------ Tier II
def _inflow_rows(u_inf, targets, n_dofs):
    """The targets' rows of the superimposed inflow u (Sec. 6.3), or 0."""
    if u_inf is None:
        return np.zeros(n_dofs)
    u = np.asarray(u_inf, dtype=np.float64)
    return u[np.concatenate([targets, u.size // 2 + np.asarray(targets)])]


def lspg_tier2(cl: Clusters, Phi, x0, delta, dt, steps, tol=1e-4, max_gn=100, u_inf=None):
    """Stage 3: LSPG over all targets with clustered sources.  Returns the
    reduced trajectory (steps+1, M) and the residual snapshots (R12).
    u_inf: optional constant inflow velocity per dof (Sec. 6.3), added to
    the right-hand side, so the residual gains -dt u at the targets."""
    Phi_t, x0_t = target_rows(Phi, x0, cl.targets)
    u_t = _inflow_rows(u_inf, cl.targets, Phi_t.shape[0])
    M = Phi.shape[1]
    xhat = np.zeros(M)
    f_prev, _ = hyperpair(xhat, cl, Phi_t, x0_t, delta)
    traj = [xhat.copy()]
    snaps = []
    for _ in range(steps):
        xprev = xhat.copy()
        first = None
        for k in range(max_gn):
            f, D = hyperpair(xhat, cl, Phi_t, x0_t, delta)
            r = Phi_t @ (xhat - xprev) - 0.5 * dt * (f + f_prev) - dt * u_t
            snaps.append(r.copy())
            C = jacobian_rows(D, Phi_t, dt)
            dx = np.linalg.lstsq(C, -r, rcond=None)[0]
            g = np.linalg.norm(C.T @ r)
            first = g if first is None else first
            xhat = xhat + dx
            eps = g / first if first > 0 else 0.0
            if (eps <= tol and k > 0) or first == 0.0:     # R9
                break
        f_prev = f
        traj.append(xhat.copy())
    return np.array(traj), np.array(snaps).T


# ------------------------------------------------------------------ Alg. 1
def greedy_sample(Phi_r, n_samples, N, preseeded=()):
    """Greedy choice of sampled bodies (Alg. 1, reading R13).  Phi_r is
    (2N, M_r); returns the body indices in the order they were chosen."""
    M_r = Phi_r.shape[1]
    chosen = list(preseeded)
    n_a = n_samples - len(chosen)
    n_d = 2 * n_samples
    n_c = min(M_r, n_d)
    n_it = min(n_c, n_a)
    n_b = 0
    for i in range(1, n_it + 1):
        n_ci = n_c // n_it + (1 if i <= n_c % n_it else 0)
        n_ai = n_a // n_it + (1 if i <= n_a % n_it else 0)
        R = Phi_r[:, n_b:n_b + n_ci]
        if i > 1 and n_b > 0:
            dofs = np.concatenate([chosen, N + np.asarray(chosen)]).astype(int)
            coef = np.linalg.lstsq(Phi_r[dofs, :n_b], R[dofs], rcond=None)[0]
            R = R - Phi_r[:, :n_b] @ coef
        err = (R[:N] ** 2).sum(axis=1) + (R[N:] ** 2).sum(axis=1)
        for _ in range(n_ai):
            err_masked = err.copy()
            err_masked[chosen] = -np.inf
            best = int(np.argmax(err_masked))      # first maximum: lowest index
            chosen.append(best)
        n_b += n_ci
    return np.array(chosen, dtype=np.int64)


def gappy_operator(Phi_r, sampled, N):
    """A = [P Phi_r]^+ (Eq. gappySolution); P picks both dofs of each body."""
    dofs = np.concatenate([sampled, N + np.asarray(sampled)])
    return np.linalg.pinv(Phi_r[dofs])


# ------------------------------------------------------------------ Alg. 4
def ptrom_online(cl: Clusters, Phi, x0, A, delta, dt, steps, tol=1e-4, max_gn=100, u_inf=None):
    """Online Gauss-Newton (Alg. 4) over HyperPair at the sampled bodies
    (cl.targets).  Returns the reduced trajectory (steps+1, M) and the
    Gauss-Newton iteration counts.  u_inf: as in ``lspg_tier2``."""
    Phi_t, x0_t = target_rows(Phi, x0, cl.targets)
    u_t = _inflow_rows(u_inf, cl.targets, Phi_t.shape[0])
    M = Phi.shape[1]
    xhat = np.zeros(M)
    f_prev, _ = hyperpair(xhat, cl, Phi_t, x0_t, delta)   # R11
    traj = [xhat.copy()]
    iters = []
    for _ in range(steps):
        xprev = xhat.copy()
        first = None
        k = 0
        while True:
            f, D = hyperpair(xhat, cl, Phi_t, x0_t, delta)
            r = Phi_t @ (xhat - xprev) - 0.5 * dt * (f + f_prev) - dt * u_t
            C = jacobian_rows(D, Phi_t, dt)
            AC, Ar = A @ C, A @ r                                    # R10
            dx = np.linalg.lstsq(AC, -Ar, rcond=None)[0]
            g = np.linalg.norm(AC.T @ Ar)                            # R9
            first = g if first is None else first
            xhat = xhat + dx
            k += 1
            eps = g / first if first > 0 else 0.0
            if (eps <= tol and k > 1) or first == 0.0 or k >= max_gn:     # R9
                break
        f_prev = f
        iters.append(k)
        traj.append(xhat.copy())
    return np.array(traj), np.array(iters)


def reconstruct(xhat, Phi, x0, rows=None):
    """x = x^0 + Phi xhat on the requested dofs (Sec. 5.3)."""
    if rows is None:
        return x0 + Phi @ xhat
    return x0[rows] + Phi[rows] @ xhat
