"""Parity of the CUDA implicit trapezoid FOM step with the FP64 oracle (GPU)."""
import numpy as np
import pytest
import torch

from oracle import direct, fom, qoi
from paper_2103_01983_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2103_01983_gb300 import ptrom
    return ptrom


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _gpu_rollout(P, x0, G, params, steps, prec):
    x = _dev(x0)
    Gt = _dev(G)
    f = P.bs_velocity(x, Gt, params.delta, prec=prec)
    work = P.fom_workspace(params, G.size)
    traj = [x0.copy()]
    stats = []
    for _ in range(steps):
        stats.append(P.fom_step(params, Gt, x, f, work=work))
        traj.append(x.cpu().numpy())
    return np.array(traj), stats, f.cpu().numpy()


def test_small_dense_fp64_matches_oracle_100_steps(P):
    """N=256 disk, delta=0.05, dt=0.01, 100 steps, dense Newton, FP64."""
    x0, G = W.disk(256, seed=0)
    params = P.fom_params(0.01, 0.05, "dense", tol=1e-12, prec="fp64")
    traj, stats, f = _gpu_rollout(P, x0, G, params, 100, "fp64")
    ref, iters = fom.rollout(x0, G, 0.05, 0.01, 100, mode="dense", tol=1e-12)
    err = np.abs(traj - ref).max()
    assert err <= 1e-10, err
    assert all(s["converged"] for s in stats)
    np.testing.assert_allclose(f, direct.velocity(traj[-1], G, 0.05), atol=1e-11)
    # linear impulse to Newton tolerance
    P0 = qoi.linear_impulse(x0, G)
    assert np.abs(qoi.linear_impulse(traj[-1], G) - P0).max() <= 1e-9


@pytest.mark.parametrize("mode", ["blockdiag", "jfnk", "dense"])
def test_modes_fp64_against_oracle(P, mode):
    x0, G = W.disk(300, seed=3)
    params = P.fom_params(0.01, 0.05, mode, tol=1e-13, prec="fp64", gmres_rtol=1e-10)
    traj, stats, _ = _gpu_rollout(P, x0, G, params, 4, "fp64")
    ref, _ = fom.rollout(x0, G, 0.05, 0.01, 4, mode="dense", tol=1e-14)
    assert np.abs(traj - ref).max() <= 1e-11


def test_jfnk_fp32c_against_oracle(P):
    """Two-cluster N=2048: JFNK with FP32 pair sums vs the FP64 dense oracle."""
    x0, G = W.two_cluster(2048, seed=0)
    params = P.fom_params(0.005, 0.02, "jfnk", prec="fp32c")
    traj, stats, _ = _gpu_rollout(P, x0, G, params, 5, "fp32c")
    ref, _ = fom.rollout(x0, G, 0.02, 0.005, 5, mode="jfnk", tol=1e-13, gmres_tol=1e-12)
    rel = np.linalg.norm(traj[-1] - ref[-1]) / np.linalg.norm(ref[-1] - x0)
    assert rel <= 1e-5, rel
    assert all(s["converged"] for s in stats)
    assert all(s["linear_iters"] > 0 for s in stats)


def test_two_vortex_rotation_on_gpu(P):
    d, delta, dt = 0.8, 0.05, 0.1
    x0, G = W.two_vortex(d, 1.0, 1.0)
    params = P.fom_params(dt, delta, "dense", tol=1e-14, prec="fp64")
    traj, _, _ = _gpu_rollout(P, x0, G, params, 10, "fp64")
    omega = 2.0 / (2 * np.pi * (d * d + delta))
    ang = np.unwrap(np.arctan2(traj[:, 3] - traj[:, 2], traj[:, 1] - traj[:, 0]))
    np.testing.assert_allclose(np.diff(ang), 2 * np.arctan(omega * dt / 2), rtol=1e-11)


def test_noconv_and_bad_params(P):
    x0, G = W.disk(64, seed=5)
    params = P.fom_params(0.01, 0.05, "blockdiag", tol=0.0, max_iter=2, prec="fp64")
    x, Gt = _dev(x0), _dev(G)
    f = P.bs_velocity(x, Gt, 0.05, prec="fp64")
    st = P.fom_step(params, Gt, x, f, allow_noconv=True)
    assert not st["converged"] and st["newton_iters"] == 2
    with pytest.raises(P.PtromError) as e:
        P.fom_step(params, Gt, x, f)
    assert e.value.status == P.ENOCONV
    bad = P.fom_params(-1.0, 0.05, "blockdiag")
    with pytest.raises(P.PtromError):
        P.fom_workspace(bad, 64)
    # NaN-seeded state -> ENAN, never a hang
    xn = x.clone()
    xn[3] = float("nan")
    good = P.fom_params(0.01, 0.05, "blockdiag", prec="fp64")
    with pytest.raises(P.PtromError) as e:
        P.fom_step(good, Gt, xn, f.clone())
    assert e.value.status == P.ENAN


def test_full_size_step_residual_sampled(P):
    """N=16384 two clusters, JFNK with FP32C pair sums (the benchmarked step):
    the oracle's FP64 trapezoid residual at 256 sampled bodies is at the level
    the FP32 velocity error allows, and the linear impulse is kept."""
    n, delta, dt = 16384, 0.02, 0.005
    x0, G = W.two_cluster(n, seed=0)
    params = P.fom_params(dt, delta, "jfnk", prec="fp32c")
    x, Gt = _dev(x0), _dev(G)
    f = P.bs_velocity(x, Gt, delta)
    work = P.fom_workspace(params, n)
    rows = np.random.default_rng(40).choice(n, 256, replace=False)
    idx = np.r_[rows, n + rows]
    xp = x0.copy()
    for step in range(3):
        st = P.fom_step(params, Gt, x, f, work=work)
        xn = x.cpu().numpy()
        fo_new = direct.velocity(xn, G, delta, targets=xn[idx])
        fo_old = direct.velocity(xp, G, delta, targets=xp[idx])
        r = xn[idx] - xp[idx] - 0.5 * dt * (fo_new + fo_old)
        step_size = np.linalg.norm(xn[idx] - xp[idx])
        assert np.linalg.norm(r) <= 1e-5 * step_size, (step, np.linalg.norm(r), step_size)
        rel_f = np.linalg.norm(f.cpu().numpy()[idx] - fo_new) / np.linalg.norm(fo_new)
        assert rel_f <= 1e-5
        np.testing.assert_allclose(qoi.linear_impulse(xn, G), qoi.linear_impulse(x0, G), atol=1e-9)
        xp = xn


def test_mixed_precision_scale_up_500_steps(P):
    """The mixed-precision scale-up workload in full: N = 16384 two clusters,
    delta = 0.02, dt = 0.005, 500 implicit steps by JFNK with FP32C pair
    sums.  Every 50 steps the library's velocity at its own state is checked
    against the FP64 oracle on 256 sampled bodies (rel-L2 <= 1e-5); the
    circulation is constant, the linear impulse (an exact invariant of the
    trapezoid rule, kept to the Newton tolerance) drifts by at most 1e-7 of
    sum |Gamma_i| |x_i|, and the angular impulse, which the trapezoid rule
    does not conserve exactly, is reported."""
    n, delta, dt, steps = 16384, 0.02, 0.005, 500
    x0, G = W.two_cluster(n, seed=0)
    params = P.fom_params(dt, delta, "jfnk", prec="fp32c")
    x, Gt = _dev(x0), _dev(G)
    f = P.bs_velocity(x, Gt, delta)
    work = P.fom_workspace(params, n)
    rows = np.random.default_rng(41).choice(n, 256, replace=False)
    idx = np.r_[rows, n + rows]
    scale = float(np.sum(np.abs(G) * np.hypot(x0[:n], x0[n:])))
    P0, I0 = qoi.linear_impulse(x0, G), qoi.angular_impulse(x0, G)
    report = []
    for k in range(1, steps + 1):
        P.fom_step(params, Gt, x, f, work=work)
        if k % 50 == 0:
            xn = x.cpu().numpy()
            fo = direct.velocity(xn, G, delta, targets=xn[idx])
            rel_f = np.linalg.norm(f.cpu().numpy()[idx] - fo) / np.linalg.norm(fo)
            dP = float(np.abs(qoi.linear_impulse(xn, G) - P0).max()) / scale
            dI = abs(qoi.angular_impulse(xn, G) - I0) / abs(I0)
            report.append((k, rel_f, dP, dI))
            assert rel_f <= 1e-5, (k, rel_f)
            assert dP <= 1e-7, (k, dP)
    assert float(Gt.sum()) == pytest.approx(float(G.sum()), abs=0)
    for k, rel_f, dP, dI in report:
        print(f"step {k:3d}: velocity rel-L2 {rel_f:.2e}, linear impulse drift {dP:.1e}, "
              f"angular impulse drift {dI:.1e}")


@pytest.mark.parametrize("restart", [1, 2, 3])
def test_jfnk_short_restart_cycles_fp64(P, restart):
    """GMRES(m) with m = 1..3 and a tight tolerance runs several cycles per
    Newton iteration (restart residual, device least squares of every cycle,
    the pipelined Arnoldi steps); the trajectory still matches the oracle."""
    x0, G = W.disk(300, seed=3)
    params = P.fom_params(0.01, 0.05, "jfnk", tol=1e-13, prec="fp64", gmres_restart=restart,
                          gmres_rtol=1e-10, gmres_max_iter=400)
    traj, stats, _ = _gpu_rollout(P, x0, G, params, 3, "fp64")
    ref, _ = fom.rollout(x0, G, 0.05, 0.01, 3, mode="dense", tol=1e-14)
    assert np.abs(traj - ref).max() <= 1e-11
    for s in stats:
        # more Krylov steps than one cycle holds: restarts happened
        assert s["linear_iters"] > restart * s["newton_iters"]
        # every counted J v is an Arnoldi step or a restart residual
        assert s["linear_iters"] <= s["jvp_evals"] <= 2 * s["linear_iters"]


def test_jfnk_iteration_cap_and_counts(P):
    """gmres_max_iter caps the Krylov steps per solve; the counts the host
    reports are the steps that ran (steps queued ahead and skipped are not
    counted) and the library's event timing holds only those launches."""
    x0, G = W.two_cluster(1024, seed=2)
    x, Gt = _dev(x0), _dev(G)
    capped = P.fom_params(0.005, 0.02, "jfnk", prec="fp64", tol=1e-6, gmres_rtol=1e-14, gmres_max_iter=3)
    f = P.bs_velocity(x, Gt, 0.02, prec="fp64")
    st = P.fom_step(capped, Gt, x, f, allow_noconv=True)
    assert st["linear_iters"] <= 3 * st["newton_iters"]
    params = P.fom_params(0.005, 0.02, "jfnk", prec="fp32c")
    x, f = _dev(x0), P.bs_velocity(_dev(x0), Gt, 0.02)
    work = P.fom_workspace(params, 1024)
    P.timing_read()
    P.timing_enable(True)
    try:
        st = P.fom_step(params, Gt, x, f, work=work)
        torch.cuda.synchronize()
        t = P.timing_read()
    finally:
        P.timing_enable(False)
    assert st["newton_iters"] >= 1 and st["linear_iters"] >= st["newton_iters"]
    assert t["jvp"][1] == st["jvp_evals"]
    assert t["velocity"][1] + t["velocity_selfjac"][1] == st["velocity_evals"]


def test_fp32_krylov_matches_fp64_krylov(P):
    """With FP32 pair sums and a loose GMRES tolerance (1e-4) the Krylov
    arithmetic runs in FP32; a tighter tolerance (1e-6) keeps it in FP64.
    Both Newton iterations stop at the same FP64 residual test
    (||r|| <= 1e-8 max(1, ||x||)), so the trajectories agree to that level."""
    x0, G = W.two_cluster(2048, seed=0)
    p32 = P.fom_params(0.005, 0.02, "jfnk", prec="fp32c", gmres_rtol=1e-4)
    p64 = P.fom_params(0.005, 0.02, "jfnk", prec="fp32c", gmres_rtol=1e-6)
    ta, sa, _ = _gpu_rollout(P, x0, G, p32, 5, "fp32c")
    tb, sb, _ = _gpu_rollout(P, x0, G, p64, 5, "fp32c")
    xnorm = np.linalg.norm(x0)
    assert all(s["converged"] and s["res_norm"] <= 1e-8 * xnorm for s in sa + sb)
    # each end state is within a Newton-tolerance-sized ball of the other
    assert np.linalg.norm(ta[-1] - tb[-1]) <= 1e-6 * xnorm


def _gpu_rollout_inflow(P, x0, G, u, params, steps, prec):
    x = _dev(x0)
    Gt = _dev(G)
    ut = _dev(u)
    f = P.bs_velocity(x, Gt, params.delta, prec=prec)
    work = P.fom_workspace(params, G.size)
    traj = [x0.copy()]
    for _ in range(steps):
        assert P.fom_step(params, Gt, x, f, work=work, u_inf=ut)["converged"]
        traj.append(x.cpu().numpy())
    return np.array(traj), f.cpu().numpy()


@pytest.mark.parametrize("mode", ["blockdiag", "jfnk", "dense"])
def test_inflow_fp64_against_oracle(P, mode):
    """Superimposed inflow (Sec. 6.3) on a non-uniform profile: every Newton
    variant matches the FP64 oracle, and f stays the pair sum."""
    x0, G = W.disk(300, seed=3)
    c = np.linspace(-1.0, 1.0, 300)
    u = np.concatenate([0.4 * np.sin(3.0 * c), 5.0 * np.sqrt(1.125 ** 2 - c * c) + 0.5])
    params = P.fom_params(0.01, 0.05, mode, tol=1e-13, prec="fp64", gmres_rtol=1e-10)
    traj, f = _gpu_rollout_inflow(P, x0, G, u, params, 4, "fp64")
    ref, _ = fom.rollout(x0, G, 0.05, 0.01, 4, mode="dense", tol=1e-14, u_inf=u)
    assert np.abs(traj - ref).max() <= 1e-11
    np.testing.assert_allclose(f, direct.velocity(traj[-1], G, 0.05), atol=1e-11)


def test_mushroom_fom_fp32c_against_oracle(P):
    """The mushroom-cloud workload (Sec. 6.3, N = 500, Gamma_max ends, the
    semicircular inflow), 40 steps of JFNK with FP32 pair sums against the
    FP64 dense oracle; Gamma = 0 moves every body by dt u per step."""
    x0, G, u = W.mushroom(-220.0, 220.0)
    M = W.MUSHROOM
    params = P.fom_params(M["dt"], M["delta"], "jfnk", prec="fp32c")
    traj, _ = _gpu_rollout_inflow(P, x0, G, u, params, 40, "fp32c")
    ref, _ = fom.rollout(x0, G, M["delta"], M["dt"], 40, mode="dense", tol=1e-13, u_inf=u)
    # each FP32C step stops at ||r|| <= 1e-8 ||x|| (positions up to 75 from
    # the origin body), so the gap may grow by that much per step
    bound = 40 * 1e-8 * np.linalg.norm(ref, axis=1).max()
    assert np.abs(traj - ref).max() <= bound, (np.abs(traj - ref).max(), bound)
    params64 = P.fom_params(M["dt"], M["delta"], "blockdiag", tol=1e-13, prec="fp64")
    still, _ = _gpu_rollout_inflow(P, x0, np.zeros(500), u, params64, 3, "fp64")
    np.testing.assert_allclose(still, x0 + np.arange(4)[:, None] * M["dt"] * u, rtol=0, atol=1e-12)


def test_batched_fom_rejects_inflow(P):
    from paper_2103_01983_gb300.ptrom import PtromError
    x0, G = W.disk(64, seed=1)
    params = P.fom_params(0.01, 0.05, "blockdiag", prec="fp64")
    ut = _dev(np.ones(128))
    q = P._with_inflow(params, ut)
    x, Gt = _dev(x0), _dev(G)
    f = P.bs_velocity(x, Gt, 0.05, prec="fp64")
    with pytest.raises(PtromError):
        P.fom_step_batched(q, [Gt], [x], [f], [P.fom_workspace(params, 64)])


@pytest.mark.parametrize("n,prec", [(4096, "fp32c"), (500, "fp64")])
def test_graph_captured_steps_match_step_by_step(P, n, prec):
    """fom_steps replays each block-diagonal Newton step from one captured CUDA
    graph; the same kernels in the same order give the step-by-step result bit
    for bit.  The time per step of both forms is printed."""
    x0, G = W.two_cluster(n, seed=90)
    params = P.fom_params(0.005, 0.02, "blockdiag", prec=prec)
    steps = 20
    Gt = _dev(G)
    xa, xb = _dev(x0), _dev(x0)
    fa, fb = P.bs_velocity(xa, Gt, 0.02, prec=prec), P.bs_velocity(xb, Gt, 0.02, prec=prec)
    wa, wb = P.fom_workspace(params, n), P.fom_workspace(params, n)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    evals = 0
    for _ in range(steps):
        evals += P.fom_step(params, Gt, xa, fa, work=wa)["velocity_evals"]
    e1.record()
    torch.cuda.synchronize()
    t_step = e0.elapsed_time(e1) / steps
    e0.record()
    st = P.fom_steps(params, Gt, xb, fb, steps, work=wb)
    e1.record()
    torch.cuda.synchronize()
    t_graph = e0.elapsed_time(e1) / steps
    print(f"N={n} {prec}: {t_step * 1e3:.0f} us per step by fom_step, {t_graph * 1e3:.0f} us by graph replay")
    assert st["steps_done"] == steps
    assert st["velocity_evals"] == evals
    assert torch.equal(xa, xb) and torch.equal(fa, fb)


def test_graph_captured_steps_stop_at_a_nonconverged_step(P):
    """With fewer captured iterations than a step needs, the rollout stops at
    that step with PTROM_ENOCONV and the library stays usable."""
    n = 1024
    x0, G = W.two_cluster(n, seed=91)
    params = P.fom_params(0.005, 0.02, "blockdiag", prec="fp32c")
    Gt, x = _dev(G), _dev(x0)
    f = P.bs_velocity(x, Gt, 0.02)
    with pytest.raises(P.PtromError) as e:
        P.fom_steps(params, Gt, x, f, 5, iters=1)
    assert e.value.status == P.ENOCONV
    x2 = _dev(x0)
    f2 = P.bs_velocity(x2, Gt, 0.02)
    st = P.fom_steps(params, Gt, x2, f2, 3)
    assert st["steps_done"] == 3
