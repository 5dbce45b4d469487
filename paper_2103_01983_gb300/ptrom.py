"""Thin Python binding of libptrom.so (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors must be CUDA float64 tensors on the current device; outputs
are allocated with torch (device memory) unless passed in.  Calls are
enqueued on torch's current CUDA stream unless ``stream`` is given.

The library is loaded on import and a missing or unloadable library raises
immediately: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libptrom.so")

FP32C = 0
FP64 = 1
TF32X3 = 2   # bs_jphi only: tensor cores, TF32 hi/lo splits
F16X3 = 3    # bs_jphi only: tensor cores, scaled FP16 hi/lo splits (delta > 0)
_PREC = {"fp32c": FP32C, "fp64": FP64, "tf32x3": TF32X3, "f16x3": F16X3, FP32C: FP32C, FP64: FP64, TF32X3: TF32X3,
         F16X3: F16X3}

_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double


class PtromError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ptrom status {status}: {msg}")
        self.status = status


JAC_BLOCKDIAG = 0
JAC_DENSE = 1
JAC_JFNK = 2
_JAC = {"blockdiag": JAC_BLOCKDIAG, "dense": JAC_DENSE, "jfnk": JAC_JFNK}

# status codes (include/ptrom.h)
OK, EINVAL, ECUDA, ENOCONV, ENAN, ETIMEOUT, ENOMEM = 0, -1, -2, -3, -4, -5, -6


class FomParams(ctypes.Structure):
    """Mirror of ptrom_fom_params."""
    _fields_ = [("dt", _d), ("delta", _d), ("tol", _d), ("max_iter", _i), ("jac_mode", _i),
                ("p_it", _i), ("prec", _i), ("gmres_restart", _i), ("gmres_max_iter", _i),
                ("gmres_rtol", _d), ("u_inf", _vp)]


class FomStats(ctypes.Structure):
    """Mirror of ptrom_fom_stats."""
    _fields_ = [("newton_iters", _i), ("linear_iters", _i), ("velocity_evals", _i),
                ("jvp_evals", _i), ("res_norm", _d), ("res_norm0", _d)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def fom_params(dt, delta, mode="blockdiag", tol=None, max_iter=100, p_it=None, prec="fp32c",
               gmres_restart=30, gmres_max_iter=200, gmres_rtol=1e-4):
    """Build a FomParams; tol defaults to 1e-12 (FP64) or 1e-8 (FP32C).

    p_it defaults to 1 (refresh every Newton iteration) for the dense and
    block-diagonal Jacobians; for JFNK the self blocks only precondition GMRES
    (the Krylov products use the exact J at the current iterate), so they are
    refreshed once per time step (p_it = max_iter)."""
    if p_it is None:
        p_it = max_iter if mode == "jfnk" else 1
    if tol is None:
        tol = 1e-12 if _prec(prec) == FP64 else 1e-8
    return FomParams(float(dt), float(delta), float(tol), int(max_iter), _JAC[mode], int(p_it),
                     _prec(prec), int(gmres_restart), int(gmres_max_iter), float(gmres_rtol))


class ModelDesc(ctypes.Structure):
    """Mirror of ptrom_model_desc (host arrays are pointers)."""
    _fields_ = [("n_s", _i), ("M", _i), ("M_r", _i), ("N_c", _i), ("dt", _d), ("delta", _d),
                ("tol", _d), ("max_gn", _i), ("qr_prec", _i),
                ("phi_s", _vp), ("x0_s", _vp), ("phi_c", _vp), ("x0_c", _vp), ("gamma_c", _vp),
                ("A", _vp), ("off", _vp), ("idx", _vp), ("u_s", _vp)]


class PtromStats(ctypes.Structure):
    _fields_ = [("gn_iters", ctypes.c_longlong), ("steps", ctypes.c_longlong), ("noconv", _i),
                ("max_iters", _i)]


class BuildParams(ctypes.Structure):
    """Mirror of ptrom_build_params."""
    _fields_ = [("M", _i), ("M_r", _i), ("n_s", _i), ("criterion", _i), ("theta", _d), ("p_c", _d),
                ("steps", _i), ("tol", _d), ("max_gn", _i), ("qr_prec", _i), ("fom", FomParams),
                ("u_infs", _vp), ("snapshots", _vp)]


class BuildInfo(ctypes.Structure):
    """Mirror of ptrom_build_info."""
    _fields_ = [("n_snapshots", _i), ("n_res_snapshots", _i), ("N_c", _i), ("N_c_all", _i),
                ("mean_list", _d), ("mean_list_all", _d), ("sigma_ratio", _d), ("seconds_fom", _d),
                ("seconds_pod", _d), ("seconds_tree", _d), ("seconds_tier2", _d), ("seconds_sample", _d)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "ptrom_last_error": ([ctypes.c_char_p, ctypes.c_size_t], _i),
        "ptrom_version": ([], _i),
        "ptrom_set_source_split": ([_i], _i),
        "ptrom_set_split_mode": ([_i], _i),
        "ptrom_tune_pairs": ([_i, _i, _d, _vp], _i),
        "ptrom_set_autotune": ([_i], _i),
        "ptrom_autotune_reset": ([], _i),
        "ptrom_test_withhold_jphi_tc": ([_i], _i),
        "bs_velocity": ([_i, _vp, _i, _vp, _vp, _d, _vp, _vp, _i, _vp], _i),
        "bs_velocity_noalloc": ([_i, _vp, _i, _vp, _vp, _d, _vp, _vp, _i, _vp], _i),
        "bs_jvp": ([_i, _vp, _vp, _d, _vp, _vp, _i, _vp], _i),
        "bs_vjp": ([_i, _vp, _vp, _d, _vp, _vp, _vp, _i, _vp], _i),
        "bs_jphi": ([_i, _vp, _vp, _d, _vp, _i, _vp, _i, _vp], _i),
        "ptrom_launch_count": ([], ctypes.c_longlong),
        "ptrom_timing_enable": ([_i], _i),
        "ptrom_timing_read": ([ctypes.POINTER(_d), ctypes.POINTER(ctypes.c_longlong), _i], _i),
        "ptrom_model_create": ([ctypes.POINTER(ModelDesc), ctypes.POINTER(_vp)], _i),
        "ptrom_free": ([_vp], None),
        "ptrom_set_param": ([_vp, _vp, _vp, _vp, _vp], _i),
        "ptrom_set_inflow": ([_vp, _vp], _i),
        "ptrom_set_inflow_full": ([_vp, _vp, _vp], _i),
        "ptrom_state_bytes": ([_vp], ctypes.c_size_t),
        "ptrom_step": ([ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                        ctypes.POINTER(_vp), _i, ctypes.POINTER(PtromStats), _vp], _i),
        "ptrom_build": ([ctypes.POINTER(BuildParams), _i, _i, _vp, _vp, ctypes.POINTER(_vp),
                         ctypes.POINTER(BuildInfo), _vp], _i),
        "ptrom_set_param_full": ([_vp, _vp, _vp, _vp], _i),
        "ptrom_reconstruct": ([_vp, _vp, _vp, _i, _vp, _vp], _i),
        "ptrom_model_query": ([_vp] + [ctypes.POINTER(_i)] * 5 + [_vp, _vp, _vp, _vp], _i),
        "fom_adjoint_workspace_bytes": ([ctypes.POINTER(FomParams), _i], ctypes.c_size_t),
        "fom_adjoint_step": ([ctypes.POINTER(FomParams), _i, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                              ctypes.POINTER(FomStats), _vp], _i),
        "bs_velocity_batched": ([_i, _vp, _vp, _vp, _vp, _vp, _vp, _i, _vp], _i),
        "fom_step_batched": ([ctypes.POINTER(FomParams), _i, _vp, _vp, _vp, _vp, _vp, _vp,
                              ctypes.POINTER(FomStats), _vp], _i),
        "ptrom_set_pod_exact_max": ([_i], _i),
        "ptrom_greedy_sample": ([_i, _i, _vp, _i, _vp], _i),
        "fom_steps": ([ctypes.POINTER(FomParams), _i, _vp, _vp, _vp, _vp, ctypes.c_size_t, _i, _i,
                       ctypes.POINTER(FomStats), ctypes.POINTER(_i), _vp], _i),
        "ptrom_model_query_training": ([_vp] + [ctypes.POINTER(_i)] * 3 + [_vp, _vp], _i),
        "ptrom_model_query_clusters": ([_vp] + [ctypes.POINTER(_i)] * 3 + [_vp] * 7, _i),
        "ptrom_gappy_operator": ([_i, _i, _vp, _i, _vp, _vp], _i),
        "ptrom_save": ([_vp, ctypes.c_char_p], _i),
        "ptrom_load": ([ctypes.c_char_p, ctypes.POINTER(_vp)], _i),
        "fom_workspace_bytes": ([ctypes.POINTER(FomParams), _i], ctypes.c_size_t),
        "fom_step": ([ctypes.POINTER(FomParams), _i, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                      ctypes.POINTER(FomStats), _vp], _i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    lib.ptrom_last_error(buf, 512)
    return buf.value.decode()


def _check(status):
    if status != 0:
        raise PtromError(status, last_error())
    return status


def _ptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float64 tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _prec(p):
    try:
        return _PREC[p]
    except KeyError:
        raise ValueError(f"prec must be 'fp32c', 'fp64', 'tf32x3' or 'f16x3', got {p!r}") from None


KERNEL_KINDS = ["velocity", "velocity_selfjac", "jvp", "vjp", "jphi", "ptrom_step", "pack", "fom_vec",
                "fom_orth"]


def launch_count() -> int:
    """Kernels launched by the library so far (process-wide)."""
    return int(lib.ptrom_launch_count())


def timing_enable(on, kinds=None) -> None:
    """Start (on) or stop event timing; kinds: optional names from KERNEL_KINDS
    to time (default: all)."""
    if not on:
        lib.ptrom_timing_enable(0)
    elif kinds is None:
        lib.ptrom_timing_enable(1)
    else:
        mask = 0
        for k in kinds:
            mask |= 1 << KERNEL_KINDS.index(k)
        lib.ptrom_timing_enable(mask if mask != 1 else 1 | (1 << 30))


def timing_read() -> dict:
    """{kind: (total_ms, launches)} of the event-timed launches since the last read."""
    k = len(KERNEL_KINDS)
    ms = (_d * k)()
    cnt = (ctypes.c_longlong * k)()
    _check(lib.ptrom_timing_read(ms, cnt, k))
    return {name: (ms[i], int(cnt[i])) for i, name in enumerate(KERNEL_KINDS)}


def greedy_sample(phi_r, n_s: int):
    """Alg. 1 on the host: phi_r a (2n, M_r) float64 numpy array; returns the
    n_s sampled body ids (numpy int32) in the order chosen."""
    import numpy as np
    P = np.ascontiguousarray(phi_r, dtype=np.float64)
    n = P.shape[0] // 2
    out = np.zeros(int(n_s), dtype=np.int32)
    _check(lib.ptrom_greedy_sample(n, P.shape[1], P.ctypes.data, int(n_s), out.ctypes.data))
    return out


def gappy_operator(phi_r, sampled):
    """A = [P Phi_r]^+ on the host: (M_r, 2 n_s) float64 numpy array."""
    import numpy as np
    P = np.ascontiguousarray(phi_r, dtype=np.float64)
    s = np.ascontiguousarray(sampled, dtype=np.int32)
    A = np.zeros((P.shape[1], 2 * s.size))
    _check(lib.ptrom_gappy_operator(P.shape[0] // 2, P.shape[1], P.ctypes.data, s.size, s.ctypes.data,
                                    A.ctypes.data))
    return A


def set_pod_exact_max(n: int) -> None:
    """POD: exact eigensolve up to min(2n, snapshots) = n, randomized above."""
    _check(lib.ptrom_set_pod_exact_max(int(n)))


def set_source_split(S: int) -> None:
    """Force the all-pairs kernels' source split (1..16; 0 = automatic)."""
    _check(lib.ptrom_set_source_split(int(S)))


def tune_pairs(n: int, delta: float, prec="fp32c", stream=None) -> None:
    """Autotune and cache the source split of the n x n all-pairs kernels."""
    _check(lib.ptrom_tune_pairs(int(n), _prec(prec), float(delta), _stream(stream)))


def set_autotune(on: bool) -> None:
    """Tune every new all-pairs launch shape on first use (off by default)."""
    _check(lib.ptrom_set_autotune(1 if on else 0))


def autotune_reset() -> None:
    _check(lib.ptrom_autotune_reset())


def test_withhold_jphi_tc(on: bool) -> None:
    """Test hook: the next tensor-core bs_jphi call withholds its tile copies
    and must come back with PTROM_ETIMEOUT (include/ptrom.h)."""
    _check(lib.ptrom_test_withhold_jphi_tc(1 if on else 0))


def set_split_mode(mode: int) -> None:
    """0 = automatic, 1 = thread-block-cluster combine, 2 = global combine."""
    _check(lib.ptrom_set_split_mode(int(mode)))


def bs_velocity(xs, Gamma, delta, xt=None, f_out=None, selfjac=False, prec="fp32c", stream=None):
    """f (2 nt) at targets xt (default: the sources themselves); with
    ``selfjac`` also the (3, nt) self blocks (D00, D01, D10)."""
    ns = Gamma.numel()
    xt = xs if xt is None else xt
    nt = xt.numel() // 2
    if f_out is None:
        f_out = torch.empty(2 * nt, dtype=torch.float64, device=xs.device)
    D = torch.empty(3 * nt, dtype=torch.float64, device=xs.device) if selfjac else None
    _check(lib.bs_velocity(nt, _ptr(xt), ns, _ptr(xs), _ptr(Gamma), float(delta), _ptr(f_out),
                           _ptr(D), _prec(prec), _stream(stream)))
    return (f_out, D.view(3, nt)) if selfjac else f_out


NOALLOC_MAX_SOURCES = 65536


def bs_velocity_noalloc(xs, Gamma, delta, f_out, xt=None, selfjac_out=None, prec="fp32c", stream=None):
    """bs_velocity without any device allocation inside the library (its
    scratch is a fixed array of NOALLOC_MAX_SOURCES sources); outputs must be
    passed in.  Calls that overlap on the GPU share that scratch and race."""
    ns = Gamma.numel()
    xt = xs if xt is None else xt
    nt = xt.numel() // 2
    _check(lib.bs_velocity_noalloc(nt, _ptr(xt), ns, _ptr(xs), _ptr(Gamma), float(delta), _ptr(f_out),
                                   _ptr(selfjac_out), _prec(prec), _stream(stream)))
    return f_out


def bs_jvp(x, Gamma, delta, v, out=None, prec="fp32c", stream=None):
    n = Gamma.numel()
    out = torch.empty_like(x) if out is None else out
    _check(lib.bs_jvp(n, _ptr(x), _ptr(Gamma), float(delta), _ptr(v), _ptr(out), _prec(prec),
                      _stream(stream)))
    return out


def bs_jphi(x, Gamma, delta, phi, prec="fp32c", stream=None):
    """(d f / d x) Phi for phi of shape (2n, M); returns (2n, M).  The library
    takes column-major storage, i.e. a contiguous (M, 2n) buffer."""
    n = Gamma.numel()
    M = phi.shape[1]
    cols = phi.t().contiguous()
    out = torch.empty_like(cols)
    _check(lib.bs_jphi(n, _ptr(x), _ptr(Gamma), float(delta), _ptr(cols), M, _ptr(out), _prec(prec),
                       _stream(stream)))
    return out.t()


def bs_vjp(x, Gamma, delta, w, want_x=True, want_gamma=True, prec="fp32c", stream=None):
    n = Gamma.numel()
    gx = torch.empty_like(x) if want_x else None
    gG = torch.empty_like(Gamma) if want_gamma else None
    _check(lib.bs_vjp(n, _ptr(x), _ptr(Gamma), float(delta), _ptr(w), _ptr(gx), _ptr(gG),
                      _prec(prec), _stream(stream)))
    return gx, gG


def fom_workspace(params, n, device="cuda"):
    nbytes = lib.fom_workspace_bytes(ctypes.byref(params), int(n))
    if nbytes == 0:
        raise PtromError(EINVAL, last_error())
    return torch.empty(int(nbytes), dtype=torch.uint8, device=device)


def _with_inflow(params, u_inf):
    """A copy of params whose u_inf is the device tensor u_inf [2n] (or none)."""
    if u_inf is None:
        return params
    q = FomParams.from_buffer_copy(params)
    q.u_inf = _ptr(u_inf).value
    return q


def fom_step(params, Gamma, x, f, work=None, stream=None, allow_noconv=False, u_inf=None):
    """One implicit trapezoid step in place on (x, f).  Returns the stats dict.
    u_inf: optional device tensor [2n], the superimposed inflow velocity
    (f stays the pair sum)."""
    n = Gamma.numel()
    params = _with_inflow(params, u_inf)
    if work is None:
        work = fom_workspace(params, n, x.device)
    st = FomStats()
    status = lib.fom_step(ctypes.byref(params), n, _ptr(Gamma), _ptr(x), _ptr(f),
                          ctypes.c_void_p(work.data_ptr()), work.numel(), ctypes.byref(st),
                          _stream(stream))
    if status == ENOCONV and allow_noconv:
        d = st.as_dict()
        d["converged"] = False
        return d
    _check(status)
    d = st.as_dict()
    d["converged"] = True
    return d


def fom_steps(params, Gamma, x, f, nsteps, iters=0, work=None, stream=None, u_inf=None):
    """nsteps block-diagonal Newton steps in place on (x, f), each replayed
    from one captured CUDA graph (iters Newton iterations per step; 0: learnt
    from a first ordinary step).  Returns the summed stats dict."""
    n = Gamma.numel()
    params = _with_inflow(params, u_inf)
    if work is None:
        work = fom_workspace(params, n, x.device)
    st = FomStats()
    done = _i()
    _check(lib.fom_steps(ctypes.byref(params), n, _ptr(Gamma), _ptr(x), _ptr(f), ctypes.c_void_p(work.data_ptr()),
                         work.numel(), int(nsteps), int(iters), ctypes.byref(st), ctypes.byref(done),
                         _stream(stream)))
    d = st.as_dict()
    d["steps_done"] = done.value
    return d


# ----------------------------------------------------------------- PTROM
def _host(a, dtype):
    import numpy as np
    return np.ascontiguousarray(a, dtype=dtype)


class PtromModel:
    """A PTROM online model on the current device (ptrom_model_create).

    Arrays are host (NumPy) arrays in the layouts of include/ptrom.h:
    phi_s (2 n_s, M), x0_s (2 n_s), phi_c (2 N_c, M), x0_c (2 N_c),
    gamma_c (N_c), A (M_r, 2 n_s), CSR lists off (n_s+1) / idx."""

    def __init__(self, phi_s, x0_s, phi_c, x0_c, gamma_c, A, off, idx, dt, delta, tol=1e-4,
                 max_gn=100, qr_prec="fp64", u_s=None):
        import numpy as np
        keep = [_host(phi_s, np.float64), _host(x0_s, np.float64), _host(phi_c, np.float64),
                _host(x0_c, np.float64), _host(gamma_c, np.float64), _host(A, np.float64),
                _host(off, np.int32), _host(idx, np.int32)]
        us = None if u_s is None else _host(u_s, np.float64)
        ns = keep[1].size // 2
        M = keep[0].shape[1]
        Mr = keep[5].shape[0]
        Nc = keep[4].size
        d = ModelDesc(ns, M, Mr, Nc, float(dt), float(delta), float(tol), int(max_gn), _prec(qr_prec),
                      *[ctypes.c_void_p(a.ctypes.data) for a in keep],
                      None if us is None else ctypes.c_void_p(us.ctypes.data))
        h = ctypes.c_void_p()
        _check(lib.ptrom_model_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.n_s, self.M, self.M_r, self.N_c = ns, M, Mr, Nc

    def set_param(self, x0_s=None, phi_c=None, x0_c=None, gamma_c=None):
        import numpy as np
        arrs = [None if a is None else _host(a, np.float64) for a in (x0_s, phi_c, x0_c, gamma_c)]
        _check(lib.ptrom_set_param(self.handle,
                                   *[None if a is None else ctypes.c_void_p(a.ctypes.data) for a in arrs]))

    @classmethod
    def _wrap(cls, handle):
        obj = cls.__new__(cls)
        obj.handle = handle
        vals = [_i() for _ in range(5)]
        _check(lib.ptrom_model_query(handle, *[ctypes.byref(v) for v in vals], None, None, None, None))
        obj.n, obj.M, obj.M_r, obj.n_s, obj.N_c = [v.value for v in vals]
        return obj

    def query(self):
        """Offline data of a built model: phi (2n, M), sigma (M), sampled (n_s), A (M_r, 2 n_s)."""
        import numpy as np
        phi = np.empty((2 * self.n, self.M))
        sig = np.empty(self.M)
        smp = np.empty(self.n_s, dtype=np.int32)
        A = np.empty((self.M_r, 2 * self.n_s))
        _check(lib.ptrom_model_query(self.handle, None, None, None, None, None,
                                     ctypes.c_void_p(phi.ctypes.data), ctypes.c_void_p(sig.ctypes.data),
                                     ctypes.c_void_p(smp.ctypes.data), ctypes.c_void_p(A.ctypes.data)))
        return {"phi": phi, "sigma": sig, "sampled": smp, "A": A}

    def query_training(self):
        """Training data of a model built in this process: phi_r (2n, M_r), the
        residual basis Alg. 1 sampled on, and tier2 (n_params, steps + 1, M),
        the Tier-II reduced trajectories."""
        import numpy as np
        Mr, npar, steps = _i(), _i(), _i()
        _check(lib.ptrom_model_query_training(self.handle, ctypes.byref(Mr), ctypes.byref(npar), ctypes.byref(steps),
                                              None, None))
        phi_r = np.empty((2 * self.n, Mr.value))
        t2 = np.empty((npar.value, steps.value + 1, self.M))
        _check(lib.ptrom_model_query_training(self.handle, None, None, None, ctypes.c_void_p(phi_r.ctypes.data),
                                              ctypes.c_void_p(t2.ctypes.data)))
        return {"phi_r": phi_r, "tier2": t2}

    def query_clusters(self):
        """The online clusters: per sampled body the list of cluster ids, each
        cluster's member bodies, and phi_c (2 N_c, M), x0_c (2 N_c), gamma_c (N_c)."""
        import numpy as np
        Nc, nl, nm = _i(), _i(), _i()
        _check(lib.ptrom_model_query_clusters(self.handle, ctypes.byref(Nc), ctypes.byref(nl), ctypes.byref(nm),
                                              *([None] * 7)))
        off = np.empty(self.n_s + 1, dtype=np.int32)
        idx = np.empty(max(nl.value, 1), dtype=np.int32)
        moff = np.empty(Nc.value + 1, dtype=np.int32)
        mem = np.empty(max(nm.value, 1), dtype=np.int32)
        phi_c = np.empty((2 * Nc.value, self.M))
        x0_c = np.empty(2 * Nc.value)
        g_c = np.empty(Nc.value)
        _check(lib.ptrom_model_query_clusters(self.handle, None, None, None,
                                              *[ctypes.c_void_p(a.ctypes.data) for a in
                                                (off, idx, moff, mem, phi_c, x0_c, g_c)]))
        lists = [idx[off[s]:off[s + 1]].tolist() for s in range(self.n_s)]
        members = [mem[moff[c]:moff[c + 1]].tolist() for c in range(Nc.value)]
        return {"lists": lists, "members": members, "phi_c": phi_c, "x0_c": x0_c, "gamma_c": g_c}

    def set_param_full(self, x0, Gamma, stream=None):
        """Reload the clusters for a new parameter (device x0 [2n], Gamma [n])."""
        _check(lib.ptrom_set_param_full(self.handle, _ptr(x0), _ptr(Gamma), _stream(stream)))

    def set_inflow(self, u_s=None):
        """Superimposed inflow at the sampled dofs (host [2 n_s]; None removes it)."""
        import numpy as np
        us = None if u_s is None else _host(u_s, np.float64)
        _check(lib.ptrom_set_inflow(self.handle, None if us is None else ctypes.c_void_p(us.ctypes.data)))

    def set_inflow_full(self, u=None, stream=None):
        """Superimposed inflow from the full per-body array (device [2n]; None removes it)."""
        _check(lib.ptrom_set_inflow_full(self.handle, None if u is None else _ptr(u), _stream(stream)))

    def reconstruct(self, xhat, rows=None, stream=None):
        """x = x^0 + Phi xhat on the listed bodies (default all) -> [chi..., psi...]."""
        if rows is None:
            rows = torch.arange(self.n, dtype=torch.int32, device=xhat.device)
        out = torch.empty(2 * rows.numel(), dtype=torch.float64, device=xhat.device)
        _check(lib.ptrom_reconstruct(self.handle, _ptr(xhat), ctypes.c_void_p(rows.data_ptr()), rows.numel(),
                                     _ptr(out), _stream(stream)))
        return out

    def save(self, path):
        """Write the model to one binary file (ptrom_save)."""
        _check(lib.ptrom_save(self.handle, os.fsencode(path)))

    @classmethod
    def load(cls, path):
        """Create a model on the current device from a ptrom_save file."""
        h = ctypes.c_void_p()
        _check(lib.ptrom_load(os.fsencode(path), ctypes.byref(h)))
        return cls._wrap(h)

    def new_state(self, device="cuda"):
        """Zero state: xhat = 0, carried velocity computed on the first step."""
        nbytes = lib.ptrom_state_bytes(self.handle)
        return torch.zeros(int(nbytes), dtype=torch.uint8, device=device)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.ptrom_free(h)
            self.handle = None


def ptrom_step(models, states, nsteps, xhat=None, hist=None, stream=None, want_stats=True):
    """Advance len(models) instances by nsteps in one launch.  models: list of
    PtromModel; states: list of uint8 device tensors from new_state();
    xhat / hist: optional lists of float64 device tensors (M) / (nsteps, M)."""
    b = len(models)
    arr = lambda xs: (_vp * b)(*[ctypes.c_void_p(x.data_ptr()) for x in xs])
    mh = (_vp * b)(*[m.handle for m in models])
    st = PtromStats()
    _check(lib.ptrom_step(mh, b, arr(states), arr(xhat) if xhat is not None else None,
                          arr(hist) if hist is not None else None, int(nsteps),
                          ctypes.byref(st) if want_stats else None, _stream(stream)))
    return {k: getattr(st, k) for k, _ in st._fields_} if want_stats else None


CRITERIA = {"bh": 0, "barnes_hut": 0, "nb": 1, "neighbor": 1}


def ptrom_build(x0s, gammas, M, M_r, n_s, steps, fom, criterion="bh", theta=0.5, p_c=1.0, tol=1e-4,
                max_gn=100, qr_prec="fp64", stream=None, u_infs=None, snapshots=None):
    """Offline training (Stages 1-4) from device tensors x0s [P, 2n], gammas [P, n]
    and optionally u_infs [P, 2n] (superimposed inflow per parameter) and
    snapshots [P * steps, 2n] (the Stage 1 states, instead of running the FOM).
    Returns (PtromModel, info dict)."""
    x0s = x0s.contiguous()
    gammas = gammas.contiguous()
    P, n = gammas.shape
    if u_infs is not None:
        u_infs = u_infs.contiguous()
        if u_infs.shape != x0s.shape or u_infs.device != x0s.device:
            raise ValueError("u_infs must be shaped like x0s, on its device")
    if snapshots is not None:
        snapshots = snapshots.contiguous()
        if tuple(snapshots.shape) != (P * int(steps), 2 * n) or snapshots.device != x0s.device:
            raise ValueError("snapshots must be [P * steps, 2n] on the device of x0s")
    bp = BuildParams(int(M), int(M_r), int(n_s), CRITERIA[criterion], float(theta), float(p_c), int(steps),
                     float(tol), int(max_gn), _prec(qr_prec), fom,
                     _ptr(u_infs), _ptr(snapshots))
    h = ctypes.c_void_p()
    info = BuildInfo()
    _check(lib.ptrom_build(ctypes.byref(bp), int(n), int(P), _ptr(x0s), _ptr(gammas), ctypes.byref(h),
                           ctypes.byref(info), _stream(stream)))
    return PtromModel._wrap(h), {k: getattr(info, k) for k, _ in info._fields_}


def fom_adjoint_workspace(params, n, device="cuda"):
    nbytes = lib.fom_adjoint_workspace_bytes(ctypes.byref(params), int(n))
    if nbytes == 0:
        raise PtromError(EINVAL, last_error())
    return torch.empty(int(nbytes), dtype=torch.uint8, device=device)


def fom_adjoint_step(params, Gamma, x_n, x_prev, lam, gGamma, work=None, stream=None):
    """lam (dL/dx^n -> dL/dx^{n-1}) and gGamma (+= dL/dGamma share) in place."""
    n = Gamma.numel()
    if work is None:
        work = fom_adjoint_workspace(params, n, x_n.device)
    st = FomStats()
    _check(lib.fom_adjoint_step(ctypes.byref(params), n, _ptr(Gamma), _ptr(x_n), _ptr(x_prev), _ptr(lam),
                                _ptr(gGamma), ctypes.c_void_p(work.data_ptr()), work.numel(), ctypes.byref(st),
                                _stream(stream)))
    return st.as_dict()


def _ptr_array(ts):
    return (_vp * len(ts))(*[ctypes.c_void_p(t.data_ptr()) for t in ts])


def bs_velocity_batched(xs, Gammas, deltas, f_outs=None, selfjac=False, prec="fp32c", stream=None):
    """Velocity of B instances (lists of per-instance tensors) in one launch."""
    B = len(xs)
    n = (_i * B)(*[g.numel() for g in Gammas])
    if f_outs is None:
        f_outs = [torch.empty_like(x) for x in xs]
    Ds = [torch.empty(3 * g.numel(), dtype=torch.float64, device=g.device) for g in Gammas] if selfjac else None
    d = (_d * B)(*[float(v) for v in deltas])
    _check(lib.bs_velocity_batched(B, n, _ptr_array(xs), _ptr_array(Gammas), d, _ptr_array(f_outs),
                                   _ptr_array(Ds) if selfjac else None, _prec(prec), _stream(stream)))
    return (f_outs, Ds) if selfjac else f_outs


def fom_step_batched(params, Gammas, xs, fs, works, stream=None):
    """One block-diagonal Newton trapezoid step for B instances (in place)."""
    B = len(xs)
    n = (_i * B)(*[g.numel() for g in Gammas])
    wb = (ctypes.c_size_t * B)(*[w.numel() for w in works])
    st = (FomStats * B)()
    status = lib.fom_step_batched(ctypes.byref(params), B, n, _ptr_array(Gammas), _ptr_array(xs),
                                  _ptr_array(fs), _ptr_array(works), wb, st, _stream(stream))
    _check(status)
    return [s.as_dict() for s in st]
