"""ctypes front end of the oracle's plain-C FP64 double loops (``bs_direct.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

All arrays use the paper's state layout (Sec. 2, Eq. 3): a state of n bodies is
[chi_1..chi_n, psi_1..psi_n].  ``Gamma`` holds circulations; the 1/(2 pi)
factor of Eq. 2 is applied inside.
"""
from __future__ import annotations

import ctypes

import numpy as np

from .build_oracle import build

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        for name, args in {
            "or_velocity": [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp],
            "or_jvp": [ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp],
            "or_vjp": [ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp, _dp],
            "or_jphi": [ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, ctypes.c_int, _dp],
            "or_jvp_rows": [ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _ip, ctypes.c_int, _dp],
            "or_vjp_rows": [ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _ip, ctypes.c_int, _dp, _dp],
        }.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = None
        lib.or_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().or_num_threads())


def velocity(x, Gamma, delta, targets=None, with_selfjac=False):
    """f (2 nt) of Eq. 2 at the targets (default: the bodies themselves).

    With ``with_selfjac`` also returns D (3, nt) = (D00, D01, D10) of the
    per-target block d f_i / d x_i (D11 = -D00).
    """
    x = _c(x)
    Gamma = _c(Gamma)
    n = Gamma.size
    xt = x if targets is None else _c(targets)
    nt = xt.size // 2
    f = np.empty(2 * nt)
    D = np.empty(3 * nt) if with_selfjac else None
    _load().or_velocity(nt, _p(xt), n, _p(x), _p(Gamma), float(delta), _p(f), _p(D))
    if with_selfjac:
        return f, D.reshape(3, nt)
    return f


def jvp(x, Gamma, delta, v, rows=None):
    """(d f / d x) v over all blocks; with ``rows`` only those bodies' rows,
    returned as [chi rows..., psi rows...]."""
    x, Gamma, v = _c(x), _c(Gamma), _c(v)
    if rows is None:
        out = np.empty_like(x)
        _load().or_jvp(Gamma.size, _p(x), _p(Gamma), float(delta), _p(v), _p(out))
        return out
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.empty(2 * rows.size)
    _load().or_jvp_rows(Gamma.size, _p(x), _p(Gamma), float(delta), _p(v),
                        rows.ctypes.data_as(_ip), rows.size, _p(out))
    return out


def vjp(x, Gamma, delta, w, rows=None):
    """((d f / d x)^T w, (d f / d Gamma)^T w); with ``rows`` only those
    bodies' entries ([chi..., psi...] and [Gamma...])."""
    x, Gamma, w = _c(x), _c(Gamma), _c(w)
    if rows is None:
        gx = np.empty_like(x)
        gG = np.empty_like(Gamma)
        _load().or_vjp(Gamma.size, _p(x), _p(Gamma), float(delta), _p(w), _p(gx), _p(gG))
        return gx, gG
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    gx = np.empty(2 * rows.size)
    gG = np.empty(rows.size)
    _load().or_vjp_rows(Gamma.size, _p(x), _p(Gamma), float(delta), _p(w),
                        rows.ctypes.data_as(_ip), rows.size, _p(gx), _p(gG))
    return gx, gG


def jphi(x, Gamma, delta, phi):
    """(d f / d x) Phi for Phi of shape (2n, M)."""
    x, Gamma = _c(x), _c(Gamma)
    phi = np.asfortranarray(phi, dtype=np.float64)
    n2, M = phi.shape
    out = np.empty((n2, M), order="F")
    _load().or_jphi(Gamma.size, _p(x), _p(Gamma), float(delta),
                    phi.ctypes.data_as(_dp), M, out.ctypes.data_as(_dp))
    return np.ascontiguousarray(out)
