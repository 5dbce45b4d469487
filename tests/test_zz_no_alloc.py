"""bs_velocity_noalloc through the C ABI (GPU; collected last on purpose).

The allocation-free entry point serves callers that may not allocate device
memory while they run; it must give what bs_velocity gives.  Two calls in a
row with different sizes check that the shared fixed scratch, which keeps the
previous call's contents, does not leak into the next result.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2103_01983_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _check_case(L, stream, x, G, delta, want_d, prec, rows=None):
    """One bs_velocity_noalloc call against bs_velocity on the same inputs."""
    from paper_2103_01983_gb300 import ptrom
    n = G.size
    xt, Gt = _dev(x), _dev(G)
    f_ref = torch.empty_like(xt)
    D_ref = torch.empty(3 * n, dtype=torch.float64, device="cuda") if want_d else None
    assert L.bs_velocity(n, _vp(xt), n, _vp(xt), _vp(Gt), ctypes.c_double(delta), _vp(f_ref),
                         _vp(D_ref), prec, stream) == 0
    f = torch.full_like(xt, float("nan"))
    D = torch.full((3 * n,), float("nan"), dtype=torch.float64, device="cuda") if want_d else None
    assert L.bs_velocity_noalloc(n, _vp(xt), n, _vp(xt), _vp(Gt), ctypes.c_double(delta), _vp(f),
                                 _vp(D), prec, stream) == 0, ptrom.last_error()
    torch.cuda.synchronize()
    tol = 1e-5 if prec == 0 else 1e-12
    assert _rel(f, f_ref) <= tol
    if want_d:
        assert _rel(D, D_ref) <= tol


def test_noalloc_matches_bs_velocity_two_calls_in_a_row():
    from paper_2103_01983_gb300 import ptrom
    L = ptrom.lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(W.two_cluster(8192, seed=50), 0.02, True), (W.disk(1500, seed=51), 0.05, False)]
    for (x, G), delta, want_d in cases:
        _check_case(L, stream, x, G, delta, want_d, 0)


def test_noalloc_fp64_records_and_the_size_limit():
    """FP64 records (the largest the fixed array holds, 48 bytes) at the
    largest accepted source count, then an FP32 call reusing the array."""
    from paper_2103_01983_gb300 import ptrom
    L = ptrom.lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = ptrom.NOALLOC_MAX_SOURCES
    x, G = W.two_cluster(n, seed=52)
    _check_case(L, stream, x, G, 0.02, False, 1)
    _check_case(L, stream, x, G, 0.02, True, 1)
    x2, G2 = W.disk(3000, seed=53)
    _check_case(L, stream, x2, G2, 0.05, True, 1)
    _check_case(L, stream, x2, G2, 0.05, False, 0)


def test_noalloc_rejects_oversize_before_launching():
    from paper_2103_01983_gb300 import ptrom
    null = ctypes.c_void_p(0)
    n = ptrom.NOALLOC_MAX_SOURCES + 1
    assert ptrom.lib.bs_velocity_noalloc(4, null, n, null, null, ctypes.c_double(0.1), null, null, 0,
                                         null) == ptrom.EINVAL
    assert "limit" in ptrom.last_error()
