"""The C-ABI library loads and exports every symbol include/*.h declares (CPU only).

Also checks argument validation that happens before any CUDA call."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "sizeof", "return"):
                names.add(name)
    return names


@pytest.fixture(scope="module")
def lib():
    from __graft_entry__ import build_library
    build_library()
    from paper_2103_01983_gb300 import ptrom
    return ptrom


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"bs_velocity", "bs_jvp", "bs_vjp", "ptrom_last_error"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib.lib, n)]
    assert not missing, missing


def test_invalid_arguments_rejected_before_any_cuda_call(lib):
    L = lib.lib
    null = ctypes.c_void_p(0)
    assert L.bs_velocity(0, null, 10, null, null, 0.1, null, null, 0, null) == -1
    assert "sizes" in lib.last_error()
    assert L.bs_velocity(4, null, 4, null, null, -1.0, null, null, 0, null) == -1
    assert L.bs_velocity(4, null, 4, null, null, 0.1, null, null, 7, null) == -1
    assert L.bs_velocity(4, null, 4, null, null, 0.1, null, null, 0, null) == -1   # NULL arrays
    assert L.bs_jvp(1, null, null, 0.1, null, null, 0, null) == -1
    assert L.bs_vjp(1, null, null, 0.1, null, null, null, 0, null) == -1
    assert L.ptrom_set_source_split(17) == -1
    assert L.ptrom_set_split_mode(3) == -1
    assert L.ptrom_set_split_mode(0) == 0
    assert L.ptrom_set_autotune(2) == -1
    assert L.ptrom_set_autotune(0) == 0
    assert L.ptrom_autotune_reset() == 0
    assert L.ptrom_test_withhold_jphi_tc(2) == -1
    assert L.ptrom_test_withhold_jphi_tc(0) == 0
    # bs_jphi: the tensor-core precisions pass the host checks, an unknown one does not
    assert L.bs_jphi(1, null, null, ctypes.c_double(0.1), null, 4, null, 2, null) == -1   # n < 2
    assert L.bs_jphi(8, null, null, ctypes.c_double(0.1), null, 4, null, 9, null) == -1   # bad prec
    assert "prec" in lib.last_error()
    assert L.bs_jphi(8, null, null, ctypes.c_double(0.1), null, 4, null, 3, null) == -1   # NULL arrays
    assert "NULL" in lib.last_error()
    assert L.ptrom_tune_pairs(1, 0, ctypes.c_double(0.02), None) == -1
    assert L.ptrom_set_source_split(0) == 0
    assert L.ptrom_set_inflow(None, None) == -1
    assert L.ptrom_set_inflow_full(None, None, None) == -1
    assert L.ptrom_set_pod_exact_max(0) == -1
    # the batched FOM takes no inflow: rejected before the instances are looked at
    fp = lib.fom_params(0.01, 0.05, "blockdiag", prec="fp64")
    fp.u_inf = 16
    one = (ctypes.c_void_p * 1)(16)
    n = (ctypes.c_int * 1)(4)
    wb = (ctypes.c_size_t * 1)(1 << 20)
    assert L.fom_step_batched(ctypes.byref(fp), 1, n, one, one, one, one, wb, None, None) == -1
    assert "u_inf" in lib.last_error()
    # ptrom_build: sizes are checked before any device work
    bp = lib.BuildParams(8, 16, 16, 0, 0.5, 1.0, 10, 1e-4, 100, 1, lib.fom_params(0.01, 0.05, "jfnk"))
    h = ctypes.c_void_p(0)
    assert L.ptrom_build(ctypes.byref(bp), 1, 1, one, one, ctypes.byref(h), None, None) == -1
    assert "sizes" in lib.last_error()


def test_model_file_errors_before_any_cuda_call(lib, tmp_path):
    """ptrom_load rejects missing, foreign, truncated and corrupted files on
    the host (the hash and the header are checked before any upload)."""
    L = lib.lib
    h = ctypes.c_void_p(0)
    assert L.ptrom_save(None, b"/nonexistent/x") == -1
    assert L.ptrom_load(None, ctypes.byref(h)) == -1
    assert L.ptrom_load(str(tmp_path / "missing.bin").encode(), ctypes.byref(h)) == -1
    assert "cannot open" in lib.last_error()
    junk = tmp_path / "junk.bin"
    junk.write_bytes(b"not a model at all, just some bytes" * 4)
    assert L.ptrom_load(str(junk).encode(), ctypes.byref(h)) == -1
    assert "checksum" in lib.last_error()
    assert not h.value
    short = tmp_path / "short.bin"
    short.write_bytes(b"PTROM")
    assert L.ptrom_load(str(short).encode(), ctypes.byref(h)) == -1
    assert "too short" in lib.last_error()


_MIRRORS = {  # C struct -> binding class name
    "ptrom_fom_params": "FomParams",
    "ptrom_fom_stats": "FomStats",
    "ptrom_model_desc": "ModelDesc",
    "ptrom_stats": "PtromStats",
    "ptrom_build_params": "BuildParams",
    "ptrom_build_info": "BuildInfo",
}


def test_binding_structs_match_the_header_layout(lib, tmp_path):
    """Every ctypes mirror has the C struct's size and every field its offset
    (the header compiled as C99 with the host compiler)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ptrom.h"', "int main(void) {"]
    for cname, pyname in _MIRRORS.items():
        cls = getattr(lib, pyname)
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    c = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    for cname, pyname in _MIRRORS.items():
        cls = getattr(lib, pyname)
        assert int(c[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(c[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)


def _fnv1a(data: bytes) -> int:
    h = 1469598103934665603
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _model_file(cl_off):
    """A built-model file in the documented layout (ptrom_io.cu), correctly
    hashed: n_s = M = M_r = N_c = 1, n = 2, with the given cluster offsets."""
    import struct
    f64 = lambda *v: struct.pack("<Q", len(v)) + struct.pack(f"<{len(v)}d", *v)
    i32 = lambda *v: struct.pack("<Q", len(v)) + struct.pack(f"<{len(v)}i", *v)
    body = b"PTROMMDL" + struct.pack("<II", 0x01020304, 2)
    body += struct.pack("<8i", 1, 1, 1, 1, 10, 0, 1, 2)            # n_s M M_r N_c max_gn qr_prec built n
    body += struct.pack("<5d", 0.01, 0.05, 1e-4, 0.0, 0.0)
    body += f64(0.1, 0.2) + f64(0.0, 0.0) + f64(0.3, 0.4) + f64(1.0, 1.0) + f64(1.0) + f64(0.5, 0.5)
    body += i32(0, 1) + i32(0) + f64()                                # off, idx, u_s (none)
    body += f64(1.0, 0.0, 0.0, 0.0) + f64(1.0) + i32(0) + i32(*cl_off) + i32() + f64(0.0, 1.0, 0.0, 0.0)
    return body + struct.pack("<Q", _fnv1a(body))


def test_model_file_with_cluster_offsets_not_from_zero_is_rejected(lib, tmp_path):
    """A crafted, correctly hashed file whose cluster-member offsets start at
    -1 would make a later reload index before the member array; ptrom_load
    rejects it on the host, before any CUDA call."""
    L = lib.lib
    h = ctypes.c_void_p(0)
    bad = tmp_path / "bad_cl_off.bin"
    bad.write_bytes(_model_file([-1, 0]))
    assert L.ptrom_load(str(bad).encode(), ctypes.byref(h)) == -1
    assert "start at 0" in lib.last_error()
    assert not h.value
