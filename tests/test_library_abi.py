"""The C-ABI library builds, loads and exports every entry point its header declares (CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _ensure_built():
    from paper_1301_1247_gb300 import build, hbs
    if not os.path.exists(hbs.LIB_PATH):
        build.build()
    return hbs.LIB_PATH


def _declared():
    src = open(os.path.join(ROOT, "include", "hbsqp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hbs_[a-z_]+)\s*\(", src)))


def test_header_declares_bound_names():
    from paper_1301_1247_gb300 import hbs
    assert sorted(hbs.EXPORTED) == _declared()


def test_library_exports_all_declared_symbols():
    path = _ensure_built()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (hbs_[a-z_]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_reports_defaults():
    _ensure_built()
    from paper_1301_1247_gb300 import hbs
    L = hbs.lib()
    for name in _declared():
        assert hasattr(L, name)
    o = hbs.default_options()
    assert o.leaf_size == 64 and o.proxy_rho == 1.5 and o.precision == 0
    assert L.hbs_last_error() is not None


def test_argument_errors_need_no_gpu():
    """Invalid arguments are rejected on the host before any CUDA call."""
    _ensure_built()
    from paper_1301_1247_gb300 import hbs
    L = hbs.lib()
    out = ctypes.c_void_p()
    g = hbs.Geometry(10, 1.0, None, None, None, None, 0)
    assert L.hbs_build(ctypes.byref(g), 10.0, 1e-12, None, None, ctypes.byref(out)) == 1
    assert L.hbs_solve(None, None, 0, None, ctypes.byref(out)) == 1
    assert L.hbs_apply_inverse(None, None, None, 1, None) == 1
    srv = ctypes.c_void_p()
    assert L.hbs_server_create(0, 0, 1, ctypes.byref(srv)) == 1
    rid = ctypes.c_int64()
    assert L.hbs_server_submit(None, 1, -0.5, ctypes.byref(rid)) == 1
    outs = (ctypes.c_void_p * 2)()
    assert L.hbs_build_batch(None, None, 2, 1e-12, None, None, outs) == 1
    fake = ctypes.c_void_p(256)
    assert L.hbs_batched_inverse(None, 8, 1, 0, None) == 1
    assert L.hbs_batched_inverse(fake, 5000, 1, 0, None) == 1
    assert L.hbs_batched_inverse(fake, 8, 1, 7, None) == 1
    passed = ctypes.c_int()
    assert L.hbs_barrier_selftest(0, 0, 0.1, ctypes.byref(passed), None) == 1
    assert L.hbs_barrier_selftest(4, 0, 0.0, ctypes.byref(passed), None) == 1


def test_fault_injection_arms_and_clears_without_gpu():
    """The host-side fault switches accept their kinds, reject bad ones, and clear."""
    _ensure_built()
    from paper_1301_1247_gb300 import hbs
    L = hbs.lib()
    assert L.hbs_fault_inject(hbs.INJECT_RANK_CAP, 5) == 0
    assert L.hbs_fault_inject(hbs.INJECT_ALLOC_FAILURE, 3) == 0
    assert L.hbs_fault_inject(hbs.INJECT_ALLOC_FAILURE, -2) == hbs.HBS_ERR_INVALID_ARG
    assert L.hbs_fault_inject(99, 0) == hbs.HBS_ERR_INVALID_ARG
    assert L.hbs_fault_inject(hbs.INJECT_CLEAR, 0) == 0


def test_load_rejects_missing_and_foreign_files_without_gpu(tmp_path):
    """hbs_load checks the file's tag before touching the device: a missing file, a file
    of random bytes and a truncated tag all give HBS_ERR_IO and no handle."""
    _ensure_built()
    from paper_1301_1247_gb300 import hbs
    L = hbs.lib()
    out = ctypes.c_void_p(1)
    assert L.hbs_load(str(tmp_path / "absent.hbs").encode(), None, ctypes.byref(out)) == hbs.HBS_ERR_IO
    assert not out.value
    junk = tmp_path / "junk.hbs"
    junk.write_bytes(bytes(range(256)) * 4)
    assert L.hbs_load(str(junk).encode(), None, ctypes.byref(out)) == hbs.HBS_ERR_IO
    short = tmp_path / "short.hbs"
    short.write_bytes(b"HBSQP\0v1")
    assert L.hbs_load(str(short).encode(), None, ctypes.byref(out)) == hbs.HBS_ERR_IO
    assert not out.value
    assert L.hbs_load(None, None, ctypes.byref(out)) == hbs.HBS_ERR_INVALID_ARG
    assert L.hbs_save(None, b"x", None) == hbs.HBS_ERR_INVALID_ARG
