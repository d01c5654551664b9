"""The C ABI library loads, exports every declared symbol, and rejects bad
arguments before touching a GPU (CPU only; no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def L():
    from paper_2409_08729_gb300.build import build_library
    build_library()
    from paper_2409_08729_gb300 import _binding
    return _binding.lib()


def declared_functions():
    names = []
    for fn in os.listdir(HEADER_DIR):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\([^;{]*\)\s*;", text, flags=re.M):
            names.append(m.group(1))
    return names


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 10
    for nm in names:
        assert hasattr(L, nm), nm


def test_version(L):
    from paper_2409_08729_gb300 import _binding
    assert L.logbessel_version().decode().count(".") == 2


@pytest.mark.parametrize("fn", ["logbessel_i", "logbessel_k"])
def test_argument_validation(L, fn):
    from paper_2409_08729_gb300 import _binding as B
    f = getattr(L, fn)
    buf = ctypes.create_string_buffer(64)
    p = ctypes.cast(buf, ctypes.c_void_p).value
    assert f(B.LB_F64, p, 1, p, p, 0, 0, None) == B.LB_OK                # n = 0: nothing to do
    assert f(B.LB_F64, p, 1, p, p, -1, 0, None) == B.LB_EINVAL           # n < 0
    assert b"n must be" in L.logbessel_last_error()
    assert f(B.LB_F64, None, 1, p, p, 5, 0, None) == B.LB_EINVAL         # NULL v
    assert b"NULL v" in L.logbessel_last_error()
    assert f(B.LB_F64, p, 1, p, None, 5, 0, None) == B.LB_EINVAL         # NULL out
    assert f(B.LB_F64, p, 2, p, p, 5, 0, None) == B.LB_EINVAL            # bad stride
    assert f(7, p, 1, p, p, 5, 0, None) == B.LB_EINVAL                   # bad dtype
    assert f(B.LB_F64, p, 1, p, p, 5, 9, None) == B.LB_EINVAL            # bad mode


def test_classify_and_region_validation(L):
    from paper_2409_08729_gb300 import _binding as B
    buf = ctypes.create_string_buffer(64)
    p = ctypes.cast(buf, ctypes.c_void_p).value
    assert L.logbessel_classify(2, B.LB_F64, p, 1, p, p, 4, 0, None) == B.LB_EINVAL
    assert L.logbessel_eval_region(0, B.LB_F64, p, 1, p, p, 4, 3, 0, None) == B.LB_EINVAL   # SPECIAL is no expression
    assert L.logbessel_eval_region(0, B.LB_F64, p, 1, p, p, 4, 99, 0, None) == B.LB_EINVAL


def test_profile_interface(L):
    from paper_2409_08729_gb300 import _binding as B
    n = L.logbessel_profile_slots()
    assert n >= 2
    name = ctypes.c_char_p()
    la, tl, ms = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double()
    assert L.logbessel_profile_get(n, ctypes.byref(name), ctypes.byref(la), ctypes.byref(tl), ctypes.byref(ms)) == B.LB_EINVAL
    assert L.logbessel_profile_get(0, ctypes.byref(name), ctypes.byref(la), ctypes.byref(tl), ctypes.byref(ms)) == B.LB_OK
    assert name.value == b"lb_tiles_kernel"
    assert L.logbessel_measure_fp64(None, None) == B.LB_EINVAL


def test_python_api_requires_cuda_tensors():
    import torch
    import paper_2409_08729_gb300 as lb
    with pytest.raises((ValueError, TypeError)):
        lb.log_i(1.0, torch.ones(3, dtype=torch.float64))


def test_workspace_entry_points_validate(L):
    """Workspace size rule and argument checks of the caller-workspace K entry points (no launch)."""
    from paper_2409_08729_gb300 import _binding as B
    assert L.logbessel_workspace_bytes(0) == 256 + 4 * 2048
    assert L.logbessel_workspace_bytes(1000) == 256 + 4 * 2048
    assert L.logbessel_workspace_bytes(5000) == 256 + 4 * 6144
    assert L.logbessel_workspace_bytes(1 << 30) == 256 + 4 * (1 << 26)
    assert L.logbessel_workspace_bytes(-1) == 0
    buf = ctypes.create_string_buffer(64)
    p = ctypes.cast(buf, ctypes.c_void_p).value
    for fn in (L.logbessel_k_ws, L.logbessel_k_dx_ws):
        assert fn(B.LB_F64, p, 1, p, p, 5, 0, None, 1 << 20, None) == B.LB_EINVAL     # NULL workspace
        assert b"workspace" in L.logbessel_last_error()
        assert fn(B.LB_F64, p, 1, p, p, 5, 0, 256 * 3 + 8, 1 << 20, None) == B.LB_EINVAL   # misaligned
        assert fn(B.LB_F64, p, 1, p, p, 5, 0, 256 * 3, 1000, None) == B.LB_EINVAL         # too small
        assert fn(B.LB_F64, p, 1, p, p, -1, 0, 256 * 3, 1 << 20, None) == B.LB_EINVAL     # n < 0
        assert fn(B.LB_F64, p, 1, p, p, 0, 0, 256 * 3, 1 << 20, None) == B.LB_OK          # nothing to do
