"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/gemm.h declares.  CPU only: no kernel is launched."""
import ctypes
import os
import re

import pytest

from paper_2305_18236_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gemm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(n for n in names if n.startswith("gemm")))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gemm_create", "gemm_destroy", "gemm", "gemm_bf16", "gemm_split_bf16",
                     "gemm_grouped", "gemm_backward", "gemm_from_host", "gemm_sync"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    assert set(declared_functions()) <= set(_lib.EXPORTED)


def test_library_is_built_for_sm103a(lib):
    # the build flags pin the one target architecture
    assert ["-gencode", "arch=compute_103a,code=sm_103a"] == build.ARCH


def test_status_strings(lib):
    for code in range(-7, 1):
        s = lib.gemm_status_string(code).decode()
        assert s.startswith("GEMM_")
    assert lib.gemm_status_string(12345).decode() == "unknown gemm_status_t"


def test_null_handle_is_argument_one(lib):
    assert lib.gemm(None, 0, 0, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, 0, None) \
        == _lib.GEMM_ERR_ARG
    assert lib.gemm_create(None) == _lib.GEMM_ERR_ARG
    assert lib.gemm_syr2k(None, 0, 0, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, 0, None) \
        == _lib.GEMM_ERR_ARG
    assert lib.gemm_syr2k_workspace_size(None, 2, 0, 4, 4) == 0
    pos = ctypes.c_int(0)
    assert lib.gemm_get_last_error_arg(None, ctypes.byref(pos)) == _lib.GEMM_ERR_ARG
    assert pos.value == 1
    assert lib.gemm_destroy(None) == _lib.GEMM_OK
    assert lib.gemm_last_error_arg(None) == 1


def test_create_without_sm103_device_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.gemm_create(ctypes.byref(h)) == _lib.GEMM_ERR_DEVICE
    assert not h.value


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_LIB", None)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()


def test_binding_row_stride_of_tensors():
    """The binding's row stride: row-major tensors give their row stride,
    a one-row tensor its width, and empty tensors (whose strides torch may
    report as 0) any valid stride; a non-contiguous last dimension raises."""
    import numpy as np
    import torch

    from paper_2305_18236_gb300.gemm import _ld

    assert _ld(torch.zeros((3, 4))) == 4
    assert _ld(torch.zeros((8, 6))[:, :5]) == 6
    assert _ld(torch.zeros((1, 7))) == 7
    for shape, want in [((0, 5), 5), ((5, 0), 1), ((0, 0), 1)]:
        t = torch.from_numpy(np.zeros(shape, np.float32))
        assert _ld(t) == want
    with pytest.raises(ValueError):
        _ld(torch.zeros((4, 6)).t())
    with pytest.raises(ValueError):
        _ld(torch.zeros(4))
