"""CPU-side checks of the C ABI library: it builds, loads without a GPU, and
exports every entry point that include/ejoin.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ejoin.h")


def declared_functions():
    with open(HEADER) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ejoin_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2312_01476_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("ejoin_create", "ejoin_destroy", "ejoin_normalize", "ejoin_threshold", "ejoin_threshold_host",
                 "ejoin_pairs_free", "ejoin_strerror", "ejoin_last_stats"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_only_calls(lib):
    lib.ejoin_strerror.restype = ctypes.c_char_p
    assert lib.ejoin_strerror(0) == b"ok"
    assert b"capacity" in lib.ejoin_strerror(3)
    lib.ejoin_padded_dim.restype = ctypes.c_int64
    assert lib.ejoin_padded_dim(1, 300) == 320   # BF16: multiple of 64
    assert lib.ejoin_padded_dim(2, 300) == 384   # e4m3: multiple of 128
    assert lib.ejoin_padded_dim(0, 300) == 320   # FP32: multiple of 32
    assert lib.ejoin_padded_dim(3, 100) == 128


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.ejoin_create(ctypes.byref(h), None)
    assert st != 0 and not h.value


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2312_01476_gb300 import ejoin
    with pytest.raises(RuntimeError):
        ejoin.load_library(str(tmp_path / "missing.so"))
