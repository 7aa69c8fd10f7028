"""The C-ABI library loads and exports every entry point include/hlc.h declares
(no compute call: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hlc_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1709_08625_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["hlc_build_tree", "hlc_assemble", "hlc_cholesky", "hlc_loglik", "hlc_serve_start",
                     "hlc_serve_submit", "hlc_serve_poll", "hlc_serve_stop", "hlc_create", "hlc_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_defaults_without_gpu(lib):
    lib.hlc_strerror.restype = ctypes.c_char_p
    assert lib.hlc_strerror(-3).decode().startswith("matrix not positive definite")
    from paper_1709_08625_gb300 import hlc

    p = hlc.params()
    assert p.leaf == 64 and p.eta == 2.0 and p.kmax == 64


def test_create_without_device_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1709_08625_gb300 import hlc

    with pytest.raises(hlc.HlcError) as e:
        hlc.Context(0)
    assert e.value.status == -5
