"""The C ABI library builds, loads on a machine without a GPU, and exports
every function that include/ce_condsim.h declares.  No compute calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ce_condsim.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ce_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import paper_2109_11044_gb300 as ce
    from paper_2109_11044_gb300.build import build
    path = build()
    return ce, ctypes.CDLL(path)


def test_header_declares_the_binding_exports():
    import paper_2109_11044_gb300 as ce
    assert _declared() == sorted(ce.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    _, so = lib
    for name in _declared():
        assert hasattr(so, name), name


def test_binding_types_every_symbol(lib):
    ce, _ = lib
    loaded = ce.load_library()
    for name in ce.EXPORTS:
        assert getattr(loaded, name).argtypes is not None or name == "ce_last_error"


def test_missing_library_fails_loudly(tmp_path):
    import paper_2109_11044_gb300 as ce
    saved = ce._lib
    ce._lib = None
    try:
        with pytest.raises(ImportError):
            ce.load_library(str(tmp_path / "nope.so"))
    finally:
        ce._lib = saved


def test_argument_errors_need_no_gpu(lib):
    """Host-side argument checks run before any CUDA call."""
    ce, so = lib
    loaded = ce.load_library()
    ctx = ctypes.c_void_p()
    g = ce._Grid(4, 0.0, 0.0, 0.1)          # m < 8
    c = ce._Cov(1.0, 0.1, 0.5, 0.05)
    assert loaded.ce_setup(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(c), 0, None) == ce.CE_ERR_ARG
    assert b"grid side" in loaded.ce_last_error(None)
    g = ce._Grid(16, 0.0, 0.0, 0.1)
    c = ce._Cov(1.0, 0.1, 0.7, 0.05)          # nu not 1/2 or 3/2
    assert loaded.ce_setup(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(c), 0, None) == ce.CE_ERR_ARG
    assert loaded.ce_philox(None, -1, 0, None, None) == ce.CE_ERR_ARG


def _declared_arities():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    out = {}
    for name, params in re.findall(r"\b(ce_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else len([p for p in params.split(",") if p.strip()])
    return out


def test_binding_argument_counts_match_the_header(lib):
    """The ctypes signature of every entry point has as many arguments as its C declaration."""
    ce, _ = lib
    loaded = ce.load_library()
    arities = _declared_arities()
    assert set(arities) == set(ce.EXPORTS)
    for name, n in arities.items():
        argtypes = getattr(loaded, name).argtypes
        assert argtypes is not None and len(argtypes) == n, (name, n, argtypes)
