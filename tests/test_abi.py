"""The C-ABI library builds, loads and exports every entry point declared in include/gabp.h.
No compute calls here (these tests run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gabp_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libgabp():
    from paper_2404_12968_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2404_12968_gb300.build import build
        build()
    return ctypes.CDLL(_lib.LIB_PATH)


def test_header_declares_the_four_core_calls():
    names = _declared_functions()
    for core in ("gabp_create", "gabp_iterate", "gabp_marginals", "gabp_residual", "gabp_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(libgabp):
    missing = [n for n in _declared_functions() if not hasattr(libgabp, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_2404_12968_gb300 as g
    exported = {n for n in dir(g) if n.startswith("gabp_")}
    # every Python wrapper carries a C name, and the core calls are all wrapped
    assert exported <= set(_declared_functions())
    for core in ("gabp_create", "gabp_iterate", "gabp_marginals", "gabp_residual", "gabp_destroy"):
        assert core in exported


def test_default_options_without_gpu(libgabp):
    from paper_2404_12968_gb300 import gabp_default_options
    o = gabp_default_options()
    assert o.precision == 0 and o.tol == pytest.approx(1e-5) and o.check_every == 50
    assert o.device == -1 and o.stream is None


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2404_12968_gb300 import _lib
    monkeypatch.setattr(_lib, "_LIB", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()
