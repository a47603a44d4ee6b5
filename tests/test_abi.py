"""The C-ABI library loads and exports every symbol include/feast_nl.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "feast_nl.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"\b(feast_nl_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["feast_nl_create", "feast_nl_set_contour", "feast_nl_solve",
              "feast_nl_get_eigpairs", "feast_nl_destroy", "feast_nl_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_1801_09794_gb300 as P
    if not os.path.exists(P.LIB_PATH):
        from paper_1801_09794_gb300.build import build
        build()
    lib = P.load_library()
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(_declared()) <= set(P.EXPORTS)
    assert P.strerror(P.FEAST_NL_ENOT_CONVERGED) == "not converged within maxit"
    assert P.strerror(99) == "unknown status"


def test_missing_library_fails_loudly(tmp_path):
    from paper_1801_09794_gb300 import _binding
    with pytest.raises(RuntimeError):
        _binding._lib_probe = None
        saved = _binding._lib
        _binding._lib = None
        try:
            _binding.load_library(str(tmp_path / "nope.so"))
        finally:
            _binding._lib = saved
