"""CPU checks of the C ABI: the library builds, loads without a GPU and exports
every entry point declared in include/wadg.h; host-only tables agree with the
oracle (no device work is issued here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "wadg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wadg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    b = g._build_module()
    if not os.path.exists(b.LIB):
        b.build()
    return ctypes.CDLL(b.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_1608_03836_gb300._lib import SIGNATURES
    assert set(_declared()) == set(SIGNATURES)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_library_rules_match_oracle_rules(lib, N):
    """Same rule, same point order on both sides (the c^2 samples and any
    quadrature-point data cross the boundary in this order)."""
    import paper_1608_03836_gb300 as W
    from oracle import polynomials as P
    rst, w, rs, wf = W.wadg_reference_rules(N)
    r2, w2 = P.tet_rule(N + 1)
    f2, wf2 = P.tri_rule(N + 1)
    assert np.abs(rst - r2).max() < 1e-14 and np.abs(w - w2).max() < 1e-14
    assert np.abs(rs - f2).max() < 1e-14 and np.abs(wf - wf2).max() < 1e-14


def test_unsupported_degree_is_rejected(lib):
    import paper_1608_03836_gb300 as W
    with pytest.raises(W.WadgError):
        W.wadg_reference_rules(7)


def test_status_strings(lib):
    import paper_1608_03836_gb300 as W
    assert W.wadg_status_string(0) == "ok"
    assert W.wadg_status_string(-4) == "invalid geometry"
