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


def test_mesh_create_rejects_bad_sizes_without_a_gpu(lib):
    """Host-side checks before any device work: an empty mesh, degrees outside
    1..6 and a volume rule whose point count no kernel is built for."""
    import paper_1608_03836_gb300 as W
    from synthetic import warped_cube
    VXYZ, EToV, geom = warped_cube(1, 2, 0.1)
    with pytest.raises(W.WadgError) as e:
        W.wadg_mesh_create(2, VXYZ, EToV[:0], None)
    assert e.value.status == -1
    for N in (0, 7):
        with pytest.raises(W.WadgError) as e:
            W.wadg_mesh_create(N, VXYZ, EToV, None)
        assert e.value.status == -8
    rst = np.zeros((5, 3)) - 0.5
    with pytest.raises(W.WadgError) as e:
        W.wadg_mesh_create(2, VXYZ, EToV, geom, rule=(rst, np.full(5, 4.0 / 15)))
    assert e.value.status == -8
