"""The offline derivation of the tabulated symmetric volume rules
(synthetic/derive_quadrature.py): the node elimination's analytic moment
derivatives, and a small derivation end to end (degree 5, about a second)."""
import math

import numpy as np
import pytest

from synthetic import derive_quadrature as D
from synthetic.quadrature import orbit


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4])
def test_orbit_terms_match_the_orbit_and_central_differences(kind):
    """The moment sums equal the monomials summed over quadrature.py's own
    orbit expansion, and the closed-form logit derivatives equal central
    differences."""
    E, _ = D._moments(11)
    z = np.random.default_rng(kind).normal(0, 1, D.NZ[kind])
    val, dz = D._orbit_terms(kind, z, E)
    P = orbit(kind, D._params(kind, D._coords(kind, z)))
    assert len(P) == D.SIZE[kind]
    want = np.prod(P[:, None, :3] ** E[None], axis=2).sum(0)
    assert np.abs(val - want).max() < 1e-14 * np.abs(want).max()
    for t in range(D.NZ[kind]):
        h = 1e-6
        zp, zm = z.copy(), z.copy()
        zp[t] += h
        zm[t] -= h
        fd = (D._orbit_terms(kind, zp, E)[0] - D._orbit_terms(kind, zm, E)[0]) / (2 * h)
        assert np.abs(fd - dz[:, t]).max() < 1e-7 * np.abs(dz[:, t]).max()


def test_elimination_derives_an_exact_degree_5_rule():
    rule = D.eliminate(5, 1, log=lambda s: None)
    assert rule is not None
    E, ex = D._moments(5)
    got = np.zeros(len(ex))
    npts = 0
    for kind, p, w in rule:
        P = orbit(kind, p)
        assert len(P) == D.SIZE[kind] and w > 0 and P.min() >= D.MIN_COORD - 1e-15
        got += w * np.prod(P[:, None, :3] ** E[None], axis=2).sum(0)
        npts += len(P)
    assert np.abs(got / ex - 1).max() < 1e-12
    assert npts <= 24
    assert math.isclose(sum(w * D.SIZE[k] for k, _, w in rule), 1.0, rel_tol=1e-13)
