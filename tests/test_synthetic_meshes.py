"""The mixed curved/affine cube of the synthetic generator (inputs of the
planar/curved split tests): elements beyond z0 keep their vertices' affine
lattice map exactly, the others are curved, the warp factor is C^1 across
z = z0, and the Jacobians stay positive and close to the affine cube's."""
import numpy as np
import pytest

from synthetic import geometry_nodes, warped_cube


@pytest.mark.parametrize("z0", [0.0, -0.75])
def test_planar_from_keeps_the_far_side_affine(z0):
    n, N = 4, 3
    VXYZ, EToV, geom = warped_cube(n, N, 0.1, planar_from=z0)
    flat = geometry_nodes(VXYZ, EToV, N, 0.0)
    dev = np.abs(geom - flat).max(axis=(1, 2))
    zmin = VXYZ[EToV][:, :, 2].min(axis=1)
    # every element whose vertices lie at z >= z0 is exactly affine
    assert np.all(dev[zmin >= z0] == 0.0)
    # those below are curved (the warp vanishes only on the cube's boundary)
    below = zmin < z0 - 1e-12
    assert below.any() and np.count_nonzero(dev[below] > 1e-6) > 0.9 * np.count_nonzero(below)
    # z is the slowest axis of the element order: the affine elements come last
    aff = np.nonzero(dev == 0.0)[0]
    assert np.all(np.diff(aff) == 1) and aff[-1] == len(EToV) - 1


def test_planar_from_warp_factor_is_c1_at_z0():
    """The factor ((z0 - z)/(1 + z0))^2 for z < z0, 0 beyond: value and slope
    vanish at z0 from both sides, so the displacement is C^1 there."""
    z0, h = -0.25, 1e-6
    VXYZ = np.array([[0.3, -0.2, z0 - h], [0.3, -0.2, z0], [0.3, -0.2, z0 + h], [0.3, -0.2, z0 - 2 * h]])
    EToV = np.array([[0, 1, 2, 3]])
    g = geometry_nodes(VXYZ, EToV, 1, 0.1, planar_from=z0)[0] - geometry_nodes(VXYZ, EToV, 1, 0.0)[0]
    d = np.abs(g).max(axis=1)
    assert d[1] == 0.0 and d[2] == 0.0
    # below z0 the displacement grows like (z0 - z)^2: second-order small
    assert d[0] < 1e-10 and d[3] < 4e-10 and d[3] > 2.0 * d[0]


def test_planar_from_jacobians_positive():
    from oracle.discretization import Mesh, RefTet
    for z0 in (0.0, -0.75):
        VXYZ, EToV, geom = warped_cube(4, 4, 0.1, planar_from=z0)
        m = Mesh(RefTet(4), VXYZ, EToV, geom)
        V0, E0, g0 = warped_cube(4, 4, 0.0)
        m0 = Mesh(RefTet(4), V0, E0, g0)
        r = m.J / m0.J
        assert r.min() > 0.9 and r.max() < 1.2, (z0, r.min(), r.max())
