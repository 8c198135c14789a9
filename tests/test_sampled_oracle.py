"""The sampled oracle used by the full-size parity tests: each column
evaluated on its element's neighbourhood equals the oracle on the whole mesh
(curved, heterogeneous c^2, two shots, every formulation)."""
import numpy as np
import pytest

from gpu_util import face_neighbours, sample_columns, sampled_oracle_rhs


@pytest.mark.parametrize("form,conservative", [("strong_weak", False), ("strong", False),
                                               ("strong_underintegrated", False), ("strong_weak", True)])
def test_sampled_columns_equal_the_whole_mesh(form, conservative):
    from oracle import wadg as OW
    from oracle.discretization import Mesh, RefTet
    from synthetic import c2_heterogeneous, random_fields, warped_cube
    N, S = 3, 2
    VXYZ, EToV, geom = warped_cube(3, N, 0.1)
    mesh = Mesh(RefTet(N), VXYZ, EToV, geom)
    E = face_neighbours(EToV)
    assert np.array_equal(E, mesh.EToE)
    Q = random_fields((4, mesh.K, S, mesh.ref.Np), 3)
    cols = sample_columns(EToV, S, 12, 0)
    assert (0, cols[0][1]) == cols[0] and cols[1][0] == mesh.K - 1
    got = sampled_oracle_rhs(VXYZ, EToV, geom, N, Q, cols, c2fun=c2_heterogeneous, form=form,
                             conservative=conservative)
    c2q = c2_heterogeneous(mesh.xq)
    for j, (k, s) in enumerate(cols):
        want = OW.rhs_nodal(mesh, Q[:, :, s], c2q=c2q, form=form, conservative=conservative)[:, k]
        assert np.abs(got[:, j] - want).max() < 1e-12 * np.abs(want).max()
