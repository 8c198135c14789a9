"""Edge cases of the stage against the FP64 oracle: exactly one tile of 128
columns, one tile and one column, a single column; and the size limits of
the tensor-core stage, refused on the host with a status code."""
import numpy as np
import pytest

from gpu_util import TOL, library_mesh, make_mesh_inputs, oracle_case, random_Q, rel_errors, to_torch

pytestmark = pytest.mark.gpu
PRECISIONS = ["fp64", "fp32", "fp32_3xbf16", "fp32_tf32"]


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_03836_gb300 as lib
    return lib


def _rhs_case(W, precision, VXYZ, EToV, geom, N, seed):
    import torch
    from oracle import wadg as OW
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision)
    Q = random_Q(m.K, 1, m.Np, seed)
    Qt = to_torch(Q, m.dtype)
    out = torch.empty_like(Qt)
    W.wadg_rhs(m, Qt, out)
    W.wadg_device_status(m)
    got = out.double().cpu().numpy()[:, :, 0]
    return rel_errors(got, OW.rhs_nodal(om, Q[:, :, 0]))


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("K", [1, 128, 129])
def test_tile_boundaries(W, precision, K):
    """The first K elements of the 384-tet cube (a conforming sub-mesh whose
    cut faces become boundary faces): a single column, exactly one 128-column
    tile, and one tile plus a one-column tail."""
    N = 4
    VXYZ, EToV, geom = make_mesh_inputs(4, N)
    l2, mx = _rhs_case(W, precision, VXYZ, EToV[:K], geom[:K], N, seed=600 + K)
    print(f"K={K} {precision}: rel L2 {l2:.3e}, max {mx:.3e}")
    assert l2 < TOL[precision] and mx < 10 * TOL[precision], (l2, mx)


def test_tensor_core_limits_are_refused(W):
    """K * shots * Np must stay below 2^31 (the 31-bit gather offsets of the
    tensor-core stage), shots <= 2^20, N <= 5 on the tensor cores: each is a
    status code from wadg_set_operators, before anything is allocated."""
    VXYZ, EToV, geom = make_mesh_inputs(2, 5)                # 48 tets, Np = 56
    m = W.wadg_mesh_create(5, VXYZ, EToV, geom)
    with pytest.raises(W.WadgError) as e:
        W.wadg_set_operators(m, "fp32_3xbf16", 1 << 20)      # 48 * 2^20 * 56 > 2^31
    assert e.value.status == -8
    with pytest.raises(W.WadgError) as e:
        W.wadg_set_operators(m, "fp32", (1 << 20) + 1)
    assert e.value.status == -1
    VXYZ, EToV, geom = make_mesh_inputs(1, 6)
    m6 = W.wadg_mesh_create(6, VXYZ, EToV, geom)
    with pytest.raises(W.WadgError) as e:
        W.wadg_set_operators(m6, "fp32_tf32", 1)
    assert e.value.status == -8
    W.wadg_set_operators(m6, "fp32", 1)                      # the CUDA-core stage takes N = 6
