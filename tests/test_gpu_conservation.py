"""Locally conservative update weights (Sec. 3, the remark after the moment
estimate) on every stage path against the oracle's conservative update."""
import numpy as np
import pytest

from gpu_util import TOL, library_mesh, make_mesh_inputs, oracle_c2, oracle_case, random_Q, rel_errors, to_torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_03836_gb300 as lib
    return lib


def _rhs(W, m, Q):
    import torch
    Qt = to_torch(Q, m.dtype)
    out = torch.empty_like(Qt)
    W.wadg_rhs(m, Qt, out)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("precision,form", [("fp64", "strong_weak"), ("fp32", "strong_weak"),
                                            ("fp32_3xbf16", "strong_weak"), ("fp32_tf32", "strong_weak"),
                                            ("fp64", "strong"), ("fp32", "strong")])
@pytest.mark.parametrize("N,n", [(3, 2), (4, 3)])
def test_conservative_rhs_matches_oracle(W, precision, form, N, n):
    """Element by element against the oracle (heterogeneous c^2, curved); the
    result is at least 3x closer to the conservative oracle than to the
    pointwise-weight one (TF32 rounding is of the size of their difference at
    N = 4, so the tolerance alone would not tell them apart)."""
    from oracle import wadg as OW
    VXYZ, EToV, geom = make_mesh_inputs(n, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, c2="heterogeneous")
    W.wadg_set_formulation(m, form)
    W.wadg_set_conservation(m, True)
    Q = random_Q(m.K, 1, m.Np, seed=300 + N)
    got = _rhs(W, m, Q).double().cpu().numpy()[:, :, 0]
    c2o = oracle_c2(om, "heterogeneous")
    want = OW.rhs_nodal(om, Q[:, :, 0], c2q=c2o, form=form, conservative=True)
    l2, mx = rel_errors(got, want)
    pointwise = OW.rhs_nodal(om, Q[:, :, 0], c2q=c2o, form=form)
    other = rel_errors(pointwise, want)[0]
    to_pointwise = rel_errors(got, pointwise)[0]
    print(f"conservative {form} N={N} K={m.K} {precision}: rel L2 {l2:.3e} (max {mx:.3e}); pointwise differs by "
          f"{other:.2e}, GPU to pointwise {to_pointwise:.2e}")
    assert l2 < TOL[precision] and mx < 10 * TOL[precision]
    assert to_pointwise > 3 * l2


@pytest.mark.parametrize("precision", ["fp64", "fp32_3xbf16"])
def test_conservation_setting_order_and_toggle(W, precision):
    """Setting the weights before or after wadg_set_operators gives the same
    result bitwise; switching back restores the pointwise result bitwise; a
    change of c^2 recomputes the conservative weights."""
    from oracle import wadg as OW
    N = 3
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    Q = random_Q(48, 1, 20, seed=9)
    m1 = library_mesh(VXYZ, EToV, geom, N, precision, c2="heterogeneous")
    plain = _rhs(W, m1, Q)
    W.wadg_set_conservation(m1, True)
    after = _rhs(W, m1, Q)
    m2 = W.wadg_mesh_create(N, VXYZ, EToV, geom)
    W.wadg_set_conservation(m2, True)
    from synthetic import c2_heterogeneous
    W.wadg_set_operators(m2, precision, 1, 1.0, 1.0, c2_heterogeneous(W.wadg_volume_points(m2)))
    before = _rhs(W, m2, Q)
    assert (after == before).all() and not (after == plain).all()
    W.wadg_set_conservation(m1, False)
    assert (_rhs(W, m1, Q) == plain).all()
    W.wadg_set_conservation(m1, True)
    W.wadg_set_operators(m1, precision, 1, 1.0, 1.0, None)     # c^2 = 1
    om = oracle_case(VXYZ, EToV, geom, N)
    got = _rhs(W, m1, Q).double().cpu().numpy()[:, :, 0]
    assert rel_errors(got, OW.rhs_nodal(om, Q[:, :, 0], conservative=True))[0] < TOL[precision]


def test_conservative_adjoint_transpose_and_c2_gradient_refused(W):
    """The adjoint operator uses the same weights: <L x, y> = <x, L^T y> in
    FP64 with the conservative weights; the c^2 gradient (recorded forward
    factors) is refused with WADG_EUNSUPPORTED."""
    import torch
    from synthetic import random_fields
    VXYZ, EToV, geom = make_mesh_inputs(2, 3)
    m = library_mesh(VXYZ, EToV, geom, 3, "fp64", shots=2, c2="heterogeneous")
    W.wadg_set_conservation(m, True)
    x = to_torch(random_fields((4, m.K, 2, m.Np), 1), torch.float64)
    y = to_torch(random_fields((4, m.K, 2, m.Np), 2), torch.float64)
    Lx, LTy = torch.empty_like(x), torch.empty_like(y)
    W.wadg_rhs(m, x, Lx)
    W.wadg_rhs_adjoint(m, y, LTy)
    a, b = float((Lx * y).sum()), float((x * LTy).sum())
    assert abs(a - b) < 1e-12 * float(Lx.norm() * y.norm())
    ystore = torch.empty((5, m.K * 2, m.Nq), dtype=torch.float64, device="cuda")
    with pytest.raises(W.WadgError) as e:
        W.wadg_step_record(m, x, torch.zeros_like(x), 0.0, 1e-3, ystore)
    assert e.value.status == -8
