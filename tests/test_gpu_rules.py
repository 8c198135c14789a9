"""The fewer-point symmetric volume rules (14 points at N = 2, 35 at N = 3,
63 at N = 4, 96 at N = 5, exact to degree 2N+1) on every stage path against
the oracle on the same rule."""
import numpy as np
import pytest

from gpu_util import TOL, library_mesh, make_mesh_inputs, oracle_c2, oracle_case, random_Q, rel_errors, to_torch

pytestmark = pytest.mark.gpu
PRECISIONS = ["fp64", "fp32", "fp32_3xbf16", "fp32_tf32"]


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_03836_gb300 as lib
    return lib


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("N,n", [(2, 3), (3, 2), (4, 2), (4, 3), (5, 2)])
def test_fewer_point_rhs_matches_oracle(W, precision, N, n):
    """Element by element against the oracle on the same rule (curved,
    heterogeneous c^2 at the rule's points)."""
    import torch
    from oracle import wadg as OW
    from synthetic import fewer_point_rule
    rule = fewer_point_rule(N)
    VXYZ, EToV, geom = make_mesh_inputs(n, N)
    om = oracle_case(VXYZ, EToV, geom, N, rule=rule)
    m = library_mesh(VXYZ, EToV, geom, N, precision, c2="heterogeneous", rule=rule)
    assert m.Nq == len(rule[1]) and np.abs(W.wadg_volume_points(m) - om.xq).max() < 1e-13
    Q = random_Q(m.K, 1, m.Np, seed=400 + N)
    Qt = to_torch(Q, m.dtype)
    out = torch.empty_like(Qt)
    W.wadg_rhs(m, Qt, out)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()[:, :, 0]
    want = OW.rhs_nodal(om, Q[:, :, 0], c2q=oracle_c2(om, "heterogeneous"))
    l2, mx = rel_errors(got, want)
    print(f"fewer-point rule N={N} Nq={m.Nq} K={m.K} {precision}: rel L2 {l2:.3e} (max {mx:.3e})")
    assert l2 < TOL[precision] and mx < 10 * TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32_3xbf16"])
def test_fewer_point_lsrk_steps_and_graph(W, precision):
    """Three LSRK steps with 2 shots against the oracle; the captured solve
    replays them bitwise."""
    import torch
    from oracle import wadg as OW
    from synthetic import fewer_point_rule
    N, S = 4, 2
    rule = fewer_point_rule(N)
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    om = oracle_case(VXYZ, EToV, geom, N, rule=rule)
    m = library_mesh(VXYZ, EToV, geom, N, precision, shots=S, c2="heterogeneous", rule=rule)
    c2o = oracle_c2(om, "heterogeneous")
    Q0 = random_Q(m.K, S, m.Np, seed=31)
    dt, nsteps = 2e-3, 3
    Qt = to_torch(Q0, m.dtype)
    Rt = torch.zeros_like(Qt)
    W.wadg_step(m, Qt, Rt, 0.0, dt, nsteps)
    Qg, Rg = to_torch(Q0, m.dtype), torch.zeros_like(Qt)
    assert W.wadg_solve(m, Qg, Rg, 0.0, nsteps * dt, dt) == nsteps
    torch.cuda.synchronize()
    assert torch.equal(Qg, Qt) and torch.equal(Rg, Rt)
    for s in range(S):
        c = om.ref.to_modal(Q0[:, :, s])
        res = np.zeros_like(c)
        for k in range(nsteps):
            c, res = OW.lsrk_step(lambda q, t: OW.rhs(om, q, c2q=c2o), c, res, k * dt, dt)
        assert rel_errors(Qt.double().cpu().numpy()[:, :, s], om.ref.to_nodal(c))[0] < TOL[precision]


def test_fewer_point_rule_refusals(W):
    """Sizes the kernels are not built for, points outside the element and
    rules not exact to 2N are refused at creation; the strong forms, the
    adjoint and batches are refused for the fewer-point sizes."""
    import torch
    from synthetic import fewer_point_rule
    VXYZ, EToV, geom = make_mesh_inputs(1, 4)
    rst, w = fewer_point_rule(4)
    with pytest.raises(W.WadgError) as e:
        W.wadg_mesh_create(4, VXYZ, EToV, geom, rule=(rst[:62], w[:62]))
    assert e.value.status == -8
    bad = rst.copy()
    bad[0] = (0.5, 0.5, 0.5)
    with pytest.raises(W.WadgError) as e:
        W.wadg_mesh_create(4, VXYZ, EToV, geom, rule=(bad, w))
    assert e.value.status == -8
    with pytest.raises(W.WadgError) as e:    # the degree-7 rule at N = 3 size but N = 4: not 63 points
        W.wadg_mesh_create(4, VXYZ, EToV, geom, rule=fewer_point_rule(3))
    assert e.value.status == -8
    m = library_mesh(VXYZ, EToV, geom, 4, "fp32", rule=(rst, w))
    with pytest.raises(W.WadgError) as e:
        W.wadg_set_formulation(m, "strong")
    assert e.value.status == -8
    lam = torch.zeros((4, m.K, 1, m.Np), dtype=torch.float32, device="cuda")
    with pytest.raises(W.WadgError) as e:
        W.wadg_rhs_adjoint(m, lam, torch.empty_like(lam))
    assert e.value.status == -8
    with pytest.raises(W.WadgError):
        W.wadg_batch_create([m])
