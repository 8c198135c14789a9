"""The tensor-core stage at N = 5 (stage_tc5.cu: two-pass faces, one pressure
accumulator, single-buffered volume operators) against the FP64 oracle:
more 128-column tiles than resident blocks with a ragged last tile and
several shots, LSRK steps, point sources with receivers, an element whose
four faces are all on the boundary; split bf16 and tf32 operands; on the
collapsed 216-point rule and on the 96-point symmetric rule."""
import numpy as np
import pytest

from gpu_util import (TOL, TRACE_FACTOR, library_mesh, make_mesh_inputs, oracle_c2, oracle_case, random_Q, rel_errors,
                      to_torch)
from synthetic import geometry_nodes

pytestmark = pytest.mark.gpu

TC = ["fp32_3xbf16", "fp32_tf32"]


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_03836_gb300 as lib
    return lib


def _gpu_rhs(W, m, Q):
    import torch
    Qt = to_torch(Q, m.dtype)
    out = torch.empty_like(Qt)
    W.wadg_rhs(m, Qt, out)
    W.wadg_device_status(m)
    return out.double().cpu().numpy()


@pytest.mark.parametrize("precision", TC)
def test_tc5_more_tiles_than_blocks(W, precision):
    """6,000 tets x 4 shots = 24,000 columns: 187.5 tiles on at most 152
    persistent blocks, the last tile ragged; heterogeneous c^2."""
    from oracle import wadg as OW
    N, S = 5, 4
    VXYZ, EToV, geom = make_mesh_inputs(10, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, shots=S, c2="heterogeneous")
    assert m.Nq == 216
    Q = random_Q(m.K, S, m.Np, seed=51)
    got = _gpu_rhs(W, m, Q)
    c2q = oracle_c2(om, "heterogeneous")
    for s in range(S):
        l2, mx = rel_errors(got[:, :, s], OW.rhs_nodal(om, Q[:, :, s], c2q=c2q))
        print(f"N=5 {precision} shot {s}: rel L2 {l2:.3e}, max {mx:.3e}")
        assert l2 < TOL[precision] and mx < 10 * TOL[precision], (s, l2, mx)


@pytest.mark.parametrize("precision", TC)
def test_tc5_lsrk_steps_match_oracle(W, precision):
    import torch
    from oracle import wadg as OW
    N = 5
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, c2="heterogeneous", tau=(1.0, 0.5))
    c2o = oracle_c2(om, "heterogeneous")
    Q0 = random_Q(m.K, 1, m.Np, seed=52)
    dt, nsteps = 1e-3, 3
    c = om.ref.to_modal(Q0[:, :, 0].astype(np.float32).astype(np.float64))
    res = np.zeros_like(c)
    for k in range(nsteps):
        c, res = OW.lsrk_step(lambda q, t: OW.rhs(om, q, c2q=c2o, tau_u=0.5), c, res, k * dt, dt)
    Qt = to_torch(Q0, m.dtype)
    Rt = torch.zeros_like(Qt)
    W.wadg_step(m, Qt, Rt, 0.0, dt, nsteps)
    W.wadg_device_status(m)
    l2, mx = rel_errors(Qt.double().cpu().numpy()[:, :, 0], om.ref.to_nodal(c))
    l2r, _ = rel_errors(Rt.double().cpu().numpy()[:, :, 0], om.ref.to_nodal(res))
    print(f"N=5 {precision}: 3 LSRK steps, Q rel L2 {l2:.3e}, res {l2r:.3e}")
    assert l2 < TOL[precision] and mx < 10 * TOL[precision] and l2r < 10 * TOL[precision], (l2, mx, l2r)


@pytest.mark.parametrize("precision", TC)
def test_tc5_sources_and_receivers_match_oracle(W, precision):
    """Two shots with a Ricker point source each (the load enters the update
    at the split of b), three receivers per shot, four steps from rest."""
    import torch
    from oracle import sources as OS
    from oracle import wadg as OW
    from synthetic import ricker, source_positions, receiver_positions
    N, S, R = 5, 2, 3
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, shots=S)
    xs = source_positions(S)
    xr = receiver_positions(S * R).reshape(S, R, 3)
    f0, t0 = 5.0, 0.05
    W.wadg_set_sources(m, xs, f0, t0)
    W.wadg_set_receivers(m, xr)
    dt, nsteps = 2e-3, 4
    Q = torch.zeros((4, m.K, S, m.Np), dtype=m.dtype, device="cuda")
    Rt = torch.zeros_like(Q)
    traces = torch.zeros((nsteps, S, R), dtype=m.dtype, device="cuda")
    W.wadg_step(m, Q, Rt, 0.0, dt, nsteps, traces)
    W.wadg_device_status(m)
    got_Q = Q.double().cpu().numpy()
    got_tr = traces.double().cpu().numpy()
    src = OS.PointSet(om, xs)
    rec = OS.PointSet(om, xr.reshape(-1, 3))
    for s in range(S):
        c = np.zeros((4, om.K, om.ref.Np))
        res = np.zeros_like(c)
        want_tr = []
        L = lambda q, t: OW.wadg_apply(om, OW.a_h(om, q) + OS.source_load(om, src, float(ricker(t, f0, t0)), s))
        for n in range(nsteps):
            c, res = OW.lsrk_step(L, c, res, n * dt, dt)
            want_tr.append(OS.sample(c[0], rec, np.arange(s * R, (s + 1) * R)))
        l2, _ = rel_errors(got_Q[:, :, s], om.ref.to_nodal(c))
        l2t, _ = rel_errors(got_tr[:, s], np.array(want_tr))
        assert l2 < TOL[precision] and l2t < TRACE_FACTOR * TOL[precision], (s, l2, l2t)


@pytest.mark.parametrize("precision", TC)
def test_tc5_single_element_all_boundary(W, precision):
    VXYZ = np.array([[-1.0, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]])
    EToV = np.array([[0, 1, 2, 3]])
    N = 5
    geom = geometry_nodes(VXYZ, EToV, N, 0.0)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision)
    Q = random_Q(1, 1, m.Np, seed=53)
    from oracle import wadg as OW
    l2, mx = rel_errors(_gpu_rhs(W, m, Q)[:, :, 0], OW.rhs_nodal(om, Q[:, :, 0]))
    assert l2 < TOL[precision] and mx < 10 * TOL[precision], (l2, mx)


@pytest.mark.parametrize("precision", TC)
def test_tc5_fewer_point_rule_matches_oracle(W, precision):
    """The 96-point symmetric rule (six volume and six update chunks of 16
    points): 6,000 tets x 2 shots (93.75 tiles, the last ragged) against the
    oracle on the same rule, heterogeneous c^2; then three LSRK steps with
    penalties (1, 0.5) on 48 tets."""
    import torch
    from oracle import wadg as OW
    from synthetic import fewer_point_rule
    N, S = 5, 2
    rule = fewer_point_rule(N)
    VXYZ, EToV, geom = make_mesh_inputs(10, N)
    om = oracle_case(VXYZ, EToV, geom, N, rule=rule)
    m = library_mesh(VXYZ, EToV, geom, N, precision, shots=S, c2="heterogeneous", rule=rule)
    assert m.Nq == 96
    Q = random_Q(m.K, S, m.Np, seed=54)
    got = _gpu_rhs(W, m, Q)
    c2q = oracle_c2(om, "heterogeneous")
    for s in range(S):
        l2, mx = rel_errors(got[:, :, s], OW.rhs_nodal(om, Q[:, :, s], c2q=c2q))
        print(f"N=5 96-point rule {precision} shot {s}: rel L2 {l2:.3e}, max {mx:.3e}")
        assert l2 < TOL[precision] and mx < 10 * TOL[precision], (s, l2, mx)
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    om = oracle_case(VXYZ, EToV, geom, N, rule=rule)
    m = library_mesh(VXYZ, EToV, geom, N, precision, c2="heterogeneous", tau=(1.0, 0.5), rule=rule)
    c2o = oracle_c2(om, "heterogeneous")
    Q0 = random_Q(m.K, 1, m.Np, seed=55)
    dt, nsteps = 1e-3, 3
    c = om.ref.to_modal(Q0[:, :, 0].astype(np.float32).astype(np.float64))
    res = np.zeros_like(c)
    for k in range(nsteps):
        c, res = OW.lsrk_step(lambda q, t: OW.rhs(om, q, c2q=c2o, tau_u=0.5), c, res, k * dt, dt)
    Qt = to_torch(Q0, m.dtype)
    Rt = torch.zeros_like(Qt)
    W.wadg_step(m, Qt, Rt, 0.0, dt, nsteps)
    W.wadg_device_status(m)
    l2, mx = rel_errors(Qt.double().cpu().numpy()[:, :, 0], om.ref.to_nodal(c))
    assert l2 < TOL[precision] and mx < 10 * TOL[precision], (l2, mx)
