"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Element-by-element comparisons of nodal values on seeded synthetic inputs,
at sizes that span several blocks and a ragged tail, for every degree the
library builds, both precisions, several shots, heterogeneous c^2, the
boundary, the LSRK step, the projection and the diagnostics.
"""
import math

import numpy as np
import pytest

from gpu_util import (TOL, TRACE_FACTOR, library_mesh, make_mesh_inputs, oracle_c2, oracle_case, random_Q, rel_errors,
                      to_torch)
from synthetic import kuhn_cube, geometry_nodes, standing_wave

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_03836_gb300 as lib
    return lib


def _oracle_rhs(omesh, Qn, c2q=None, tau=(1.0, 1.0)):
    from oracle import wadg as OW
    return OW.rhs_nodal(omesh, Qn, c2q=c2q, tau_p=tau[0], tau_u=tau[1])


def _gpu_rhs(W, m, Q):
    import torch
    Qt = to_torch(Q, m.dtype)
    out = torch.empty_like(Qt)
    W.wadg_rhs(m, Qt, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_3xbf16", "fp32_tf32"])
@pytest.mark.parametrize("N,n", [(1, 3), (2, 2), (3, 2), (4, 2), (5, 2), (6, 1)])
def test_rhs_matches_oracle(W, precision, N, n):
    if precision in ("fp32_3xbf16", "fp32_tf32") and N > 5:
        pytest.skip("the tensor-core stage is built for N <= 5")
    VXYZ, EToV, geom = make_mesh_inputs(n, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, c2="heterogeneous")
    Q = random_Q(m.K, 1, m.Np, seed=100 + N)
    want = _oracle_rhs(om, Q[:, :, 0], c2q=oracle_c2(om, "heterogeneous"))
    got = _gpu_rhs(W, m, Q)[:, :, 0]
    W.wadg_device_status(m)
    l2, mx = rel_errors(got, want)
    print(f"N={N} {precision}: rel L2 {l2:.3e}, rel max {mx:.3e}")
    assert l2 < TOL[precision] and mx < 10 * TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp32_3xbf16"])
@pytest.mark.parametrize("N,n", [(2, 8), (4, 8)])
def test_smooth_fields_rhs_matches_oracle(W, precision, N, n):
    """The standing wave at t = 0.3 projected by the oracle (smooth in every
    element), on the fewer-point rule: the RHS of smooth fields is a small
    difference of large volume and face terms and a derivative of nearly
    constant data, which amplifies the rounding of the operands (by about 1/h
    for element means left in).  Split bf16 with the element means taken out
    of its products stays at 4-7e-5 here (3.4e-4 and 2e-4 with them in, at
    N = 4 and 2 on 3,072 tets); the bar is 1.2e-4, and 4e-5 for FP32 (its
    p field reaches 1.5e-5)."""
    from oracle import wadg as OW
    from synthetic import standing_wave, fewer_point_rule
    rule = fewer_point_rule(N)
    VXYZ, EToV, geom = make_mesh_inputs(n, N)
    om = oracle_case(VXYZ, EToV, geom, N, rule=rule)
    c = OW.wadg_projection(om, standing_wave(om.xq, 0.3))
    Q = om.ref.to_nodal(c)[:, :, None, :]
    m = library_mesh(VXYZ, EToV, geom, N, precision, rule=rule)
    got = _gpu_rhs(W, m, Q)[:, :, 0]
    W.wadg_device_status(m)
    want = _oracle_rhs(om, Q[:, :, 0])
    bar = {"fp32": 4e-5, "fp32_3xbf16": 1.2e-4}[precision]
    for f in range(4):
        l2, _ = rel_errors(got[f], want[f])
        print(f"smooth N={N} n={n} {precision} field {f}: rel L2 {l2:.3e}")
        assert l2 < bar, (f, l2)


def test_volume_points_match_oracle_geometry(W):
    VXYZ, EToV, geom = make_mesh_inputs(2, 4)
    om = oracle_case(VXYZ, EToV, geom, 4)
    m = library_mesh(VXYZ, EToV, geom, 4)
    xq = W.wadg_volume_points(m)
    assert np.abs(xq - om.xq).max() < 1e-14


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_3xbf16", "fp32_tf32"])
def test_shots_and_ragged_tail(W, precision):
    """S = 3 shots of different data on one mesh; K*S = 162 is not a multiple of
    the block width, so the last block is ragged."""
    N, S = 3, 3
    VXYZ, EToV = kuhn_cube(3)
    geom = geometry_nodes(VXYZ, EToV, N, 0.1)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, shots=S)
    Q = random_Q(m.K, S, m.Np, seed=7)
    got = _gpu_rhs(W, m, Q)
    for s in range(S):
        want = _oracle_rhs(om, Q[:, :, s])
        l2, mx = rel_errors(got[:, :, s], want)
        assert l2 < TOL[precision] and mx < 10 * TOL[precision], (s, l2, mx)


@pytest.mark.parametrize("precision", ["fp32", "fp32_3xbf16", "fp32_tf32"])
def test_more_tiles_than_blocks(W, precision):
    """6,000 tets x 4 shots = 24,000 columns: more 128-column tiles (187.5)
    than resident blocks, so persistent blocks take several tiles, the last
    one ragged; heterogeneous c^2."""
    N, S = 4, 4
    VXYZ, EToV, geom = make_mesh_inputs(10, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, shots=S, c2="heterogeneous")
    Q = random_Q(m.K, S, m.Np, seed=31)
    got = _gpu_rhs(W, m, Q)
    W.wadg_device_status(m)
    c2q = oracle_c2(om, "heterogeneous")
    for s in range(S):
        l2, mx = rel_errors(got[:, :, s], _oracle_rhs(om, Q[:, :, s], c2q=c2q))
        assert l2 < TOL[precision] and mx < 10 * TOL[precision], (s, l2, mx)


def test_single_element_all_boundary(W):
    VXYZ = np.array([[-1.0, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]])
    EToV = np.array([[0, 1, 2, 3]])
    N = 4
    geom = geometry_nodes(VXYZ, EToV, N, 0.0)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, "fp64")
    Q = random_Q(1, 1, m.Np, seed=3)
    l2, mx = rel_errors(_gpu_rhs(W, m, Q)[:, :, 0], _oracle_rhs(om, Q[:, :, 0]))
    assert l2 < TOL["fp64"]


@pytest.mark.parametrize("tau", [(0.0, 0.0), (1.0, 0.5)])
def test_penalty_parameters(W, tau):
    VXYZ, EToV, geom = make_mesh_inputs(2, 3)
    om = oracle_case(VXYZ, EToV, geom, 3)
    m = library_mesh(VXYZ, EToV, geom, 3, "fp64", tau=tau)
    Q = random_Q(m.K, 1, m.Np, seed=11)
    l2, _ = rel_errors(_gpu_rhs(W, m, Q)[:, :, 0], _oracle_rhs(om, Q[:, :, 0], tau=tau))
    assert l2 < TOL["fp64"]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_3xbf16", "fp32_tf32"])
def test_lsrk_steps_match_oracle(W, precision):
    import torch
    from oracle import wadg as OW
    N = 3
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, c2="heterogeneous")
    c2o = oracle_c2(om, "heterogeneous")
    Q0 = random_Q(m.K, 1, m.Np, seed=21)
    dt, nsteps = 2e-3, 3
    ref = om.ref
    c = ref.to_modal(Q0[:, :, 0])
    res = np.zeros_like(c)
    for s in range(nsteps):
        c, res = OW.lsrk_step(lambda q, t: OW.rhs(om, q, c2q=c2o), c, res, s * dt, dt)
    Qt = to_torch(Q0, m.dtype)
    Rt = torch.zeros_like(Qt)
    W.wadg_step(m, Qt, Rt, 0.0, dt, nsteps)
    torch.cuda.synchronize()
    l2, mx = rel_errors(Qt.double().cpu().numpy()[:, :, 0], ref.to_nodal(c))
    l2r, _ = rel_errors(Rt.double().cpu().numpy()[:, :, 0], ref.to_nodal(res))
    assert l2 < TOL[precision] and l2r < 10 * TOL[precision], (l2, l2r)


def test_projection_energy_and_error_match_oracle(W):
    import torch
    from oracle import wadg as OW
    N = 4
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, "fp64")
    xq = W.wadg_volume_points(m)
    fq = standing_wave(xq, 0.1)                         # (4, K, Nq) at the library's points
    Q = torch.empty((4, m.K, 1, m.Np), dtype=torch.float64, device="cuda")
    W.wadg_project(m, to_torch(fq[:, :, None, :], torch.float64), Q)
    c = OW.wadg_projection(om, standing_wave(om.xq, 0.1))
    l2, _ = rel_errors(Q.cpu().numpy()[:, :, 0], om.ref.to_nodal(c))
    assert l2 < TOL["fp64"]
    E = W.wadg_energy(m, Q)
    assert abs(E - OW.quadrature_energy(om, c)) < 1e-12 * E
    ex = standing_wave(xq, 0.1)
    err = W.wadg_l2_error(m, Q, to_torch(ex[:, :, None, :], torch.float64), 1)
    vals = np.einsum("qm,km->kq", om.ref.Vq, c[0]) - standing_wave(om.xq, 0.1)[0]
    want = math.sqrt(float(np.sum(om.ref.w_q * om.J * vals ** 2)))
    assert abs(err - want) < 1e-9 * want


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_energy_matches_oracle_with_heterogeneous_wave_speed(W, precision):
    """wadg_energy (FP64 reduction) against the oracle's 1/2 int (p^2/c^2 +
    |u|^2) with c^2 = 1 + 0.5 sin sin sin at the volume points, two shots of
    random fields (the oracle sees the same values the library holds)."""
    from oracle import wadg as OW
    N, S = 3, 2
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, shots=S, c2="heterogeneous")
    Q = random_Q(m.K, S, m.Np, seed=17)
    Qt = to_torch(Q, m.dtype)
    Qh = Qt.double().cpu().numpy()
    c2q = oracle_c2(om, "heterogeneous")
    want = sum(OW.quadrature_energy(om, om.ref.to_modal(Qh[:, :, s]), c2q=c2q) for s in range(S))
    got = W.wadg_energy(m, Qt)
    assert abs(got - want) < 1e-12 * want, (got, want)


def test_bad_arguments_are_rejected(W):
    import torch
    VXYZ, EToV, geom = make_mesh_inputs(1, 2)
    m = library_mesh(VXYZ, EToV, geom, 2, "fp64")
    Q = torch.zeros((4, m.K, 1, m.Np), dtype=torch.float64, device="cuda")
    with pytest.raises(W.WadgError):
        W.wadg_rhs(m, Q, Q)                                  # aliasing
    bad = EToV.copy()
    bad[0, [2, 3]] = bad[0, [3, 2]]                           # inverted element
    with pytest.raises(W.WadgError) as e:
        W.wadg_mesh_create(2, VXYZ, bad, None)
    assert e.value.status == -4
    with pytest.raises(W.WadgError) as e:
        W.wadg_mesh_create(7, VXYZ, EToV, None)
    assert e.value.status == -8


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_3xbf16", "fp32_tf32"])
def test_sources_and_receivers_match_oracle(W, precision):
    """Two shots, each driven by a Ricker point source at its own seeded
    position, three receivers per shot, four LSRK steps from rest."""
    import torch
    from oracle import sources as OS
    from oracle import wadg as OW
    from synthetic import ricker, source_positions, receiver_positions
    N, S, R = 3, 2, 3
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


def test_bounded_wait_expiry_is_reported(W):
    """A device wait that nothing completes gives up after its budget and the
    host reads WADG_ETIMEOUT; the context stays usable and the flag clears."""
    import torch
    VXYZ, EToV, geom = make_mesh_inputs(1, 3)
    m = library_mesh(VXYZ, EToV, geom, 3, "fp32_3xbf16")
    W.wadg_selftest_bounded_wait(m, 2000)
    with pytest.raises(W.WadgError) as e:
        W.wadg_device_status(m)
    assert e.value.status == -6
    Q = torch.zeros((4, m.K, 1, m.Np), dtype=torch.float32, device="cuda")
    out = torch.empty_like(Q)
    W.wadg_rhs(m, Q, out)
    W.wadg_device_status(m)
    assert float(out.abs().max()) == 0.0
