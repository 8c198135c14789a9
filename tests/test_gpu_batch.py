"""Batches of meshes of uneven size and degree: one persistent launch per
stage gives bitwise the per-mesh results, and each mesh of the batch matches
the FP64 oracle's steps of that mesh alone; the autotuner and the captured
solve keep them."""
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


def _meshes(W, spec):
    ms = []
    for i, (n, N, S) in enumerate(spec):
        VXYZ, EToV, geom = make_mesh_inputs(n, N)
        ms.append(library_mesh(VXYZ, EToV, geom, N, "fp32", shots=S, c2="heterogeneous"))
    return ms


def test_batch_step_equals_per_mesh_steps(W):
    import torch
    spec = [(2, 2, 1), (3, 5, 1), (2, 3, 2), (1, 6, 1), (2, 4, 1), (2, 1, 3)]
    ms = _meshes(W, spec)
    Q0 = [to_torch(random_Q(m.K, m.S, m.Np, 40 + i), torch.float32) for i, m in enumerate(ms)]
    dt, ns = 1e-3, 3
    ref = []
    for m, q in zip(ms, Q0):
        Q, R = q.clone(), torch.zeros_like(q)
        W.wadg_step(m, Q, R, 0.0, dt, ns)
        ref.append((Q, R))
    b = W.wadg_batch_create(ms)
    info = W.wadg_batch_info(b)
    assert info["meshes"] == len(ms) and info["items"] > 0
    Qs = [q.clone() for q in Q0]
    Rs = [torch.zeros_like(q) for q in Q0]
    g = W.wadg_batch_autotune(b, Qs, Rs)
    assert 1 <= g
    W.wadg_batch_step(b, Qs, Rs, 0.0, dt, ns)
    torch.cuda.synchronize()
    for (Qr, Rr), Q, R, q0 in zip(ref, Qs, Rs, Q0):
        assert torch.equal(Qr, Q) and torch.equal(Rr, R)
        assert not torch.equal(Q, q0)
    # captured solve, replayed twice from the same start
    for _ in range(2):
        Qg = [q.clone() for q in Q0]
        Rg = [torch.zeros_like(q) for q in Q0]
        n = W.wadg_batch_solve(b, Qg, Rg, 0.0, dt * ns, dt)
        torch.cuda.synchronize()
        assert n == ns
        for (Qr, Rr), Q, R in zip(ref, Qg, Rg):
            assert torch.equal(Qr, Q) and torch.equal(Rr, R)
    # every tile rule (tile widths and register caps differ), stepped and as a
    # captured solve that is captured again after the rule changes
    for rule in (2, 0, 1):
        W.wadg_batch_set_rule(b, rule)
        info = W.wadg_batch_info(b)
        assert info["rule"] == rule and 1 <= info["grid"] <= info["items"]
        Qs = [q.clone() for q in Q0]
        Rs = [torch.zeros_like(q) for q in Q0]
        W.wadg_batch_step(b, Qs, Rs, 0.0, dt, ns)
        Qg = [q.clone() for q in Q0]
        Rg = [torch.zeros_like(q) for q in Q0]
        W.wadg_batch_solve(b, Qg, Rg, 0.0, dt * ns, dt)
        torch.cuda.synchronize()
        for (Qr, Rr), Q, R, Q2, R2 in zip(ref, Qs, Rs, Qg, Rg):
            assert torch.equal(Qr, Q) and torch.equal(Rr, R)
            assert torch.equal(Qr, Q2) and torch.equal(Rr, R2)
    with pytest.raises(W.WadgError) as e:
        W.wadg_batch_set_rule(b, 3)
    assert e.value.status == -1


def test_batch_step_matches_oracle(W):
    """Four meshes of uneven size and degree (N = 2..5, one with two shots,
    heterogeneous c^2) stepped together by the persistent batch launch: every
    mesh's state after three LSRK steps against the FP64 oracle's steps of
    that mesh alone, element by element, at the FP32 bar."""
    import torch
    from oracle import wadg as OW
    spec = [(2, 2, 1), (1, 5, 1), (2, 3, 2), (2, 4, 1)]
    ms = _meshes(W, spec)
    Q0 = [random_Q(m.K, m.S, m.Np, 60 + i) for i, m in enumerate(ms)]
    Qs = [to_torch(q, torch.float32) for q in Q0]
    Rs = [torch.zeros_like(q) for q in Qs]
    b = W.wadg_batch_create(ms)
    dt, ns = 1e-3, 3
    W.wadg_batch_step(b, Qs, Rs, 0.0, dt, ns)
    torch.cuda.synchronize()
    for (n, N, S), q0, Q, R in zip(spec, Q0, Qs, Rs):
        VXYZ, EToV, geom = make_mesh_inputs(n, N)
        om = oracle_case(VXYZ, EToV, geom, N)
        c2o = oracle_c2(om, "heterogeneous")
        q0 = q0.astype(np.float32).astype(np.float64)
        got_Q = Q.double().cpu().numpy()
        got_R = R.double().cpu().numpy()
        for s in range(S):
            c = om.ref.to_modal(q0[:, :, s])
            res = np.zeros_like(c)
            for k in range(ns):
                c, res = OW.lsrk_step(lambda q, t: OW.rhs(om, q, c2q=c2o), c, res, k * dt, dt)
            l2, mx = rel_errors(got_Q[:, :, s], om.ref.to_nodal(c))
            l2r, _ = rel_errors(got_R[:, :, s], om.ref.to_nodal(res))
            assert l2 < TOL["fp32"] and mx < 10 * TOL["fp32"] and l2r < 10 * TOL["fp32"], (N, s, l2, mx, l2r)


def test_batch_rejects_other_precisions(W):
    VXYZ, EToV, geom = make_mesh_inputs(1, 2)
    m = library_mesh(VXYZ, EToV, geom, 2, "fp64")
    with pytest.raises(W.WadgError) as e:
        W.wadg_batch_create([m])
    assert e.value.status == -5


@pytest.mark.parametrize("precision", ["fp32_3xbf16", "fp32_tf32"])
def test_tensor_core_batch_equals_per_mesh_steps(W, precision):
    """Tensor-core batches: meshes of N = 2..5 (two of N = 4 on the collapsed
    rule share a class, one on the 63-point rule and one with two shots are
    classes of their own) stepped as combined meshes, bitwise equal to
    per-mesh wadg_step, stepped and as a captured solve replayed twice; every
    member against the oracle's steps of that mesh alone."""
    import torch
    from synthetic import fewer_point_rule
    spec = [(2, 2, 1, None), (3, 4, 1, None), (2, 4, 1, None), (2, 4, 1, 4), (1, 5, 1, None), (2, 3, 2, None),
            (4, 4, 1, None)]
    ms = []
    for n, N, S, rule_N in spec:
        VXYZ, EToV, geom = make_mesh_inputs(n, N)
        rule = fewer_point_rule(rule_N) if rule_N else None
        ms.append(library_mesh(VXYZ, EToV, geom, N, precision, shots=S, c2="heterogeneous", rule=rule))
    Q0 = [to_torch(random_Q(m.K, m.S, m.Np, 90 + i), torch.float32) for i, m in enumerate(ms)]
    dt, ns = 1e-3, 3
    ref = []
    for m, q in zip(ms, Q0):
        Q, R = q.clone(), torch.zeros_like(q)
        W.wadg_step(m, Q, R, 0.0, dt, ns)
        ref.append((Q, R))
    b = W.wadg_batch_create(ms)
    info = W.wadg_batch_info(b)
    assert info["meshes"] == len(ms) and info["rule"] == -1
    classes = {}
    for m in ms:
        classes[(m.N, m.Nq, m.S)] = classes.get((m.N, m.Nq, m.S), 0) + m.K * m.S
    assert len(classes) == 5 and info["items"] == sum((c + 127) // 128 for c in classes.values())
    Qs = [q.clone() for q in Q0]
    Rs = [torch.zeros_like(q) for q in Q0]
    W.wadg_batch_step(b, Qs, Rs, 0.0, dt, ns)
    torch.cuda.synchronize()
    for m in ms:
        W.wadg_device_status(m)
    for (Qr, Rr), Q, R, q0 in zip(ref, Qs, Rs, Q0):
        assert torch.equal(Qr, Q) and torch.equal(Rr, R)
        assert not torch.equal(Q, q0)
    # each member against the FP64 oracle's steps of that mesh alone
    from oracle import wadg as OW
    for (n, N, S, rule_N), m, q0, Q in zip(spec, ms, Q0, Qs):
        VXYZ, EToV, geom = make_mesh_inputs(n, N)
        om = oracle_case(VXYZ, EToV, geom, N, rule=fewer_point_rule(rule_N) if rule_N else None)
        c2o = oracle_c2(om, "heterogeneous")
        q0n, got = q0.double().cpu().numpy(), Q.double().cpu().numpy()
        for s in range(S):
            c = om.ref.to_modal(q0n[:, :, s])
            res = np.zeros_like(c)
            for k in range(ns):
                c, res = OW.lsrk_step(lambda q, t: OW.rhs(om, q, c2q=c2o), c, res, k * dt, dt)
            l2, mx = rel_errors(got[:, :, s], om.ref.to_nodal(c))
            assert l2 < TOL[precision] and mx < 10 * TOL[precision], (N, s, l2, mx)
    for _ in range(2):
        Qg = [q.clone() for q in Q0]
        Rg = [torch.zeros_like(q) for q in Q0]
        n = W.wadg_batch_solve(b, Qg, Rg, 0.0, dt * ns, dt)
        torch.cuda.synchronize()
        assert n == ns
        for (Qr, Rr), Q, R in zip(ref, Qg, Rg):
            assert torch.equal(Qr, Q) and torch.equal(Rr, R)
    W.wadg_batch_destroy(b)


def test_tensor_core_batch_refuses_mixed_precisions(W):
    VXYZ, EToV, geom = make_mesh_inputs(1, 2)
    a = library_mesh(VXYZ, EToV, geom, 2, "fp32_3xbf16")
    c = library_mesh(VXYZ, EToV, geom, 2, "fp32")
    for pair in ([a, c], [c, a]):
        with pytest.raises(W.WadgError) as e:
            W.wadg_batch_create(pair)
        assert e.value.status == -5
