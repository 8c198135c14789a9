"""wadg_solve (captured CUDA graph) and the full c0 solve against stored oracle values."""
import json
import os

import numpy as np
import pytest

from gpu_util import library_mesh, make_mesh_inputs, random_Q, to_torch
from synthetic import standing_wave

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c0_standing_wave.json")


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_03836_gb300 as lib
    return lib


@pytest.mark.parametrize("N", [3, 5])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_3xbf16", "fp32_tf32"])
def test_solve_graph_equals_steps(W, precision, N):
    """The captured graph replays exactly the launches of wadg_step: bitwise
    equal results, also on a second (replayed) call, with sources/receivers
    (N = 5 runs the N = 5 tensor-core stage in the tensor-core precisions)."""
    import torch
    from synthetic import source_positions, receiver_positions
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, shots=2, c2="heterogeneous")
    W.wadg_set_sources(m, source_positions(2), 5.0, 0.05)
    W.wadg_set_receivers(m, receiver_positions(4).reshape(2, 2, 3))
    Q0 = to_torch(random_Q(m.K, 2, m.Np, 4), m.dtype)
    T, dtmax = 0.05, 0.004
    nst = int(np.ceil(T / dtmax))
    outs = []
    for rep in range(2):
        Q, R = Q0.clone(), torch.zeros_like(Q0)
        tr = torch.zeros((nst, 2, 2), dtype=m.dtype, device="cuda")
        n = W.wadg_solve(m, Q, R, 0.0, T, dtmax, tr)
        outs.append((Q.clone(), R.clone(), tr.clone(), n))
    Qs, Rs = Q0.clone(), torch.zeros_like(Q0)
    trs = torch.zeros((nst, 2, 2), dtype=m.dtype, device="cuda")
    W.wadg_step(m, Qs, Rs, 0.0, T / nst, nst, trs)
    torch.cuda.synchronize()
    for Q, R, tr, n in outs:
        assert n == nst
        assert torch.equal(Q, Qs) and torch.equal(R, Rs) and torch.equal(tr, trs)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_c0_standing_wave_matches_oracle_solve(W, precision):
    """c0: 48 tets, N = 3, T = 0.25.  The FP64 GPU error equals the oracle's
    (same discrete solution) to 1e-9 relative; FP32 is within 1.05x of it
    (equal L2 error)."""
    import torch
    g = json.load(open(GOLDEN))
    VXYZ, EToV, geom = make_mesh_inputs(2, 3)
    m = library_mesh(VXYZ, EToV, geom, 3, precision)
    xq = W.wadg_volume_points(m)
    Q = torch.empty((4, m.K, 1, m.Np), dtype=m.dtype, device="cuda")
    W.wadg_project(m, to_torch(standing_wave(xq, 0.0)[:, :, None, :], torch.float64), Q)
    R = torch.zeros_like(Q)
    n = W.wadg_solve(m, Q, R, 0.0, g["T"], g["dt_cfl"])
    assert n == g["nsteps"]
    err = W.wadg_l2_error(m, Q, to_torch(standing_wave(xq, g["T"])[:, :, None, :], torch.float64), 1)
    want = g["wadg"]["l2_error_p_volume_rule"]
    tol = 1e-9 if precision == "fp64" else 0.05
    assert abs(err - want) < tol * want, (err, want)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_3xbf16"])
def test_step_host_equals_step(W, precision):
    """wadg_step_host on pinned host tensors gives exactly wadg_step's result."""
    import torch
    VXYZ, EToV, geom = make_mesh_inputs(2, 3)
    m = library_mesh(VXYZ, EToV, geom, 3, precision, shots=2, c2="heterogeneous")
    Q0 = to_torch(random_Q(m.K, 2, m.Np, 12), m.dtype)
    Qd, Rd = Q0.clone(), torch.zeros_like(Q0)
    W.wadg_step(m, Qd, Rd, 0.0, 0.003, 4)
    Qh, Rh = Q0.cpu().pin_memory(), torch.zeros_like(Q0).cpu().pin_memory()
    W.wadg_step_host(m, Qh, Rh, 0.0, 0.003, 4)
    torch.cuda.synchronize()
    assert torch.equal(Qh, Qd.cpu()) and torch.equal(Rh, Rd.cpu())


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_3xbf16"])
def test_step_does_not_read_the_incoming_residual(W, precision):
    """LSRK(5,4) has a_1 = 0: a step with a residual full of NaN gives exactly
    the result of a step from a zero residual (device and host entry points)."""
    import torch
    VXYZ, EToV, geom = make_mesh_inputs(2, 3)
    m = library_mesh(VXYZ, EToV, geom, 3, precision, shots=2, c2="heterogeneous")
    Q0 = to_torch(random_Q(m.K, 2, m.Np, 13), m.dtype)
    Qa, Ra = Q0.clone(), torch.zeros_like(Q0)
    Qb, Rb = Q0.clone(), torch.full_like(Q0, float("nan"))
    W.wadg_step(m, Qa, Ra, 0.0, 0.003, 2)
    W.wadg_step(m, Qb, Rb, 0.0, 0.003, 2)
    torch.cuda.synchronize()
    assert torch.equal(Qa, Qb) and torch.equal(Ra, Rb)
    Qh, Rh = Q0.cpu().pin_memory(), torch.full_like(Q0, float("nan")).cpu().pin_memory()
    W.wadg_step_host(m, Qh, Rh, 0.0, 0.003, 2)
    assert torch.equal(Qh, Qa.cpu()) and torch.equal(Rh, Ra.cpu())
    Qn = Q0.cpu().pin_memory()
    W.wadg_step_host(m, Qn, None, 0.0, 0.003, 2)  # the residual stays on the device
    assert torch.equal(Qn, Qa.cpu())


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_3xbf16"])
def test_resume_from_a_host_checkpoint_equals_the_uninterrupted_run(W, precision):
    """Checkpoint / resume: six steps in one call against three steps, a dump
    of (Q, res) to host memory, and three more steps from fresh device buffers
    restored from the dump, started at t0 + 3 dt.  With point sources (two
    shots) and dt a power of two, every stage time t0 + n dt + c_s dt is the
    same double in both runs, and the two runs agree bit for bit, receiver
    traces included."""
    import torch
    from synthetic import source_positions, receiver_positions
    N, S, R = 3, 2, 2
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, shots=S)
    W.wadg_set_sources(m, source_positions(S), 5.0, 0.02)
    W.wadg_set_receivers(m, receiver_positions(S * R).reshape(S, R, 3))
    dt = 2.0 ** -9
    Q0 = to_torch(random_Q(m.K, S, m.Np, seed=91), m.dtype) * 1e-3
    Qa, Ra = Q0.clone(), torch.zeros_like(Q0)
    tra = torch.zeros((6, S, R), dtype=m.dtype, device="cuda")
    W.wadg_step(m, Qa, Ra, 0.0, dt, 6, tra)
    Qb, Rb = Q0.clone(), torch.zeros_like(Q0)
    trb = torch.zeros((3, S, R), dtype=m.dtype, device="cuda")
    W.wadg_step(m, Qb, Rb, 0.0, dt, 3, trb)
    dump = (Qb.cpu(), Rb.cpu())                      # the checkpoint, on the host
    del Qb, Rb
    Qc, Rc = dump[0].cuda(), dump[1].cuda()
    trc = torch.zeros((3, S, R), dtype=m.dtype, device="cuda")
    W.wadg_step(m, Qc, Rc, 0.0 + 3 * dt, dt, 3, trc)
    torch.cuda.synchronize()
    W.wadg_device_status(m)
    assert not torch.equal(Qc, Q0)
    assert torch.equal(Qa, Qc) and torch.equal(Ra, Rc)
    assert torch.equal(tra[:3], trb) and torch.equal(tra[3:], trc)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_blow_up_is_reported_by_the_energy(W, precision):
    """Blow-up detector: a state with a non-finite value gives WADG_EUNSTABLE
    from the energy reduction (both entry points); a finite state does not."""
    import torch
    N = 2
    VXYZ, EToV, geom = make_mesh_inputs(2, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision)
    Q = to_torch(random_Q(m.K, 1, m.Np, seed=92), m.dtype)
    assert np.isfinite(W.wadg_energy(m, Q)) and W.wadg_energy(m, Q) > 0
    for bad in (float("nan"), float("inf")):
        Qb = Q.clone()
        Qb[2, m.K // 2, 0, 3] = bad
        for fn in (W.wadg_energy, W.wadg_energy_noalloc):
            with pytest.raises(W.WadgError) as e:
                fn(m, Qb)
            assert e.value.status == -7
    assert W.wadg_energy(m, Q) > 0
