"""The partitioned stage on the CUDA path: each rank's local mesh (owned
elements and ghosts, paper_1608_03836_gb300.partition) is created through the
C ABI, its ghosts are filled by the exchange plan, and the library's
right-hand side of every owned column equals, bit for bit, the one of the
whole mesh.  The ranks run one after another on one GPU (no kernel waits on
another); the exchange is the plan's copies between their buffers, in the
order the messages of halo_exchange would carry them."""
import numpy as np
import pytest

from gpu_util import library_mesh, make_mesh_inputs, random_Q, to_torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_03836_gb300 as lib
    return lib


def _exchange(Qs, rms):
    """In-process halo exchange: rank s's send list to r fills r's receive
    list from s (both in increasing global id): whole columns, or the
    face-node values of the shared faces when the plan has them."""
    import torch
    for r, rm in enumerate(rms):
        for s, idx in rm.recv.items():
            dev = Qs[r].device
            if rm.recv_nodes:
                p, n = (torch.as_tensor(a, device=dev) for a in rm.recv_nodes[s])
                ps, ns = (torch.as_tensor(a, device=dev) for a in rms[s].send_nodes[r])
                Qs[r][:, p, :, n] = Qs[s][:, ps, :, ns]
            else:
                src = torch.as_tensor(rms[s].send[r], device=dev)
                Qs[r][:, torch.as_tensor(idx, device=dev)] = Qs[s][:, src]


def _setup(W, n, N, nparts, precision, S, traces=True):
    from paper_1608_03836_gb300 import partition as P
    VXYZ, EToV, geom = make_mesh_inputs(n, N)
    part = P.slab_partition(VXYZ, EToV, nparts)
    rms = [P.build_rank_mesh(EToV, part, r, N=N if traces else None) for r in range(nparts)]
    full = library_mesh(VXYZ, EToV, geom, N, precision, shots=S, c2="heterogeneous")
    subs = [library_mesh(*P.local_inputs(VXYZ, EToV, geom, rm), N, precision, shots=S, c2="heterogeneous")
            for rm in rms]
    return full, subs, rms


@pytest.mark.parametrize("traces", [True, False])
@pytest.mark.parametrize("precision,N,n,nparts,S", [
    ("fp64", 3, 3, 2, 1), ("fp32", 4, 3, 3, 2), ("fp32_3xbf16", 4, 4, 2, 1), ("fp32_3xbf16", 3, 4, 3, 2),
    ("fp32_tf32", 2, 4, 4, 1), ("fp32_3xbf16", 5, 3, 2, 1)])
def test_partitioned_rhs_is_bitwise_the_whole_mesh_rhs(W, precision, N, n, nparts, S, traces):
    """With the trace exchange only the shared faces' nodes of a ghost are
    filled and its other nodes stay NaN: an owned column that read any of
    them would not be finite."""
    import torch
    full, subs, rms = _setup(W, n, N, nparts, precision, S, traces)
    Q = to_torch(random_Q(full.K, S, full.Np, seed=70 + N), full.dtype)
    ref = torch.empty_like(Q)
    W.wadg_rhs(full, Q, ref)
    # each rank starts from its owned columns; ghosts are NaN until the exchange
    Qs = []
    for rm in rms:
        q = torch.full((4, len(rm.elems), S, full.Np), float("nan"), dtype=full.dtype, device="cuda")
        own = torch.as_tensor(rm.owned, device="cuda")
        q[:, own] = Q[:, torch.as_tensor(rm.elems[rm.owned], device="cuda")]
        Qs.append(q)
    _exchange(Qs, rms)
    for m, q, rm in zip(subs, Qs, rms):
        own = torch.as_tensor(rm.owned, device="cuda")
        assert not torch.isnan(q[:, own]).any() and (traces or not torch.isnan(q).any())
        out = torch.empty_like(q)
        W.wadg_rhs(m, q, out)
        torch.cuda.synchronize()
        own = torch.as_tensor(rm.owned, device="cuda")
        assert torch.equal(out[:, own], ref[:, torch.as_tensor(rm.elems[rm.owned], device="cuda")])


@pytest.mark.parametrize("precision", ["fp64", "fp32_3xbf16"])
def test_partitioned_lsrk_step_with_an_exchange_per_stage(W, precision):
    """One LSRK(5,4) step composed of right-hand-side launches with a halo
    exchange before each stage equals, bit for bit, the same composition on
    the whole mesh."""
    import torch
    from oracle.wadg import LSRK_A, LSRK_B
    N, S, dt = 3, 1, 1e-3
    full, subs, rms = _setup(W, 3, N, 2, precision, S)
    Q0 = to_torch(random_Q(full.K, S, full.Np, seed=81), full.dtype)
    Q, R, rf = Q0.clone(), torch.zeros_like(Q0), torch.empty_like(Q0)
    for s in range(5):
        W.wadg_rhs(full, Q, rf)
        R = float(LSRK_A[s]) * R + dt * rf
        Q = Q + float(LSRK_B[s]) * R
    Qs = [Q0[:, torch.as_tensor(rm.elems, device="cuda")].clone() for rm in rms]
    Rs = [torch.zeros_like(q) for q in Qs]
    for s in range(5):
        _exchange(Qs, rms)
        for i, (m, rm) in enumerate(zip(subs, rms)):
            r = torch.empty_like(Qs[i])
            W.wadg_rhs(m, Qs[i], r)
            own = torch.as_tensor(rm.owned, device="cuda")
            Rs[i][:, own] = float(LSRK_A[s]) * Rs[i][:, own] + dt * r[:, own]
            Qs[i][:, own] = Qs[i][:, own] + float(LSRK_B[s]) * Rs[i][:, own]
    torch.cuda.synchronize()
    for q, rm in zip(Qs, rms):
        own = torch.as_tensor(rm.owned, device="cuda")
        assert torch.equal(q[:, own], Q[:, torch.as_tensor(rm.elems[rm.owned], device="cuda")])
