"""Element partitioning across ranks (paper_1608_03836_gb300.partition), on
CPU: the local meshes, the halo-exchange plan, and two gloo ranks stepping a
partitioned mesh with one halo exchange per stage.  The arithmetic of a stage
is the oracle's here, which sums each element's face terms in the order of
its mesh's face list, so a local mesh changes the result at round-off (about
1e-16 relative on the right-hand side): the comparisons with the whole mesh
use 1e-13.  The CUDA path's partitioned stage, whose per-column order is
fixed, is compared bit for bit in test_gpu_partition.py."""
import os
import socket

import numpy as np
import pytest

from synthetic import warped_cube, c2_heterogeneous, random_fields

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def part_mod():
    import __graft_entry__ as g
    b = g._build_module()
    if not os.path.exists(b.LIB):
        b.build()
    from paper_1608_03836_gb300 import partition
    return partition


def _oracle_face_neighbours(EToV):
    from gpu_util import face_neighbours
    return face_neighbours(EToV)


@pytest.mark.parametrize("n,nparts", [(2, 2), (3, 2), (3, 3), (4, 4)])
def test_local_meshes_and_exchange_plan(part_mod, n, nparts):
    """Every element is owned once; a rank's ghosts are exactly the face
    neighbours of its elements owned elsewhere; the local mesh is in global
    order; each message's send and receive lists name the same elements in
    the same order."""
    VXYZ, EToV, geom = warped_cube(n, 1, 0.1)
    K = len(EToV)
    E = _oracle_face_neighbours(EToV)
    assert np.array_equal(part_mod.face_neighbours(EToV), E)
    part = part_mod.slab_partition(VXYZ, EToV, nparts)
    assert K % nparts == 0 and np.array_equal(np.bincount(part, minlength=nparts), np.full(nparts, K // nparts))
    rms = [part_mod.build_rank_mesh(EToV, part, r) for r in range(nparts)]
    owned = np.concatenate([rm.elems[rm.owned] for rm in rms])
    assert np.array_equal(np.sort(owned), np.arange(K))
    for rm in rms:
        assert np.all(np.diff(rm.elems) > 0)
        mine = rm.elems[rm.owned]
        assert np.all(part[mine] == rm.rank)
        nb = E[mine].ravel()
        want = np.unique(nb[(nb >= 0) & (part[np.maximum(nb, 0)] != rm.rank)])
        assert np.array_equal(rm.elems[rm.ghosts], want)
        assert sorted(np.concatenate([rm.owned, rm.ghosts])) == list(range(len(rm.elems)))
        for s, idx in rm.send.items():
            assert np.array_equal(rm.elems[idx], rms[s].elems[rms[s].recv[rm.rank]])
        for s, idx in rm.recv.items():
            assert np.all(part[rm.elems[idx]] == s)
    # the trace plan: each message's (element, node) pairs agree on both
    # sides, and name exactly the nodes of the faces shared across the cut
    N = 3
    fn = part_mod.face_node_indices(N)
    assert all(len(f) == (N + 1) * (N + 2) // 2 for f in fn)
    rmt = [part_mod.build_rank_mesh(EToV, part, r, N=N) for r in range(nparts)]
    for rm in rmt:
        for s, (p, nd) in rm.send_nodes.items():
            q, nq = rmt[s].recv_nodes[rm.rank]
            assert np.array_equal(rm.elems[p], rmt[s].elems[q]) and np.array_equal(nd, nq)
            for g in np.unique(rm.elems[p]):
                want = np.unique(np.concatenate([fn[f] for f in range(4) if E[g, f] >= 0 and part[E[g, f]] == s]))
                assert np.array_equal(nd[rm.elems[p] == g], want)
            assert len(p) < len(rm.send[s]) * (N + 1) * (N + 2) * (N + 3) // 6   # fewer values than whole columns
    # the slabs are slabs: owned centroids of rank r lie below those of rank r + 1
    cz = VXYZ[EToV, 2].mean(1)
    for r in range(nparts - 1):
        assert cz[part == r].max() <= cz[part == r + 1].min() + 1e-12


def test_local_rhs_equals_the_whole_mesh_rhs(part_mod):
    """With the ghosts holding their owners' values, the oracle right-hand side
    of every owned element on its rank's local mesh equals the one on the
    whole mesh to round-off (the local mesh keeps every shared face's owner
    and points; a face taken from the wrong side would differ at O(1))."""
    from oracle import wadg as OW
    from oracle.discretization import Mesh, RefTet
    N = 2
    VXYZ, EToV, geom = warped_cube(3, N, 0.1)
    ref = RefTet(N)
    full = Mesh(ref, VXYZ, EToV, geom)
    c = random_fields((4, full.K, ref.Np), 11)
    rf = OW.rhs(full, c, c2q=c2_heterogeneous(full.xq))
    part = part_mod.slab_partition(VXYZ, EToV, 3)
    for r in range(3):
        rm = part_mod.build_rank_mesh(EToV, part, r)
        V, Ev, G = part_mod.local_inputs(VXYZ, EToV, geom, rm)
        sub = Mesh(ref, V, Ev, G)
        rs = OW.rhs(sub, c[:, rm.elems], c2q=c2_heterogeneous(sub.xq))
        d = np.abs(rs[:, rm.owned] - rf[:, rm.elems[rm.owned]]).max()
        assert d <= 1e-13 * np.abs(rf).max()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_worker(rank, ws, port, nsteps, out):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch
    import torch.distributed as dist
    from oracle import wadg as OW
    from oracle.discretization import Mesh, RefTet
    from paper_1608_03836_gb300 import partition as P
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    N = 2
    VXYZ, EToV, geom = warped_cube(3, N, 0.1)
    ref = RefTet(N)
    part = P.slab_partition(VXYZ, EToV, ws)
    rm = P.build_rank_mesh(EToV, part, rank, N=N)
    sub = Mesh(ref, *P.local_inputs(VXYZ, EToV, geom, rm))
    c2q = c2_heterogeneous(sub.xq)
    # nodal fields (the library's layout); this rank starts from its owned
    # columns only; the ghosts' shared-face nodes come from the trace
    # exchange, their other nodes stay 0 (the trace on a face depends only on
    # the face's nodes)
    c0 = ref.to_nodal(random_fields((4, len(EToV), ref.Np), 12))
    q = torch.zeros((4, len(rm.elems), 1, ref.Np), dtype=torch.float64)
    q[:, rm.owned, 0] = torch.from_numpy(c0[:, rm.elems[rm.owned]])
    res = torch.zeros_like(q)
    dt, exchanges = 1e-3, 0
    for _ in range(nsteps):
        for s in range(5):
            P.halo_exchange(q, rm)
            exchanges += 1
            r = ref.to_nodal(OW.rhs(sub, ref.to_modal(q[:, :, 0].numpy()), c2q=c2q))
            o = rm.owned
            res[:, o, 0] = float(OW.LSRK_A[s]) * res[:, o, 0] + dt * torch.from_numpy(r[:, o])
            q[:, o, 0] = q[:, o, 0] + float(OW.LSRK_B[s]) * res[:, o, 0]
    out[rank] = (rm.elems[rm.owned].copy(), q[:, rm.owned, 0].numpy().copy(), exchanges)
    dist.destroy_process_group()


def test_two_gloo_ranks_step_like_the_whole_mesh(part_mod):
    """Two ranks (gloo), two LSRK(5,4) steps with a trace exchange (the
    shared faces' node values) before each stage, each rank starting from its
    owned columns only: the owned columns gathered from both ranks equal the
    same steps on the whole mesh to round-off."""
    import torch.multiprocessing as mp
    from oracle import wadg as OW
    from oracle.discretization import Mesh, RefTet
    ws, port, nsteps = 2, _free_port(), 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_worker, args=(ws, port, nsteps, out), nprocs=ws, join=True)
        res = dict(out)
    N = 2
    VXYZ, EToV, geom = warped_cube(3, N, 0.1)
    full = Mesh(RefTet(N), VXYZ, EToV, geom)
    c2q = c2_heterogeneous(full.xq)
    c = random_fields((4, full.K, full.ref.Np), 12)
    r = np.zeros_like(c)
    for k in range(nsteps):
        c, r = OW.lsrk_step(lambda q, t: OW.rhs(full, q, c2q=c2q), c, r, k * 1e-3, 1e-3)
    c = full.ref.to_nodal(c)
    got = np.full_like(c, np.nan)
    for rank in range(ws):
        ids, q, nex = res[rank]
        got[:, ids] = q
        assert nex == 5 * nsteps
    assert np.isfinite(got).all()
    assert np.abs(got - c).max() <= 1e-13 * np.abs(c).max()
