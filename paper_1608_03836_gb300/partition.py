"""Element partitioning of a mesh across ranks, with the halo exchange of one
stage (host-side bookkeeping; the stage itself runs in the library's kernels).

The right-hand side of an element depends only on the element and its four
face neighbours (Sec. 4.1: the numerical flux couples an element to its
neighbours through their traces on the shared faces).  A rank therefore owns
a set of elements and holds, beside them, a copy of every face neighbour
owned by another rank (a ghost).  Before each stage the owners send the
current fields of those elements (the halo exchange); the rank then evaluates
the stage on its local mesh and keeps the results of the elements it owns.

The local mesh lists its elements (owned and ghosts) in increasing global
order.  Every shared face is integrated at the face points of its owner, the
element of lower index, so keeping the global order keeps every face's owner
and points, and an owned element's right-hand side is bitwise the one of the
whole mesh.  Ghost results are discarded: a ghost's own neighbours on other
ranks are missing from the local mesh.

Fields are the library's layout [4][K][S][Np] on the equispaced node lattice
(include/wadg.h).  The library's stage reads of a neighbour only the values
at the nodes of the shared face (it gathers them in the owner's node order
and interpolates them to the face points), so with the degree N given the
exchange moves, per message, the face-node values of the shared faces only:
4 Nfp S values per cut face instead of 4 Np S per ghost element (Nfp = 15,
Np = 35 at N = 4); the other nodes of a ghost are never read.  Without N it
moves whole (element, shot) columns.  Messages are torch.distributed
point-to-point (gloo on CPU tensors, NCCL on CUDA tensors).

One exchange per stage runs before the stage.  At the sizes of a GB300 rack
the halo is small beside the stage (two z-slabs of the 196,608-tet cube
exchange about 0.5 MB per stage and direction in FP32 at N = 4, against a
0.56 ms stage), so the exchange is not overlapped with the interior
elements: that would need the stage split over element subsets, and the
copies between the subsets would cost more than the exchange.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_FACE_VERTS = np.array(((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)))


def face_neighbours(EToV) -> np.ndarray:
    """Face neighbours (K, 4) of a conforming tetrahedral mesh, matched by
    their sorted vertex triples; -1 on the boundary."""
    EToV = np.asarray(EToV, dtype=np.int64)
    K = len(EToV)
    tri = np.sort(EToV[:, _FACE_VERTS], axis=2).reshape(-1, 3)
    nv = int(EToV.max()) + 1 if K else 1
    key = (tri[:, 0] * nv + tri[:, 1]) * nv + tri[:, 2]
    order = np.argsort(key, kind="stable")
    sk = key[order]
    i = np.nonzero(sk[1:] == sk[:-1])[0]
    a, b = order[i], order[i + 1]
    E = -np.ones(4 * K, dtype=np.int64)
    E[a] = b // 4
    E[b] = a // 4
    return E.reshape(K, 4)


def face_node_indices(N: int) -> list:
    """Node indices of the four reference faces (t = -1, s = -1, r + s + t = -1,
    r = -1, the face order of include/wadg.h) on the equispaced lattice of
    degree N, node (i, j, k) at sum_{k' < k} (N-k'+1)(N-k'+2)/2 + j (N-k+1) -
    j (j-1)/2 + i (the library's node order)."""
    faces = [[], [], [], []]
    n = 0
    for k in range(N + 1):
        for j in range(N + 1 - k):
            for i in range(N + 1 - j - k):
                if k == 0:
                    faces[0].append(n)
                if j == 0:
                    faces[1].append(n)
                if i + j + k == N:
                    faces[2].append(n)
                if i == 0:
                    faces[3].append(n)
                n += 1
    return [np.array(f, dtype=np.int64) for f in faces]


def slab_partition(VXYZ, EToV, nparts: int, axis: int = 2) -> np.ndarray:
    """Rank of every element: slabs along one coordinate axis of equal element
    counts (elements sorted by their vertex centroid; ties by index)."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    VXYZ = np.asarray(VXYZ, dtype=np.float64)
    EToV = np.asarray(EToV, dtype=np.int64)
    K = len(EToV)
    cz = VXYZ[EToV, axis].mean(axis=1)
    order = np.lexsort((np.arange(K), cz))
    part = np.empty(K, dtype=np.int64)
    part[order] = (np.arange(K) * nparts) // max(K, 1)
    return part


@dataclass
class RankMesh:
    """One rank's local mesh.  elems: global ids of its elements (owned and
    ghosts) in increasing order; owned / ghosts: positions in elems; send[s]:
    positions of owned elements that rank s holds as ghosts, recv[s]: positions
    of the ghosts that rank s owns, both in increasing global id (so that the
    two sides of a message agree).  With the degree given, send_nodes[s] and
    recv_nodes[s] are (positions, nodes) pairs: the nodes of each such element
    on its faces shared with an element of the other rank, in increasing
    (global id, node)."""
    rank: int
    elems: np.ndarray
    owned: np.ndarray
    ghosts: np.ndarray
    send: dict = field(default_factory=dict)
    recv: dict = field(default_factory=dict)
    send_nodes: dict = field(default_factory=dict)
    recv_nodes: dict = field(default_factory=dict)


def build_rank_mesh(EToV, part, rank: int, EToE=None, N=None) -> RankMesh:
    """The local mesh of `rank` under the element-to-rank map `part`; with the
    degree N, also the face-node lists of the trace exchange."""
    EToV = np.asarray(EToV, dtype=np.int64)
    part = np.asarray(part, dtype=np.int64)
    E = face_neighbours(EToV) if EToE is None else np.asarray(EToE, dtype=np.int64)
    mine = np.nonzero(part == rank)[0]
    nb = E[mine].ravel()
    nb = nb[nb >= 0]
    ghost_ids = np.unique(nb[part[nb] != rank])
    elems = np.union1d(mine, ghost_ids)
    pos = {int(g): i for i, g in enumerate(elems)}
    owned = np.array([pos[int(g)] for g in mine], dtype=np.int64)
    ghosts = np.array([pos[int(g)] for g in ghost_ids], dtype=np.int64)
    rm = RankMesh(rank, elems, owned, ghosts)
    # receive: my ghosts grouped by owner
    for s in np.unique(part[ghost_ids]) if len(ghost_ids) else []:
        ids = ghost_ids[part[ghost_ids] == s]
        rm.recv[int(s)] = np.array([pos[int(g)] for g in ids], dtype=np.int64)
    # send: my elements that are ghosts elsewhere, grouped by the holder
    for s in np.unique(part):
        s = int(s)
        if s == rank:
            continue
        theirs = np.nonzero(part == s)[0]
        tn = E[theirs].ravel()
        tn = np.unique(tn[(tn >= 0)])
        ids = tn[part[tn] == rank]
        if len(ids):
            rm.send[s] = np.array([pos[int(g)] for g in ids], dtype=np.int64)
    if N is not None:
        fn = face_node_indices(N)

        def pairs(ids, other):
            # nodes of element g on its faces whose neighbour rank `other` owns
            P, Nd = [], []
            for g in ids:
                nodes = np.unique(np.concatenate(
                    [fn[f] for f in range(4) if E[g, f] >= 0 and part[E[g, f]] == other]))
                P.append(np.full(len(nodes), pos[int(g)], dtype=np.int64))
                Nd.append(nodes)
            return np.concatenate(P), np.concatenate(Nd)
        for s, idx in rm.send.items():
            rm.send_nodes[s] = pairs(rm.elems[idx], s)
        for s, idx in rm.recv.items():
            rm.recv_nodes[s] = pairs(rm.elems[idx], rank)
    return rm


def local_inputs(VXYZ, EToV, geom, rm: RankMesh):
    """Vertex table, connectivity and curved geometry nodes of the local mesh
    (for wadg_mesh_create); the vertex table is shared, unused vertices are
    ignored."""
    return VXYZ, np.asarray(EToV)[rm.elems], (None if geom is None else np.asarray(geom)[rm.elems])


def halo_exchange(Q, rm: RankMesh, group=None) -> None:
    """Fill the ghosts of the local fields Q [4][K_local][S][Np] from their
    owners (torch.distributed isend/irecv, one message per neighbouring rank
    and direction): the face-node values of the shared faces when the plan
    has them (build_rank_mesh with N), else whole columns.  Every rank of the
    partition must call it."""
    import torch
    import torch.distributed as dist
    dev = Q.device
    traces = bool(rm.send_nodes) or bool(rm.recv_nodes)

    def take(plan, s):
        if traces:
            p, n = plan[s]
            return torch.as_tensor(p, device=dev), torch.as_tensor(n, device=dev)
        return torch.as_tensor(plan[s], device=dev)

    reqs, bufs = [], []
    for s in sorted(rm.send):
        ix = take(rm.send_nodes if traces else rm.send, s)
        buf = (Q[:, ix[0], :, ix[1]] if traces else Q[:, ix]).contiguous()   # [M, 4, S] or [4, M, S, Np]
        bufs.append(buf)
        reqs.append(dist.isend(buf, s, group=group))
    incoming = []
    for s in sorted(rm.recv):
        ix = take(rm.recv_nodes if traces else rm.recv, s)
        shape = ((len(ix[0]), Q.shape[0], Q.shape[2]) if traces else
                 (Q.shape[0], len(ix)) + tuple(Q.shape[2:]))
        buf = torch.empty(shape, dtype=Q.dtype, device=dev)
        incoming.append((ix, buf))
        reqs.append(dist.irecv(buf, s, group=group))
    for r in reqs:
        r.wait()
    for ix, buf in incoming:
        if traces:
            Q[:, ix[0], :, ix[1]] = buf
        else:
            Q[:, ix] = buf

