"""Shared helpers of the GPU parity tests: build the same seeded case for the
CUDA library (through its C ABI) and for the FP64 oracle, and compare.

Inputs come from the synthetic generators only; expected values come from
the oracle only.  Nothing computed by the CUDA path is fed to the oracle.
"""
from __future__ import annotations

import numpy as np

from synthetic import warped_cube, c2_heterogeneous, random_fields

# Parity bars (relative L2 over all compared values, and max-abs relative to
# the largest expected value).  FP64: the target 1e-11.  FP32: unit roundoff
# 6e-8 amplified by dot products of up to 3 Nq terms and the operator norms of
# V_q^a / P_q; measured 5e-7 at N <= 4, 7e-7 at N = 5, 1.1e-6 at N = 6 (the
# worst case), so the bar is 2e-6: a tenfold regression anywhere fails.
# Split bf16 (x = hi + lo with bf16 parts of 8 significant bits, three
# products hi*hi + hi*lo + lo*hi): |lo| <= 2^-8 |x|, the residual of the split
# and the dropped lo*lo are each <= 2^-16 relative, so each product carries
# about 2^-16 = 1.5e-5 before amplification; measured 1.2e-5 on the RHS and
# 2.6e-5 on receiver samples of p (a few point values, less averaging): 3e-5.
# TF32 (10-bit mantissa, round to nearest): each operand to 2^-11 = 4.9e-4,
# each product to about 1e-3, three products in series (interpolate, weight,
# project) and the same amplification: 5e-3 (measured 7e-4 to 1e-3).
TOL = {"fp64": 1e-11, "fp32": 2e-6, "fp32_3xbf16": 3e-5, "fp32_tf32": 5e-3}
# Receiver samples p(x_r) = sum_n l_n(x_r) p_n weight every nodal error by the
# Lagrange basis values at x_r (their absolute sum is the Lebesgue function of
# the node lattice, above 1 inside the element), and a relative L2 over a few
# samples does not average the nodal errors as the norm over all nodes does:
# their bar is TRACE_FACTOR times the state's (split bf16, N = 3, measured
# 3.2e-5 on the traces against 6.6e-6 on the state).
TRACE_FACTOR = 4


def make_mesh_inputs(n, N, amp=0.1):
    return warped_cube(n, N, amp)


def oracle_case(VXYZ, EToV, geom, N, rule=None):
    from oracle.discretization import Mesh, RefTet
    ref = RefTet(N, volume_rule=rule)
    return Mesh(ref, VXYZ, EToV, geom)


def library_mesh(VXYZ, EToV, geom, N, precision="fp64", shots=1, c2="one", tau=(1.0, 1.0), rule=None):
    import paper_1608_03836_gb300 as W
    m = W.wadg_mesh_create(N, VXYZ, EToV, geom, rule=rule)
    c2q = None
    if isinstance(c2, np.ndarray):
        c2q = c2
    elif c2 == "heterogeneous":
        c2q = c2_heterogeneous(W.wadg_volume_points(m))
    W.wadg_set_operators(m, precision, shots, tau[0], tau[1], c2q)
    return m


def oracle_c2(omesh, c2):
    if isinstance(c2, np.ndarray):
        return c2
    if c2 == "one":
        return None
    if c2 == "heterogeneous":
        return c2_heterogeneous(omesh.xq)
    return c2


def rel_errors(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    l2 = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300)
    mx = np.abs(got - want).max() / max(np.abs(want).max(), 1e-300)
    return l2, mx


def to_torch(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def random_Q(K, S, Np, seed):
    return random_fields((4, K, S, Np), seed)


FACE_VERTS = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))


def face_neighbours(EToV):
    """EToE (K, 4) from matching sorted vertex triples, -1 on the boundary."""
    EToV = np.asarray(EToV, dtype=np.int64)
    K = len(EToV)
    tri = np.sort(EToV[:, np.array(FACE_VERTS)], axis=2).reshape(-1, 3)
    nv = int(EToV.max()) + 1
    key = (tri[:, 0] * nv + tri[:, 1]) * nv + tri[:, 2]
    order = np.argsort(key, kind="stable")
    sk = key[order]
    i = np.nonzero(sk[1:] == sk[:-1])[0]
    a, b = order[i], order[i + 1]
    E = -np.ones(4 * K, dtype=np.int64)
    E[a] = b // 4
    E[b] = a // 4
    return E.reshape(K, 4)


def sample_columns(EToV, S, count, seed):
    """Seeded (element, shot) columns: the first and last element, elements
    with a boundary face, and random ones."""
    rng = np.random.default_rng(seed)
    K = len(EToV)
    bd = np.nonzero((face_neighbours(EToV) < 0).any(1))[0]
    ks = [0, K - 1] + list(rng.choice(bd, size=min(len(bd), count // 4), replace=False))
    ks += list(rng.choice(K, size=count - len(ks), replace=False))
    return [(int(k), int(rng.integers(S))) for k in ks]


def sampled_oracle_rhs(VXYZ, EToV, geom, N, Q, cols, c2fun=None, c2q_all=None, rule=None, **kw):
    """The oracle's RHS at sampled columns (k, s) of a large mesh, nodal,
    shape (4, len(cols), Np).  The RHS of element k depends only on k and its
    face neighbours, so each column is evaluated on that sub-mesh; its
    elements keep their increasing global order, so every shared face keeps
    its owner (the lower index) and its quadrature points.  c^2 at the volume
    points: c2fun(x), or per-point values c2q_all (K, Nq), or 1."""
    from oracle import wadg as OW
    from oracle.discretization import Mesh, RefTet
    EToV = np.asarray(EToV)
    ref = RefTet(N, volume_rule=rule)
    E = face_neighbours(EToV)
    out = []
    for k, s in cols:
        ks = np.unique(np.concatenate([[k], E[k][E[k] >= 0]]))
        sub = Mesh(ref, VXYZ, EToV[ks], geom[ks])
        c2q = c2q_all[ks] if c2q_all is not None else (None if c2fun is None else c2fun(sub.xq))
        r = OW.rhs_nodal(sub, Q[:, ks, s], c2q=c2q, **kw)
        out.append(r[:, int(np.nonzero(ks == k)[0][0])])
    return np.stack(out, 1)
