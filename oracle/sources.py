"""Point sources and receivers for the oracle (FP64, modal).

Test infrastructure (see the package header).  A point source delta(x - x_s)
f(t) in the pressure equation contributes f(t) v(x_s) to the right-hand side
tested against v (the weak form of Sec. 4.1 with a source term), i.e. the
basis values at the source's reference coordinates in its element; the mass
inverse (exact or weight-adjusted, Sec. 4) is applied afterwards.  A receiver
samples the pressure polynomial at its point.

Point location: Newton's method on x_h(x^) = x in every element whose
geometry-node bounding box (padded by 5 %) holds the point; among the
elements where it converges, the one in which the point is most interior
(largest smallest barycentric coordinate) is chosen.  The CUDA library uses
the same selection rule, so both sides agree on which element owns a point
lying near a shared face.
"""
from __future__ import annotations

import numpy as np

from . import polynomials as P
from .discretization import Mesh


def _geom_nodes(mesh: Mesh):
    return mesh.ref.to_nodal(np.moveaxis(mesh.Xmodal, 2, 0)).transpose(1, 2, 0)  # (K, Np, 3)


def locate(mesh: Mesh, x) -> tuple[int, np.ndarray]:
    x = np.asarray(x, dtype=np.float64)
    X = _geom_nodes(mesh)
    lo, hi = X.min(axis=1), X.max(axis=1)
    pad = 0.05 * (hi - lo) + 1e-12
    cand = np.where(np.all((x >= lo - pad) & (x <= hi + pad), axis=1))[0]
    best, best_k, best_r = -np.inf, -1, None
    for k in cand:
        r = np.array([-0.5, -0.5, -0.5])
        ok = False
        for _ in range(50):
            V = P.dubiner_tet(mesh.ref.N, *r[:, None])                   # (1, Np)
            xr = (V @ mesh.Xmodal[k])[0]
            Jm = mesh.jacobian_matrix(np.array([k]), r[None, :])[0, 0]    # (3 x_i, 3 a)
            try:
                d = np.linalg.solve(Jm, xr - x)
            except np.linalg.LinAlgError:
                break
            r = r - d
            if np.abs(r).max() > 10:
                break
            if np.abs(d).max() < 1e-14:
                ok = True
                break
        if not ok:
            continue
        lam = min((1 + r[0]) / 2, (1 + r[1]) / 2, (1 + r[2]) / 2, -(1 + r.sum()) / 2)
        if lam > best and lam > -1e-10:
            best, best_k, best_r = lam, int(k), r.copy()
    if best_k < 0:
        raise ValueError(f"point {x} is not inside the mesh")
    return best_k, best_r


def point_basis(mesh: Mesh, r) -> np.ndarray:
    """Modal basis values at reference point r, (Np,)."""
    return P.dubiner_tet(mesh.ref.N, *np.asarray(r, dtype=np.float64)[:, None])[0]


class PointSet:
    """Located points: element index and modal basis values per point."""

    def __init__(self, mesh: Mesh, xyz):
        xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
        self.elem = np.empty(len(xyz), dtype=np.int64)
        self.phi = np.empty((len(xyz), mesh.ref.Np))
        for i, x in enumerate(xyz):
            k, r = locate(mesh, x)
            self.elem[i] = k
            self.phi[i] = point_basis(mesh, r)


def source_load(mesh: Mesh, src: PointSet, amplitude: float, shot: int) -> np.ndarray:
    """Modal load vector of shot `shot`'s point source times its amplitude, (4, K, Np)."""
    b = np.zeros((4, mesh.K, mesh.ref.Np))
    b[0, src.elem[shot]] += amplitude * src.phi[shot]
    return b


def sample(c_p: np.ndarray, rec: PointSet, idx) -> np.ndarray:
    """Pressure at receivers idx: sum_m c_m psi_m(x^_r) in the receiver's element."""
    idx = np.atleast_1d(idx)
    return np.einsum("rm,rm->r", c_p[rec.elem[idx]], rec.phi[idx])
