"""Reference element, mesh connectivity and isoparametric geometry (FP64, modal).

Test infrastructure (see the package header).

Passages followed (Chan, Hewett & Warburton, arXiv:1608.03836):
  * Sec. 2: reference tetrahedron, P^N space, map x = Phi^k(x^) with Jacobian J.
  * Sec. 4.1: J dx^_a/dx_i are cofactors of dx/dx^ (polynomial for an
    isoparametric map); surface integrals are taken over reference faces with
    the surface Jacobian J^f.
  * Sec. 4 and Sec. 6.2: volume rule exact to degree 2N+1.
  * Sec. 6.4 (strong-weak surface kernel): the element and its neighbour use
    values at the same ("neighbouring") face quadrature points.  With the
    collapsed rule used here the point set is not symmetric, so every shared
    face is integrated at the points of one owner, the element with the lower
    index; the other element evaluates its own polynomial at those physical
    points.

Geometry here is computed independently of the CUDA library: the oracle uses
the modal basis for the interpolant, numpy's det/inv for J and the metric,
and a direct cross product of the face tangents for n J^f (the library uses
cofactors and Nanson's formula).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import polynomials as P

# Reference vertices and faces of the bi-unit tetrahedron (Sec. 2).
REF_VERTS = np.array([[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])
FACE_VERTS = [(0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)]
PERMS = list(itertools.permutations(range(3)))


def own_lattice(N: int) -> np.ndarray:
    """Equispaced lattice (interface node set), i fastest then j then k."""
    pts = [(-1 + 2 * i / N, -1 + 2 * j / N, -1 + 2 * k / N)
           for k in range(N + 1) for j in range(N + 1 - k) for i in range(N + 1 - j - k)]
    return np.array(pts)


def face_param(f: int, rs: np.ndarray) -> np.ndarray:
    """Reference-tet coordinates of reference-triangle points (r,s) on face f.

    x^ = -(r+s)/2 v_A + (1+r)/2 v_B + (1+s)/2 v_C with (A,B,C) = FACE_VERTS[f].
    """
    A, B, C = (REF_VERTS[v] for v in FACE_VERTS[f])
    lam = np.stack([-(rs[:, 0] + rs[:, 1]) / 2, (1 + rs[:, 0]) / 2, (1 + rs[:, 1]) / 2], 1)
    return lam[:, :1] * A + lam[:, 1:2] * B + lam[:, 2:3] * C


def face_bary(rs: np.ndarray) -> np.ndarray:
    return np.stack([-(rs[:, 0] + rs[:, 1]) / 2, (1 + rs[:, 0]) / 2, (1 + rs[:, 1]) / 2], 1)


# Sign that makes the cross product of the face tangents (d/dr x d/ds of the
# face parametrisation) point outward, for each reference face.
FACE_ORIENT = np.array([-1.0, 1.0, 1.0, -1.0])


class RefTet:
    """Modal reference operators for degree N (M^ = I in this basis)."""

    def __init__(self, N: int, qdeg_pts: int | None = None, face_pts: int | None = None, volume_rule=None):
        """Collapsed rules with qdeg_pts points per direction on the volume
        and face_pts on the faces (defaults: N+1, exact to degree 2N+1;
        face_pts defaults to qdeg_pts), or an explicit volume rule
        volume_rule = (rst (n, 3), w (n,)) on the reference tetrahedron with the
        default face rule."""
        self.N = N
        self.Np = (N + 1) * (N + 2) * (N + 3) // 6
        self.Nfp = (N + 1) * (N + 2) // 2
        nq = N + 1 if qdeg_pts is None else qdeg_pts
        nf = nq if face_pts is None else face_pts
        if volume_rule is None:
            self.rst_q, self.w_q = P.tet_rule(nq)           # degree 2 nq - 1 volume rule
        else:
            self.rst_q = np.asarray(volume_rule[0], dtype=np.float64)
            self.w_q = np.asarray(volume_rule[1], dtype=np.float64)
        self.Nq = len(self.w_q)
        self.rs_f, self.w_f = P.tri_rule(nf)                # degree 2 nf - 1 face rule
        self.Nfq = len(self.w_f)
        self.lattice = own_lattice(N)
        self.Vn = P.dubiner_tet(N, *self.lattice.T)         # nodal <- modal
        self.Vn_inv = np.linalg.inv(self.Vn)                # modal <- nodal
        self.Vq = P.dubiner_tet(N, *self.rst_q.T)
        self.Vq_a = np.stack(P.dubiner_tet_grad(N, *self.rst_q.T))   # (3, Nq, Np)
        # Face points on the 4 faces, each parametrised by the reference triangle.
        self.rst_f = np.stack([face_param(f, self.rs_f) for f in range(4)])   # (4, Nfq, 3)
        self.Vf = np.stack([P.dubiner_tet(N, *self.rst_f[f].T) for f in range(4)])
        # Tangents of the face parametrisations, d x^/d r_f and d x^/d s_f.
        self.face_tangents = []
        for f in range(4):
            A, B, C = (REF_VERTS[v] for v in FACE_VERTS[f])
            self.face_tangents.append(((B - A) / 2.0, (C - A) / 2.0))

    def to_modal(self, q_nodal):
        return q_nodal @ self.Vn_inv.T

    def to_nodal(self, c_modal):
        return c_modal @ self.Vn.T


class Mesh:
    """Conforming tetrahedral mesh with isoparametric geometry of degree N."""

    def __init__(self, ref: RefTet, VXYZ, EToV, geom_xyz):
        self.ref = ref
        self.VXYZ = np.asarray(VXYZ, dtype=np.float64)
        self.EToV = np.asarray(EToV, dtype=np.int64)
        self.K = len(self.EToV)
        X = np.asarray(geom_xyz, dtype=np.float64)           # (K, Np, 3) at the lattice
        self.geom_xyz = X
        self.Xmodal = np.einsum("mn,knd->kmd", ref.Vn_inv, X)  # modal coefficients of x_h
        self._connect()
        self._geometry()

    # -- connectivity ---------------------------------------------------
    def _connect(self):
        K = self.K
        faces = {}
        self.EToE = -np.ones((K, 4), dtype=np.int64)
        self.EToF = -np.ones((K, 4), dtype=np.int64)
        for k in range(K):
            for f, fv in enumerate(FACE_VERTS):
                key = tuple(sorted(int(self.EToV[k, v]) for v in fv))
                if key in faces:
                    k2, f2 = faces.pop(key)
                    self.EToE[k, f], self.EToF[k, f] = k2, f2
                    self.EToE[k2, f2], self.EToF[k2, f2] = k, f
                else:
                    faces[key] = (k, f)
        # sigma[k,f]: for my face vertex slot m, the owner face slot holding the
        # same global vertex.  Owner = lower element index (self on boundary).
        self.owner = np.where((self.EToE < 0) | (self.EToE > np.arange(K)[:, None]),
                              np.arange(K)[:, None], self.EToE)
        self.owner_face = np.where(self.owner == np.arange(K)[:, None],
                                   np.arange(4)[None, :], self.EToF)
        self.sigma = np.zeros((K, 4, 3), dtype=np.int64)
        for k in range(K):
            for f in range(4):
                ko, fo = self.owner[k, f], self.owner_face[k, f]
                mine = [int(self.EToV[k, v]) for v in FACE_VERTS[f]]
                theirs = [int(self.EToV[ko, v]) for v in FACE_VERTS[fo]]
                self.sigma[k, f] = [theirs.index(g) for g in mine]

    def face_points_ref(self, k: int, f: int) -> np.ndarray:
        """My reference coordinates of the owner's face quadrature points on face f."""
        lam_owner = face_bary(self.ref.rs_f)                 # barycentric on the owner face
        lam_mine = lam_owner[:, self.sigma[k, f]]
        verts = REF_VERTS[list(FACE_VERTS[f])]
        return lam_mine @ verts

    # -- geometry -------------------------------------------------------
    def jacobian_matrix(self, k_idx, rst):
        """dx/dx^ at reference points rst, (len(k_idx), npts, 3 [x_i], 3 [a])."""
        dr, ds, dt = P.dubiner_tet_grad(self.ref.N, *rst.T)
        D = np.stack([dr, ds, dt], axis=-1)                  # (npts, Np, 3[a])
        return np.einsum("pma,kmi->kpia", D, self.Xmodal[k_idx])

    def _geometry(self):
        ref, K = self.ref, self.K
        allk = np.arange(K)
        Jm = self.jacobian_matrix(allk, ref.rst_q)           # (K, Nq, 3, 3)
        self.J = np.linalg.det(Jm)                           # (K, Nq)
        if np.any(self.J <= 0):
            raise ValueError("non-positive Jacobian")
        inv = np.linalg.inv(Jm)                              # inv[..., a, i] = dx^_a/dx_i
        self.G = self.J[..., None, None] * inv               # G[k,q,a,i] = J dx^_a/dx_i
        self.xq = np.einsum("pm,kmd->kpd", ref.Vq, self.Xmodal)
        # Face normals times surface Jacobian at the owner's points, in my
        # element: n J^f = orient * (dx/dr_f x dx/ds_f).
        Nfq = ref.Nfq
        self.nJ = np.zeros((K, 4, Nfq, 3))
        self.face_rst = np.zeros((K, 4, Nfq, 3))
        groups = {}
        for k in range(K):
            for f in range(4):
                groups.setdefault((f, tuple(self.sigma[k, f])), []).append(k)
        self.face_groups = {key: np.array(v) for key, v in groups.items()}
        for (f, sig), ks in self.face_groups.items():
            pts = self.face_points_ref(ks[0], f)
            self.face_rst[ks, f] = pts
            Jm_f = self.jacobian_matrix(ks, pts)             # (nk, Nfq, 3, 3)
            ta, tb = ref.face_tangents[f]
            # The owner's parametrisation seen from my element is the affine
            # image of my face parametrisation under the vertex permutation;
            # it has |det| = 1, so |cross| is unchanged and only the direction
            # sign matters, which FACE_ORIENT fixes for outward normals.
            xr = np.einsum("kpia,a->kpi", Jm_f, ta)
            xs = np.einsum("kpia,a->kpi", Jm_f, tb)
            self.nJ[ks, f] = FACE_ORIENT[f] * np.cross(xr, xs)
        self.Jf = np.linalg.norm(self.nJ, axis=-1)
        # Basis values of my polynomial at the owner's face points, per group.
        self.face_V = {key: P.dubiner_tet(ref.N, *self.face_points_ref(ks[0], key[0]).T)
                       for key, ks in self.face_groups.items()}
