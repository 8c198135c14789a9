"""Kuhn-split warped-cube meshes and the seeded data that drive them.

Everything here is an *input* to the WADG solver: the cube [-1,1]^3 cut into
n^3 hexahedra, each hexahedron split into 6 tetrahedra along the main
diagonal (Kuhn split), and the degree-N isoparametric geometry given as
physical coordinates of the equispaced degree-N lattice of every element,
displaced by a smooth warp that vanishes on the cube boundary.

Node-set convention (shared interface format, documented in include/wadg.h):
on the bi-unit reference tetrahedron {r,s,t >= -1, r+s+t <= -1} the lattice
node (i,j,k), i+j+k <= N, sits at (r,s,t) = (-1+2i/N, -1+2j/N, -1+2k/N); nodes
are ordered with i fastest, then j, then k.  Vertex order of the reference
element: v0=(-1,-1,-1), v1=(1,-1,-1), v2=(-1,1,-1), v3=(-1,-1,1).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

# Angular frequency of the standing wave cos(pi x/2)cos(pi y/2)cos(pi z/2)
# with c^2 = 1: omega^2 = 3 (pi/2)^2.
OMEGA = math.sqrt(3.0) * math.pi / 2.0

# The five workloads: sizes, orders, warp amplitude and material.
CONFIGS = {
    "c0": dict(n=2, N=3, warp=0.1, c2="one", T=0.25,
               desc="48 tets, N=3, FP64, standing wave to T=0.25"),
    "c1": dict(n=32, N=4, warp=0.1, c2="heterogeneous", steps=200,
               desc="196,608 tets, N=4, heterogeneous c^2, FP64 and FP32"),
    "c2": dict(n=24, N=5, warp=0.1, c2="one", T=0.5,
               desc="82,944 tets, N=5, FP32 fields, tensor-core products"),
    "c3": dict(n=16, N=4, warp=0.1, c2="one", shots=64, receivers=8,
               desc="24,576 tets, N=4, 64 Ricker shots, 8 receivers each"),
    "c4": dict(n=16, N=3, warp=0.1, c2="perturbed", steps=300, receivers=16,
               desc="24,576 tets, N=3, adjoint of a receiver misfit"),
}


def lattice_tet(N: int) -> np.ndarray:
    """Equispaced degree-N lattice on the reference tetrahedron, (Np, 3)."""
    pts = []
    for k in range(N + 1):
        for j in range(N + 1 - k):
            for i in range(N + 1 - j - k):
                pts.append((-1.0 + 2.0 * i / N, -1.0 + 2.0 * j / N, -1.0 + 2.0 * k / N))
    return np.array(pts, dtype=np.float64)


def lattice_tri(N: int) -> np.ndarray:
    """Equispaced degree-N lattice on the reference triangle, (Nfp, 2); i fastest."""
    pts = []
    for j in range(N + 1):
        for i in range(N + 1 - j):
            pts.append((-1.0 + 2.0 * i / N, -1.0 + 2.0 * j / N))
    return np.array(pts, dtype=np.float64)


def kuhn_cube(n: int):
    """Vertices and positively oriented tetrahedra of the Kuhn-split cube.

    Returns (VXYZ (Nv,3) float64, EToV (K,4) int64).  Hex (i,j,k) is split
    into the 6 tetrahedra v000 -> v000+e_a -> v000+e_a+e_b -> v111 over the
    permutations (a,b,c) of the axes; every hex uses the same diagonal, so the
    triangulation is conforming.  Element order: hex index i + n(j + n k),
    then the 6 permutations in lexicographic order.  Tets with negative
    orientation have their last two vertices swapped.
    """
    g = np.linspace(-1.0, 1.0, n + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    VXYZ = np.stack([X.ravel(order="F"), Y.ravel(order="F"), Z.ravel(order="F")], axis=1)

    def vid(i, j, k):
        return i + (n + 1) * (j + (n + 1) * k)

    eye = np.eye(3, dtype=np.int64)
    tets = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                base = np.array([i, j, k])
                for perm in itertools.permutations(range(3)):
                    p0 = base
                    p1 = p0 + eye[perm[0]]
                    p2 = p1 + eye[perm[1]]
                    p3 = p2 + eye[perm[2]]
                    tets.append([vid(*p0), vid(*p1), vid(*p2), vid(*p3)])
    EToV = np.array(tets, dtype=np.int64)
    v = VXYZ[EToV]
    d = np.einsum("ki,ki->k", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), v[:, 3] - v[:, 0])
    neg = d < 0
    EToV[neg, 2], EToV[neg, 3] = EToV[neg, 3].copy(), EToV[neg, 2].copy()
    return VXYZ, EToV


def warp_displacement(x: np.ndarray, amplitude: float) -> np.ndarray:
    """Smooth warp d(x) that vanishes on the boundary of [-1,1]^3.

    With C = cos(pi x/2)cos(pi y/2)cos(pi z/2):
    d = a C (1, cos(pi(x-1/2)/2), cos(pi(y-1/2)/2)).
    """
    C = np.cos(np.pi * x[..., 0] / 2) * np.cos(np.pi * x[..., 1] / 2) * np.cos(np.pi * x[..., 2] / 2)
    d = np.empty_like(x)
    d[..., 0] = amplitude * C
    d[..., 1] = amplitude * C * np.cos(np.pi * (x[..., 0] - 0.5) / 2)
    d[..., 2] = amplitude * C * np.cos(np.pi * (x[..., 1] - 0.5) / 2)
    return d


def geometry_nodes(VXYZ, EToV, N: int, amplitude: float, planar_from: float | None = None) -> np.ndarray:
    """Physical coordinates of each element's equispaced lattice, warped; (K, Np, 3).

    planar_from = z0: the warp is multiplied by ((z0 - z) / (1 + z0))^2 for
    z < z0 and by 0 beyond (C^1 across z = z0), so that the elements with
    z >= z0 stay affine: a mesh of curved and planar elements.  z is the
    slowest axis of the element order, so the affine elements come last."""
    rst = lattice_tet(N)
    lam = np.stack([-(1.0 + rst.sum(1)) / 2, (1 + rst[:, 0]) / 2,
                    (1 + rst[:, 1]) / 2, (1 + rst[:, 2]) / 2], axis=1)  # (Np, 4)
    x = np.einsum("nv,kvd->knd", lam, VXYZ[EToV])
    if amplitude != 0.0:
        d = warp_displacement(x, amplitude)
        if planar_from is not None:
            x0 = float(planar_from)
            d = d * (np.minimum(x[..., 2] - x0, 0.0) / (1.0 + x0))[..., None] ** 2
        x = x + d
    return np.ascontiguousarray(x)


def warped_cube(n: int, N: int, amplitude: float = 0.1, planar_from: float | None = None):
    """(VXYZ, EToV, geom_xyz) of the warped Kuhn cube; planar_from: see
    geometry_nodes (a cube curved for z < z0 and planar beyond)."""
    VXYZ, EToV = kuhn_cube(n)
    return VXYZ, EToV, geometry_nodes(VXYZ, EToV, N, amplitude, planar_from)


def standing_wave(x: np.ndarray, t: float):
    """Exact (p, u1, u2, u3) of the standing wave with c^2 = 1, rho = 1.

    p = C cos(omega t), u = -grad C sin(omega t)/omega, with
    C = cos(pi x/2)cos(pi y/2)cos(pi z/2); p = 0 on the cube boundary.
    """
    h = np.pi / 2
    cx, cy, cz = np.cos(h * x[..., 0]), np.cos(h * x[..., 1]), np.cos(h * x[..., 2])
    sx, sy, sz = np.sin(h * x[..., 0]), np.sin(h * x[..., 1]), np.sin(h * x[..., 2])
    C = cx * cy * cz
    st, ct = math.sin(OMEGA * t), math.cos(OMEGA * t)
    p = C * ct
    u1 = h * sx * cy * cz * st / OMEGA
    u2 = h * cx * sy * cz * st / OMEGA
    u3 = h * cx * cy * sz * st / OMEGA
    return np.stack([p, u1, u2, u3], axis=0)


def c2_heterogeneous(x: np.ndarray) -> np.ndarray:
    """c^2(x) = 1 + 0.5 sin(pi x) sin(pi y) sin(pi z)."""
    return 1.0 + 0.5 * np.sin(np.pi * x[..., 0]) * np.sin(np.pi * x[..., 1]) * np.sin(np.pi * x[..., 2])


def c2_perturbed_samples(shape, seed: int = 20161608) -> np.ndarray:
    """c^2 = 1 + 0.1 xi, xi ~ U[-1,1] i.i.d. per volume quadrature point."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return 1.0 + 0.1 * rng.uniform(-1.0, 1.0, size=shape)


def ricker(t, f0: float = 5.0, t0: float | None = None):
    """Ricker wavelet (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = t - t0."""
    if t0 is None:
        t0 = 1.2 / f0
    tau = np.asarray(t, dtype=np.float64) - t0
    a = (np.pi * f0 * tau) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def source_positions(S: int, base_seed: int = 1608) -> np.ndarray:
    """S source points, shot s drawn uniformly in [-0.8,0.8]^3 with seed base_seed+s."""
    out = np.empty((S, 3))
    for s in range(S):
        rng = np.random.Generator(np.random.PCG64(base_seed + s))
        out[s] = rng.uniform(-0.8, 0.8, size=3)
    return out


def receiver_positions(R: int, seed: int = 1608) -> np.ndarray:
    """R receiver points drawn uniformly in [-0.8,0.8]^3."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return rng.uniform(-0.8, 0.8, size=(R, 3))


def random_fields(shape, seed: int) -> np.ndarray:
    """Seeded standard-normal test data (e.g. nodal fields for parity tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(shape)
