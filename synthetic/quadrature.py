"""Tabulated symmetric quadrature rules on the tetrahedron with fewer points
than the collapsed Gauss rules, for the volume rule of the method (exact to
degree 2N+1, Sec. 4 and Sec. 6.2).

The paper takes its volume rules from published tables with far fewer points
than a collapsed (N+1)^3 rule; those tables are not available here, so these
rules were derived for this project (derive_quadrature.py) and are stored as
data: an input to the method, like the mesh.  Neither the oracle nor the CUDA
library derives them; each expands the same points and weights and checks
them on its own (the oracle's tests integrate every monomial up to the degree
against its closed form; the library checks P_q V_q = I).

A rule is a list of orbits of the tetrahedron's 24 vertex permutations, each
orbit a barycentric representative and one weight (weights of the
unit-measure simplex, summing to 1):
  kind 0: (1/4, 1/4, 1/4, 1/4)          1 point
  kind 1: (a, a, a, 1 - 3a)             4 points
  kind 2: (a, a, 1/2 - a, 1/2 - a)      6 points
  kind 3: (a, a, b, 1 - 2a - b)        12 points
  kind 4: (a, b, c, 1 - a - b - c)     24 points
"""
from __future__ import annotations

import itertools

import numpy as np

# degree -> [(kind, params, weight)]
SYMMETRIC_RULES = {
    5: [  # 14 points
        (1, (0.3108859192633007,), 0.11268792571801467),
        (1, (0.09273525031089097,), 0.0734930431163615),
        (2, (0.4544962958743488,), 0.04254602077708256),
    ],
    7: [  # 35 points
        (0, (), 0.09548528946629624),
        (1, (0.315701149778696,), 0.04232958120934625),
        (2, (0.4495101774013517,), 0.03189692783303701),
        (3, (0.18883383102579784, 0.5751716375871425), 0.037207130728271594),
        (3, (0.02126547254136205, 0.8108302410985377), 0.008110770829903139),
    ],
    9: [  # 63 points
        (0, (), 0.04151770610161335),
        (1, (0.18298314266204588,), 0.02653856689831988),
        (1, (0.04336357653612531,), 0.007902280000115433),
        (2, (0.39231266615734883,), 0.03434015143753869),
        (3, (0.3467224667488717, 0.2738681019897694), 0.011008782708640634),
        (3, (0.17740783585839787, 0.03864425096987643), 0.02270494969802471),
        (3, (0.031904877425252984, 0.7186038497123036), 0.009405679271801907),
        (3, (0.45903648723540347, 0.0023447430466212007), 0.008103754794817194),
    ],
    11: [  # 96 points (node elimination, seed 100; two orbits at the 1e-3 coordinate bound)
        (1, (0.11804884106967635,), 0.016865718825243983),
        (1, (0.3261574903033582,), 0.01217401352789134),
        (1, (0.06378982468749753,), 0.00700752014248011),
        (1, (0.2931439460454494,), 0.022889376166740832),
        (1, (0.1898897187337074,), 0.0235347681957092),
        (2, (0.10148308055102657,), 0.024818904562489367),
        (3, (0.1334760764817837, 0.001), 0.0038388762804312786),
        (3, (0.013388986005848574, 0.8280685599040966), 0.001794978837598775),
        (3, (0.21750416078041412, 0.04034730197691247), 0.01859369075436357),
        (3, (0.4410289816644533, 0.0028897837578749025), 0.0061188001373923785),
        (2, (0.001,), 0.0012466022509926321),
        (3, (0.04335010420207233, 0.6323945671172728), 0.012033132370589441),
        (1, (0.022818137544555552,), 0.0012919077805852474),
    ],
}


def _representative(kind: int, p) -> tuple:
    if kind == 0:
        return (0.25, 0.25, 0.25, 0.25)
    if kind == 1:
        return (p[0], p[0], p[0], 1.0 - 3.0 * p[0])
    if kind == 2:
        return (p[0], p[0], 0.5 - p[0], 0.5 - p[0])
    if kind == 3:
        return (p[0], p[0], p[1], 1.0 - 2.0 * p[0] - p[1])
    if kind == 4:
        return (p[0], p[1], p[2], 1.0 - p[0] - p[1] - p[2])
    raise ValueError(kind)


def orbit(kind: int, p) -> np.ndarray:
    """The distinct vertex permutations of an orbit's representative, (n, 4)
    barycentric coordinates in lexicographic order of the permuted tuple."""
    rep = _representative(kind, p)
    pts = sorted(set(itertools.permutations(rep)))
    return np.array(pts)


def symmetric_rule(degree: int):
    """Points and weights on the bi-unit reference tetrahedron (vertices
    (-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1)): rst (n, 3) and w (n,),
    weights summing to its volume 4/3."""
    lam, w = [], []
    for kind, p, wt in SYMMETRIC_RULES[degree]:
        pts = orbit(kind, p)
        lam.append(pts)
        w.append(np.full(len(pts), wt))
    lam = np.vstack(lam)
    rst = -1.0 + 2.0 * lam[:, 1:4]
    return rst, np.concatenate(w) * (4.0 / 3.0)


def fewer_point_rule(N: int):
    """The symmetric volume rule exact to degree 2N+1 for N = 2 (14 points),
    N = 3 (35 points), N = 4 (63 points) and N = 5 (96 points)."""
    return symmetric_rule(2 * N + 1)
