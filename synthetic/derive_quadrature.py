"""Derives the symmetric tetrahedral rules stored in quadrature.py (run once,
offline; about ten minutes for degree 9).

For a fixed orbit structure (kinds as in quadrature.py) the orbit parameters
and weights are fitted to the exact moments of every monomial
l1^a l2^b l3^c (a + b + c <= degree) of the barycentric coordinates,
mean over the simplex a! b! c! 3! / (a + b + c + 3)!, by bounded nonlinear
least squares from seeded random starts; a start that comes within 1e-6 is
polished, and a rule is accepted when every moment is met to 1e-14 with
positive weights and interior points.  Prints the orbit table.

    python -m synthetic.derive_quadrature 9 0 1 1 2 3 3 3 3
    python -m synthetic.derive_quadrature 7 0 1 2 3 3
    python -m synthetic.derive_quadrature 5 1 1 2
"""
from __future__ import annotations

import math
import sys

import numpy as np

from .quadrature import orbit

NPAR = {0: 0, 1: 1, 2: 1, 3: 2, 4: 3}


def _unpack(struct, x):
    pts, ws, i = [], [], 0
    for kind in struct:
        p = x[i:i + NPAR[kind]]
        i += NPAR[kind]
        w = x[i]
        i += 1
        o = orbit(kind, p)
        pts.append(o)
        ws.append(np.full(len(o), w))
    return np.vstack(pts), np.concatenate(ws)


def _moments(degree):
    E = np.array([(a, b, c) for a in range(degree + 1) for b in range(degree + 1 - a)
                  for c in range(degree + 1 - a - b)])
    ex = np.array([math.factorial(a) * math.factorial(b) * math.factorial(c) * 6.0 / math.factorial(a + b + c + 3)
                   for a, b, c in E])
    return E, ex


def _residual(x, struct, E, ex):
    P, w = _unpack(struct, x)
    V = np.prod(P[:, None, :3] ** E[None, :, :], axis=2)
    return V.T @ w - ex


def derive(degree, struct, seed=0, max_tries=100000):
    from scipy.optimize import least_squares
    E, ex = _moments(degree)
    rng = np.random.default_rng(seed)
    npts = sum(len(orbit(k, (0.1, 0.2, 0.3)[:NPAR[k]])) for k in struct)
    for _ in range(max_tries):
        x, lo, hi = [], [], []
        for kind in struct:
            if kind == 1:
                x += [rng.uniform(0.01, 0.33)]; lo += [1e-9]; hi += [1 / 3 - 1e-9]
            elif kind == 2:
                x += [rng.uniform(0.01, 0.49)]; lo += [1e-9]; hi += [0.5 - 1e-9]
            elif kind == 3:
                a = rng.uniform(0.01, 0.45)
                x += [a, rng.uniform(0.01, max(0.02, 1 - 2 * a - 0.01))]; lo += [1e-9, 1e-9]; hi += [0.5, 1.0]
            elif kind == 4:
                b = rng.dirichlet(np.ones(4))
                x += list(b[:3]); lo += [1e-9] * 3; hi += [1.0] * 3
            x += [rng.uniform(0.3, 1.5) / npts]; lo += [1e-12]; hi += [1.0]
        x = np.clip(x, np.array(lo) + 1e-12, np.array(hi) - 1e-12)
        r = least_squares(_residual, x, args=(struct, E, ex), bounds=(lo, hi), xtol=1e-15, ftol=1e-15, gtol=1e-15,
                          max_nfev=400)
        P, w = _unpack(struct, r.x)
        err = np.abs(r.fun).max()
        if err < 1e-6 and P.min() > 1e-6 and w.min() > 0:
            r = least_squares(_residual, r.x, args=(struct, E, ex), bounds=(lo, hi), xtol=3e-16, ftol=3e-16,
                              gtol=3e-16, max_nfev=20000)
            P, w = _unpack(struct, r.x)
            err = np.abs(r.fun).max()
        if err < 1e-14 and P.min() > 1e-8 and w.min() > 0:
            return r.x
    return None


if __name__ == "__main__":
    deg = int(sys.argv[1])
    struct = [int(c) for c in sys.argv[2:]]
    x = derive(deg, struct)
    if x is None:
        sys.exit("no rule found")
    i = 0
    for kind in struct:
        p = tuple(float(v) for v in x[i:i + NPAR[kind]])
        i += NPAR[kind]
        print(f"        ({kind}, {p!r}, {float(x[i])!r}),")
        i += 1
