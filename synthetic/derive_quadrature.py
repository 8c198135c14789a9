"""Derives the symmetric tetrahedral rules stored in quadrature.py (run once,
offline).

Two methods, both fitting orbit parameters and weights to the exact moments
of every monomial l1^a l2^b l3^c (a + b + c <= degree) of the barycentric
coordinates, mean over the simplex a! b! c! 3! / (a + b + c + 3)!:

* derive(): for a fixed orbit structure (kinds as in quadrature.py), bounded
  nonlinear least squares from seeded random starts; a start that comes
  within 1e-6 is polished, and a rule is accepted when every moment is met to
  1e-14 with positive weights and interior points (about ten minutes for
  degree 9).

      python -m synthetic.derive_quadrature 9 0 1 1 2 3 3 3 3
      python -m synthetic.derive_quadrature 7 0 1 2 3 3
      python -m synthetic.derive_quadrature 5 1 1 2

* eliminate(): node elimination.  A seeded random set of candidate orbits
  (no 24-point orbits) gets non-negative weights from NNLS on the moment
  equations; the orbits NNLS keeps are polished to an exact rule, and then,
  one move at a time, an orbit is removed or replaced by a smaller kind (two
  equal coordinates merged) and the rule re-polished, a move being kept when
  every moment is still met to 1e-13.  Each orbit is parametrised by logits
  of its distinct barycentric coordinates (1e-3 plus a scaled softmax, so
  every coordinate stays >= 1e-3: points well inside) and by the logarithm
  of its weight (so weights stay positive).
  The degree-11 rule (N = 5):

      python -m synthetic.derive_quadrature --eliminate 11 SEED
"""
from __future__ import annotations

import itertools
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


# ---- node elimination ----

SIZE = {0: 1, 1: 4, 2: 6, 3: 12, 4: 24}    # points per orbit kind
CANDIDATES = {0: 1, 1: 40, 2: 30, 3: 100}  # candidate orbits drawn per kind
MIN_COORD = 1e-3                            # lower bound of every barycentric coordinate
# Each kind as classes of equal barycentric coordinates: class multiplicities
# (the last class has logit 0) and the class labels of the representative.
# Kind 2 puts the pair (a, a) and the pair (1/2 - a, 1/2 - a) in two classes
# of two, whose values sum to 1/2 under this softmax.
CLASSES = {0: ((4,), (0, 0, 0, 0)), 1: ((3, 1), (0, 0, 0, 1)), 2: ((2, 2), (0, 0, 1, 1)),
           3: ((2, 1, 1), (0, 0, 1, 2)), 4: ((1, 1, 1, 1), (0, 1, 2, 3))}
NZ = {k: len(m) - 1 for k, (m, _) in CLASSES.items()}  # logits per kind
# the orbit's points as class labels of their four coordinates
ARRANGEMENTS = {k: np.array(sorted(set(itertools.permutations(lab)))) for k, (_, lab) in CLASSES.items()}


def _class_values(kind, z):
    """u_c = exp(y_c) / sum_c' m_c' exp(y_c'), y = (z, 0): the distinct
    barycentric coordinates of the orbit, positive, sum_c m_c u_c = 1."""
    m = np.array(CLASSES[kind][0], dtype=float)
    y = np.append(np.asarray(z, dtype=float), 0.0)
    e = np.exp(y - y.max())
    return e / (m * e).sum()


def _params(kind, u):
    """quadrature.py's orbit parameters from the class values."""
    n = {0: 0, 1: 1, 2: 1, 3: 2, 4: 3}[kind]
    return tuple(float(v) for v in u[:n])


def _logits(kind, u):
    """Logits of given class values (inverse of _class_values)."""
    u = np.clip(np.asarray(u, dtype=float), 1e-9, None)
    return [math.log(u[c] / u[-1]) for c in range(len(u) - 1)]


def _orbit_terms(kind, z, E):
    """Sum over the orbit's points of every monomial l1^a l2^b l3^c of E and
    its derivatives in the logits.  A point of class labels L has the
    coordinates x_c = MIN_COORD + s u[L_c] (s = 1 - 4 MIN_COORD, so every
    coordinate is >= MIN_COORD and they sum to 1), and with
    du_q/dz_t = u_q (delta_qt - m_t u_t):
    d(prod x_c^E_c)/dz_t = prod x_c^E_c * sum_c E_c s u[L_c] / x_c (delta(L_c, t) - m_t u_t)."""
    m = np.array(CLASSES[kind][0], dtype=float)
    u = _class_values(kind, z)
    s = 1.0 - 4.0 * MIN_COORD
    L = ARRANGEMENTS[kind][:, :3]
    x = MIN_COORD + s * u[L]                      # (points, 3)
    mv = np.exp(np.log(x) @ E.T)                  # (points, monomials)
    val = mv.sum(0)
    ratio = s * u[L] / x
    dz = np.empty((len(E), NZ[kind]))
    for t in range(NZ[kind]):
        coef = ratio * ((L == t) - m[t] * u[t])   # (points, 3)
        dz[:, t] = (mv * (coef @ E.T)).sum(0)
    return val, dz


def _coords(kind, z):
    """The distinct barycentric coordinates of the orbit."""
    return MIN_COORD + (1.0 - 4.0 * MIN_COORD) * _class_values(kind, z)


def _split(kinds, x):
    out, i = [], 0
    for k in kinds:
        out.append((k, x[i:i + NZ[k]], x[i + NZ[k]]))
        i += NZ[k] + 1
    return out


def _fun_jac(kinds, E, ex):
    cache = {}

    def terms(x):
        key = x.tobytes()
        if key not in cache:
            cache.clear()
            r = -ex.copy()
            J = np.empty((len(ex), len(x)))
            i = 0
            for k, z, lw in _split(kinds, x):
                val, dz = _orbit_terms(k, z, E)
                w = math.exp(min(lw, 50.0))
                r += w * val
                J[:, i:i + NZ[k]] = w * dz
                J[:, i + NZ[k]] = w * val
                i += NZ[k] + 1
            cache[key] = (r / ex, J / ex[:, None])
        return cache[key]
    return (lambda x: terms(x)[0]), (lambda x: terms(x)[1])


def _polish(kinds, x, E, ex, nfev):
    """Levenberg-Marquardt on the relative moment residuals; returns the
    parameters and the largest relative residual."""
    from scipy.optimize import least_squares
    f, jac = _fun_jac(kinds, E, ex)
    r = least_squares(f, x, jac=jac, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=nfev)
    return r.x, np.abs(r.fun).max()


def _smaller_kinds(kind, z):
    """Replacements of an orbit by one of a smaller kind, two classes of
    coordinates merged (their mean)."""
    u = _class_values(kind, z)   # merged in the class values (the map to coordinates is affine)
    out = []
    if kind == 4:
        s = np.sort(u)
        for i in range(3):   # (a, a, b, d) from the two closest coordinates
            rest = [s[t] for t in range(4) if t not in (i, i + 1)]
            out.append((3, _logits(3, (0.5 * (s[i] + s[i + 1]), rest[0], rest[1]))))
    elif kind == 3:
        a, b, d = u
        out.append((1, _logits(1, ((2 * a + b) / 3, d))))
        out.append((1, _logits(1, ((2 * a + d) / 3, b))))
        out.append((2, _logits(2, (a, 0.5 * (b + d)))))
    elif kind in (1, 2):
        out.append((0, []))
    return out


def eliminate(degree, seed, log=print):
    """Node elimination from a seeded candidate set; returns [(kind, params,
    weight)] (weights of the unit-measure simplex) or None."""
    from scipy.optimize import nnls
    E, ex = _moments(degree)
    rng = np.random.default_rng(seed)
    kinds, zs = [], []
    for k, n in CANDIDATES.items():
        for _ in range(n):
            kinds.append(k)
            zs.append(rng.normal(0, 1.5, NZ[k]))
    A = np.stack([_orbit_terms(k, z, E)[0] for k, z in zip(kinds, zs)], 1) / ex[:, None]
    w, _ = nnls(A, np.ones(len(ex)), maxiter=20000)
    keep = np.nonzero(w > 1e-14)[0]
    kinds = [kinds[i] for i in keep]
    x = np.array([v for i in keep for v in list(zs[i]) + [math.log(w[i])]])
    x, err = _polish(kinds, x, E, ex, 2000)
    if err > 1e-12:
        return None
    log(f"{len(kinds)} orbits, {sum(SIZE[k] for k in kinds)} points")
    while True:
        parts = _split(kinds, x)
        sig = [math.exp(lw) * SIZE[k] / (NZ[k] + 1) for k, z, lw in parts]
        moves = [(SIZE[parts[j][0]], j, None) for j in np.argsort(sig)]
        for j, (k, z, lw) in enumerate(parts):
            moves += [(SIZE[k] - SIZE[k2], j, (k2, z2)) for k2, z2 in _smaller_kinds(k, z)]
        moves.sort(key=lambda mv: -mv[0])
        for _, j, rep in moves:
            nk, nx = [], []
            for t, (k, z, lw) in enumerate(parts):
                if t == j:
                    if rep is None:
                        continue
                    k, z = rep
                nk.append(k)
                nx += list(z) + [lw]
            nx, e2 = _polish(nk, np.array(nx), E, ex, 1000)
            if e2 < 1e-13:
                kinds, x = nk, nx
                log(f"{len(nk)} orbits, {sum(SIZE[k] for k in nk)} points")
                break
        else:
            break
    return [(k, _params(k, _coords(k, z)), float(math.exp(lw))) for k, z, lw in _split(kinds, x)]


if __name__ == "__main__":
    if sys.argv[1] == "--eliminate":
        rule = eliminate(int(sys.argv[2]), int(sys.argv[3]))
        if rule is None:
            sys.exit("no rule found")
        print(f"        # {sum(SIZE[k] for k, _, _ in rule)} points")
        for kind, p, w in rule:
            print(f"        ({kind}, {p!r}, {w!r}),")
        sys.exit(0)
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
