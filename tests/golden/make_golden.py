"""Write the stored expected values of the GPU solve tests, from the oracle only.

c0_standing_wave.json: the 48-tet warped cube (2^3 hexahedra x 6), N = 3,
warp amplitude 0.1, c^2 = 1, standing wave p = C cos(omega t), u = -grad C
sin(omega t)/omega, WADG pseudo-projection of the initial data, LSRK(5,4) to
T = 0.25 with dt = T / ceil(T / dt_cfl), dt_cfl = 0.5 min_k (min J / max J^f) /
(N+1)^2.  Stores dt, nsteps, the L2 errors of p at T in the volume rule
(degree 2N+1) and in a rich rule (degree 2N+7), and the exact-inverse DG error.

Run: python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import wadg as OW  # noqa: E402
from oracle.discretization import Mesh, RefTet  # noqa: E402
from synthetic import standing_wave, warped_cube  # noqa: E402


def c0():
    N, n, T = 3, 2, 0.25
    VXYZ, EToV, geom = warped_cube(n, N, 0.1)
    ref = RefTet(N)
    mesh = Mesh(ref, VXYZ, EToV, geom)
    h = mesh.J.min(1) / mesh.Jf.reshape(mesh.K, -1).max(1)
    dt_cfl = 0.5 * h.min() / (N + 1) ** 2
    nsteps = int(math.ceil(T / dt_cfl))
    dt = T / nsteps
    out = {"config": "48 tets, N=3, warp 0.1, c2=1, standing wave, T=0.25", "T": T, "dt_cfl": dt_cfl,
           "nsteps": nsteps, "dt": dt}
    for variant in ("wadg", "exact"):
        if variant == "wadg":
            c = OW.wadg_projection(mesh, standing_wave(mesh.xq, 0.0))
        else:
            c = OW.l2_projection(mesh, lambda x: standing_wave(x, 0.0))
        res = np.zeros_like(c)
        for s in range(nsteps):
            c, res = OW.lsrk_step(lambda q, t: OW.rhs(mesh, q, variant=variant), c, res, s * dt, dt)
        rich = OW.l2_error(mesh, c, lambda x: standing_wave(x, T))
        vals = np.einsum("qm,km->kq", ref.Vq, c[0]) - standing_wave(mesh.xq, T)[0]
        qrule = math.sqrt(float(np.sum(ref.w_q * mesh.J * vals ** 2)))
        out[variant] = {"l2_error_p_rich_rule": rich, "l2_error_p_volume_rule": qrule}
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "c0_standing_wave.json"), "w") as f:
        json.dump(c0(), f, indent=1)
    print(open(os.path.join(HERE, "c0_standing_wave.json")).read())
