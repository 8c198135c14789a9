"""Discrete adjoint of the WADG time stepping, for receiver misfits (FP64).

Test infrastructure (see the package header).  The paper has no adjoint; this
is the exact transpose of the discrete forward map built from the oracle's own
operators (Sec. 4.1 strong-weak form, Sec. 4 / Sec. 6.2 weight-adjusted
inverse, Sec. 7 c^2 weighting, Sec. 5.2 LSRK).  It is meant for tiny meshes:
the right-hand side operator is assembled as a dense matrix column by column
(brute force), and its transpose is the matrix transpose.

Forward, per stage s: res = a_s res + dt (L c + f_s); c = c + b_s res, with
L the modal WADG operator and f_s the source load at the stage time after the
weight-adjusted inverse.  Reverse, per stage s = 5..1:
    mu = lam_res + b_s lam_c;  lam_c += dt L^T mu;  lam_res = a_s mu,
and, because r_p = V_q^T diag(w c^2 / J) V_q b_p in the orthonormal basis,
    dJ/dc^2_q += dt w_q (V_q mu_p)_q (V_q b_p)_q / J_q,
with b_p the pressure load vector (strong-weak terms plus source) at the
stage's input.
"""
from __future__ import annotations

import numpy as np

from . import wadg as OW
from . import sources as OS


def dense_operator(mesh, c2q=None, tau=(1.0, 1.0)) -> np.ndarray:
    """Matrix of the modal RHS c -> rhs(c) (WADG), shape (4 K Np, 4 K Np)."""
    n = 4 * mesh.K * mesh.ref.Np
    L = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        L[:, j] = OW.rhs(mesh, e.reshape(4, mesh.K, mesh.ref.Np), c2q=c2q, tau_p=tau[0], tau_u=tau[1]).ravel()
    return L


class MisfitProblem:
    """Receiver misfit J = sum_n sum_r p_h(x_r, t_n)^2 after every step, one shot."""

    def __init__(self, mesh, c2q, src_xyz, rec_xyz, f0, t0, dt, nsteps):
        from synthetic import ricker
        self.mesh, self.c2q, self.dt, self.nsteps = mesh, c2q, dt, nsteps
        self.src = OS.PointSet(mesh, np.atleast_2d(src_xyz))
        self.rec = OS.PointSet(mesh, rec_xyz)
        self.R = len(self.rec.elem)
        self.amp = lambda t: float(ricker(t, f0, t0))

    def _load(self, c, t):
        return OW.a_h(self.mesh, c) + OS.source_load(self.mesh, self.src, self.amp(t), 0)

    def forward(self, p0_modal, c2q=None, keep=False):
        mesh = self.mesh
        c2q = self.c2q if c2q is None else c2q
        c = np.zeros((4, mesh.K, mesh.ref.Np))
        c[0] = p0_modal
        res = np.zeros_like(c)
        traces, stages = [], []
        for n in range(self.nsteps):
            t = n * self.dt
            for s in range(5):
                ts = t + OW.LSRK_C[s] * self.dt
                if keep:
                    stages.append((c.copy(), ts))
                res = OW.LSRK_A[s] * res + self.dt * OW.wadg_apply(mesh, self._load(c, ts), c2q)
                c = c + OW.LSRK_B[s] * res
            traces.append(OS.sample(c[0], self.rec, np.arange(self.R)))
        traces = np.array(traces)
        return (traces, stages) if keep else traces

    def misfit(self, p0_modal, c2q=None):
        return float(np.sum(self.forward(p0_modal, c2q) ** 2))

    def gradients(self, p0_modal):
        """(J, dJ/dp0_modal (K, Np), dJ/dc^2 (K, Nq)) by the discrete adjoint."""
        mesh, ref, dt = self.mesh, self.mesh.ref, self.dt
        traces, stages = self.forward(p0_modal, keep=True)
        L = dense_operator(mesh, self.c2q)
        shape = (4, mesh.K, ref.Np)
        lam_c = np.zeros(shape)
        lam_r = np.zeros(shape)
        dc2 = np.zeros((mesh.K, ref.Nq))
        g = 2.0 * traces
        for n in reversed(range(self.nsteps)):
            for r in range(self.R):
                lam_c[0, self.rec.elem[r]] += g[n, r] * self.rec.phi[r]
            for s in reversed(range(5)):
                c_in, ts = stages[5 * n + s]
                mu = lam_r + OW.LSRK_B[s] * lam_c
                lam_c = lam_c + dt * (L.T @ mu.ravel()).reshape(shape)
                lam_r = OW.LSRK_A[s] * mu
                b_p = self._load(c_in, ts)[0]
                vm = np.einsum("qm,km->kq", ref.Vq, mu[0])
                vb = np.einsum("qm,km->kq", ref.Vq, b_p)
                dc2 += dt * ref.w_q * vm * vb / mesh.J
        return float(np.sum(traces ** 2)), lam_c[0], dc2
