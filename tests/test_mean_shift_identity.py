"""The identity behind the tensor-core stage's mean shift, checked on the
oracle's operators (CPU): for element k with element means pbar_k, ubar_k of
its nodal fields, the strong-weak functional a_h (Sec. 4.1) satisfies

    a_h,k(Q) = a_h,k[fields Q - Qbar_k, averages {u} - ubar_k, jumps of Q]
               + sum_i ubar_k,i a_h,k(p = 0, u = e_i everywhere),

where the last state has {u} = e_i on every face and no jumps, so its value
on element k depends on element k alone; the mean of p drops out (p enters
only through derivatives and jumps).  The update is linear, so the same
holds for the right-hand side with the update applied."""
import numpy as np
import pytest

from oracle import wadg as OW
from oracle.discretization import Mesh, RefTet
from synthetic import warped_cube, fewer_point_rule


def _shifted_a_h(mesh, c, means):
    """a_h with the volume fields less their element means and {u} less the
    element's own velocity mean; the jumps from the unshifted traces."""
    ref = mesh.ref
    K = mesh.K
    Qn = ref.to_nodal(c)
    cs = ref.to_modal(Qn - means[:, :, None])
    w = ref.w_q
    p, u = cs[0], cs[1:]
    uq = np.einsum("qm,ikm->ikq", ref.Vq, u)
    dpq = np.einsum("aqm,km->akq", ref.Vq_a, p)
    U = np.einsum("kqai,ikq->akq", mesh.G, uq)
    gp = np.einsum("kqai,akq->ikq", mesh.G, dpq)
    out = np.zeros_like(c)
    out[0] = np.einsum("aqm,akq->km", ref.Vq_a, w * U)
    out[1:] = -np.einsum("qm,ikq->ikm", ref.Vq, w * gp)
    minus, plus = OW.traces(mesh, c)
    # the flux with {u} less ubar_k: shift both traces' average, keep the jumps
    shift = np.zeros_like(minus)
    shift[1:] = means[1:, :, None, None] * np.ones((1, K, 4, ref.Nfq))
    F = OW.fluxes(mesh, minus - shift, plus - shift)
    for (f, sig), ks in mesh.face_groups.items():
        out[:, ks] += np.einsum("fkp,pm->fkm", F[:, ks, f] * ref.w_f, mesh.face_V[(f, sig)])
    return out


@pytest.mark.parametrize("N", [2, 4])
def test_mean_shift_identity(N):
    VXYZ, EToV, geom = warped_cube(2, N, 0.1)
    mesh = Mesh(RefTet(N, volume_rule=fewer_point_rule(N)), VXYZ, EToV, geom)
    ref = mesh.ref
    rng = np.random.default_rng(11)
    Qn = rng.standard_normal((4, mesh.K, ref.Np)) + rng.standard_normal((4, mesh.K, 1)) * 3.0
    c = ref.to_modal(Qn)
    means = Qn.mean(axis=2)
    D = []
    for i in range(3):
        e = np.zeros((4, mesh.K, ref.Np))
        e[1 + i] = 1.0
        D.append(OW.a_h(mesh, ref.to_modal(e)))
    want = OW.a_h(mesh, c)
    got = _shifted_a_h(mesh, c, means) + sum(means[1 + i][None, :, None] * D[i] for i in range(3))
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    # the constant-velocity state's velocity rows vanish: its jumps and the
    # derivatives of p are zero
    assert max(np.abs(d[1:]).max() for d in D) < 1e-12 * np.abs(want).max()
    # and its pressure row is the discrete divergence of a constant: zero at
    # N = 2 (every integrand is integrated exactly), not at N = 4 (the face
    # integrand n J^f phi has degree 3N - 2 > 2N + 1)
    dp = max(np.abs(d[0]).max() for d in D)
    assert (dp < 1e-12) if N == 2 else (dp > 1e-8)
