"""Parity at the full workload sizes, in the launch configuration that
bench.py times (the persistent tensor-core stage on all SMs, the CUDA-core
stage over all columns), on sampled columns that the oracle evaluates one by
one from each element's neighbourhood:

  * warped cube 32^3 x 6 = 196,608 tets, N = 4, heterogeneous c^2: FP64, FP32,
    split bf16 and TF32 tensor cores, also on the 63-point volume rule; the
    strong form and the conservative
    weights in FP32; one LSRK step (tensor cores and CUDA cores) against five
    RHS launches composed on the device;
  * 24^3 x 6 = 82,944 tets, N = 5: FP32, split bf16 and TF32 on the collapsed
    rule, and FP64 and both tensor precisions on the 96-point rule;
  * 16^3 x 6 = 24,576 tets, N = 4, 64 shots as columns, split bf16;
  * 16^3 x 6 tets, N = 3, FP32, c^2 perturbed by 10 % per point.
"""
import numpy as np
import pytest

from gpu_util import TOL, rel_errors, sample_columns, sampled_oracle_rhs, to_torch

pytestmark = pytest.mark.gpu
SAMPLES = 32


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_03836_gb300 as lib
    return lib


_CUBES = {}


def cube(n, N):
    if (n, N) not in _CUBES:
        from synthetic import warped_cube
        _CUBES[(n, N)] = warped_cube(n, N, 0.1)
    return _CUBES[(n, N)]


def run_sampled(W, n, N, precision, S=1, c2="heterogeneous", form="strong_weak", conservative=False, seed=0,
                rule=None):
    import torch
    from synthetic import c2_heterogeneous, random_fields
    VXYZ, EToV, geom = cube(n, N)
    m = W.wadg_mesh_create(N, VXYZ, EToV, geom, rule=rule)
    xq = W.wadg_volume_points(m)
    c2q, c2fun = None, None
    if isinstance(c2, np.ndarray):
        c2q = c2
    elif c2 == "heterogeneous":
        c2q, c2fun = c2_heterogeneous(xq), c2_heterogeneous
    W.wadg_set_operators(m, precision, S, 1.0, 1.0, c2q)
    if form != "strong_weak":
        W.wadg_set_formulation(m, form)
    if conservative:
        W.wadg_set_conservation(m, True)
    Q = random_fields((4, m.K, S, m.Np), 700 + seed)
    Qt = to_torch(Q, m.dtype)
    out = torch.empty_like(Qt)
    W.wadg_rhs(m, Qt, out)
    W.wadg_device_status(m)
    got = out.double().cpu().numpy()
    cols = sample_columns(EToV, S, SAMPLES, seed)
    want = sampled_oracle_rhs(VXYZ, EToV, geom, N, Q, cols, c2fun=c2fun,
                              c2q_all=c2 if isinstance(c2, np.ndarray) else None, rule=rule, form=form,
                              conservative=conservative)
    g = np.stack([got[:, k, s] for k, s in cols], 1)
    l2, mx = rel_errors(g, want)
    print(f"n={n} N={N} K={m.K} Nq={m.Nq} S={S} {precision} {form}{' conservative' if conservative else ''}: "
          f"{len(cols)} sampled columns, rel L2 {l2:.3e}, max {mx:.3e}")
    assert l2 < TOL[precision] and mx < 10 * TOL[precision]
    return m


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_3xbf16", "fp32_tf32"])
def test_c1_rhs_sampled(W, precision):
    run_sampled(W, 32, 4, precision, seed=1)


@pytest.mark.parametrize("precision,form,conservative", [("fp32", "strong", False), ("fp64", "strong", False),
                                                        ("fp32", "strong_weak", True)])
def test_c1_variants_sampled(W, precision, form, conservative):
    run_sampled(W, 32, 4, precision, form=form, conservative=conservative, seed=2)


def test_c1_conservative_tensor_cores_on_the_fewer_point_rule_sampled(W):
    from synthetic import fewer_point_rule
    run_sampled(W, 32, 4, "fp32_3xbf16", conservative=True, seed=7, rule=fewer_point_rule(4))


@pytest.mark.parametrize("precision", ["fp32_3xbf16", "fp32"])
def test_c1_lsrk_step_composes_rhs(W, precision):
    """One wadg_step (the LSRK mode of the stage, as bench.py times it) equals
    five wadg_rhs launches composed with the LSRK(5,4) coefficients on the
    device, to 10x the parity tolerance of one RHS (the two paths round the
    products of slightly different stage inputs differently)."""
    import torch
    from synthetic import c2_heterogeneous, random_fields
    from oracle.wadg import LSRK_A, LSRK_B
    VXYZ, EToV, geom = cube(32, 4)
    m = W.wadg_mesh_create(4, VXYZ, EToV, geom)
    W.wadg_set_operators(m, precision, 1, 1.0, 1.0, c2_heterogeneous(W.wadg_volume_points(m)))
    Q0 = to_torch(random_fields((4, m.K, 1, m.Np), 703), torch.float32)
    Q, R = Q0.clone(), torch.zeros_like(Q0)
    dt = 1e-3
    W.wadg_step(m, Q, R, 0.0, dt, 1)
    q, res, r = Q0.clone(), torch.zeros_like(Q0), torch.empty_like(Q0)
    for s in range(5):
        W.wadg_rhs(m, q, r)
        res = float(LSRK_A[s]) * res + dt * r
        q = q + float(LSRK_B[s]) * res
    torch.cuda.synchronize()
    W.wadg_device_status(m)
    eq = float((Q - q).norm()) / float((q - Q0).norm())
    er = float((R - res).norm()) / float(res.norm())
    print(f"{precision}: one LSRK step vs composed RHS: Q {eq:.3e} (of the increment), res {er:.3e}")
    assert eq < 10 * TOL[precision] and er < 10 * TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32_3xbf16", "fp32_tf32"])
def test_c1_fewer_point_rule_sampled(W, precision):
    from synthetic import fewer_point_rule
    run_sampled(W, 32, 4, precision, seed=6, rule=fewer_point_rule(4))


@pytest.mark.parametrize("precision", ["fp32", "fp32_3xbf16", "fp32_tf32"])
def test_c2_rhs_sampled(W, precision):
    run_sampled(W, 24, 5, precision, seed=3)


@pytest.mark.parametrize("precision", ["fp64", "fp32_3xbf16", "fp32_tf32"])
def test_c2_fewer_point_rule_sampled(W, precision):
    from synthetic import fewer_point_rule
    run_sampled(W, 24, 5, precision, seed=8, rule=fewer_point_rule(5))


def test_c3_shots_sampled(W):
    run_sampled(W, 16, 4, "fp32_3xbf16", S=64, c2="one", seed=4)


def test_c4_rhs_sampled(W):
    from synthetic import c2_perturbed_samples
    VXYZ, EToV, geom = cube(16, 3)
    c2q = c2_perturbed_samples((len(EToV), 64), seed=11)
    run_sampled(W, 16, 3, "fp32", c2=c2q, seed=5)
