"""Tiles of affine elements on the planar tensor-core kernel (Sec. 6 runs the
planar and the curvilinear elements in separate kernels): on a cube curved
for z < 0 and affine beyond, the split launch matches the oracle, agrees with
the single curved launch to FP32 rounding, replays bit for bit in a captured
solve, and reports its tile counts."""
import numpy as np
import pytest

from gpu_util import TOL, library_mesh, oracle_c2, oracle_case, random_Q, rel_errors, to_torch
from synthetic import warped_cube

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_03836_gb300 as lib
    return lib


def _half_planar(n, N):
    return warped_cube(n, N, 0.1, planar_from=0.0)


def _rhs(W, m, Q):
    import torch
    Qt = to_torch(Q, m.dtype)
    out = torch.empty_like(Qt)
    W.wadg_rhs(m, Qt, out)
    torch.cuda.synchronize()
    W.wadg_device_status(m)
    return out.double().cpu().numpy()


def test_planar_tile_counts(W):
    VXYZ, EToV, geom = _half_planar(4, 3)
    # 384 elements, z >= 0 affine; S = 1: tiles [0,128) [128,256) [256,384)
    # of which the last is all affine; S = 3: 9 tiles, columns 576.. affine.
    # Fewer tiles than SMs: one launch is cheaper, so the plan runs none on
    # the planar kernel
    for prec, S, want in (("fp32_3xbf16", 1, (192, 1, 3)), ("fp32_tf32", 3, (192, 4, 9)),
                          ("fp32", 1, (192, 0, 0)), ("fp64", 1, (192, 0, 0))):
        m = library_mesh(VXYZ, EToV, geom, 3, prec, shots=S)
        info = W.wadg_planar_info(m)
        assert (info["affine_elements"], info["planar_tiles"], info["tiles"]) == want, (prec, S, info)
        assert info["planar_launch_tiles"] == 0
        W.wadg_set_planar_split(m, "all")
        assert W.wadg_planar_info(m)["planar_launch_tiles"] == want[1]
        W.wadg_set_planar_split(m, "off")
        assert W.wadg_planar_info(m)["planar_launch_tiles"] == 0
        with pytest.raises(W.WadgError):
            W.wadg_set_planar_split(m, 3)
    # the warped cube has no affine element; the affine cube has only affine
    # ones, and its one tile runs on the planar kernel
    Vw, Ew, Gw = warped_cube(2, 3, 0.1)
    assert W.wadg_planar_info(library_mesh(Vw, Ew, Gw, 3, "fp32_3xbf16"))["affine_elements"] == 0
    Va, Ea, Ga = warped_cube(2, 3, 0.0)
    info = W.wadg_planar_info(library_mesh(Va, Ea, Ga, 3, "fp32_3xbf16"))
    assert info == {"affine_elements": 48, "planar_tiles": 1, "tiles": 1, "planar_launch_tiles": 1}


@pytest.mark.parametrize("precision", ["fp32_3xbf16", "fp32_tf32"])
@pytest.mark.parametrize("N,n,S", [(1, 4, 2), (2, 4, 1), (3, 4, 3), (4, 4, 1)])
def test_split_rhs_matches_oracle_and_single_launch(W, precision, N, n, S):
    VXYZ, EToV, geom = _half_planar(n, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, precision, shots=S, c2="heterogeneous")
    W.wadg_set_planar_split(m, "all")
    info = W.wadg_planar_info(m)
    assert 0 < info["planar_launch_tiles"] == info["planar_tiles"] < info["tiles"], info
    Q = random_Q(m.K, S, m.Np, seed=300 + N)
    got = _rhs(W, m, Q)
    c2o = oracle_c2(om, "heterogeneous")
    from oracle import wadg as OW
    for s in range(S):
        want = OW.rhs_nodal(om, Q[:, :, s], c2q=c2o)
        l2, mx = rel_errors(got[:, :, s], want)
        print(f"N={N} S={S} {precision} shot {s}: rel L2 {l2:.3e}, rel max {mx:.3e}")
        assert l2 < TOL[precision] and mx < 10 * TOL[precision], (s, l2, mx)
    # the curved kernel on every tile: the planar kernel's constant G and
    # n J^f are the curved tables' values, so the two differ by FP32 rounding
    W.wadg_set_planar_split(m, "off")
    one = _rhs(W, m, Q)
    d = np.abs(got - one).max() / np.abs(one).max()
    assert d < 2e-6, d
    # the curved tiles' columns see the same kernel either way
    curved_cols = np.arange(m.K * S) < (info["tiles"] - info["planar_tiles"]) * 128
    ks = np.nonzero(curved_cols.reshape(m.K, S).all(1))[0]
    assert np.array_equal(got[:, ks], one[:, ks])
    # the plan keeps a mesh of fewer tiles than SMs on the curved kernel
    W.wadg_set_planar_split(m, True)
    assert W.wadg_planar_info(m)["planar_launch_tiles"] == 0
    assert np.array_equal(_rhs(W, m, Q), one)


def test_planned_split_at_scale(W):
    """N = 1, 24,576 tets curved for z < -0.75 and affine beyond, 8 shots:
    1,536 tiles, the last 1,344 all affine.  The plan runs the planar kernel
    on part of them (1,232 on 152 SMs: 8.1 rounds instead of 8.8, the first
    112 affine tiles joining the 192 curved ones in two curved rounds); the
    results equal the curved kernel's on every tile to rounding (at N = 1 bit
    for bit: an affine map's factors are the same at every point), and bit
    for bit on the curved launch's tiles."""
    import torch
    N, S = 1, 8
    VXYZ, EToV, geom = warped_cube(16, N, 0.1, planar_from=-0.75)
    m = library_mesh(VXYZ, EToV, geom, N, "fp32_3xbf16", shots=S, c2="heterogeneous")
    G = torch.cuda.get_device_properties(0).multi_processor_count
    info = W.wadg_planar_info(m)
    assert info["tiles"] == 1536 and info["planar_tiles"] == 1344, info
    npl = info["planar_launch_tiles"]
    assert 0 < npl <= 1344, npl
    if G == 152:
        assert npl == 1232, npl
    Q = random_Q(m.K, S, m.Np, seed=303)
    got = _rhs(W, m, Q)
    W.wadg_set_planar_split(m, "off")
    one = _rhs(W, m, Q)
    assert np.abs(got - one).max() < 2e-6 * np.abs(one).max()
    # the affine tiles are the last 1,344; the planar launch takes the first
    # npl of them, the curved launch the others and the 192 curved tiles
    cols = np.arange(m.K * S) // 128
    stay = (cols < 192) | (cols >= 192 + npl)
    g4, o4 = got.reshape(4, -1, m.Np), one.reshape(4, -1, m.Np)
    assert np.array_equal(g4[:, stay], o4[:, stay])
    # half affine: the plan saves nothing and keeps one launch
    m2 = library_mesh(*_half_planar(16, N), N, "fp32_3xbf16", shots=S)
    info2 = W.wadg_planar_info(m2)
    assert info2["planar_tiles"] == 768 and (G != 152 or info2["planar_launch_tiles"] == 0), info2


def test_split_steps_match_oracle_and_replay(W):
    import torch
    from oracle import wadg as OW
    N, S = 4, 2
    VXYZ, EToV, geom = _half_planar(4, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, "fp32_3xbf16", shots=S, c2="heterogeneous")
    W.wadg_set_planar_split(m, "all")
    assert W.wadg_planar_info(m)["planar_launch_tiles"] > 0
    c2o = oracle_c2(om, "heterogeneous")
    Q0 = random_Q(m.K, S, m.Np, seed=91)
    dt, nsteps = 1e-3, 3
    Qt = to_torch(Q0, m.dtype)
    Rt = torch.zeros_like(Qt)
    W.wadg_step(m, Qt, Rt, 0.0, dt, nsteps)
    Qg, Rg = to_torch(Q0, m.dtype), torch.zeros_like(Qt)
    assert W.wadg_solve(m, Qg, Rg, 0.0, nsteps * dt, dt) == nsteps
    torch.cuda.synchronize()
    W.wadg_device_status(m)
    assert torch.equal(Qg, Qt) and torch.equal(Rg, Rt)
    for s in range(S):
        c = om.ref.to_modal(Q0[:, :, s].astype(np.float32).astype(np.float64))
        res = np.zeros_like(c)
        for k in range(nsteps):
            c, res = OW.lsrk_step(lambda q, t: OW.rhs(om, q, c2q=c2o), c, res, k * dt, dt)
        l2, mx = rel_errors(Qt.double().cpu().numpy()[:, :, s], om.ref.to_nodal(c))
        assert l2 < TOL["fp32_3xbf16"] and mx < 10 * TOL["fp32_3xbf16"], (s, l2, mx)

