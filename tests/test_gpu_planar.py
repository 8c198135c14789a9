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
@pytest.mark.parametrize("N,n,S,fewer", [(1, 4, 2, False), (2, 4, 1, False), (3, 4, 3, False), (4, 4, 1, False),
                                         (5, 4, 1, False), (5, 4, 2, True)])
def test_split_rhs_matches_oracle_and_single_launch(W, precision, N, n, S, fewer):
    """fewer: the fewer-point volume rule (96 points at N = 5) instead of the
    collapsed one."""
    from synthetic import fewer_point_rule
    rule = fewer_point_rule(N) if fewer else None
    VXYZ, EToV, geom = _half_planar(n, N)
    om = oracle_case(VXYZ, EToV, geom, N, rule=rule)
    m = library_mesh(VXYZ, EToV, geom, N, precision, shots=S, c2="heterogeneous", rule=rule)
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



def test_split_with_sources_receivers_and_compensation_matches_oracle(W):
    """Two shots on the half-planar cube, one Ricker point source in an
    affine element (z > 0) and one in a curved element, three receivers per
    shot, compensated state updates, every affine tile on the planar kernel:
    four LSRK steps from rest against the oracle's."""
    import torch
    from gpu_util import TRACE_FACTOR
    from oracle import sources as OS
    from oracle import wadg as OW
    from synthetic import ricker, receiver_positions
    N, S, R = 3, 2, 3
    VXYZ, EToV, geom = _half_planar(4, N)
    om = oracle_case(VXYZ, EToV, geom, N)
    m = library_mesh(VXYZ, EToV, geom, N, "fp32_3xbf16", shots=S)
    W.wadg_set_planar_split(m, "all")
    W.wadg_set_compensation(m, True)
    assert W.wadg_planar_info(m)["planar_launch_tiles"] > 0
    xs = np.array([[0.11, -0.23, 0.42], [-0.31, 0.17, -0.46]])
    xr = receiver_positions(S * R).reshape(S, R, 3)
    f0, t0 = 5.0, 0.05
    W.wadg_set_sources(m, xs, f0, t0)
    W.wadg_set_receivers(m, xr)
    dt, nsteps = 2e-3, 4
    Q = torch.zeros((4, m.K, S, m.Np), dtype=m.dtype, device="cuda")
    Rt = torch.zeros_like(Q)
    traces = torch.zeros((nsteps, S, R), dtype=m.dtype, device="cuda")
    W.wadg_step(m, Q, Rt, 0.0, dt, nsteps, traces)
    W.wadg_device_status(m)
    got_Q = Q.double().cpu().numpy()
    got_tr = traces.double().cpu().numpy()
    src = OS.PointSet(om, xs)
    rec = OS.PointSet(om, xr.reshape(-1, 3))
    for s in range(S):
        c = np.zeros((4, om.K, om.ref.Np))
        res = np.zeros_like(c)
        want_tr = []
        L = lambda q, t: OW.wadg_apply(om, OW.a_h(om, q) + OS.source_load(om, src, float(ricker(t, f0, t0)), s))
        for n in range(nsteps):
            c, res = OW.lsrk_step(L, c, res, n * dt, dt)
            want_tr.append(OS.sample(c[0], rec, np.arange(s * R, (s + 1) * R)))
        l2, _ = rel_errors(got_Q[:, :, s], om.ref.to_nodal(c))
        l2t, _ = rel_errors(got_tr[:, s], np.array(want_tr))
        assert l2 < TOL["fp32_3xbf16"] and l2t < TRACE_FACTOR * TOL["fp32_3xbf16"], (s, l2, l2t)


def test_planned_split_full_size_sampled(W):
    """The headline size with 7/8 of its tiles affine: 196,608 tets curved
    for z < -0.75, N = 4, the 63-point rule, heterogeneous c^2, split bf16,
    the planned split (1,232 tiles on the planar kernel on 152 SMs); 48
    sampled columns (the first and last element, boundary elements, random
    ones, and elements of the planar launch, of the moved affine tiles and
    at the curved/affine interface) against the oracle's RHS evaluated on
    each column's neighbourhood."""
    import torch
    from gpu_util import sample_columns, sampled_oracle_rhs
    from synthetic import c2_heterogeneous, fewer_point_rule, random_fields
    N = 4
    rule = fewer_point_rule(N)
    VXYZ, EToV, geom = warped_cube(32, N, 0.1, planar_from=-0.75)
    m = W.wadg_mesh_create(N, VXYZ, EToV, geom, rule=rule)
    W.wadg_set_operators(m, "fp32_3xbf16", 1, 1.0, 1.0, c2_heterogeneous(W.wadg_volume_points(m)))
    info = W.wadg_planar_info(m)
    nc = info["tiles"] - info["planar_tiles"]
    npl = info["planar_launch_tiles"]
    assert npl > 0 and info["planar_tiles"] == 1344, info
    Q = random_fields((4, m.K, 1, m.Np), 777)
    Qt = to_torch(Q, m.dtype)
    out = torch.empty_like(Qt)
    W.wadg_rhs(m, Qt, out)
    W.wadg_device_status(m)
    got = out.double().cpu().numpy()
    cols = sample_columns(EToV, 1, 32, 17)
    rng = np.random.default_rng(18)
    # planar launch: tiles [nc, nc + npl); moved affine tiles: [nc + npl, tiles); interface: tile nc
    extra = list(rng.integers(nc * 128, (nc + npl) * 128, 6)) + list(rng.integers((nc + npl) * 128, m.K, 4))
    extra += list(range(nc * 128 - 3, nc * 128 + 3))
    cols += [(int(k), 0) for k in extra]
    want = sampled_oracle_rhs(VXYZ, EToV, geom, N, Q, cols, c2fun=c2_heterogeneous, rule=rule)
    g = np.stack([got[:, k, s] for k, s in cols], 1)
    l2, mx = rel_errors(g, want)
    print(f"planned split at full size: {len(cols)} sampled columns, rel L2 {l2:.3e}, max {mx:.3e}")
    assert l2 < TOL["fp32_3xbf16"] and mx < 10 * TOL["fp32_3xbf16"]
