"""The allocation-free energy entry point (wadg_energy_noalloc).

Some callers cannot allocate device memory when they want the energy: code
inside a framework whose allocator owns the device memory, and real-time loops
that must not wait on the driver's allocator.  wadg_energy_noalloc serves them
from a fixed scratch array in the library image.  This file is collected last
so that a run stopping at the first failure has already run every other test;
it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from gpu_util import TOL, library_mesh, make_mesh_inputs, random_Q, to_torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_03836_gb300 as lib
    return lib


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_energy_matches_wadg_energy_twice(W, precision):
    VXYZ, EToV, geom = make_mesh_inputs(2, 4)
    m = library_mesh(VXYZ, EToV, geom, 4, precision, shots=2, c2="heterogeneous")
    for call, seed in enumerate((31, 32)):
        Q = to_torch(random_Q(m.K, 2, m.Np, seed), m.dtype)
        want = W.wadg_energy(m, Q)
        got = W.wadg_energy_noalloc(m, Q)
        assert abs(got - want) <= TOL["fp64"] * abs(want), (call, got, want)


def test_noalloc_energy_rejects_too_many_columns(W):
    import torch
    VXYZ, EToV, geom = make_mesh_inputs(1, 1)          # 6 tets, N = 1
    shots = (1 << 20) // 6 + 1                           # K*S = 1048578 > 2^20
    m = library_mesh(VXYZ, EToV, geom, 1, "fp32", shots=shots)
    Q = torch.zeros((4, m.K, shots, m.Np), dtype=torch.float32, device="cuda")
    with pytest.raises(W.WadgError) as e:
        W.wadg_energy_noalloc(m, Q)
    assert e.value.status == -1
    assert "1048576" in str(e.value)
