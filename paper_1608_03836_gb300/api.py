"""Python binding of the WADG C ABI (argument marshalling only).

Every function has the name of the C entry point it calls (include/wadg.h).
Device buffers are torch CUDA tensors (PyTorch supplies device memory and
streams); host arrays are numpy.  All arithmetic runs in the library's CUDA
kernels: nothing here computes on the data.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import WadgError, load

WADG_FP64, WADG_FP32, WADG_FP32_TF32, WADG_FP32_3XBF16 = 0, 1, 2, 3
PRECISIONS = {"fp64": WADG_FP64, "fp32": WADG_FP32, "fp32_tf32": WADG_FP32_TF32, "fp32_3xbf16": WADG_FP32_3XBF16}


def _check(status: int, where: str, mesh=None):
    if status != 0:
        detail = ""
        if mesh is not None:
            detail = (load().wadg_last_error(mesh.handle) or b"").decode()
        raise WadgError(status, where, detail)


def _dptr(arr: np.ndarray):
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class MeshHandle:
    """Owns a wadg_mesh*; freed by wadg_mesh_destroy."""

    def __init__(self, handle: ctypes.c_void_p):
        self.handle = handle
        info = (ctypes.c_int64 * 8)()
        _check(load().wadg_mesh_info(handle, info), "wadg_mesh_info")
        self.N, self.K, self.Np, self.Nq, self.Nfp, self.Nfq = (int(v) for v in info[:6])
        self.S = 1
        self.precision = None
        self.R = 0

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == WADG_FP64 else torch.float32

    def field_shape(self):
        return (4, self.K, self.S, self.Np)

    def __del__(self):
        try:
            if self.handle:
                load().wadg_mesh_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def wadg_version() -> int:
    return load().wadg_version()


def wadg_mesh_create(N: int, VXYZ, EToV, geom_xyz=None, rule=None) -> MeshHandle:
    """rule: None (the collapsed (N+1)^3 volume rule) or (rst (nq, 3), w (nq,))
    on the reference tetrahedron (wadg_mesh_create_rule)."""
    lib = load()
    V = np.ascontiguousarray(VXYZ, dtype=np.float64)
    E = np.ascontiguousarray(EToV, dtype=np.int64)
    G = None if geom_xyz is None else np.ascontiguousarray(geom_xyz, dtype=np.float64)
    out = ctypes.c_void_p()
    if rule is None:
        st = lib.wadg_mesh_create(int(N), V.shape[0], _dptr(V), E.shape[0],
                                  E.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  None if G is None else _dptr(G), ctypes.byref(out))
    else:
        rst, w = rule
        R = np.ascontiguousarray(np.column_stack([np.asarray(rst, dtype=np.float64), np.asarray(w, dtype=np.float64)]))
        st = lib.wadg_mesh_create_rule(int(N), V.shape[0], _dptr(V), E.shape[0],
                                       E.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                       None if G is None else _dptr(G), R.shape[0], _dptr(R), ctypes.byref(out))
    _check(st, "wadg_mesh_create")
    return MeshHandle(out)


def wadg_set_operators(mesh: MeshHandle, precision="fp64", shots: int = 1, tau_p: float = 1.0,
                       tau_u: float = 1.0, c2q=None):
    prec = PRECISIONS.get(precision, precision)
    c2 = None if c2q is None else np.ascontiguousarray(c2q, dtype=np.float64)
    if c2 is not None and c2.size != mesh.K * mesh.Nq:
        raise ValueError("c2q must have K*Nq values")
    st = load().wadg_set_operators(mesh.handle, int(prec), int(shots), float(tau_p), float(tau_u),
                                   None if c2 is None else _dptr(c2))
    _check(st, "wadg_set_operators", mesh)
    if int(shots) != mesh.S or int(prec) != mesh.precision:
        mesh.R = 0                          # the library drops sources and receivers then
    mesh.S = int(shots)
    mesh.precision = int(prec)
    mesh.tau_p, mesh.tau_u = float(tau_p), float(tau_u)


def wadg_device_status(mesh: MeshHandle, stream=None):
    """Raises WadgError (WADG_ETIMEOUT) if a bounded device wait expired."""
    _check(load().wadg_device_status(mesh.handle, _stream(stream)), "wadg_device_status", mesh)


def wadg_selftest_bounded_wait(mesh: MeshHandle, max_iters: int = 1000, stream=None):
    """Launch the bounded-wait failure-path test (see include/wadg.h)."""
    _check(load().wadg_selftest_bounded_wait(mesh.handle, int(max_iters), _stream(stream)),
           "wadg_selftest_bounded_wait", mesh)


def wadg_reference_rules(N: int):
    Nq, Nfq = (N + 1) ** 3, (N + 1) ** 2
    rst, w, rs, wf = np.zeros((Nq, 3)), np.zeros(Nq), np.zeros((Nfq, 2)), np.zeros(Nfq)
    _check(load().wadg_reference_rules(int(N), _dptr(rst), _dptr(w), _dptr(rs), _dptr(wf)), "wadg_reference_rules")
    return rst, w, rs, wf


def wadg_volume_points(mesh: MeshHandle) -> np.ndarray:
    out = np.zeros((mesh.K, mesh.Nq, 3))
    _check(load().wadg_volume_points(mesh.handle, _dptr(out)), "wadg_volume_points", mesh)
    return out


def _check_field(mesh, t, name, dtype=None, last=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    want = dtype if dtype is not None else mesh.dtype
    if t.dtype != want:
        raise TypeError(f"{name} must be {want}, got {t.dtype}")
    n = 4 * mesh.K * mesh.S * (last if last is not None else mesh.Np)
    if t.numel() != n:
        raise ValueError(f"{name} must have {n} elements [4][K][S][..], got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def wadg_project(mesh: MeshHandle, fq, Q, stream=None):
    import torch
    a = _check_field(mesh, fq, "fq", torch.float64, mesh.Nq)
    b = _check_field(mesh, Q, "Q")
    _check(load().wadg_project(mesh.handle, a, b, _stream(stream)), "wadg_project", mesh)


def wadg_rhs(mesh: MeshHandle, Q, dQdt, stream=None):
    a = _check_field(mesh, Q, "Q")
    b = _check_field(mesh, dQdt, "dQdt")
    _check(load().wadg_rhs(mesh.handle, a, b, _stream(stream)), "wadg_rhs", mesh)


def wadg_step(mesh: MeshHandle, Q, res, t0: float, dt: float, nsteps: int, traces=None, stream=None):
    a = _check_field(mesh, Q, "Q")
    b = _check_field(mesh, res, "res")
    tr = None
    if traces is not None:
        if traces.dtype != mesh.dtype or not traces.is_cuda or traces.numel() < nsteps * mesh.S * mesh.R:
            raise ValueError("traces must be a CUDA tensor of nsteps*S*R values in the mesh precision")
        tr = ctypes.c_void_p(traces.data_ptr())
    _check(load().wadg_step(mesh.handle, a, b, float(t0), float(dt), int(nsteps), tr, _stream(stream)),
           "wadg_step", mesh)


FORMULATIONS = {"strong_weak": 0, "strong": 1, "strong_underintegrated": 2}


def wadg_set_formulation(mesh: MeshHandle, form: str):
    """'strong_weak' (default), 'strong' (energy-stable rules) or
    'strong_underintegrated' (the degree 2N+1 rules); see include/wadg.h."""
    _check(load().wadg_set_formulation(mesh.handle, FORMULATIONS[form]), "wadg_set_formulation", mesh)


def wadg_set_conservation(mesh: MeshHandle, on: bool):
    """Locally conservative update weights (True) or the pointwise ones
    (False, the default); see include/wadg.h."""
    _check(load().wadg_set_conservation(mesh.handle, 1 if on else 0), "wadg_set_conservation", mesh)


def wadg_set_compensation(mesh: MeshHandle, on=True):
    """Compensated summation of the FP32 state in the LSRK steps: True or 1
    (the carry cleared at every call), 2 (the carry kept across calls), False
    or 0 (plain FP32 updates, the default); see include/wadg.h."""
    _check(load().wadg_set_compensation(mesh.handle, int(on)), "wadg_set_compensation", mesh)


def wadg_compensation_carry(mesh: MeshHandle, lo, store: bool, stream=None):
    """Copy the compensation carry into lo (store=True) or from lo into the
    mesh (store=False); lo is a float32 tensor of the shape of Q, on the host
    or the device."""
    import torch
    if lo.dtype != torch.float32 or lo.numel() != 4 * mesh.K * mesh.S * mesh.Np or not lo.is_contiguous():
        raise ValueError("lo must be a contiguous float32 tensor of 4*K*S*Np values")
    _check(load().wadg_compensation_carry(mesh.handle, ctypes.c_void_p(lo.data_ptr()), 0 if store else 1,
                                          _stream(stream)), "wadg_compensation_carry", mesh)


PLANAR_SPLIT = {False: 0, True: 1, "off": 0, "planned": 1, "all": 2}


def wadg_set_planar_split(mesh: MeshHandle, on=True):
    """Tiles of affine elements on the planar tensor-core kernel: True or
    "planned" (the default: as the tile counts pay), "all" (every all-affine
    tile), False or "off" (every tile on the curved kernel); see
    include/wadg.h."""
    mode = PLANAR_SPLIT[on] if isinstance(on, (bool, str)) else int(on)
    _check(load().wadg_set_planar_split(mesh.handle, mode), "wadg_set_planar_split", mesh)


def wadg_planar_info(mesh: MeshHandle) -> dict:
    info = (ctypes.c_int64 * 4)()
    _check(load().wadg_planar_info(mesh.handle, info), "wadg_planar_info", mesh)
    return {"affine_elements": info[0], "planar_tiles": info[1], "tiles": info[2], "planar_launch_tiles": info[3]}


def wadg_step_host(mesh: MeshHandle, Q, res, t0: float, dt: float, nsteps: int, stream=None):
    """wadg_step on host tensors (CPU, contiguous, the mesh precision; pinned
    memory gives the fastest copies): Q copied in, stepped, Q and res copied
    back; res=None keeps the residual on the device."""
    shape = tuple(mesh.field_shape())
    for name, x in (("Q", Q), ("res", res)):
        if x is None and name == "res":
            continue
        if x.is_cuda or x.dtype != mesh.dtype or tuple(x.shape) != shape or not x.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CPU tensor {shape} of {mesh.dtype}")
    rp = None if res is None else ctypes.c_void_p(res.data_ptr())
    _check(load().wadg_step_host(mesh.handle, ctypes.c_void_p(Q.data_ptr()), rp,
                                 float(t0), float(dt), int(nsteps), _stream(stream)), "wadg_step_host", mesh)


def wadg_solve(mesh: MeshHandle, Q, res, t0: float, T: float, dt_max: float, traces=None, stream=None) -> int:
    """Solve to t0 + T with a captured CUDA graph; returns the number of steps."""
    a = _check_field(mesh, Q, "Q")
    b = _check_field(mesh, res, "res")
    n = ctypes.c_int()
    _check(load().wadg_solve(mesh.handle, a, b, float(t0), float(T), float(dt_max),
                             None if traces is None else ctypes.c_void_p(traces.data_ptr()), ctypes.byref(n),
                             _stream(stream)), "wadg_solve", mesh)
    return n.value


def wadg_set_sources(mesh: MeshHandle, xyz, f0: float = 5.0, t0: float | None = None):
    if xyz is None:
        _check(load().wadg_set_sources(mesh.handle, None, float(f0), 0.0), "wadg_set_sources", mesh)
        return
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(mesh.S, 3)
    t0 = 1.2 / f0 if t0 is None else t0
    _check(load().wadg_set_sources(mesh.handle, _dptr(x), float(f0), float(t0)), "wadg_set_sources", mesh)


def wadg_set_receivers(mesh: MeshHandle, xyz):
    if xyz is None:
        _check(load().wadg_set_receivers(mesh.handle, 0, None), "wadg_set_receivers", mesh)
        mesh.R = 0
        return
    x = np.ascontiguousarray(xyz, dtype=np.float64)
    R = x.shape[-2]
    x = x.reshape(mesh.S, R, 3)
    _check(load().wadg_set_receivers(mesh.handle, int(R), _dptr(x)), "wadg_set_receivers", mesh)
    mesh.R = int(R)


def wadg_energy(mesh: MeshHandle, Q, stream=None) -> float:
    a = _check_field(mesh, Q, "Q")
    E = ctypes.c_double()
    _check(load().wadg_energy(mesh.handle, a, ctypes.byref(E), _stream(stream)), "wadg_energy", mesh)
    return E.value


def wadg_energy_noalloc(mesh: MeshHandle, Q, stream=None) -> float:
    """wadg_energy without any allocation (fixed library scratch; see include/wadg.h)."""
    a = _check_field(mesh, Q, "Q")
    E = ctypes.c_double()
    _check(load().wadg_energy_noalloc(mesh.handle, a, ctypes.byref(E), _stream(stream)), "wadg_energy_noalloc",
           mesh)
    return E.value


def wadg_l2_error(mesh: MeshHandle, Q, exact_q, field_mask: int = 1, stream=None) -> float:
    import torch
    a = _check_field(mesh, Q, "Q")
    b = _check_field(mesh, exact_q, "exact_q", torch.float64, mesh.Nq)
    e = ctypes.c_double()
    _check(load().wadg_l2_error(mesh.handle, a, b, int(field_mask), ctypes.byref(e), _stream(stream)),
           "wadg_l2_error", mesh)
    return e.value


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def wadg_rhs_adjoint(mesh: MeshHandle, lam, out, stream=None):
    a = _check_field(mesh, lam, "lambda")
    b = _check_field(mesh, out, "out")
    _check(load().wadg_rhs_adjoint(mesh.handle, a, b, _stream(stream)), "wadg_rhs_adjoint", mesh)


def wadg_step_record(mesh: MeshHandle, Q, res, t0: float, dt: float, ystore=None, traces=None, stream=None):
    a = _check_field(mesh, Q, "Q")
    b = _check_field(mesh, res, "res")
    if ystore is not None and (ystore.dtype != mesh.dtype or ystore.numel() != 5 * mesh.K * mesh.S * mesh.Nq):
        raise ValueError("ystore must hold 5*K*S*Nq values in the mesh precision")
    if traces is not None and (traces.dtype != mesh.dtype or traces.numel() < mesh.S * mesh.R):
        raise ValueError("traces must hold S*R values in the mesh precision")
    _check(load().wadg_step_record(mesh.handle, a, b, float(t0), float(dt), _ptr(ystore), _ptr(traces),
                                   _stream(stream)), "wadg_step_record", mesh)


def wadg_step_adjoint(mesh: MeshHandle, lamQ, lamR, dt: float, ystore=None, dc2=None, stream=None):
    import torch
    a = _check_field(mesh, lamQ, "lamQ")
    b = _check_field(mesh, lamR, "lamR")
    if dc2 is not None and (dc2.dtype != torch.float64 or dc2.numel() != mesh.K * mesh.Nq):
        raise ValueError("dc2 must be a float64 tensor of K*Nq values")
    _check(load().wadg_step_adjoint(mesh.handle, a, b, float(dt), _ptr(ystore), _ptr(dc2), _stream(stream)),
           "wadg_step_adjoint", mesh)


def wadg_receivers_adjoint(mesh: MeshHandle, weights, lamQ, stream=None):
    a = _check_field(mesh, lamQ, "lamQ")
    if weights.dtype != mesh.dtype or weights.numel() != mesh.S * mesh.R or not weights.is_contiguous():
        raise ValueError("weights must be a contiguous S*R tensor in the mesh precision")
    _check(load().wadg_receivers_adjoint(mesh.handle, _ptr(weights), a, _stream(stream)), "wadg_receivers_adjoint",
           mesh)


def wadg_segment_adjoint(mesh: MeshHandle, Q, res, t0: float, dt: float, nsteps: int, weights, lamQ, lamR,
                         ystore=None, dc2=None, stream=None):
    import torch
    a = _check_field(mesh, lamQ, "lamQ")
    b = _check_field(mesh, lamR, "lamR")
    q = r = None
    if ystore is not None:
        q = _check_field(mesh, Q, "Q")
        r = _check_field(mesh, res, "res")
        if ystore.dtype != mesh.dtype or ystore.numel() != nsteps * 5 * mesh.K * mesh.S * mesh.Nq \
                or not ystore.is_contiguous():
            raise ValueError("ystore must hold nsteps*5*K*S*Nq contiguous values in the mesh precision")
    if dc2 is not None and (dc2.dtype != torch.float64 or dc2.numel() != mesh.K * mesh.Nq):
        raise ValueError("dc2 must be a float64 tensor of K*Nq values")
    if weights is not None and (weights.dtype != mesh.dtype or weights.numel() != nsteps * mesh.S * mesh.R
                                or not weights.is_contiguous()):
        raise ValueError("weights must be a contiguous nsteps*S*R tensor in the mesh precision")
    _check(load().wadg_segment_adjoint(mesh.handle, q, r, float(t0), float(dt), int(nsteps), _ptr(weights), a, b,
                                       _ptr(ystore), _ptr(dc2), _stream(stream)), "wadg_segment_adjoint", mesh)


class BatchHandle:
    """Owns a wadg_batch*; keeps its meshes alive."""

    def __init__(self, handle, meshes):
        self.handle = handle
        self.meshes = list(meshes)

    def __del__(self):
        try:
            if self.handle:
                load().wadg_batch_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def _bcheck(status, where, batch=None):
    if status != 0:
        detail = ""
        if batch is not None and batch.handle:
            detail = (load().wadg_batch_last_error(batch.handle) or b"").decode()
        raise WadgError(status, where, detail)


def _ptr_array(batch, tensors, name):
    if len(tensors) != len(batch.meshes):
        raise ValueError(f"{name}: one buffer per mesh")
    arr = (ctypes.c_void_p * len(tensors))()
    for i, (m, t) in enumerate(zip(batch.meshes, tensors)):
        arr[i] = _check_field(m, t, f"{name}[{i}]")
    return arr


def wadg_batch_create(meshes) -> BatchHandle:
    arr = (ctypes.c_void_p * len(meshes))(*[m.handle for m in meshes])
    out = ctypes.c_void_p()
    _bcheck(load().wadg_batch_create(arr, len(meshes), ctypes.byref(out)), "wadg_batch_create")
    return BatchHandle(out, meshes)


def wadg_batch_info(batch: BatchHandle) -> dict:
    info = (ctypes.c_int64 * 5)()
    _bcheck(load().wadg_batch_info(batch.handle, info), "wadg_batch_info", batch)
    return {"meshes": info[0], "items": info[1], "grid": info[2], "max_grid": info[3], "rule": info[4]}


def wadg_batch_set_grid(batch: BatchHandle, grid: int):
    _bcheck(load().wadg_batch_set_grid(batch.handle, int(grid)), "wadg_batch_set_grid", batch)


def wadg_batch_set_rule(batch: BatchHandle, rule: int):
    _bcheck(load().wadg_batch_set_rule(batch.handle, int(rule)), "wadg_batch_set_rule", batch)


def wadg_batch_autotune(batch: BatchHandle, Q, res, stream=None) -> int:
    g = ctypes.c_int()
    _bcheck(load().wadg_batch_autotune(batch.handle, _ptr_array(batch, Q, "Q"), _ptr_array(batch, res, "res"),
                                       ctypes.byref(g), _stream(stream)), "wadg_batch_autotune", batch)
    return g.value


def wadg_batch_step(batch: BatchHandle, Q, res, t0: float, dt: float, nsteps: int, stream=None):
    _bcheck(load().wadg_batch_step(batch.handle, _ptr_array(batch, Q, "Q"), _ptr_array(batch, res, "res"),
                                   float(t0), float(dt), int(nsteps), _stream(stream)), "wadg_batch_step", batch)


def wadg_batch_solve(batch: BatchHandle, Q, res, t0: float, T: float, dt_max: float, stream=None) -> int:
    n = ctypes.c_int()
    _bcheck(load().wadg_batch_solve(batch.handle, _ptr_array(batch, Q, "Q"), _ptr_array(batch, res, "res"),
                                    float(t0), float(T), float(dt_max), ctypes.byref(n), _stream(stream)),
            "wadg_batch_solve", batch)
    return n.value


def wadg_batch_destroy(batch: BatchHandle):
    if batch.handle:
        load().wadg_batch_destroy(batch.handle)
        batch.handle = None


def wadg_batch_last_error(batch: BatchHandle) -> str:
    return (load().wadg_batch_last_error(batch.handle) or b"").decode()


def wadg_mesh_destroy(mesh: MeshHandle):
    if mesh.handle:
        load().wadg_mesh_destroy(mesh.handle)
        mesh.handle = None


def wadg_status_string(status: int) -> str:
    return load().wadg_status_string(int(status)).decode()


def wadg_last_error(mesh: MeshHandle) -> str:
    return (load().wadg_last_error(mesh.handle) or b"").decode()
