"""Throughput of the WADG right-hand side + LSRK update on GB300.

Workload (the configuration the headline metric is quoted on): the warped
Kuhn cube with 32^3 hexahedra x 6 = 196,608 curved tetrahedra, degree N = 4
(Np = 35), heterogeneous c^2 = 1 + 0.5 sin(pi x) sin(pi y) sin(pi z) at the
volume quadrature points, standing-wave initial data.  One step = one LSRK(5,4)
time step = 5 fused stage launches (strong-weak volume + surface terms,
weight-adjusted update, Runge-Kutta update).  DOF = 4 K Np S scalar unknowns;
value = DOF * stages / second.

The headline line is the mixed-precision path (FP32 fields, the dense
products on the tensor cores with split bf16 operands); the plain FP64 path
and the FP32 CUDA-core path are measured on the same mesh, data and dt and
reported under "variants", and "accuracy" gives the L2 error of each against
the analytic solution.  Inputs (1.1 GB of FP32 geometric factors alone) are
larger than the 129 MB L2, so no flush is needed between iterations.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(n=32, N=4, warp=0.1, c2="heterogeneous")
METRIC = "WADG RHS DOF*stage/s (RHS + weight-adjusted update + LSRK stage)"
UNIT = "DOF*stage/s"


def algorithmic(N: int, S: int, s: int, nq: int | None = None):
    """Per element and stage: algorithmic bytes (fields read/written once,
    geometric factors read once, neighbour reads counted as L2 hits) and flops
    (dense reference-operator products); nq: points of the volume rule
    (default the collapsed (N+1)^3)."""
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    Nq, Nfq = ((N + 1) ** 3 if nq is None else nq), (N + 1) ** 2
    B = s * (16 * Np * S + 11 * Nq + 12 * Nfq) + 32
    F = (24 + 16) * Nq * Np * S + 16 * Np * 4 * Nfq * S
    return B, F


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured", float(d.get("sm_max_mhz", 2070.0))
    except Exception:
        return 6800.0, "fallback", 2070.0


def headline_config(ws: int) -> dict:
    """The workload both arms report on (the native arm times all of it, the
    reference arm a bounded sample, described in its cpu_baseline)."""
    n, N = WORKLOAD["n"], WORKLOAD["N"]
    K = 6 * n ** 3
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    rule = headline_rule()
    nq = (N + 1) ** 3 if rule is None else len(rule[1])
    # FP32 geometric factors as the tensor-core stage reads them (11 rows per
    # volume point, padded to groups of 4 points)
    geo_gb = K * 11 * ((nq + 3) // 4 * 4) * 4 / 1e9
    l2 = (f"inputs larger than L2 ({geo_gb:.2f} GB FP32 geometric factors)" if geo_gb > 0.129 else
          f"geometric factors ({geo_gb:.3f} GB) fit in the 129 MB L2: not an L2-flushed measurement")
    return {"workload": f"warped Kuhn cube {n}^3x6 = {K} curved tets, N={N} (Np={Np}), "
                        f"{nq}-point symmetric volume rule exact to degree {2 * N + 1}, heterogeneous c^2, 1 shot, "
                        "LSRK(5,4) step = 5 fused stage launches",
            "volume_points": nq, "elements": K, "N": N, "shots": 1, "dof": 4 * K * Np,
            "l2": l2, "parallelism": f"replicas{ws}"}


def headline_rule():
    """The volume rule of the workload: the fewer-point symmetric rule exact
    to degree 2N+1 where one is tabulated (N = 2..5), else the collapsed rule."""
    from synthetic import fewer_point_rule
    return fewer_point_rule(WORKLOAD["N"]) if WORKLOAD["N"] in (2, 3, 4, 5) else None


TC_SOURCES = ("paper_1608_03836_gb300/csrc/stage_tc.cu", "paper_1608_03836_gb300/csrc/stage_tc_kernel.cuh",
              "paper_1608_03836_gb300/csrc/tc_ops.cuh", "paper_1608_03836_gb300/csrc/tc_stage_common.cuh")
TC_PROFILE = "profiles/stage_tc_kernel_63pt_n20_full.md"


def tc_source_hash() -> str:
    """Hash of the kernel sources without their comments and blank lines (a
    comment edit does not change the kernel the counters were taken on)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for rel in TC_SOURCES:
        with open(os.path.join(ROOT, rel)) as f:
            for line in f:
                code = re.sub(r"//.*$", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def tc_traffic_per_element():
    """DRAM bytes per element and launch of the tensor-core stage from the
    committed ncu summary (lines 'source_hash: ...' and
    'dram_bytes_per_element: ...'), or None when the kernel source has changed
    since the capture."""
    try:
        vals = {}
        with open(os.path.join(ROOT, TC_PROFILE)) as f:
            for ln in f:
                if ":" in ln and ln.split(":")[0].strip() in ("source_hash", "dram_bytes_per_element"):
                    k, v = ln.split(":", 1)
                    vals[k.strip()] = v.strip().strip("`")
        if vals.get("source_hash") != tc_source_hash():
            return None
        return float(vals["dram_bytes_per_element"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # the timed region starts once the sampler is producing (every 20 ms)
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_case(W, precision, rank, rule=None):
    import torch
    from synthetic import warped_cube, c2_heterogeneous, standing_wave
    VXYZ, EToV, geom = warped_cube(WORKLOAD["n"], WORKLOAD["N"], WORKLOAD["warp"])
    m = W.wadg_mesh_create(WORKLOAD["N"], VXYZ, EToV, geom, rule=rule)
    xq = W.wadg_volume_points(m)
    W.wadg_set_operators(m, precision, 1, 1.0, 1.0, c2_heterogeneous(xq))
    fq = torch.from_numpy(standing_wave(xq, 0.0)[:, :, None, :]).cuda()
    Q = torch.empty((4, m.K, 1, m.Np), dtype=m.dtype, device="cuda")
    W.wadg_project(m, fq, Q)
    del fq
    return m, Q


def dt_for(m):
    # CFL-type step: 0.5 h_min / (c_max (N+1)^2) with h = hex side / 2
    h = 2.0 / WORKLOAD["n"]
    return 0.5 * (h / 2) / (math.sqrt(1.5) * (WORKLOAD["N"] + 1) ** 2)


def time_steps(W, m, Q, steps, warmup):
    """Device time of `steps` LSRK steps (one C-ABI call) and of one stage launch."""
    import torch
    R = torch.zeros_like(Q)
    dt = dt_for(m)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        W.wadg_step(m, Q, R, 0.0, dt, 1)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    W.wadg_step(m, Q, R, 0.0, dt, steps)
    stop.record(stream)
    torch.cuda.synchronize()
    total_ms = start.elapsed_time(stop)
    # one stage launch alone, averaged (same stream, same kernel)
    out = torch.empty_like(Q)
    reps = 5
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        W.wadg_rhs(m, Q, out)
    b.record(stream)
    torch.cuda.synchronize()
    return total_ms, a.elapsed_time(b) / reps


def batched_shots(W, steps):
    """Shots as columns: the 16^3 x 6 = 24,576-tet N=4 cube with 64 shots
    sharing the geometry, each with its own Ricker point source (f0 = 5,
    seeded position in [-0.8, 0.8]^3) and 8 receivers sampled after every
    step, from zero fields; FP32 and FP32 + split-bf16 tensor cores; DOF =
    4 K Np S; CUDA events around one wadg_step call of `steps` steps after 3
    warm-up steps."""
    import torch
    from synthetic import warped_cube, source_positions, receiver_positions
    n, N, S, R = 16, 4, 64, 8
    VXYZ, EToV, geom = warped_cube(n, N, 0.1)
    rule = headline_rule()
    out = {"workload": f"warped cube 16^3x6 = {len(EToV)} tets, N=4, 64 shots (columns K*S = {len(EToV) * S}), "
                       f"{'collapsed' if rule is None else str(len(rule[1])) + '-point'} volume rule, one Ricker "
                       "point source (f0 = 5) and 8 receivers per shot"}
    for prec in ("fp32", "fp32_3xbf16"):
        m = W.wadg_mesh_create(N, VXYZ, EToV, geom, rule=rule)
        W.wadg_set_operators(m, prec, S, 1.0, 1.0, None)
        W.wadg_set_sources(m, source_positions(S), 5.0, 0.24)
        W.wadg_set_receivers(m, receiver_positions(R * S).reshape(S, R, 3))
        Q = torch.zeros((4, m.K, S, m.Np), dtype=torch.float32, device="cuda")
        Rs = torch.zeros_like(Q)
        dt = 0.5 * (1.0 / n) / (N + 1) ** 2
        tr = torch.zeros((steps, S, R), dtype=torch.float32, device="cuda")
        W.wadg_step(m, Q, Rs, 0.0, dt, 3)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        W.wadg_step(m, Q, Rs, 3 * dt, dt, steps, tr)
        b.record()
        torch.cuda.synchronize()
        W.wadg_device_status(m)
        ms = a.elapsed_time(b) / steps
        dof = 4 * m.K * S * m.Np
        out[prec] = {"value": dof * 5 / (ms * 1e-3), "ms_per_step": ms, "stage_ms": ms / 5,
                     "max_abs_trace": float(tr.abs().max())}
        del Q, Rs, m, tr
        torch.cuda.empty_cache()
    out["accuracy_vs_fp64"] = shots_accuracy(W)
    return out


def shots_accuracy(W, S=4, nsteps=120, t_start=0.1):
    """The batched-shot paths against FP64 on the same shots: the first S of
    the 64 shots (same sources, receivers, mesh and rule), from zero fields at
    t_start (the wavelet, centred at t0 = 0.24, is below 1 % of its peak
    there) for nsteps steps; relative L2 difference from the FP64 run of the
    final p (all shots) and of the receiver traces."""
    import torch
    from synthetic import warped_cube, source_positions, receiver_positions
    n, N, R = 16, 4, 8
    VXYZ, EToV, geom = warped_cube(n, N, 0.1)
    rule = headline_rule()
    dt = 0.5 * (1.0 / n) / (N + 1) ** 2
    runs = {}
    for prec in ("fp64", "fp32", "fp32_3xbf16", "fp32_tf32"):
        m = W.wadg_mesh_create(N, VXYZ, EToV, geom, rule=rule)
        W.wadg_set_operators(m, prec, S, 1.0, 1.0, None)
        W.wadg_set_sources(m, source_positions(64)[:S], 5.0, 0.24)
        W.wadg_set_receivers(m, receiver_positions(R * 64).reshape(64, R, 3)[:S])
        Q = torch.zeros((4, m.K, S, m.Np), dtype=m.dtype, device="cuda")
        Rs = torch.zeros_like(Q)
        tr = torch.zeros((nsteps, S, R), dtype=m.dtype, device="cuda")
        W.wadg_step(m, Q, Rs, t_start, dt, nsteps, tr)
        torch.cuda.synchronize()
        W.wadg_device_status(m)
        runs[prec] = (Q[0].double().cpu().numpy(), tr.double().cpu().numpy())
        del Q, Rs, tr, m
        torch.cuda.empty_cache()
    p64, t64 = runs["fp64"]
    out = {"workload": f"first {S} of the 64 shots, {nsteps} steps of dt = {dt:.3e} from t = {t_start}",
           "fp64_max_abs_trace": float(np.abs(t64).max())}
    for prec in ("fp32", "fp32_3xbf16", "fp32_tf32"):
        p, t = runs[prec]
        out[prec] = {"p_rel_l2_vs_fp64": float(np.linalg.norm(p - p64) / np.linalg.norm(p64)),
                     "traces_rel_l2_vs_fp64": float(np.linalg.norm(t - t64) / np.linalg.norm(t64))}
    return out


def uneven_batch(W, steps, small=False, tensor_cores=False):
    """12 meshes of uneven size and degree (n_i = 4 + round(12 i/11) hexes per
    side, N_i = 2 + (i mod 5)) stepped by one persistent launch per stage
    (autotuned grid), against the same meshes stepped one after another.
    small=True: the same degrees on n_i = 2 + (i mod 4) (48 to 384 tets per
    mesh), where the per-mesh launches dominate.  tensor_cores=True: the same
    sizes with N_i = 2 + (i mod 4) (the tensor-core stage is built for N <= 5)
    in split bf16 on the fewer-point rules where tabulated, one combined
    launch per degree class and stage against per-mesh tensor-core steps."""
    import torch
    from synthetic import warped_cube, random_fields, fewer_point_rule
    ms, Qs, Rs = [], [], []
    dof = 0
    for i in range(12):
        n = 2 + (i % 4) if small else 4 + int(round(12 * i / 11))
        N = 2 + (i % 4) if tensor_cores else 2 + (i % 5)
        VXYZ, EToV, geom = warped_cube(n, N, 0.1)
        rule = fewer_point_rule(N) if tensor_cores and N in (2, 3, 4, 5) else None
        m = W.wadg_mesh_create(N, VXYZ, EToV, geom, rule=rule)
        W.wadg_set_operators(m, "fp32_3xbf16" if tensor_cores else "fp32", 1, 1.0, 1.0, None)
        ms.append(m)
        Qs.append(torch.from_numpy(random_fields((4, m.K, 1, m.Np), 10 + i).astype(np.float32)).cuda() * 1e-3)
        Rs.append(torch.zeros_like(Qs[-1]))
        dof += 4 * m.K * m.Np
    b = W.wadg_batch_create(ms)
    grid = W.wadg_batch_autotune(b, Qs, Rs)
    dt = 1e-4
    stream = torch.cuda.current_stream()
    W.wadg_batch_step(b, Qs, Rs, 0.0, dt, 3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    W.wadg_batch_step(b, Qs, Rs, 0.0, dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / steps
    e0.record(stream)
    for _ in range(steps):
        for m, Q, R in zip(ms, Qs, Rs):
            W.wadg_step(m, Q, R, 0.0, dt, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / steps
    info = W.wadg_batch_info(b)
    for m in ms:
        W.wadg_device_status(m)
    classes = len({(m.N, m.Nq) for m in ms})
    return {"workload": "12 warped cubes, " + ("n = 2..5" if small else "n = 4..16") +
                        (", N = 2..5, split bf16 tensor cores (fewer-point rules at N = 2..5)" if tensor_cores
                         else ", N = 2..6, FP32"),
            "dof": dof, "items": info["items"], "tile_rule": info["rule"],
            "grid": grid, "value": dof * 5 / (t_batch * 1e-3), "ms_per_step": t_batch,
            "sequential_ms_per_step": t_seq, "speedup": t_seq / t_batch,
            "launches_per_step": 5 * classes if tensor_cores else 5, "sequential_launches_per_step": 60}


def adjoint_timing(W, nsteps=300, checkpoint=20):
    """The differentiation configuration: warped cube 16^3 x 6 = 24,576 tets,
    N = 3, FP32 (CUDA cores, collapsed rule), c^2 perturbed by 10 % per volume
    point (seeded), 16 seeded receivers, 300 LSRK(5,4) steps from the
    projected standing wave; misfit = sum of squared receiver pressures.
    Times the forward pass (traces, a checkpoint every 20 steps) and the
    backward pass (gradients with respect to the initial pressure and c^2:
    each segment recomputed forward with the stage factors recorded, then the
    discrete adjoint steps), CUDA events on the current stream, after a
    2-step warm-up pass."""
    import torch
    from synthetic import warped_cube, c2_perturbed_samples, receiver_positions, standing_wave
    from paper_1608_03836_gb300.adjoint import receiver_traces
    n, N = 16, 3
    VXYZ, EToV, geom = warped_cube(n, N, 0.1)
    m = W.wadg_mesh_create(N, VXYZ, EToV, geom)
    c2q = c2_perturbed_samples((len(EToV), (N + 1) ** 3), seed=4)
    W.wadg_set_operators(m, "fp32", 1, 1.0, 1.0, c2q)
    W.wadg_set_receivers(m, receiver_positions(16).reshape(1, 16, 3))
    xq = W.wadg_volume_points(m)
    Q = torch.empty((4, m.K, 1, m.Np), dtype=m.dtype, device="cuda")
    W.wadg_project(m, torch.from_numpy(standing_wave(xq, 0.0)[:, :, None, :]).cuda(), Q)
    dt = 0.5 * (1.0 / n) / ((N + 1) ** 2 * 1.1 ** 0.5)
    p0 = Q[0].clone().requires_grad_(True)
    c2 = torch.tensor(c2q, dtype=torch.float64, device="cuda", requires_grad=True)
    # warm-up: the first autograd backward pass of a process carries a
    # one-time cost of several seconds outside the library
    (receiver_traces(m, p0, c2, dt, 2, checkpoint=checkpoint) ** 2).sum().backward()
    p0.grad, c2.grad = None, None
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    ev[0].record()
    tr = receiver_traces(m, p0, c2, dt, nsteps, checkpoint=checkpoint)
    ev[1].record()
    loss = (tr.double() ** 2).sum()
    loss.backward()
    ev[2].record()
    torch.cuda.synchronize()
    W.wadg_device_status(m)
    fwd, bwd = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    dof = 4 * m.K * m.Np
    return {"workload": f"warped cube 16^3x6 = {m.K} tets, N={N}, FP32, c^2 perturbed 10 %, 16 receivers, "
                        f"{nsteps} steps, checkpoint every {checkpoint}",
            "forward_ms": fwd, "backward_ms": bwd, "backward_over_forward": bwd / fwd,
            "forward_dof_stage_per_s": dof * 5 * nsteps / (fwd * 1e-3),
            "misfit": float(loss.detach()), "grad_p0_norm": float(p0.grad.norm()), "grad_c2_norm": float(c2.grad.norm())}


def accuracy(W):
    """Equal L2 error: the same mesh, standing wave (c^2 = 1), same dt and
    steps in every precision; L2 error of p against the analytic solution at T
    by the volume rule.  Two meshes: 8^3 x 6 tets at N = 3 (discretisation
    error well above FP32 rounding) and 16^3 x 6 tets at N = 4 (discretisation
    error near the FP32 floor).  All on the fewer-point symmetric volume rule
    (35 points at N = 3, 63 at N = 4) except fp64_collapsed_rule (the (N+1)^3
    rule); fp64_conservative: the FP64 path with the locally conservative
    update weights."""
    import torch
    from synthetic import warped_cube, standing_wave
    out = {}
    for n, N in ((8, 3), (16, 4)):
        T = 0.1
        VXYZ, EToV, geom = warped_cube(n, N, 0.1)
        h = 2.0 / n
        dt_max = 0.5 * (h / 2) / (N + 1) ** 2
        case = {"workload": f"warped cube {n}^3x6, N={N}, c^2=1, standing wave to T={T}, dt_max={dt_max:.3e}"}
        from synthetic import fewer_point_rule
        for prec in ("fp64", "fp32", "fp32_3xbf16", "fp32_tf32", "fp64_conservative", "fp64_collapsed_rule"):
            collapsed = prec.endswith("_collapsed_rule")
            m = W.wadg_mesh_create(N, VXYZ, EToV, geom, rule=None if collapsed else fewer_point_rule(N))
            W.wadg_set_operators(m, prec.split("_c")[0], 1, 1.0, 1.0, None)
            if prec.endswith("_conservative"):
                W.wadg_set_conservation(m, True)
            xq = W.wadg_volume_points(m)
            Q = torch.empty((4, m.K, 1, m.Np), dtype=m.dtype, device="cuda")
            W.wadg_project(m, torch.from_numpy(standing_wave(xq, 0.0)[:, :, None, :]).cuda(), Q)
            R = torch.zeros_like(Q)
            nsteps = W.wadg_solve(m, Q, R, 0.0, T, dt_max)
            err = W.wadg_l2_error(m, Q, torch.from_numpy(standing_wave(xq, T)[:, :, None, :]).cuda(), 1)
            case[prec] = {"l2_error_p": err, "nsteps": nsteps}
        e64 = case["fp64"]["l2_error_p"]
        for prec in ("fp32", "fp32_3xbf16", "fp32_tf32", "fp64_conservative", "fp64_collapsed_rule"):
            case[prec]["ratio_to_fp64"] = case[prec]["l2_error_p"] / e64
            case[prec]["equal_l2_error"] = bool(case[prec]["l2_error_p"] <= 1.05 * e64)
        out[f"n{n}_N{N}"] = case
    return out


EQUAL_ERROR_CASES = ((32, 2), (16, 3), (24, 3), (8, 4), (12, 4))


def best_at_equal_error(case):
    """The fastest FP32-field path of one equal-error case that keeps the
    FP64 error (within 1.05x), with its speed-up over FP64; None when no path
    does."""
    ok = [(v["speedup_over_fp64"], k) for k, v in case.items()
          if isinstance(v, dict) and v.get("equal_l2_error")]
    if not ok:
        return None
    sp, k = max(ok)
    return {"variant": k, "speedup_over_fp64": sp, "ratio_to_fp64": case[k]["ratio_to_fp64"]}


def equal_error(W, T=0.25):
    """The headline comparison: plain FP64 against the mixed-precision paths
    on the same mesh, N, data (standing wave, c^2 = 1), dt and number of
    steps; each whole solve to T is one captured graph (wadg_solve), timed
    with CUDA events after an untimed first solve; error = L2 error of p
    against the analytic solution by the volume rule.  'Equal' means within
    1.05x of the FP64 error.  Meshes (n^3 x 6 tets) and degrees where the
    discretisation error lies well above the FP32 rounding floor; the
    fewer-point volume rules where tabulated (N = 2..5), else the (N+1)^3
    rule.  The FP32-field paths run with plain FP32 state updates and, in
    the '_compensated' rows, with compensated summation of the state
    (wadg_set_compensation).  'headline' names the case with the most DOF
    where the plain split-bf16 and FP32 paths keep equal error."""
    import torch
    from synthetic import warped_cube, standing_wave, fewer_point_rule
    out = {}
    for n, N in EQUAL_ERROR_CASES:
        VXYZ, EToV, geom = warped_cube(n, N, 0.1)
        rule = fewer_point_rule(N) if N in (2, 3, 4, 5) else None
        dt_max = 0.5 * (1.0 / n) / (N + 1) ** 2
        case = {"workload": f"warped cube {n}^3x6 = {len(EToV)} tets, N={N}, "
                            f"{'collapsed' if rule is None else str(len(rule[1])) + '-point'} volume rule, c^2=1, "
                            f"standing wave to T={T}, dt_max={dt_max:.3e}"}
        for name in ("fp64", "fp32_3xbf16", "fp32", "fp32_tf32", "fp32_3xbf16_compensated", "fp32_compensated"):
            prec = name.replace("_compensated", "")
            m = W.wadg_mesh_create(N, VXYZ, EToV, geom, rule=rule)
            W.wadg_set_operators(m, prec, 1, 1.0, 1.0, None)
            if name.endswith("_compensated"):
                W.wadg_set_compensation(m, True)
            xq = W.wadg_volume_points(m)
            f0 = torch.from_numpy(standing_wave(xq, 0.0)[:, :, None, :]).cuda()
            Q = torch.empty((4, m.K, 1, m.Np), dtype=m.dtype, device="cuda")
            R = torch.zeros_like(Q)
            W.wadg_project(m, f0, Q)
            W.wadg_solve(m, Q, R, 0.0, T, dt_max)       # captures the graph
            W.wadg_project(m, f0, Q)
            R.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            nsteps = W.wadg_solve(m, Q, R, 0.0, T, dt_max)
            b.record()
            torch.cuda.synchronize()
            W.wadg_device_status(m)
            ms = a.elapsed_time(b)
            err = W.wadg_l2_error(m, Q, torch.from_numpy(standing_wave(xq, T)[:, :, None, :]).cuda(), 1)
            dof = 4 * m.K * m.Np
            case[name] = {"l2_error_p": err, "nsteps": nsteps, "solve_ms": ms,
                          "value": dof * 5 * nsteps / (ms * 1e-3)}
            del Q, R, f0, m
            torch.cuda.empty_cache()
        e64, v64 = case["fp64"]["l2_error_p"], case["fp64"]["value"]
        for prec in ("fp32_3xbf16", "fp32", "fp32_tf32", "fp32_3xbf16_compensated", "fp32_compensated"):
            case[prec]["ratio_to_fp64"] = case[prec]["l2_error_p"] / e64
            case[prec]["equal_l2_error"] = bool(case[prec]["l2_error_p"] <= 1.05 * e64)
            case[prec]["speedup_over_fp64"] = case[prec]["value"] / v64
        case["dof"] = 4 * len(EToV) * (N + 1) * (N + 2) * (N + 3) // 6
        case["best_at_equal_error"] = best_at_equal_error(case)
        out[f"n{n}_N{N}"] = case
    eq = [k for k, c in out.items() if c["fp32_3xbf16"]["equal_l2_error"] and c["fp32"]["equal_l2_error"]]
    if eq:
        k = max(eq, key=lambda k: out[k]["dof"])
        c = out[k]
        out["headline"] = {"case": k, "fp64_value": c["fp64"]["value"], "mixed_value": c["fp32_3xbf16"]["value"],
                           "speedup": c["fp32_3xbf16"]["speedup_over_fp64"],
                           "fp64_l2_error_p": c["fp64"]["l2_error_p"],
                           "mixed_l2_error_p": c["fp32_3xbf16"]["l2_error_p"],
                           "error_ratio": c["fp32_3xbf16"]["ratio_to_fp64"]}
    return out


def algorithmic_form(N: int, S: int, s: int, form: str) -> int:
    """Algorithmic bytes per element and stage of a formulation: the strong
    form reads its 9 geometric factors at (max(N+1, 2N-1))^3 volume points and
    its normals at (2N)^2 points per face, the update's two weights at the
    degree 2N+1 points; the others read the strong-weak set (algorithmic())."""
    if form != "strong":
        return algorithmic(N, S, s)[0]
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    nv, nf = max(N + 1, 2 * N - 1), 2 * N
    return s * (16 * Np * S + 9 * nv ** 3 + 2 * (N + 1) ** 3 + 12 * nf ** 2) + 32


def formulations(W, steps):
    """The three formulations on the headline mesh (warped cube, N = 4,
    heterogeneous c^2, the collapsed rule that the strong forms are built for)
    on the CUDA-core stage, FP32 and FP64: LSRK step time, one LSRK launch
    (step / 5) with its algorithmic bytes against the measured HBM copy
    bandwidth, and one RHS launch."""
    import torch
    hbm, _, _ = peaks()
    out = {}
    for prec, nsteps in (("fp32", max(2, steps // 2)), ("fp64", max(2, steps // 5))):
        m, Q = build_case(W, prec, 0)
        s = 4 if prec == "fp32" else 8
        dof = 4 * m.K * m.Np
        rows = {}
        for form in ("strong_weak", "strong", "strong_underintegrated"):
            W.wadg_set_formulation(m, form)
            tot, st = time_steps(W, m, Q, nsteps, 3)
            B = algorithmic_form(WORKLOAD["N"], 1, s, form)
            ls = tot / nsteps / 5  # one LSRK-mode launch, from the timed steps
            rows[form] = {"value": dof * 5 / (tot / nsteps * 1e-3), "ms_per_step": tot / nsteps, "stage_ms": ls,
                          "rhs_launch_ms": st, "algorithmic_bytes_per_element": B,
                          "achieved_gbs": B * m.K / (ls * 1e-3) / 1e9,
                          "hbm_frac": B * m.K / (ls * 1e-3) / 1e9 / hbm}
        W.wadg_device_status(m)
        for form in ("strong", "strong_underintegrated"):
            rows[form]["time_vs_strong_weak"] = rows[form]["ms_per_step"] / rows["strong_weak"]["ms_per_step"]
        out[prec] = rows
        del Q, m
        torch.cuda.empty_cache()
    out["workload"] = (f"warped cube {WORKLOAD['n']}^3x6, N=4, heterogeneous c^2, CUDA-core stage; strong: "
                       "7^3 volume and 8^2 face points per element for its volume and surface terms")
    return out


def planar_study(W, steps, meshes=("half_planar", "mostly_planar", "affine")):
    """Planar and curved tiles in separate kernels (Sec. 6) on the headline
    workload's tensor-core stage (N = 4, split bf16, 63-point rule,
    heterogeneous c^2): cubes warped for z < 0 (half the elements affine,
    half the tiles planar) and for z < -0.75 (7/8 of the tiles planar), and
    the affine cube (every tile planar), each with the split as planned, with every all-affine tile on
    the planar kernel, and off.  LSRK step time and one LSRK launch
    (step / 5)."""
    import torch
    from synthetic import warped_cube, c2_heterogeneous, standing_wave
    n, N = WORKLOAD["n"], WORKLOAD["N"]
    out = {}
    for name, planar_from, amp in (("half_planar", 0.0, WORKLOAD["warp"]),
                                   ("mostly_planar", -0.75, WORKLOAD["warp"]), ("affine", None, 0.0)):
        if name not in meshes:
            continue
        VXYZ, EToV, geom = warped_cube(n, N, amp, planar_from=planar_from)
        m = W.wadg_mesh_create(N, VXYZ, EToV, geom, rule=headline_rule())
        xq = W.wadg_volume_points(m)
        W.wadg_set_operators(m, "fp32_3xbf16", 1, 1.0, 1.0, c2_heterogeneous(xq))
        fq = torch.from_numpy(standing_wave(xq, 0.0)[:, :, None, :]).cuda()
        Q = torch.empty((4, m.K, 1, m.Np), dtype=m.dtype, device="cuda")
        W.wadg_project(m, fq, Q)
        del fq
        rows = {}
        dof = 4 * m.K * m.Np
        for mode in ("planned", "all", "off"):
            W.wadg_set_planar_split(m, mode)
            tot, st = time_steps(W, m, Q, steps, 3)
            rows[mode] = {"value": dof * 5 / (tot / steps * 1e-3), "ms_per_step": tot / steps,
                          "stage_ms": tot / steps / 5, "rhs_launch_ms": st, "info": W.wadg_planar_info(m)}
        W.wadg_device_status(m)
        for mode in ("planned", "all"):
            rows[f"time_{mode}_vs_off"] = rows[mode]["ms_per_step"] / rows["off"]["ms_per_step"]
        out[name] = rows
        del Q, m
        torch.cuda.empty_cache()
    out["workload"] = (f"Kuhn cube {n}^3x6, N={N}, fp32_3xbf16, the fewer-point rule, heterogeneous c^2; half_planar: "
                       "warp times (z/1)^2 for z < 0, none beyond; mostly_planar: warp times ((z + 0.75)/0.25)^2 for "
                       "z < -0.75, none beyond; affine: no warp")
    return out


def c2_study(W):
    """The precision configuration: warped cube 24^3 x 6 = 82,944 tets, N = 5,
    c^2 = 1, standing wave to T = 0.5, on the 96-point symmetric volume rule
    and on the collapsed 216-point rule.  For every precision (FP64, FP32 on
    the CUDA cores, FP32 fields with split-bf16 or tf32 tensor-core products),
    the L2 error of p against the analytic solution, the relative L2
    difference of the nodal p from the FP64 solution on the same rule (the
    FP64 path equals the oracle's discrete solution to 1e-11) and the
    throughput of the whole solve (one captured graph; the FP32-field paths
    are timed on a second solve after an untimed first one, each FP64 solve,
    one to three minutes, once)."""
    import torch
    from synthetic import warped_cube, standing_wave, fewer_point_rule
    n, N, T = 24, 5, 0.5
    VXYZ, EToV, geom = warped_cube(n, N, 0.1)
    h = 2.0 / n
    dt_max = 0.5 * (h / 2) / (N + 1) ** 2
    out = {"workload": f"warped cube {n}^3x6 = {len(EToV)} tets, N={N}, c^2=1, "
                       f"standing wave to T={T}, dt_max={dt_max:.3e}"}
    for rule_name, rule in (("96-point rule", fewer_point_rule(N)), ("collapsed 216-point rule", None)):
        rows = {}
        ref = None
        for prec in ("fp64", "fp32", "fp32_3xbf16", "fp32_tf32"):
            m = W.wadg_mesh_create(N, VXYZ, EToV, geom, rule=rule)
            W.wadg_set_operators(m, prec, 1, 1.0, 1.0, None)
            xq = W.wadg_volume_points(m)
            f0 = torch.from_numpy(standing_wave(xq, 0.0)[:, :, None, :]).cuda()
            Q = torch.empty((4, m.K, 1, m.Np), dtype=m.dtype, device="cuda")
            R = torch.zeros_like(Q)
            if prec != "fp64":
                W.wadg_project(m, f0, Q)
                W.wadg_solve(m, Q, R, 0.0, T, dt_max)
                R.zero_()
            W.wadg_project(m, f0, Q)
            stream = torch.cuda.current_stream()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            nsteps = W.wadg_solve(m, Q, R, 0.0, T, dt_max)
            b.record(stream)
            torch.cuda.synchronize()
            W.wadg_device_status(m)
            ms = a.elapsed_time(b)
            err = W.wadg_l2_error(m, Q, torch.from_numpy(standing_wave(xq, T)[:, :, None, :]).cuda(), 1)
            dof = 4 * m.K * m.Np
            row = {"l2_error_p": err, "nsteps": nsteps, "solve_ms": ms, "volume_points": m.Nq,
                   "dof_stage_per_s": dof * 5 * nsteps / (ms * 1e-3)}
            p = Q[0].double().cpu().numpy()
            if ref is None:
                ref = p
            else:
                row["rel_l2_diff_vs_fp64_nodal"] = float(np.linalg.norm(p - ref) / np.linalg.norm(ref))
                row["ratio_to_fp64"] = err / rows["fp64"]["l2_error_p"]
                row["speedup_over_fp64"] = row["dof_stage_per_s"] / rows["fp64"]["dof_stage_per_s"]
            rows[prec] = row
            del Q, R, f0, m
            torch.cuda.empty_cache()
        out[rule_name] = rows
    return out


def e2e_steps(W, m, Q, steps):
    """Same metric end to end through the C ABI with host buffers: every step
    one wadg_step_host call (the state Q copied from pinned host memory to the
    device, one LSRK step, Q copied back; the LSRK residual is integrator
    scratch that a step does not read, kept on the device; the call returns
    when the copies are done).  Returns the time per step and the bytes
    copied in and out per step."""
    import torch
    Qh = Q.cpu().pin_memory()
    dt = dt_for(m)
    stream = torch.cuda.current_stream()
    W.wadg_step_host(m, Qh, None, 0.0, dt, 1)  # warm-up (allocates the library's device copies)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(steps):
        W.wadg_step_host(m, Qh, None, 0.0, dt, 1)
    b.record(stream)
    torch.cuda.synchronize()
    nq = Q.numel() * Q.element_size()
    return a.elapsed_time(b) / steps, nq, nq


def _limit_blas_threads():
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        from threadpoolctl import threadpool_limits
        return threadpool_limits(1)
    except Exception:
        return None


SAMPLE_N = 16  # hexahedra per cube side in the oracle's sample (16^3 x 6 = 24,576 tets, 1/8 of the workload)


def _sample_elements(EToV, part: int, nparts: int):
    """Elements [k0, k1) of an equal split and their face neighbours (faces
    matched by sorted vertex triples), in increasing global order, and the
    positions of the owned ones in that list."""
    K = len(EToV)
    k0, k1 = part * K // nparts, (part + 1) * K // nparts
    if nparts == 1:
        return np.arange(K), np.arange(K)
    faces = np.array(((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)))
    tri = np.sort(np.asarray(EToV)[:, faces], axis=2).reshape(-1, 3)
    nv = int(np.max(EToV)) + 1
    key = (tri[:, 0] * nv + tri[:, 1]) * nv + tri[:, 2]
    own = np.zeros(K, dtype=bool)
    own[k0:k1] = True
    mine = np.isin(key, key[np.repeat(own, 4)])
    ks = np.unique(np.nonzero(mine)[0] // 4)
    return ks, np.nonzero((ks >= k0) & (ks < k1))[0]


class OracleSample:
    """The FP64 oracle, as it stands, on a bounded sample of the workload: the
    same recipe (warped cube, N = 4, heterogeneous c^2, the workload's volume
    rule) on a 16^3-hex cube (24,576 tets, 1/8 of the workload).  One stage =
    oracle RHS (strong-weak terms + matrix-free weight-adjusted inverse) + LSRK
    update, one thread.  part/nparts: the process owns an equal share of the
    elements and evaluates them on the sub-mesh of those elements and their
    face neighbours in increasing global order (every shared face keeps its
    owner and its points, so an owned element's stage is the whole mesh's);
    the neighbours' results are discarded.  nparts = 1: the whole sample."""

    def __init__(self, part: int = 0, nparts: int = 1):
        self._limit = _limit_blas_threads()
        from oracle import wadg as OW
        from oracle.discretization import Mesh, RefTet
        from synthetic import warped_cube, c2_heterogeneous, random_fields
        self.OW = OW
        N = WORKLOAD["N"]
        VXYZ, EToV, geom = warped_cube(SAMPLE_N, N, WORKLOAD["warp"])
        ks, self.owned = _sample_elements(EToV, part, nparts)
        self.ref = RefTet(N, volume_rule=headline_rule())
        self.mesh = Mesh(self.ref, VXYZ, EToV[ks], geom[ks])
        self.c2 = c2_heterogeneous(self.mesh.xq)
        self.c = self.ref.to_modal(random_fields((4, len(EToV), self.ref.Np), 1)[:, ks])
        self.res = np.zeros_like(self.c)
        self.K_sample = len(EToV)
        self.dof = 4 * len(self.owned) * self.ref.Np
        self.s = 0

    def stage(self) -> float:
        t0 = time.perf_counter()
        r = self.OW.rhs(self.mesh, self.c, c2q=self.c2)
        self.res = self.OW.LSRK_A[self.s % 5] * self.res + 1e-4 * r
        self.c = self.c + self.OW.LSRK_B[self.s % 5] * self.res
        self.s += 1
        return time.perf_counter() - t0

    def describe(self, stages, seconds, cores=1):
        return (f"a sample of the workload: warped cube {SAMPLE_N}^3 x 6 = {self.K_sample} tets, N={self.ref.N}, "
                f"{self.ref.Nq}-point volume rule, heterogeneous c^2, FP64, {stages} stages in {seconds:.1f} s "
                f"({cores} {'process' if cores == 1 else 'processes'} of one thread each; "
                "DOF*stage/s over the sample's DOF)")


def _oracle_part(part, nparts, nstages, barrier, queue):
    """One process of the all-core oracle run: build its part (not timed),
    one warm-up stage, then nstages stages between wall-clock stamps taken
    after every process has reached the barrier."""
    try:
        o = OracleSample(part, nparts)
        o.stage()
        barrier.wait(timeout=300)
        t0 = time.time()
        for _ in range(nstages):
            o.stage()
        queue.put((part, t0, time.time(), o.dof, o.describe(nstages, 0.0, nparts), None))
    except Exception as e:  # reported to the parent, which raises
        queue.put((part, 0.0, 0.0, 0, "", repr(e)))


def oracle_all_cores(nstages: int, cores: int | None = None):
    """The oracle on `cores` host cores (default: every core this process may
    run on), element-parallel over spawned processes: returns (DOF*stage/s
    over the sample's DOF, wall seconds of the timed stages, cores, text)."""
    import multiprocessing as mp
    cores = cores or len(os.sched_getaffinity(0))
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(cores), ctx.Queue()
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    procs = [ctx.Process(target=_oracle_part, args=(p, cores, nstages, barrier, queue)) for p in range(cores)]
    for pr in procs:
        pr.start()
    import queue as _q
    out = []
    try:
        while len(out) < cores:
            try:
                out.append(queue.get(timeout=5))
            except _q.Empty:
                if not any(pr.is_alive() for pr in procs):
                    raise RuntimeError("oracle processes exited without reporting")
    finally:
        for pr in procs:
            pr.join(timeout=60)
            if pr.is_alive():
                pr.kill()
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    errs = [e for *_, e in out if e]
    if errs:
        raise RuntimeError(f"oracle process failed: {errs[0]}")
    wall = max(o[2] for o in out) - min(o[1] for o in out)
    dof = sum(o[3] for o in out)
    text = out[0][4].replace(" in 0.0 s", f" in {wall:.1f} s")
    return dof * nstages / wall, wall, cores, text


def cpu_baseline(budget_s: float = 20.0):
    """The oracle on every host core (element-parallel processes) and on one
    core, on the 16^3 sample; the line's value is the all-core one."""
    o = OracleSample()
    o.stage()  # warm-up
    stages, t = 0, 0.0
    while t < budget_s and stages < 25:
        t += o.stage()
        stages += 1
    one = {"value": o.dof * stages / t, "cores": 1, "sample": o.describe(stages, t)}
    del o
    # about as much work per process as the single-core run did in total
    v, wall, cores, text = oracle_all_cores(max(5, stages))
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": text, "single_core": one}


def max_over_ranks(ms: float, ws: int) -> float:
    """Largest of the ranks' timings (every rank gets it); ws = 1 returns ms."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(dof_per_rank: int, stages: int, ms: float, ws: int) -> float:
    """Whole-job DOF*stage/s: all ranks' work over the slowest rank's time."""
    return ws * dof_per_rank * stages / (ms * 1e-3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """Reference arm: the oracle on every host core (element-parallel
    processes) on the 16^3 sample of the workload; one step = one LSRK step
    (5 stages) of the sample."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    v, wall, cores, text = oracle_all_cores(5 * (args.warmup + args.steps))
    steps = args.warmup + args.steps
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / steps,
            "higher_is_better": True, "scaling": "weak", "dtype": "f64", "data": "synthetic", "vs_baseline": None,
            "config": headline_config(ws),
            "reference_sample": (f"timed on the {SAMPLE_N}^3 x 6 = {6 * SAMPLE_N ** 3}-tet sample of the workload "
                                 "(value normalised by the sample's DOF); ms_per_step is one LSRK step (5 stages) "
                                 "of the sample on all host cores; the warm-up steps are timed with the others"),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": text, "value": v},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--c2", action="store_true",
                    help="run only the N = 5 precision study (82,944 tets, T = 0.5) and print its JSON")
    ap.add_argument("--forms", action="store_true",
                    help="run only the formulation comparison on the headline mesh and print its JSON")
    ap.add_argument("--batch", action="store_true",
                    help="run only the uneven-batch study (12 meshes, N = 2..6, large and small) and print its JSON")
    ap.add_argument("--equal-error", action="store_true",
                    help="run only the equal-L2-error comparison (FP64 vs mixed precision, whole solves) and print it")
    ap.add_argument("--planar", action="store_true",
                    help="run only the planar/curved kernel split study (half-planar and affine cubes) and print it")
    ap.add_argument("--planar-meshes", default="half_planar,mostly_planar,affine",
                    help="meshes of the planar study (comma-separated subset of half_planar, mostly_planar, affine)")
    ap.add_argument("--n", type=int, default=WORKLOAD["n"],
                    help="hexahedra per cube side (default: the headline workload; smaller for profiling)")
    ap.add_argument("--N", type=int, default=WORKLOAD["N"],
                    help="polynomial degree (default: the headline workload's 4; 5 runs the N = 5 tensor-core stage)")
    args = ap.parse_args()
    WORKLOAD["n"] = args.n
    WORKLOAD["N"] = args.N
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_1608_03836_gb300 as W
    if args.c2:
        if rank == 0:
            print(json.dumps({"c2_precision_study": c2_study(W)}))
        return
    if args.forms:
        if rank == 0:
            print(json.dumps({"formulations": formulations(W, args.steps)}))
        return
    if args.planar:
        if rank == 0:
            print(json.dumps({"planar_split": planar_study(W, max(2, args.steps), args.planar_meshes.split(","))}))
        return
    if args.equal_error:
        if rank == 0:
            print(json.dumps({"equal_error": equal_error(W)}))
        return
    if args.batch:
        if rank == 0:
            print(json.dumps({"uneven_batch": uneven_batch(W, max(2, args.steps)),
                              "uneven_batch_small": uneven_batch(W, max(2, args.steps), small=True),
                              "uneven_batch_tc": uneven_batch(W, max(2, args.steps), tensor_cores=True),
                              "uneven_batch_tc_small": uneven_batch(W, max(2, args.steps), small=True,
                                                                    tensor_cores=True)}))
        return

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    headline = "fp32_3xbf16"
    rule = headline_rule()
    m, Q = build_case(W, headline, rank, rule=rule)
    Np, K = m.Np, m.K
    dof = 4 * K * Np
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        total_ms, stage_ms = time_steps(W, m, Q, args.steps, args.warmup)
    barrier()
    W.wadg_device_status(m)
    total_ms = max_over_ranks(total_ms, ws)
    ms_per_step = total_ms / args.steps
    value = job_value(dof, 5, ms_per_step, ws)
    e2e_ms, h2d, d2h = e2e_steps(W, m, Q, max(2, args.steps // 2))
    e2e_value = ws * dof * 5 / (e2e_ms * 1e-3)
    hbm, peak_kind, sm_max = peaks()
    nq = m.Nq
    B, F = algorithmic(WORKLOAD["N"], 1, 4, nq=nq)
    # the dominant kernel as the timed region launches it: five LSRK-mode
    # stage launches per step (B counts Q and res read and written)
    lsrk_ms = ms_per_step / 5
    achieved_gbs = B * K / (lsrk_ms * 1e-3) / 1e9
    achieved_tf = F * K / (lsrk_ms * 1e-3) / 1e12
    tpe = tc_traffic_per_element() if (WORKLOAD["N"], nq) == (4, 63) else None
    variants = {headline: {"value": value, "ms_per_step": ms_per_step, "stage_ms": lsrk_ms, "rhs_launch_ms": stage_ms,
                           "achieved_tflops": achieved_tf, "achieved_gbs": achieved_gbs,
                           "dtype": "f32 fields, bf16x3 tensor products", "volume_points": nq}}
    del Q, m
    torch.cuda.empty_cache()

    # the same precision on the collapsed (N+1)^3 rule
    mc, Qc = build_case(W, headline, rank)
    tcl, scl = time_steps(W, mc, Qc, args.steps, 3)
    W.wadg_device_status(mc)
    Bc, _ = algorithmic(WORKLOAD["N"], 1, 4)
    lcl = tcl / args.steps / 5
    variants[headline + "_collapsed_rule"] = {
        "value": ws * dof * 5 / (tcl / args.steps * 1e-3), "ms_per_step": tcl / args.steps, "stage_ms": lcl,
        "rhs_launch_ms": scl,
        "achieved_gbs": Bc * K / (lcl * 1e-3) / 1e9, "hbm_frac": Bc * K / (lcl * 1e-3) / 1e9 / hbm,
        "algorithmic_bytes_per_element": Bc, "volume_points": mc.Nq,
        "dtype": "f32 fields, bf16x3 tensor products"}
    del Qc, mc
    torch.cuda.empty_cache()

    mtf, Qtf = build_case(W, "fp32_tf32", rank, rule=rule)
    ttf, stf = time_steps(W, mtf, Qtf, args.steps, 3)
    W.wadg_device_status(mtf)
    ltf = ttf / args.steps / 5
    variants["fp32_tf32"] = {"value": ws * dof * 5 / (ttf / args.steps * 1e-3), "ms_per_step": ttf / args.steps,
                             "stage_ms": ltf, "rhs_launch_ms": stf, "achieved_gbs": B * K / (ltf * 1e-3) / 1e9,
                             "hbm_frac": B * K / (ltf * 1e-3) / 1e9 / hbm,
                             "dtype": "f32 fields, tf32 tensor products"}
    del Qtf, mtf
    torch.cuda.empty_cache()

    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s, CUDA-core FMA
    m32, Q32 = build_case(W, "fp32", rank, rule=rule)
    t32, s32 = time_steps(W, m32, Q32, args.steps, 3)
    l32 = t32 / args.steps / 5
    variants["fp32"] = {"value": ws * dof * 5 / (t32 / args.steps * 1e-3), "ms_per_step": t32 / args.steps,
                        "stage_ms": l32, "rhs_launch_ms": s32, "achieved_tflops": F * K / (l32 * 1e-3) / 1e12,
                        "achieved_gbs": B * K / (l32 * 1e-3) / 1e9, "dtype": "f32",
                        "alu_frac": F * K / (l32 * 1e-3) / 1e12 / fp32_peak}
    del Q32, m32
    torch.cuda.empty_cache()
    if not args.no_fp64:
        m64, Q64 = build_case(W, "fp64", rank, rule=rule)
        t64, s64 = time_steps(W, m64, Q64, max(1, args.steps // 5), 3)
        ms64 = t64 / max(1, args.steps // 5)
        B64, _ = algorithmic(WORKLOAD["N"], 1, 8, nq=nq)
        l64 = ms64 / 5
        variants["fp64"] = {"value": ws * dof * 5 / (ms64 * 1e-3), "ms_per_step": ms64, "stage_ms": l64,
                            "rhs_launch_ms": s64, "achieved_tflops": F * K / (l64 * 1e-3) / 1e12,
                            "achieved_gbs": B64 * K / (l64 * 1e-3) / 1e9, "dtype": "f64"}
        variants["fp64"]["headline_speedup"] = value / variants["fp64"]["value"]
        del Q64, m64
        torch.cuda.empty_cache()

    extras = {}
    if not args.no_extras:
        extras["batched_shots"] = batched_shots(W, max(2, args.steps // 3))
        extras["uneven_batch"] = uneven_batch(W, max(2, args.steps))
        extras["uneven_batch_small"] = uneven_batch(W, max(2, args.steps), small=True)
        extras["uneven_batch_tc"] = uneven_batch(W, max(2, args.steps), tensor_cores=True)
        extras["uneven_batch_tc_small"] = uneven_batch(W, max(2, args.steps), small=True, tensor_cores=True)
        extras["accuracy"] = accuracy(W)
        extras["equal_error"] = equal_error(W)
        extras["formulations"] = formulations(W, args.steps)
        extras["adjoint"] = adjoint_timing(W)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3/f32", "data": "synthetic",
        "config": headline_config(ws),
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                     "frac": achieved_gbs / hbm,
                     "traffic": None if tpe is None else tpe * K,
                     "peak_kind": peak_kind,
                     "kernel": (f"stage_tc_kernel<{WORKLOAD['N']},1,0,{nq}>" if WORKLOAD["N"] <= 4 else
                                f"stage_tc5_kernel<1,0,{nq}>") + " (one launch = one LSRK stage over all elements)",
                     "launch_ms": lsrk_ms,
                     "launch_ms_from": "the timed region: ms_per_step / 5 launches (CUDA events on the launching stream)",
                     "algorithmic_bytes_per_element": B,
                     # the tensor-core stage's mean correction, 3 x Np FP32 values per element read in
                     # the epilogue: part of the traffic, not of the method's algorithmic bytes
                     "mean_correction_bytes_per_element": 12 * (WORKLOAD["N"] + 1) * (WORKLOAD["N"] + 2) * (WORKLOAD["N"] + 3) // 6,
                     "tensor": {"achieved_fp32_equiv_tflops": achieved_tf,
                                "note": "flops counted once per product; each runs as three bf16 MMAs "
                                        "(four in the update, whose operators carry a third part)"}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 5 * args.steps,
        "clocks": clk.summary(),
        "variants": variants,
        **extras,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))


if __name__ == "__main__":
    main()
