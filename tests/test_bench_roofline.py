"""The roofline arithmetic of bench.py on CPU: the algorithmic bytes and flops
per element and stage that the reported roofline divides by, recounted from
the arrays one LSRK stage touches and from the products it applies."""
import pytest


def _bench():
    import bench
    return bench


def _bytes_from_layout(N, S, s, nq):
    """One LSRK stage reads Q and res and writes res and Q_out (4 fields x Np
    values per column each), reads the 11 geometric rows per volume point
    (9 G_ai, c^2/J, 1/J) and n J^f (3 components) at the 4 Nfq face points,
    and the element's connectivity (counted as 32 bytes)."""
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    Nfq = (N + 1) ** 2
    fields = 4 * (4 * Np * S * s)
    vgeo = 11 * nq * s
    fgeo = 3 * 4 * Nfq * s
    return fields + vgeo + fgeo + 32


def _flops_from_products(N, S, nq):
    """2 flops per multiply-add of each dense product of the method: volume
    (3 V_q u_i, 3 V_q^a p, 3 (V_q^a)^T, 3 V_q^T: 12 products of nq x Np),
    update (4 fields x (V_q, P_q): 8 products of nq x Np), faces (4 traces
    interpolated and 4 fluxes lifted per face: 8 products of Np x Nfq on each
    of the 4 faces)."""
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    Nfq = (N + 1) ** 2
    return 2 * (12 + 8) * nq * Np * S + 2 * 8 * Np * 4 * Nfq * S


@pytest.mark.parametrize("N,S,s,nq", [(4, 1, 4, 63), (4, 1, 8, 63), (4, 1, 4, 125), (4, 1, 8, 125),
                                      (5, 1, 4, 216), (4, 64, 4, 125), (3, 1, 4, 64), (3, 1, 4, 35)])
def test_algorithmic_bytes_and_flops(N, S, s, nq):
    B, F = _bench().algorithmic(N, S, s, nq=nq)
    assert B == _bytes_from_layout(N, S, s, nq)
    assert F == _flops_from_products(N, S, nq)


def test_headline_figures():
    """The per-element figures the roofline of the headline workload uses:
    6,244 B and 144,200 flops (FP32, N = 4, 63 points); 8,972 B with the 125
    points; 12,456 B in FP64."""
    b = _bench()
    assert b.algorithmic(4, 1, 4, nq=63) == (6244, 144200)
    assert b.algorithmic(4, 1, 4)[0] == 8972 and b.algorithmic(4, 1, 4)[1] == 231000
    assert b.algorithmic(4, 1, 8, nq=63)[0] == 12456
    # the strong form: 9 factors at 7^3 points, 2 weights at 5^3, n J^f at 8^2 per face
    assert b.algorithmic_form(4, 1, 4, "strong") == 4 * (16 * 35 + 9 * 343 + 2 * 125 + 12 * 64) + 32 == 18692
    assert b.algorithmic_form(4, 1, 4, "strong_weak") == 8972


def test_job_value_counts_every_rank():
    b = _bench()
    assert b.job_value(4 * 196608 * 35, 5, 2.0, 1) == pytest.approx(4 * 196608 * 35 * 5 / 2e-3)
    assert b.job_value(100, 5, 2.0, 4) == pytest.approx(4 * b.job_value(100, 5, 2.0, 1))


def test_both_arms_report_the_same_config():
    """The reference arm (the oracle on a bounded sample, on every host core)
    prints the native arm's config; the sample is named beside it and
    described in its cpu_baseline."""
    import json
    import os
    import subprocess
    import sys
    b = _bench()
    cfg = b.headline_config(1)
    assert cfg["elements"] == 196608 and cfg["volume_points"] == 63 and cfg["dof"] == 4 * 196608 * 35
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["impl"] == "reference" and line["config"] == cfg
    assert line["metric"] == b.METRIC and line["unit"] == b.UNIT and line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and "sample" in line["cpu_baseline"]["sample"]
    # every host core, element-parallel; the sample it times is named beside the config
    assert line["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
    assert "16^3 x 6 = 24576-tet sample" in line["reference_sample"]
