"""Host logic of bench.py that the reported numbers depend on (CPU only):
the algorithmic-bytes model of the exact evaluation and the traffic table.
"""

import numpy as np

import bench
import synth
from oracle import acom_oracle as O


def test_pattern_shell_rows_counts_the_rows_the_image_reaches():
    """The non-zero shell rows that the select kernel's compulsory bytes are
    counted from: every row where the oracle's polar image of the pattern is
    non-zero is counted, and the count exceeds those rows by less than 1 %
    (rows the tent reaches only at weight zero)."""
    W = bench.W
    scan = synth.grain_scan(1002, H=6, W=6, peaks="uniform10-60")
    prm = O.PlanParams(W["S"], W["dq"], W["N"], W["delta"], lam=W["lam"])
    rows = []
    for b in range(scan.n_patterns):
        X = O.polar_image(*scan.pattern(b), prm)
        rows.append(int((np.abs(X).sum(axis=1) > 0).sum()))
    est = bench.pattern_shell_rows(scan)
    assert est >= np.mean(rows) - 1e-9
    assert est <= 1.01 * np.mean(rows)


def test_traffic_table_is_tied_to_its_sources():
    """A traffic figure is reported only for the captured kernel sources,
    precision and workload, and scaled only where it grows with the
    patterns of a launch."""
    for name, (byts, pats, files, digest, prec, wl, prop) in bench.TRAFFIC_PER_LAUNCH.items():
        assert byts > 0 and pats > 0 and len(digest) == 16
        ok = bench.sources_hash(files) == digest and bench.W["name"] == wl
        t = bench.kernel_traffic(name, pats, prec)
        assert (t == byts) if ok else (t is None)
        half = bench.kernel_traffic(name, pats / 2, prec)
        if ok:
            assert (half == byts / 2) if prop else (half is None)
        assert bench.kernel_traffic(name, pats, "bf16" if prec != "bf16" else "fp16") is None


def test_reference_arm_line_keys(monkeypatch, capsys):
    """The reference arm prints the contract's keys, with the GPU arm's
    workload description (a tiny scan and sample keep this fast)."""
    import argparse
    import json
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("LOCAL_RANK", "0")
    import time
    monkeypatch.setattr(bench, "oracle_plans", lambda stride=1: _tiny_plans())
    t0 = time.perf_counter()
    # the worker processes build every 64th zone axis of the workload's plan
    bench.reference_arm(argparse.Namespace(warmup=1, steps=2, gpus=1, scan="4x4",
                                           oracle_stride=64))
    wall = time.perf_counter() - t0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    # ms_per_step is the time of the sample each step ran: it fits the run
    assert 0 < line["ms_per_step"] * line["steps"] / 1e3 <= wall
    assert line["cpu_baseline"]["cores"] >= 1
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert {"workload", "patterns_per_gpu", "peaks_nnz", "zone_axes", "shells",
            "n_phi"} <= set(line["config"])
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def _tiny_plans():
    """A small oracle plan (6-degree grid, 40 shells, 72 bins) standing in for
    the workload's plans, so that the test exercises the arm, not the oracle's
    speed."""
    refl = O.reflections(np.eye(3) * 4.08, [[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]],
                         [79.0] * 4, [0.25] * 4, 1.5)
    v0, v1, v2, om = O.cubic_triangle()
    za = O.zone_axis_grid(v0, v1, v2, 6.0, om)
    return [O.orientation_plan(refl, za, O.PlanParams(40, 0.0375, 72, 0.08, lam=0.01969))]


def test_sweep_oracle_subset_agreement(monkeypatch):
    """The sweep's oracle agreement: the patterns are matched by oracle worker
    processes against the plan of the given step, and each run's choices are
    compared with the oracle's argmax (its own argmax agrees on every
    pattern; a choice moved off the argmax to a lower value does not).  A
    small plan (6-degree grid, 40 shells, 72 bins) keeps this fast."""
    tiny = dict(bench.W, S=40, dq=0.0375, N=72, delta=0.08, q_max=1.5)
    monkeypatch.setattr(bench, "W", tiny)
    scan = synth.grain_scan(1002, H=3, W=3, peaks="uniform10-60")
    refl = O.reflections(np.eye(3) * 4.08, [[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]],
                         [79.0] * 4, [0.25] * 4, 1.5)
    v0, v1, v2, om = O.cubic_triangle()
    za = O.zone_axis_grid(v0, v1, v2, 6.0, om)
    plan = O.orientation_plan(refl, za, O.PlanParams(40, 0.0375, 72, 0.08, lam=tiny["lam"]))
    idx = np.array([0, 4, 8])
    own, off = [], []
    for b in idx:
        mt = O.match_pattern(plan, *scan.pattern(int(b)))
        own.append((mt.za, mt.k, mt.mirror))
        C = mt.Cm if mt.mirror else mt.C
        k2 = int(np.argmin(C[mt.za]))             # the axis' lowest bin
        off.append((mt.za, k2, mt.mirror))
    got = bench.oracle_subset_agreement(scan, idx, 6.0, len(za), [own, off], cores=2)
    assert got[0] == "3/3"
    assert got[1] == "0/3"
