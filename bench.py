#!/usr/bin/env python
"""Benchmark of the sparse correlation match on one or more GB300s.

Workload: the 256 x 256 fcc-Au scan (65,536 patterns with 10-60 Bragg peaks
each in CSR, 200 Voronoi grains at random orientations) matched against the
1-degree plan (903 zone axes, 150 shells of 0.01 1/A, 360 phi3 bins).  One
step is the whole path: plan build (reflections, plan raster + transform,
normalisation) and the match of every pattern (sparse polar raster +
transform, shell contraction, inverse transform + argmax, refinement).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp16|bf16|fp32]
  python bench.py --impl reference ...   # the FP64 CPU oracle as the reference arm
  python bench.py --workload mixed ...   # two phases in one plan (see below)
  python bench.py --workload refine ...  # coarse 3-degree match + continuous refinement
  python bench.py --workload sweep ...   # 512x512 scan: 1 and 0.5 degree plans x precisions

The default precision is FP16 operands (per-pattern and per-plan power-of-two
scaling) on the tensor cores for the certified bound, with every winner
evaluated exactly in FP32; bf16 takes BF16 operands instead, fp32 the FP32
CUDA-core contraction.  Under torchrun (N > 1)
every rank matches its own scan (weak scaling, scan seed + rank); there is no
collective on the data path; rank 0 prints one JSON line.

--workload mixed: 65,536 independent patterns drawn 50/50 from fcc Au and hcp
Mg (peaks above 1e-3 of the strongest, at most 40) matched against one plan
holding the Au 2-degree grid (231 axes) and the Mg 1-degree grid (1770 axes),
75 shells of 0.02 1/A, 180 bins; every pattern gets each phase's best score
and a phase decision.

--workload refine: the same 256x256 scan matched on the 3-degree plan (105
axes) and then refined (20 Gauss-Newton steps of the continuous kinematical
score, from the match, from the runner-up zone axis outside the match's grid
neighbourhood, and from the Friedel twin of each); the line also carries the
plain FP32 1-degree grid path measured in the same run.

--workload sweep: a 512x512 grain scan (262,144 patterns, Poisson(30) peaks
clipped to 5..80) against the 1-degree (903 axes) and 0.5-degree (3486 axes)
plans with FP32, BF16, FP16 and E4M3 contraction operands; the line's value is
the 0.5-degree FP16 step and its "sweep" object holds every combination, each
with its argmax agreement with the oracle on the same 1,000 sampled patterns.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "patterns indexed/s on 1 GB300, % of roofline, mean misorientation (deg)"
W = dict(name="au_scan_256x256_1deg", phases=(("Au", 1.0),), Z=903, step=1.0, S=150, dq=0.01,
         N=360, seed=1002, H=256, Wd=256, grains=200, delta=0.08, lam=0.01969, q_max=1.5,
         text=("fcc Au 256x256 scan (65,536 patterns, 10-60 peaks each, CSR, 200 Voronoi "
               "grains) vs 1-degree plan (903 zone axes, 150 shells x 0.01 1/A, 360 phi3 bins)"))
REFINE = dict(name="au_scan_256x256_3deg_refined", phases=(("Au", 3.0),), Z=105, step=3.0,
              refine=True, precision="bf16",
              text=("fcc Au 256x256 scan (65,536 patterns, 10-60 peaks each, CSR, 200 Voronoi "
                    "grains, continuous orientations) matched on the 3-degree plan (105 zone "
                    "axes, 150 shells x 0.01 1/A, 360 phi3 bins), then refined: 20 Gauss-Newton "
                    "steps of the continuous kinematical score from the match, the runner-up "
                    "axis and their Friedel twins"))
SWEEP = dict(name="au_scan_512x512_halfdeg_sweep", phases=(("Au", 0.5),), Z=3486, step=0.5,
             seed=1005, H=512, Wd=512, peaks="poisson30", sweep=True,
             text=("fcc Au 512x512 scan (262,144 patterns, Poisson(30) peaks clipped to 5..80, "
                   "CSR, 200 Voronoi grains) vs the 0.5-degree plan (3486 zone axes, 150 shells "
                   "x 0.01 1/A, 360 phi3 bins); sweep over 1 and 0.5 degree plans and FP32, "
                   "BF16 and FP16 operands"))
MIXED = dict(name="au2deg_mg1deg_mixed_65536", phases=(("Au", 2.0), ("Mg", 1.0)), Z=231 + 1770,
             step=None, S=75, dq=0.02, N=180, seed=1003, n_patterns=65536,
             text=("65,536 patterns, 50/50 fcc Au / hcp Mg (peaks > 1e-3 of the strongest, "
                   "at most 40, CSR) vs one plan of the Au 2-degree (231 axes) and Mg "
                   "1-degree (1770 axes) grids, 75 shells x 0.02 1/A, 180 phi3 bins"))
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default=None, choices=["bf16", "fp16", "fp32"],
                    help="contraction operands (default: the workload's, fp16 for au_scan "
                         "and mixed, bf16 for refine)")
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--exhaustive", action="store_true",
                    help="inverse-transform every zone axis (no certified pruning)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=16)
    ap.add_argument("--scan", default=None,
                    help="scan size HxW (default: the workload's; smaller sizes are for "
                         "profiling captures only)")
    ap.add_argument("--workload", default="au_scan",
                    choices=["au_scan", "mixed", "refine", "sweep"])
    args = ap.parse_args()
    if args.workload == "mixed":
        W.update(MIXED)
    elif args.workload == "refine":
        W.update(REFINE)
    elif args.workload == "sweep":
        W.update(SWEEP)
    if args.scan is None:
        args.scan = f"{W['H']}x{W['Wd']}"
    elif "n_patterns" not in W:
        # a scan of another size, same recipe: the workload text names its size
        H, Wd = (int(v) for v in args.scan.split("x"))
        old = f"{W['H']}x{W['Wd']} scan ({W['H'] * W['Wd']:,} patterns"
        assert old in W["text"]
        W["text"] = W["text"].replace(old, f"{H}x{Wd} scan ({H * Wd:,} patterns")
    if args.precision is None:
        args.precision = W.get("precision", "fp16")
    return args


def make_scan(seed, args):
    import synth
    if "n_patterns" in W:
        return synth.mixed_patterns(seed, n_patterns=W["n_patterns"])
    H, Wd = (int(v) for v in args.scan.split("x"))
    return synth.grain_scan(seed, H=H, W=Wd, peaks=W.get("peaks", "uniform10-60"))


def pattern_shell_rows(scan):
    """Mean number of shell rows per pattern that its sparse polar image can
    make non-zero: shells s with |r_m - q_s| < delta for some peak m, q_s =
    (s + 1) dq.  These are the only rows of a pattern's spectra that the exact
    evaluation multiplies (a zero row contributes exactly 0)."""
    S, dq, delta = W["S"], W["dq"], W["delta"]
    rp = np.asarray(scan.row_ptr, dtype=np.int64)
    B = len(rp) - 1
    r = np.hypot(np.asarray(scan.qx, np.float64), np.asarray(scan.qy, np.float64))
    b = np.repeat(np.arange(B), np.diff(rp))
    lo = np.clip(np.floor((r - delta) / dq - 1.0).astype(np.int64) + 1, 0, S)
    hi = np.clip(np.ceil((r + delta) / dq - 1.0).astype(np.int64) - 1, -1, S - 1)
    ok = hi >= lo
    diff = np.zeros((B, S + 1), np.int32)
    np.add.at(diff, (b[ok], lo[ok]), 1)
    np.add.at(diff, (b[ok], hi[ok] + 1), -1)
    return float((np.cumsum(diff[:, :S], axis=1) > 0).sum() / max(B, 1))


def peaks_file():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the
    timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(self.rows),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- accuracy

def cubic_ops():
    import itertools
    ops = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1.0, -1.0), repeat=3):
            M = np.zeros((3, 3))
            for r in range(3):
                M[r, perm[r]] = signs[r]
            if np.linalg.det(M) > 0:
                ops.append(M)
    return np.array(ops)


def hexagonal_ops():
    """The 12 proper rotations of 622 (c along z, a along x)."""
    ops = []
    for k in range(6):
        c, s = math.cos(k * math.pi / 3), math.sin(k * math.pi / 3)
        Rz = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])
        ops += [Rz, Rz @ np.diag([1.0, -1.0, -1.0])]
    return np.array(ops)


def misorientation(m_est, m_true, ops=None, spread=None):
    """Mean symmetry-reduced misorientation (deg), also reduced over the
    in-plane Friedel twin m Rz(pi), and the zone-axis tilt error.  With a
    dict ``spread``, also the median misorientation and the fraction of
    patterns within 0.1 and 1 degree go into it."""
    ops = cubic_ops() if ops is None else ops
    me = m_est.astype(np.float64)
    # re-orthonormalise the FP32-stored matrices before taking angles
    u, _, vt = np.linalg.svd(me)
    me = u @ vt
    SM = np.einsum("sij,bjk->sbik", ops, me)

    def angles(M):                      # rotation angle of m_true^T M, robust near 0
        D = np.einsum("bji,sbjk->sbik", m_true, M)
        tr = np.trace(D, axis1=2, axis2=3)
        v = np.stack([D[..., 2, 1] - D[..., 1, 2], D[..., 0, 2] - D[..., 2, 0],
                      D[..., 1, 0] - D[..., 0, 1]], -1)
        return np.degrees(2 * np.arctan2(np.linalg.norm(v, axis=-1) / 2, (1 + tr) / 2))

    a1 = angles(SM)
    ang = a1.min(axis=0)
    Rz = np.diag([-1.0, -1.0, 1.0])
    ang2 = np.minimum(a1, angles(np.einsum("sbik,kl->sbil", SM, Rz))).min(axis=0)
    we = np.einsum("sij,bj->sbi", ops, me[:, :, 2])
    c = np.abs(np.einsum("sbi,bi->sb", we, m_true[:, :, 2])).max(axis=0)
    tilt = np.degrees(np.arccos(np.clip(c, -1, 1)))
    if spread is not None:
        spread.update({"median_misorientation_deg": float(np.median(ang)),
                       "frac_within_0.1_deg": float(np.mean(ang <= 0.1)),
                       "frac_within_1_deg": float(np.mean(ang <= 1.0))})
    return float(ang.mean()), float(ang2.mean()), float(tilt.mean())


# ------------------------------------------------------------- oracle leg

def oracle_plans(stride=1):
    """The oracle's plan of every phase of the workload (every stride-th
    zone axis)."""
    from oracle import acom_oracle as O
    plans = []
    for phase, step in W["phases"]:
        if phase == "Au":
            refl = O.reflections(np.eye(3) * 4.08,
                                 [[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]],
                                 [79.0] * 4, [0.25] * 4, W["q_max"])
            v0, v1, v2, om = O.cubic_triangle()
        else:
            a, c = 3.21, 5.21
            L = np.array([[a, 0, 0], [-a / 2, a * math.sqrt(3) / 2, 0], [0, 0, c]])
            refl = O.reflections(L, [[1 / 3, 2 / 3, .25], [2 / 3, 1 / 3, .75]], [12.0] * 2,
                                 [0.3] * 2, W["q_max"])
            v0, v1, v2, om = O.hexagonal_triangle()
        za = O.zone_axis_grid(v0, v1, v2, step, om)[::stride]
        plans.append(O.orientation_plan(refl, za, O.PlanParams(W["S"], W["dq"], W["N"],
                                                               W["delta"], lam=W["lam"])))
    return plans


def oracle_refine(plan, mt, qx, qy, I):
    """The oracle's grid refinement of match ``mt`` followed by its
    continuous refinement (match and Friedel twin)."""
    from oracle import acom_oracle as O
    rf = O.refine(mt, plan.za, W["step"])
    refl = O.reflections(np.eye(3) * 4.08, [[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]],
                         [79.0] * 4, [0.25] * 4, W["q_max"])
    return O.refine_with_twin(rf.m, qx, qy, I, refl, W["lam"], O.RefineParams())


def oracle_match(plans, qx, qy, I):
    """The oracle's best over all phases' axes (global axis index)."""
    from oracle import acom_oracle as O
    if len(plans) == 1:
        return O.match_pattern(plans[0], qx, qy, I)
    mm = O.match_multi(plans, qx, qy, I)
    return O.best_match(np.concatenate([m.C for m in mm.matches]),
                        np.concatenate([m.Cm for m in mm.matches]))


def host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# Oracle worker processes (spawn: the parent has initialised CUDA).  Each
# builds the workload's oracle plans once; a match needs their spectra only,
# so the real plans are dropped to halve the worker's memory.
_POOL_PLANS = None


def _pool_init(w, stride=1):
    global _POOL_PLANS
    W.update(w)
    plans = oracle_plans(stride)
    for q in plans:
        q.P = None
    _POOL_PLANS = plans


def _pool_ready(_):
    time.sleep(0.3)
    return os.getpid()


def _pool_match(task):
    """The oracle's match of one pattern; with the GPU's choice (za, k,
    mirror) given, also whether that choice is the oracle's or a documented
    tie (the oracle's value there within 1e-5 relative of its best)."""
    (qx, qy, I), choice = task
    mt = oracle_match(_POOL_PLANS, qx, qy, I)
    if W.get("refine"):
        oracle_refine(_POOL_PLANS[0], mt, qx, qy, I)
    ok = None
    if choice is not None:
        # one choice (z, k, mirror), or a list of them (one per GPU run)
        oks = []
        for z, k, m in (choice if isinstance(choice, list) else [choice]):
            val = (mt.Cm if m else mt.C)[z, k]
            oks.append((z, k, m) == (mt.za, mt.k, mt.mirror) or val >= mt.score * (1 - 1e-5))
        ok = oks if isinstance(choice, list) else oks[0]
    return int(mt.za), int(mt.k), int(mt.mirror), float(mt.score), ok


def oracle_pool(cores, stride=1, w=None):
    """A pool of ``cores`` oracle workers with the plans of workload ``w``
    (default: the current one) built (every ``stride``-th zone axis; returns
    after every worker has finished its set-up) and the time that took; fewer
    workers where host memory would not hold every worker's plans."""
    import multiprocessing as mp
    w = dict(W) if w is None else w
    per = sum(8 * 1.1 * w["Z"] * w["S"] * (w["N"] // 2 + 1) * 2 for _ in w["phases"]) + 0.5e9
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        cores = max(1, min(cores, int(0.5 * avail / per)))
    except (ValueError, OSError):
        pass
    t0 = time.perf_counter()
    pool = mp.get_context("spawn").Pool(cores, initializer=_pool_init, initargs=(w, stride))
    pool.map(_pool_ready, range(4 * cores), chunksize=1)
    return pool, cores, time.perf_counter() - t0


def cpu_baseline(scan, gpu_res, n_sample):
    """The oracle as it stands on this host's cores, on a bounded sample of
    the workload, extrapolated to the whole scan: (1) one core: the full plan
    build timed once, then n_sample patterns matched; (2) every core: one
    worker process per core, each with the plans built (timed: the set-up
    runs on all workers at once), then 4 patterns per worker matched across
    the pool (wall time).  Returns the all-core figure with the single-core
    one inside, and the argmax agreement of the sampled patterns with the GPU."""
    t0 = time.perf_counter()
    plans = oracle_plans()
    t_plan = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    idx = rng.choice(scan.n_patterns, n_sample, replace=False)
    agree = 0
    t0 = time.perf_counter()
    for b in idx:
        mt = oracle_match(plans, *scan.pattern(b))
        if W.get("refine"):
            oracle_refine(plans[0], mt, *scan.pattern(b))
        z, k, m = (int(gpu_res["za_idx"][b]), int(gpu_res["phi3_bin"][b]),
                   int(gpu_res["mirror"][b]))
        val = (mt.Cm if m else mt.C)[z, k]
        agree += int((z, k, m) == (mt.za, mt.k, mt.mirror) or val >= mt.score * (1 - 1e-5))
    t_match = (time.perf_counter() - t0) / n_sample
    del plans
    B = scan.n_patterns
    single = {"value": B / (t_plan + B * t_match), "unit": "patterns/s", "cores": 1,
              "sample": (f"full {W['Z']}-axis plan build timed once ({t_plan:.1f} s) + "
                         f"{n_sample} sampled patterns matched ({t_match * 1e3:.0f} ms each), "
                         f"extrapolated to {B} patterns")}
    pool, cores, t_setup = oracle_pool(host_cores())
    try:
        idx2 = rng.choice(scan.n_patterns, 4 * cores, replace=False)
        tasks = [(scan.pattern(b), (int(gpu_res["za_idx"][b]), int(gpu_res["phi3_bin"][b]),
                                    int(gpu_res["mirror"][b]))) for b in idx2]
        t0 = time.perf_counter()
        got = pool.map(_pool_match, tasks, chunksize=1)
        t_all = (time.perf_counter() - t0) / len(idx2)
    finally:
        pool.close()
        pool.join()
    agree += sum(int(g[4]) for g in got)
    value = B / (t_setup + B * t_all)
    return {"value": value, "unit": "patterns/s", "cores": cores, "kind": "oracle",
            "sample": (f"FP64 NumPy oracle, {cores} worker processes (one per host core): "
                       f"set-up with every worker building the {W['Z']}-axis plans at once "
                       f"({t_setup:.1f} s) + {len(idx2)} sampled patterns matched across the "
                       f"pool ({t_all * 1e3:.1f} ms wall per pattern), extrapolated to {B} "
                       f"patterns"),
            "single_core": single}, f"{agree}/{n_sample + len(idx2)}"


def workload_config(scan):
    """The workload keys of the JSON line's config, shared by both arms."""
    return {"workload": W["text"], "patterns_per_gpu": scan.n_patterns,
            "peaks_nnz": int(scan.row_ptr[-1]), "zone_axes": W["Z"], "shells": W["S"],
            "n_phi": W["N"], "step": "plan build + match of every pattern"}


def rank_seed(rank):
    """Scan seed of ``rank`` under weak scaling: every rank its own scan."""
    return W["seed"] + rank


def reference_arm(args):
    """--impl reference: the oracle timed on the host cores (rank 0 only).
    Set-up (untimed): a pool of one oracle worker per core with the
    workload's plans built.  Each step runs a bounded sample of the workload:
    the plan build on every 16th zone axis (one core) and 2 patterns per
    worker matched across the pool; ms_per_step is the time of that sample,
    and value the sample's rates extrapolated to the whole step (the full
    plan build and every pattern of the scan)."""
    from paper_2111_00171_gb300.ranks import rank_env
    if rank_env()[1] != 0:
        return
    scan = make_scan(W["seed"], args)
    pool, cores, _ = oracle_pool(host_cores(), getattr(args, "oracle_stride", 1))
    Z = W["Z"]
    rng = np.random.default_rng(1)
    vals = []
    tot = 0.0
    try:
        for it in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            nsub = sum(len(p.za) for p in oracle_plans(16))
            t_sub = time.perf_counter() - t0
            bs = rng.choice(scan.n_patterns, 2 * cores, replace=False)
            t1 = time.perf_counter()
            pool.map(_pool_match, [(scan.pattern(b), None) for b in bs], chunksize=1)
            t_p = (time.perf_counter() - t1) / len(bs)
            if it >= args.warmup:
                B = scan.n_patterns
                vals.append(B / (t_sub * Z / nsub + B * t_p))
                tot += time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    v = float(np.mean(vals))
    sample = (f"FP64 NumPy oracle on {cores} host cores; each step: plan build on every 16th "
              f"of {Z} zone axes (one core) + {2 * cores} patterns matched across {cores} "
              f"worker processes; value extrapolates those rates to the full plan build and "
              f"all {scan.n_patterns} patterns; ms_per_step is the sample's own time")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "patterns/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(scan),
            "cpu_baseline": {"value": v, "unit": "patterns/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "patterns/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------- GPU arm

def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    import torch.distributed as dist

    import synth
    from paper_2111_00171_gb300 import acom
    from paper_2111_00171_gb300.ranks import barrier, max_over_ranks, rank_env

    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib = acom.load_library()
    prec = {"bf16": acom.ACOM_PREC_BF16, "fp16": acom.ACOM_PREC_FP16,
            "fp32": acom.ACOM_PREC_FP32}[args.precision]

    scan = make_scan(rank_seed(rank), args)
    B = scan.n_patterns
    mixed = len(W["phases"]) > 1
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_in = (dev(scan.row_ptr), dev(scan.qx), dev(scan.qy), dev(scan.I))
    h_in = tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                 for a in (scan.row_ptr, scan.qx, scan.qy, scan.I))
    h2d = sum(t.numel() * t.element_size() for t in h_in)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def make_plan():
        parts = []
        for phase, step_deg in W["phases"]:
            v, om = acom.cubic_triangle() if phase == "Au" else acom.hexagonal_triangle()
            cr = acom.au_crystal() if phase == "Au" else acom.mg_crystal()
            parts.append(acom.Plan(cr, v, om, step_deg, W["S"], W["dq"], W["N"],
                                   delta=W["delta"], lam=W["lam"], q_max=W["q_max"],
                                   precision=prec))
        if len(parts) == 1:
            return parts[0]
        p = acom.Plan.concat(parts)
        for q in parts:
            q.close()
        return p

    out_keys = ("za_idx", "phi3_bin", "mirror", "score", "score_cos", "phi3", "orient") + \
        (("phase", "phase_score") if mixed else ())

    stats = {}

    def step(inputs, out):
        p = make_plan()
        stats["k0"] = p.info["k0"]
        p.match(*inputs, chunk=args.chunk, out=out, exhaustive=args.exhaustive,
                phase_scores=mixed, tile_order=tuned["tile_order"] if tuned else 0,
                cta_pairs=tuned["cta_pairs"] if tuned else 0)
        stats["evaluated"] = p.get_info()["last_evaluated"]
        if W.get("refine"):
            p.refine(*inputs, out["orient"], orient_alt=out["runner_orient"])
            stats["refine_pairs"] = p.get_info()["last_refine_pairs"]
        p.close()
        return out

    probe = make_plan()
    out = probe.alloc_result(B, phase_scores=mixed, runner=bool(W.get("refine")))
    # the contraction's schedule (chunk, tile order) by acom_autotune on this
    # scan, unless --chunk fixes it or the FP32 / exhaustive paths run
    tuned = None
    if args.chunk == 0 and not args.exhaustive and args.precision != "fp32":
        tuned, trials = probe.autotune(*d_in)
        args.chunk = tuned["chunk"]
    probe.close()
    for _ in range(args.warmup):
        step(d_in, out)
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs
    lib.acom_profile_reset()
    lib.acom_profile_enable(1)
    launches0 = lib.acom_kernel_launches()
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier()
    torch.cuda.synchronize()
    ev = []
    w0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()                                      # L2 flush, outside the events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(d_in, out)
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    barrier()
    ck = clocks.stop() if clocks else None
    launches = lib.acom_kernel_launches() - launches0
    lib.acom_profile_enable(0)
    prof = read_profile(lib, acom)
    dev_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev))

    # ---- e2e: host buffers through the public API, copies inside the region
    d_buf = tuple(torch.empty_like(t, device="cuda") for t in h_in)
    h_out = {k: torch.empty(out[k].shape, dtype=out[k].dtype).pin_memory() for k in out_keys}
    d2h = sum(t.numel() * t.element_size() for t in h_out.values())
    barrier()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d, h in zip(d_buf, h_in):
            d.copy_(h, non_blocking=True)
        step(d_buf, out)
        for k in out_keys:
            h_out[k].copy_(out[k], non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms = max_over_ranks(e2e_ms)
    barrier()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    res = {k: out[k].cpu().numpy() for k in out_keys}
    grid_path = grid_fp32_path(args, acom, scan, d_in, flush, stream) if W.get("refine") else None
    sweep = sweep_combos(args, acom, lib, scan, d_in, flush, stream) if W.get("sweep") else None
    if mixed:
        ph = res["phase"]
        ok = ph == scan.phase
        accuracy = {"phase_decision_correct": float(ok.mean())}
        for p, (name, _) in enumerate(W["phases"]):
            sel = ok & (scan.phase == p)
            if not sel.any():
                continue
            m, mt, t = misorientation(res["orient"][sel], scan.truth[sel],
                                      cubic_ops() if name == "Au" else hexagonal_ops())
            accuracy[name] = {"mean_misorientation_deg": m, "mean_misorientation_friedel_deg": mt,
                              "mean_za_tilt_deg": t, "patterns": int(sel.sum())}
    else:
        spread = {}
        mis, mis_twin, tilt = misorientation(res["orient"], scan.truth, spread=spread)
        accuracy = {"mean_misorientation_deg": mis, "mean_misorientation_friedel_deg": mis_twin,
                    "mean_za_tilt_deg": tilt, **spread}
    peaks, src = peaks_file()
    K = args.steps
    value = world * B * K / (dev_ms / 1e3)
    roof = roofline(prof, peaks, src, B, K, args.precision, int(scan.row_ptr[-1]),
                    stats.get("refine_pairs", 0),
                    None if args.exhaustive else pattern_shell_rows(scan), stats.get("k0", 0))
    line = {"metric": METRIC, "value": value, "unit": "patterns/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": dev_ms / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp16": "f16", "bf16": "bf16"}[args.precision],
            "data": "synthetic",
            "config": {**workload_config(scan), "precision": args.precision,
                       "chunk": args.chunk or (1024 if args.exhaustive else 8192),
                       "autotuned": ({"chunk": tuned["chunk"], "tile_order": tuned["tile_order"],
                                      "cta_pairs": tuned["cta_pairs"],
                                      "trials_ms": {f"{t['chunk']}/{t['tile_order']}/{t['cta_pairs']}":
                                                    round(t["ms"], 2) for t in trials}}
                                     if tuned else None),
                       "mode": "exhaustive" if args.exhaustive else "certified pruning",
                       "axes_evaluated_per_pattern": stats.get("evaluated", 0) / B,
                       "l2": "flushed between steps (256 MiB write outside the timed events)",
                       "wall_ms_per_step": wall * 1e3 / K},
            "roofline": roof,
            "e2e": {"value": world * B * K / (e2e_ms / 1e3), "unit": "patterns/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": ck,
            "kernels_ms_per_step": {n: round(ms / K, 3) for n, (c, ms) in prof.items() if c},
            "accuracy": accuracy}
    if grid_path is not None:
        line["grid_fp32_1deg"] = grid_path
    if sweep is not None:
        line["sweep"] = sweep
    if not args.no_cpu_baseline and world == 1:
        cb, agree = cpu_baseline(scan, res, args.cpu_sample)
        line["cpu_baseline"] = cb
        line["accuracy"]["oracle_argmax_agreement"] = agree
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def sweep_combos(args, acom, lib, scan, d_in, flush, stream, n_oracle=1000):
    """Every (plan step, precision) of the sweep: patterns/s of plan build +
    match (CUDA events, L2 flushed; one warm-up and one timed step for the
    combinations beside the line's own), the contraction's fraction of its
    roofline, axes evaluated, misorientation, and the oracle's argmax
    agreement on a subset of n_oracle sampled patterns per plan (matched by
    the oracle on every host core after the GPU runs of that plan).  E4M3
    operands run the uncertified top-8 rescoring (their certified margin is
    about a quarter of the bound)."""
    import torch
    peaks, src = peaks_file()
    v, om = acom.cubic_triangle()
    cr = acom.au_crystal()
    B = scan.n_patterns
    F, S, N = W["N"] // 2 + 1, W["S"], W["N"]
    fp32_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    out_rows = []
    idx = np.random.default_rng(0).choice(B, min(n_oracle, B), replace=False)
    for step_deg, Z in ((1.0, 903), (0.5, 3486)):
        rows, choices = [], []
        for prec in ("fp32", "bf16", "fp16", "fp8"):
            code = {"bf16": acom.ACOM_PREC_BF16, "fp16": acom.ACOM_PREC_FP16,
                    "fp32": acom.ACOM_PREC_FP32, "fp8": acom.ACOM_PREC_FP8}[prec]
            top = 8 if prec == "fp8" else 0

            def plan():
                return acom.Plan(cr, v, om, step_deg, S, W["dq"], N, delta=W["delta"],
                                 lam=W["lam"], q_max=W["q_max"], precision=code)
            probe = plan()
            out = probe.alloc_result(B)
            probe.close()
            info = {}

            def step():
                p = plan()
                p.match(*d_in, out=out, rescore_top=top)
                info["ev"] = p.get_info()["last_evaluated"]
                p.close()
            step()
            torch.cuda.synchronize()
            lib.acom_profile_reset()
            lib.acom_profile_enable(1)
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            lib.acom_profile_enable(0)
            prof = read_profile(lib, acom)
            name = "contract_fp32" if prec == "fp32" else "contract_tc"
            cnt, cms = prof.get(name, (0, 0.0))
            flops = 8.0 * Z * S * F * B
            tflops = flops / (cms / 1e3) / 1e12 if cms else 0.0
            # E4M3's dense rate is twice BF16's (4.5 vs 2.25 PFLOP/s nominal)
            peak = fp32_peak if prec == "fp32" else peaks["bf16_tflops"] * \
                (2.0 if prec == "fp8" else 1.0)
            mis, mis_twin, tilt = misorientation(out["orient"].cpu().numpy(), scan.truth)
            res = {k: out[k].cpu().numpy() for k in ("za_idx", "phi3_bin", "mirror")}
            choices.append([(int(res["za_idx"][b]), int(res["phi3_bin"][b]),
                             int(res["mirror"][b])) for b in idx])
            rows.append({"plan_step_deg": step_deg, "zone_axes": Z, "precision": prec,
                             "mode": "top-8 rescoring, not certified" if top
                                     else "certified pruning",
                             "patterns_per_s": B / (ms / 1e3), "ms_per_step": ms,
                             "contraction_tflops": tflops, "contraction_frac": tflops / peak,
                             "contraction_bound": "alu" if prec == "fp32" else "tensor",
                             "axes_evaluated_per_pattern": info["ev"] / B,
                             "mean_misorientation_deg": mis,
                             "mean_misorientation_friedel_deg": mis_twin})
        for row, agree in zip(rows, oracle_subset_agreement(scan, idx, step_deg, Z, choices)):
            row["oracle_argmax_agreement"] = agree
        out_rows += rows
    return out_rows


def oracle_subset_agreement(scan, idx, step_deg, Z, choices, cores=None):
    """The oracle's argmax on patterns ``idx`` against the fcc Au plan of
    this step, matched on every host core, compared with each GPU run's
    choices (``choices[r][i]`` for pattern ``idx[i]``; ties within 1e-5 of the
    oracle's best count as agreement): one "agreed/total" per run."""
    w = dict(W, phases=(("Au", step_deg),), Z=Z, step=step_deg)
    pool, _, _ = oracle_pool(cores or host_cores(), w=w)
    try:
        tasks = [(scan.pattern(int(b)), [c[i] for c in choices]) for i, b in enumerate(idx)]
        got = pool.map(_pool_match, tasks, chunksize=4)
    finally:
        pool.close()
        pool.join()
    return [f"{sum(int(g[4][r]) for g in got)}/{len(idx)}" for r in range(len(choices))]


def grid_fp32_path(args, acom, scan, d_in, flush, stream):
    """The plain FP32 path on the 1-degree grid (plan build + match with the
    FP32 contraction and grid refinement) on the same scan: its patterns/s
    (CUDA events, same L2 flush) and misorientation."""
    import torch
    v, om = acom.cubic_triangle()
    cr = acom.au_crystal()

    def plan():
        return acom.Plan(cr, v, om, 1.0, W["S"], W["dq"], W["N"], delta=W["delta"],
                         lam=W["lam"], q_max=W["q_max"], precision=acom.ACOM_PREC_FP32)
    B = scan.n_patterns
    probe = plan()
    out = probe.alloc_result(B)
    probe.close()

    def step():
        p = plan()
        p.match(*d_in, out=out)
        p.close()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    mis, mis_twin, tilt = misorientation(out["orient"].cpu().numpy(), scan.truth)
    return {"value": B * args.steps / (ms / 1e3), "unit": "patterns/s",
            "ms_per_step": ms / args.steps, "zone_axes": 903, "precision": "fp32",
            "accuracy": {"mean_misorientation_deg": mis, "mean_misorientation_friedel_deg": mis_twin,
                         "mean_za_tilt_deg": tilt}}


def read_profile(lib, acom):
    import ctypes as C

    class Entry(C.Structure):
        _fields_ = [("name", C.c_char_p), ("launches", C.c_int64), ("total_ms", C.c_double)]
    lib.acom_profile_read.restype = C.c_int32
    lib.acom_profile_read.argtypes = [C.POINTER(Entry), C.c_int32]
    n = lib.acom_profile_read(None, 0)
    arr = (Entry * n)()
    lib.acom_profile_read(arr, n)
    return {e.name.decode(): (e.launches, e.total_ms) for e in arr}


# DRAM bytes (read + write) of one launch of the captured size (the second
# field, in patterns), from a single-pass ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the full-size run, with a hash of the kernel's
# sources at capture time, the precision and the workload of the captured
# run: a changed kernel, or another precision or workload, reports no
# traffic.  The last field says whether the traffic grows in proportion to
# the patterns of a launch (then another chunk size is scaled); the
# contraction's does not (the plan is re-read once per tile wave).
TRAFFIC_PER_LAUNCH = {
    "select_exact": (5.341e9 + 20.85e6, 32768, ("match_prune.cu",), "5542e2567c0d4a2d", "fp16",
                     "au_scan_256x256_1deg", True),
    "raster_patterns": (21.56e6 + 8.031e9, 32768, ("raster.cu",), "65f790beeba11713", "fp16",
                        "au_scan_256x256_1deg", True),
    "contract_tc": (7.005e9 + 115.2e6, 32768, ("match_tc.cu",), "98bbb62117c87ae7", "fp16",
                    "au_scan_256x256_1deg", False),
}


def sources_hash(files):
    import hashlib
    d = os.path.join(ROOT, "paper_2111_00171_gb300", "csrc")
    m = hashlib.sha256()
    for f in tuple(files) + ("acom_internal.cuh", "fft_warp.cuh"):
        with open(os.path.join(d, f), "rb") as fh:
            m.update(fh.read())
    return m.hexdigest()[:16]


def kernel_traffic(name, pats, precision):
    """DRAM bytes of one launch of ``pats`` patterns: the captured launch's,
    scaled to ``pats`` where traffic grows in proportion, else None."""
    t = TRAFFIC_PER_LAUNCH.get(name)
    if t is None or sources_hash(t[2]) != t[3] or precision != t[4] or W["name"] != t[5]:
        return None
    if abs(pats - t[1]) < 0.5:
        return t[0]
    return t[0] * pats / t[1] if t[6] else None


def kernel_roofline(name, cnt, ms, peaks, src, B, K, nnz, precision, refine_pairs=0,
                    rows_nz=None, k0=0):
    """Achieved rate of one kernel class: algorithmic work per launch over its
    event-timed average launch duration."""
    Z, S, N = W["Z"], W["S"], W["N"]
    F = N // 2 + 1
    avg_s = ms / cnt / 1e3 if cnt else float("nan")
    pats = B * K / cnt if cnt else 0          # patterns per launch
    fp32_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    if name == "contract_tc":
        # the kernel runs for a few ms at a time within a short step, at the
        # maximum SM clock (clocks sampled beside): the burst peak applies
        work, unit, bound, peak = 8.0 * Z * S * F * pats, "TFLOP/s", "tensor", \
            peaks["bf16_tflops"]
        note = (f"8 Z S F flops per pattern; bf16 burst peak, which FP16 operands "
                f"share ({src})")
        if k0:
            note += (f"; the kernel skips shells 0..{k0 - 1}, where every plan row is zero "
                     f"(it executes {W['S'] - k0} of the {W['S']} shells counted)")
    elif name == "contract_fp32":
        work, unit, bound, peak = 8.0 * Z * S * F * pats, "TFLOP/s", "alu", fp32_peak
        note = "8 Z S F flops per pattern; FP32 FMA peak 152 SMs x 128 lanes x 2 x max clock"
    elif name == "select_exact":
        # compulsory HBM bytes: each pattern's FP32 shell-major spectra on
        # the shells its peaks reach (rows_nz of S, re/im) read once, and the
        # plan's FP32 spectra once per launch; the repeated reads of an axis'
        # spectra are served by L2
        rows = S if rows_nz is None else rows_nz
        work = (rows * F * 8 * pats + Z * S * F * 8) / 1e9
        unit, bound, peak = "GB/s", "hbm", peaks["hbm_gbs"]
        note = (f"pattern FP32 spectra on its non-zero shells ({rows:.1f} of {S} on average) "
                f"once per pattern + plan FP32 spectra once per launch; HBM peak ({src})")
    elif name == "refine_orient" and refine_pairs:
        # every (contributing reflection, peak) pair of every score evaluation:
        # 13 FP32 operations and one exp (counted by the kernel itself)
        work = 13.0 * refine_pairs * (K / cnt)
        unit, bound, peak = "TFLOP/s", "alu", fp32_peak
        note = ("13 flop per (reflection, peak) pair summed (the kernel counts the pairs); "
                "FP32 FMA peak 152 SMs x 128 lanes x 2 x max clock")
    elif name == "raster_patterns":
        # algorithmic bytes: CSR in (8 B row pointer + 12 B per peak) and the
        # spectra out: the contraction's operand (re/im, F frequencies: 16-bit
        # on the shells from the plan's first non-zero shell k0 on, which are
        # all the tensor-core contraction reads; FP32 frequency-major on all S
        # shells for the FP32 contraction) and the FP32 shell-major rows
        # select reads, those of the shells the pattern's peaks reach (rows_nz
        # of S; the raster writes no other row)
        rows = S if rows_nz is None else rows_nz
        op_shells = S if precision == "fp32" else S - k0
        out_b = op_shells * F * 2 * (4 if precision == "fp32" else 2) + rows * F * 8
        work = (nnz / B * 12 + 8 + out_b) * pats / 1e9
        unit, bound, peak = "GB/s", "hbm", peaks["hbm_gbs"]
        note = (f"CSR in + contraction operand on {op_shells} shells out + FP32 shell-major "
                f"spectra on the {rows:.1f} of {S} shells the peaks reach per pattern; "
                f"HBM peak ({src})")
    else:
        return None
    ach = work / avg_s / (1e12 if unit == "TFLOP/s" else 1.0)
    return {"kernel": name, "bound": bound, "achieved": ach, "peak": peak, "unit": unit,
            "frac": ach / peak, "traffic": kernel_traffic(name, pats, precision),
            "avg_launch_ms": avg_s * 1e3,
            "launches": cnt, "peak_source": note}


def roofline(prof, peaks, src, B, K, precision, nnz, refine_pairs=0, rows_nz=None, k0=0):
    """The dominant kernel's roofline (the largest event-timed total among
    the kernels with a stated roofline), plus every other kernel's share."""
    rows = []
    for name, (cnt, ms) in prof.items():
        if cnt == 0:
            continue
        r = kernel_roofline(name, cnt, ms, peaks, src, B, K, nnz, precision, refine_pairs,
                            rows_nz, k0)
        if r is not None:
            r["total_ms"] = ms
            rows.append(r)
    top = max(rows, key=lambda r: r["total_ms"])
    top = dict(top)
    top["others"] = {r["kernel"]: {"frac": r["frac"], "bound": r["bound"]}
                     for r in rows if r["kernel"] != top["kernel"]}
    return top


if __name__ == "__main__":
    main()
