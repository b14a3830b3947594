"""The FP64 oracle fanned out over host processes, for parity tests that
compare hundreds to thousands of patterns.

The pool uses the spawn start method (the test process has already
initialised CUDA; a forked child of it can hang).  Each worker builds the
oracle's plan once and then matches the patterns it is sent; the spectra are
all a match needs, so the worker drops the real plan P to halve its memory.
"""

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

_PLAN = None


def _init(name, phase):
    global _PLAN
    from gpu_common import oracle_plan
    plan = oracle_plan(name, phase)
    plan.P = None
    _PLAN = plan


def _match(batch):
    from oracle import acom_oracle as O
    out = []
    for b, qx, qy, I, (z, k, m) in batch:
        mt = O.match_pattern(_PLAN, qx, qy, I)
        val = float((mt.Cm if m else mt.C)[z, k])
        out.append((int(b), int(mt.za), int(mt.k), int(mt.mirror), float(mt.score), val))
    return out


def oracle_matches(name, scan, idx, choices, workers=16, phase="Au", per_task=8):
    """The oracle's (za, k, mirror, score) of patterns ``idx`` of ``scan``
    against the oracle plan ``name``, and the oracle's correlation at the
    GPU's choice (za, k, mirror) of each: {b: (za, k, mirror, score, value)}."""
    n = max(1, min(workers, os.cpu_count() or 1, len(idx)))
    tasks = []
    for i in range(0, len(idx), per_task):
        tasks.append([(b, *scan.pattern(b), tuple(int(v) for v in choices[j]))
                      for j, b in enumerate(idx[i:i + per_task], start=i)])
    res = {}
    with ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"),
                             initializer=_init, initargs=(name, phase)) as ex:
        for part in ex.map(_match, tasks):
            for b, za, k, m, score, val in part:
                res[b] = (za, k, m, score, val)
    return res
