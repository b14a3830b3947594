"""Shared set-up of the GPU parity tests: the same seeded inputs for the
library and for the FP64 oracle, and the comparison rules."""

import functools
import math

import numpy as np

import synth
from oracle import acom_oracle as O

LAM = 0.01969
DELTA = 0.08
AU_POS = [[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]]

# workloads: name -> (step_deg, n_shells, dq, n_phi)
CONFIGS = {
    "au_2deg_75x180": (2.0, 75, 0.02, 180),      # 100 random patterns, 231 zone axes
    "au_1deg_150x360": (1.0, 150, 0.01, 360),    # 256x256 Voronoi scan, 903 zone axes
    "au_6deg_40x72": (6.0, 40, 0.0375, 72),      # tiny case for quick checks
    "au_halfdeg_150x360": (0.5, 150, 0.01, 360),  # 512x512 sweep scan, 3486 zone axes
    "au_6deg_200x72": (6.0, 200, 0.0075, 72),     # contraction K range over two ring stages
}


def au_refl():
    return O.reflections(np.eye(3) * 4.08, AU_POS, [79.0] * 4, [0.25] * 4, 1.5)


def mg_refl():
    s = synth.mg_hcp()
    return O.reflections(s.lattice, s.frac_pos, [12.0] * 2, [0.3] * 2, 1.5)


@functools.lru_cache(maxsize=None)
def oracle_plan(name, phase="Au"):
    step, S, dq, N = CONFIGS[name]
    if phase == "Au":
        v0, v1, v2, om = O.cubic_triangle()
        refl = au_refl()
    else:
        v0, v1, v2, om = O.hexagonal_triangle()
        refl = mg_refl()
    za = O.zone_axis_grid(v0, v1, v2, step, om)
    return O.orientation_plan(refl, za, O.PlanParams(S, dq, N, DELTA, lam=LAM))


def gpu_plan(name, phase="Au", precision=0):
    from paper_2111_00171_gb300 import acom
    step, S, dq, N = CONFIGS[name]
    if phase == "Au":
        v, om = acom.cubic_triangle()
        cr = acom.au_crystal()
    else:
        v, om = acom.hexagonal_triangle()
        cr = acom.mg_crystal()
    return acom.Plan(cr, v, om, step, S, dq, N, delta=DELTA, lam=LAM, q_max=1.5,
                     precision=precision)


def to_dev(scan):
    import torch
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return d(scan.row_ptr), d(scan.qx), d(scan.qy), d(scan.I)


def check_argmax(mt, za, k, mir, tie_rel=1e-5):
    """The GPU's (zone axis, bin, mirror) is the oracle's, or an oracle
    value within tie_rel of the oracle's best (a documented tie)."""
    if (za, k, mir) == (mt.za, mt.k, mt.mirror):
        return True
    val = (mt.Cm if mir else mt.C)[za, k]
    return val >= mt.score - tie_rel * abs(mt.score)


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(1e-30, np.max(np.abs(b))))
