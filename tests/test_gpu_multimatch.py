"""Several matches per pattern (acom_match_multi) through the C ABI against
the oracle's match_multiple: each round's (zone axis, phi3 bin, mirror) the
oracle's up to documented ties, each score the full pattern's correlation at
that match within 1e-4, and "no further orientation" where the oracle
stops."""

import math

import numpy as np
import pytest

import synth
from oracle import acom_oracle as O

from gpu_common import LAM, au_refl, check_argmax, gpu_plan, oracle_plan, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _overlapping_scan(op, n, seed):
    """n patterns, each the peaks of two noiseless patterns at grid
    orientations superimposed."""
    refl = au_refl()
    rng = np.random.default_rng(seed)
    N = op.params.n_phi
    rows = []
    for _ in range(n):
        zs = rng.choice(len(op.za), 2, replace=False)
        pats = [O.kinematical_pattern(refl, O.orientation_matrix(
            op.za[z], -2 * math.pi * int(rng.integers(N)) / N, int(rng.integers(2))), LAM, 0.02,
            1e-3) for z in zs]
        rows.append(tuple(np.concatenate([p[i] for p in pats]) for i in range(3)))
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r[0]) for r in rows])
    cat = lambda i: np.concatenate([r[i] for r in rows]).astype(np.float32)
    return synth.Scan(rp, cat(0), cat(1), cat(2), np.tile(np.eye(3), (n, 1, 1)),
                      np.zeros(n, np.int32), (synth.au_fcc(),), "overlapping grid patterns")


def _compare(res, scan, op, n_matches, r_del):
    """Round by round against the oracle.  A round resolved differently at a
    documented tie deletes different peaks, so the pattern's later rounds are
    not compared."""
    refl = au_refl()
    got = [{k: r[k].cpu().numpy() for k in ("za_idx", "phi3_bin", "mirror", "score")} for r in res]
    ties = 0
    for b in range(scan.n_patterns):
        qx, qy, I = (a.astype(np.float64) for a in scan.pattern(b))
        ref = O.match_multiple(op, refl, qx, qy, I, n_matches, r_del, LAM, 0.02)
        C, Cm = O.correlogram(op.P_hat, O.polar_image(qx, qy, I, op.params))
        for j in range(n_matches):
            za = int(got[j]["za_idx"][b])
            if j >= len(ref):
                assert za == -1, (b, j)
                continue
            mt = ref[j]
            k, mir = int(got[j]["phi3_bin"][b]), int(got[j]["mirror"][b])
            assert check_argmax(mt.match, za, k, mir), (b, j, za, mt.za)
            full = (Cm if mir else C)[za, k]            # the full pattern at the GPU's match
            assert got[j]["score"][b] == pytest.approx(full, rel=1e-4, abs=1e-6 * abs(full)), (b, j)
            if (za, k, mir) != (mt.za, mt.k, mt.mirror):
                ties += 1
                break
    return ties


@pytest.mark.parametrize("exhaustive", [False, True], ids=["pruned", "exhaustive"])
def test_overlapping_patterns_match_oracle(exhaustive):
    plan = gpu_plan("au_2deg_75x180")
    op = oracle_plan("au_2deg_75x180")
    scan = _overlapping_scan(op, 24, 51)
    res = plan.match_multi(*to_dev(scan), n_matches=2, r_del=0.04, exhaustive=exhaustive)
    _compare(res, scan, op, 2, 0.04)
    plan.close()


def test_random_patterns_three_rounds_match_oracle():
    plan = gpu_plan("au_2deg_75x180")
    op = oracle_plan("au_2deg_75x180")
    scan = synth.random_patterns(1201, n_patterns=40)
    res = plan.match_multi(*to_dev(scan), n_matches=3, r_del=0.04)
    _compare(res, scan, op, 3, 0.04)
    # the peaks are not changed: a plain match afterwards equals the first match
    import torch
    r = plan.match(*to_dev(scan))
    torch.cuda.synchronize()
    assert torch.equal(r["za_idx"], res[0]["za_idx"])
    plan.close()
