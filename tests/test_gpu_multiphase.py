"""Several phases in one plan (acom_plan_concat) through the C ABI, against
the oracle's one-match-per-phase (match_multi) on seeded mixed Au / Mg
patterns.

Tolerances as for one phase: every phase's best score within 1e-4 relative
of the oracle's; the winning (zone axis, phi3 bin, mirror) the oracle's up to
documented ties (within 1e-5 relative of the best); the phase decision the
oracle's unless the two phases' best scores tie within 1e-5.
"""

import math

import numpy as np
import pytest

import synth
from oracle import acom_oracle as O

from gpu_common import CONFIGS, check_argmax, gpu_plan, oracle_plan, to_dev

pytestmark = pytest.mark.gpu

CONFIGS.setdefault("mg_2deg_75x180", (2.0, 75, 0.02, 180))
CONFIGS.setdefault("mg_1deg_75x180", (1.0, 75, 0.02, 180))     # 1770 axes


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _concat(names, precision=0):
    from paper_2111_00171_gb300 import acom
    parts = [gpu_plan(n, phase=ph, precision=precision) for n, ph in names]
    return parts, acom.Plan.concat(parts)


@pytest.fixture(scope="module")
def two_phase():
    parts, cat = _concat([("au_2deg_75x180", "Au"), ("mg_2deg_75x180", "Mg")])
    yield parts, cat
    cat.close()
    for p in parts:
        p.close()


def _oracles(mg="mg_2deg_75x180"):
    return [oracle_plan("au_2deg_75x180"), oracle_plan(mg, phase="Mg")]


def _global(mm):
    """The best over the concatenated axes (ties: lowest global index)."""
    C = np.concatenate([m.C for m in mm.matches])
    Cm = np.concatenate([m.Cm for m in mm.matches])
    return O.best_match(C, Cm)


def test_concat_layout(two_phase):
    import torch
    (au, mg), cat = two_phase
    za, zm = au.info["n_za"], mg.info["n_za"]
    assert cat.info["n_phases"] == 2 and cat.info["n_za"] == za + zm
    np.testing.assert_array_equal(cat.phases(), [0, za, za + zm])
    np.testing.assert_array_equal(cat.zone_axes(), np.vstack([au.zone_axes(), mg.zone_axes()]))
    sp = cat.spectra()
    assert torch.equal(sp[:za], au.spectra()) and torch.equal(sp[za:], mg.spectra())
    scan = synth.mixed_patterns(1004, n_patterns=40)
    u = cat.bounds(*to_dev(scan)).cpu().numpy()
    ua = au.bounds(*to_dev(scan)).cpu().numpy()
    um = mg.bounds(*to_dev(scan)).cpu().numpy()
    np.testing.assert_allclose(u, np.hstack([ua, um]), rtol=1e-6, atol=1e-7 * np.abs(u).max())


def _compare(r, scan, oplans, n_check=None):
    za = r["za_idx"].cpu().numpy()
    kk = r["phi3_bin"].cpu().numpy()
    mi = r["mirror"].cpu().numpy()
    sc = r["score"].cpu().numpy()
    ph = r["phase"].cpu().numpy()
    ps = r["phase_score"].cpu().numpy()
    z0 = len(oplans[0].za)
    rows = range(scan.n_patterns) if n_check is None else n_check
    agree = 0
    for b in rows:
        mm = O.match_multi(oplans, *scan.pattern(b))
        np.testing.assert_allclose(ps[b], mm.phase_scores, rtol=1e-4, err_msg=str(b))
        g = _global(mm)
        assert check_argmax(g, za[b], kk[b], mi[b]), (b, (za[b], kk[b], mi[b]), (g.za, g.k, g.mirror))
        assert ph[b] == (1 if za[b] >= z0 else 0)
        if ph[b] != mm.phase:           # a tie between the phases' bests
            assert abs(mm.phase_scores[0] - mm.phase_scores[1]) <= 1e-5 * mm.phase_scores.max(), b
        assert math.isclose(sc[b], mm.match.score, rel_tol=1e-4), b
        agree += int(ph[b] == scan.phase[b])
    return agree


@pytest.mark.parametrize("chunk", [0, 48])
@pytest.mark.parametrize("exhaustive", [True, False], ids=["exhaustive", "pruned"])
def test_multi_phase_match_matches_oracle(two_phase, exhaustive, chunk):
    """100 mixed patterns (chunk 48: two full chunks and a ragged tail):
    per-phase best scores, winner and phase decision against the oracle."""
    _, cat = two_phase
    scan = synth.mixed_patterns(1003, n_patterns=100)
    r = cat.match(*to_dev(scan), phase_scores=True, exhaustive=exhaustive, chunk=chunk)
    agree = _compare(r, scan, _oracles())
    print(f"phase decision equals the generating phase for {agree}/100 patterns")
    assert agree >= 90


def test_per_phase_certification_only_when_asked(two_phase):
    """Without per-phase scores the search certifies the overall winner only:
    the same winners (up to ties) and scores, no more evaluations.  An axis
    scored in batches of different sizes is summed over shells in a different
    split, so scores agree to FP32 rounding, not bit for bit."""
    import torch
    _, cat = two_phase
    scan = synth.mixed_patterns(1005, n_patterns=200)
    a = cat.match(*to_dev(scan), phase_scores=True)
    torch.cuda.synchronize()
    ev_a = cat.get_info()["last_evaluated"]
    b = cat.match(*to_dev(scan))
    torch.cuda.synchronize()
    ev_b = cat.get_info()["last_evaluated"]
    np.testing.assert_allclose(a["score"].cpu().numpy(), b["score"].cpu().numpy(), rtol=2e-6)
    ka = np.stack([a[k].cpu().numpy().astype(np.int64) for k in ("za_idx", "phi3_bin", "mirror")], 1)
    kb = np.stack([b[k].cpu().numpy().astype(np.int64) for k in ("za_idx", "phi3_bin", "mirror")], 1)
    op = _oracles()
    for i in np.nonzero(np.any(ka != kb, axis=1))[0]:
        g = _global(O.match_multi(op, *scan.pattern(i)))
        assert check_argmax(g, *ka[i]) and check_argmax(g, *kb[i]), i
    print(f"axes evaluated: {ev_a / 200:.2f} per pattern with per-phase scores, "
          f"{ev_b / 200:.2f} without")
    assert ev_b <= ev_a


@pytest.mark.parametrize("precision", [2], ids=["fp16"])
def test_mixed_full_size(precision):
    """The mixed workload at full size: fcc Au on the 2-degree grid plus hcp
    Mg on the 1-degree grid (231 + 1770 axes, 75 shells, 180 bins) in one
    plan, 65,536 patterns drawn 50/50.  Certified FP16 pruning returns the
    FP32 path's winners and per-phase scores; sampled patterns are checked
    against the oracle one by one."""
    import time

    import torch
    (p32s, cat32) = _concat([("au_2deg_75x180", "Au"), ("mg_1deg_75x180", "Mg")])
    (p16s, cat16) = _concat([("au_2deg_75x180", "Au"), ("mg_1deg_75x180", "Mg")], precision)
    assert cat16.info["n_za"] == 231 + 1770
    scan = synth.mixed_patterns(1003, n_patterns=65536)
    inp = to_dev(scan)
    a = cat32.match(*inp, phase_scores=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = cat16.match(*inp, phase_scores=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ev = cat16.get_info()["last_evaluated"] / scan.n_patterns
    ka = np.stack([a[k].cpu().numpy().astype(np.int64) for k in ("za_idx", "phi3_bin", "mirror")], 1)
    kb = np.stack([b[k].cpu().numpy().astype(np.int64) for k in ("za_idx", "phi3_bin", "mirror")], 1)
    np.testing.assert_allclose(b["phase_score"].cpu().numpy(), a["phase_score"].cpu().numpy(),
                               rtol=1e-5)
    np.testing.assert_allclose(b["score"].cpu().numpy(), a["score"].cpu().numpy(), rtol=1e-5)
    diff = np.nonzero(np.any(ka != kb, axis=1))[0]
    assert len(diff) <= 0.001 * len(ka), len(diff)
    op = _oracles("mg_1deg_75x180")
    for i in diff:          # every difference must be a documented tie in the oracle
        g = _global(O.match_multi(op, *scan.pattern(i)))
        assert check_argmax(g, *ka[i]) and check_argmax(g, *kb[i]), i
    rng = np.random.default_rng(3)
    sample = rng.choice(scan.n_patterns, 8, replace=False)
    _compare(b, scan, op, n_check=sample)
    ph = b["phase"].cpu().numpy()
    acc = float(np.mean(ph == scan.phase))
    print(f"mixed 65536: {scan.n_patterns / dt:.0f} patterns/s (match call incl. sync), "
          f"{ev:.2f} axes evaluated per pattern, phase decision = generating phase for "
          f"{100 * acc:.2f} %")
    assert acc > 0.9
    for p in (cat32, cat16, *p32s, *p16s):
        p.close()
