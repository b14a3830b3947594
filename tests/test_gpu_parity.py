"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs.

Tolerances: plan and pattern spectra within 1e-5 of their largest magnitude
(FP32 tent and transform against FP64); correlation scores within 1e-4
relative; the argmax (zone axis, phi3 bin, mirror) exact except documented
ties, where the oracle's own value at the GPU's choice is within 1e-5
relative of its maximum.
"""

import math

import numpy as np
import pytest

import synth
from oracle import acom_oracle as O

from gpu_common import (CONFIGS, check_argmax, gpu_plan, oracle_plan, rel_err, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def c1():
    plan = gpu_plan("au_2deg_75x180")
    yield plan
    plan.close()


def test_zone_axes_match_oracle(c1):
    op = oracle_plan("au_2deg_75x180")
    za = c1.zone_axes()
    assert za.shape == op.za.shape == (231, 3)
    np.testing.assert_allclose(za, op.za, atol=1e-12)
    assert c1.info["n_reflections"] == 258


def test_plan_spectra_match_oracle(c1):
    op = oracle_plan("au_2deg_75x180")
    sp = c1.spectra().cpu().numpy()
    ref = np.stack([op.P_hat.real, op.P_hat.imag], axis=-1)
    assert sp.shape == ref.shape
    assert rel_err(sp, ref) < 1e-5
    # every slice unit-norm (Parseval on the spectrum)
    N = op.params.n_phi
    w = np.full(N // 2 + 1, 2.0)
    w[0] = w[-1] = 1.0
    e = (w * (sp[..., 0] ** 2 + sp[..., 1] ** 2)).sum(axis=(1, 2)) / N
    np.testing.assert_allclose(e, 1.0, rtol=1e-5)


def test_polar_spectra_match_oracle(c1):
    scan = synth.random_patterns(1001, n_patterns=100)
    sp, xn = c1.polar_spectra(*to_dev(scan))
    sp = sp.cpu().numpy()
    xn = xn.cpu().numpy()
    prm = oracle_plan("au_2deg_75x180").params
    for b in range(scan.n_patterns):
        X = O.polar_image(*scan.pattern(b), prm)
        Xh = np.fft.rfft(X, axis=1)
        ref = np.stack([Xh.real, Xh.imag], axis=-1)
        assert rel_err(sp[b], ref) < 1e-5, b
        assert math.isclose(xn[b], np.sqrt((X * X).sum()), rel_tol=1e-5)


def _match_and_compare(plan, oplan, scan, chunk=0, tie_rel=1e-5, check_refine=True,
                       exhaustive=True):
    r = plan.match(*to_dev(scan), za_scores=True, chunk=chunk, exhaustive=exhaustive)
    za = r["za_idx"].cpu().numpy()
    kk = r["phi3_bin"].cpu().numpy()
    mi = r["mirror"].cpu().numpy()
    sc = r["score"].cpu().numpy()
    zs = r["za_scores"].cpu().numpy()
    orient = r["orient"].cpu().numpy()
    nb = O.za_neighbours(oplan.za, plan.step_deg)
    worst = {"za_scores": 0.0, "score": 0.0, "phi3_over_tol": 0.0}
    for b in range(scan.n_patterns):
        mt = O.match_pattern(oplan, *scan.pattern(b))
        worst["score"] = max(worst["score"], abs(sc[b] - mt.score) / abs(mt.score) if mt.score else 0)
        if exhaustive:
            worst["za_scores"] = max(worst["za_scores"], rel_err(zs[b], mt.za_scores))
            assert rel_err(zs[b], mt.za_scores) < 1e-4, b
        else:
            # exact where evaluated, an upper bound elsewhere
            assert np.all(zs[b] >= mt.za_scores - 1e-5 * abs(mt.score)), b
            assert math.isclose(zs[b][za[b]], mt.za_scores[za[b]], rel_tol=1e-4), b
        assert check_argmax(mt, za[b], kk[b], mi[b], tie_rel), (b, (za[b], kk[b], mi[b]),
                                                                 (mt.za, mt.k, mt.mirror))
        assert math.isclose(sc[b], mt.score, rel_tol=1e-4), b
        if check_refine and (za[b], kk[b], mi[b]) == (mt.za, mt.k, mt.mirror):
            rf = O.refine(mt, oplan.za, plan.step_deg, nb)
            # a neighbour within 1e-4 of the 0.9 threshold may flip: allow it
            best = mt.za_scores[mt.za]
            near = [abs(mt.za_scores[z2] / best - 0.9) < 1e-4 for z2 in nb[mt.za]]
            if any(near):
                continue
            # the parabola vertex divides by a second difference: propagate a
            # relative error eps of each correlation value into dk
            N = oplan.params.n_phi
            Cz = (mt.Cm if mt.mirror else mt.C)[mt.za]
            cm, c0, cp = Cz[(mt.k - 1) % N], Cz[mt.k], Cz[(mt.k + 1) % N]
            den = cm - 2 * c0 + cp
            eps = 2e-5 * abs(c0)
            ddk = (2 * eps / (2 * abs(den)) + abs(rf.dk) * 4 * eps / abs(den)) if den < 0 else 0.0
            tol = math.degrees(2 * math.pi / N * min(ddk, 0.5)) + 2e-3
            d_phi = abs(math.degrees(float(r["phi3"][b].cpu()) - rf.phi3))
            d_phi = min(d_phi, 360 - d_phi)
            # small-angle distance ||dM||_F / sqrt(2); acos of the trace is
            # ill-conditioned near the identity for FP32-stored matrices
            ang = math.degrees(np.linalg.norm(rf.m - orient[b].astype(np.float64)) / math.sqrt(2))
            worst["phi3_over_tol"] = max(worst["phi3_over_tol"], d_phi / tol, ang / tol)
            assert d_phi < tol, (b, d_phi, tol, den / c0, rf.dk)
            assert ang < tol, (b, ang, tol, den / c0, rf.dk)
    print("parity worst:", worst)
    return r


@pytest.mark.parametrize("exhaustive", [True, False], ids=["exhaustive", "pruned"])
def test_match_matches_oracle_random_patterns(c1, exhaustive):
    scan = synth.random_patterns(1001, n_patterns=100)
    _match_and_compare(c1, oracle_plan("au_2deg_75x180"), scan, exhaustive=exhaustive)
    if not exhaustive:
        # the bound leaves a few percent of the axes for full evaluation
        assert c1.get_info()["last_evaluated"] < 0.1 * 100 * 231


@pytest.mark.parametrize("exhaustive", [True, False], ids=["exhaustive", "pruned"])
def test_match_ragged_chunks(c1, exhaustive):
    """100 patterns in chunks of 48: two full chunks and a ragged tail."""
    scan = synth.random_patterns(1011, n_patterns=100)
    _match_and_compare(c1, oracle_plan("au_2deg_75x180"), scan, chunk=48, exhaustive=exhaustive)


def test_edge_cases_empty_and_degenerate(c1):
    import torch
    # pattern 0: no peaks; 1: one peak; 2: peaks beyond the last shell;
    # 3: zero intensities; 4: a normal pattern
    base = synth.random_patterns(5, n_patterns=1)
    px, py, pI = base.pattern(0)
    rows = [([], [], []), ([0.49], [0.0], [5.0]), ([2.5, -3.0], [0.1, 0.2], [1.0, 1.0]),
            (list(px), list(py), [0.0] * len(px)), (list(px), list(py), list(pI))]
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r[0]) for r in rows])
    qx = np.concatenate([np.asarray(r[0], np.float32) for r in rows])
    qy = np.concatenate([np.asarray(r[1], np.float32) for r in rows])
    I = np.concatenate([np.asarray(r[2], np.float32) for r in rows])
    scan = synth.Scan(rp, qx, qy, I, np.tile(np.eye(3), (len(rows), 1, 1)),
                      np.zeros(len(rows), np.int32), (synth.au_fcc(),), "edge cases")
    oplan = oracle_plan("au_2deg_75x180")
    r = c1.match(*to_dev(scan), za_scores=True)
    sc = r["score"].cpu().numpy()
    za = r["za_idx"].cpu().numpy()
    for b in (0, 2, 3):
        assert sc[b] == 0.0 and za[b] == 0          # all-zero correlation: lowest index
    for b in (1, 4):
        mt = O.match_pattern(oplan, *scan.pattern(b))
        assert math.isclose(sc[b], mt.score, rel_tol=1e-4)
    assert np.all(np.isfinite(r["orient"].cpu().numpy()))
    # empty batch
    e = c1.match(torch.zeros(1, dtype=torch.int64, device="cuda"),
                 torch.zeros(0, device="cuda"), torch.zeros(0, device="cuda"),
                 torch.zeros(0, device="cuda"))
    assert e["score"].numel() == 0


def test_bad_input_reported(c1):
    import torch
    from paper_2111_00171_gb300.acom import AcomError
    scan = synth.random_patterns(3, n_patterns=4)
    rp, qx, qy, I = to_dev(scan)
    bad = rp.clone()
    bad[2] = bad[3] + 1                               # decreasing row_ptr
    with pytest.raises(AcomError) as ei:
        c1.match(bad, qx, qy, I)
    assert ei.value.status == 6
    nan = qx.clone()
    nan[0] = float("nan")
    with pytest.raises(AcomError) as ei:
        c1.match(rp, nan, qy, I)
    assert ei.value.status == 6
    # the plan still works after a reported error
    r = c1.match(rp, qx, qy, I)
    torch.cuda.synchronize()
    assert torch.isfinite(r["score"]).all()


@pytest.mark.parametrize("exhaustive", [True, False], ids=["exhaustive", "pruned"])
def test_deterministic(c1, exhaustive):
    scan = synth.random_patterns(77, n_patterns=64)
    a = c1.match(*to_dev(scan), za_scores=True, exhaustive=exhaustive)
    b = c1.match(*to_dev(scan), za_scores=True, exhaustive=exhaustive)
    for k in a:
        assert (a[k].cpu() == b[k].cpu()).all(), k


def test_pruned_equals_exhaustive(c1):
    """Certified pruning returns the exhaustive winner; scores agree to FP32
    rounding (the two paths sum in different orders)."""
    scan = synth.random_patterns(91, n_patterns=200)
    a = c1.match(*to_dev(scan), exhaustive=True)
    b = c1.match(*to_dev(scan), exhaustive=False)
    ka = np.stack([a[k].cpu().numpy().astype(np.int64) for k in ("za_idx", "phi3_bin", "mirror")], 1)
    kb = np.stack([b[k].cpu().numpy().astype(np.int64) for k in ("za_idx", "phi3_bin", "mirror")], 1)
    np.testing.assert_allclose(a["score"].cpu().numpy(), b["score"].cpu().numpy(), rtol=1e-5)
    diff = np.nonzero(np.any(ka != kb, axis=1))[0]
    # the two paths sum in different orders, so exact (symmetry) ties resolve
    # either way; a few per cent of random patterns have one
    assert len(diff) <= len(ka) // 20, diff
    oplan = oracle_plan("au_2deg_75x180")
    for i in diff:          # a difference must be an FP32-level tie in the oracle (R10)
        mt = O.match_pattern(oplan, *scan.pattern(i))
        assert check_argmax(mt, *ka[i]) and check_argmax(mt, *kb[i]), (i, ka[i], kb[i])
    same = np.setdiff1d(np.arange(len(ka)), diff)
    np.testing.assert_allclose(a["orient"].cpu().numpy()[same], b["orient"].cpu().numpy()[same],
                               atol=1e-4)


def test_hexagonal_plan_and_match():
    """Mg-like hcp on a 6-degree grid over the 1/24-sphere region."""
    from gpu_common import CONFIGS as CF
    CF.setdefault("mg_6deg_40x72", (6.0, 40, 0.0375, 72))
    plan = gpu_plan("mg_6deg_40x72", phase="Mg")
    op = oracle_plan("mg_6deg_40x72", phase="Mg")
    np.testing.assert_allclose(plan.zone_axes(), op.za, atol=1e-12)
    sp = plan.spectra().cpu().numpy()
    assert rel_err(sp, np.stack([op.P_hat.real, op.P_hat.imag], -1)) < 1e-5
    scan = synth.random_patterns(31, n_patterns=20, crystal=synth.mg_hcp())
    _match_and_compare(plan, op, scan, check_refine=False)
    _match_and_compare(plan, op, scan, check_refine=False, exhaustive=False)
    plan.close()


@pytest.fixture(scope="module")
def full_scan():
    return synth.grain_scan(1002)


def test_full_size_scan_sampled(full_scan):
    """The 256x256 scan against the 1-degree plan (903 zone axes, 150
    shells, 360 bins) in the launch configuration of the benchmark; sampled
    patterns are compared with the oracle one by one."""
    plan = gpu_plan("au_1deg_150x360")
    op = oracle_plan("au_1deg_150x360")
    import torch
    r = plan.match(*to_dev(full_scan), za_scores=False)
    torch.cuda.synchronize()
    n_eval = plan.get_info()["last_evaluated"]
    assert n_eval < 0.05 * 903 * full_scan.n_patterns, n_eval
    za = r["za_idx"].cpu().numpy()
    kk = r["phi3_bin"].cpu().numpy()
    mi = r["mirror"].cpu().numpy()
    sc = r["score"].cpu().numpy()
    assert np.all(np.isfinite(sc)) and np.all(za < 903)
    rng = np.random.default_rng(0)
    for b in rng.choice(full_scan.n_patterns, 12, replace=False):
        mt = O.match_pattern(op, *full_scan.pattern(b))
        assert check_argmax(mt, za[b], kk[b], mi[b]), b
        assert math.isclose(sc[b], mt.score, rel_tol=1e-4), b
    plan.close()


# ---------------------------------------------- tensor-core paths: BF16, FP16

TC_PRECISIONS = [1, 2]
TC_IDS = ["bf16", "fp16"]
# relative error of the bounds against FP32: BF16 rounds each operand to 2^-8,
# FP16 to 2^-11, so a product is off by at most 2^-7 and 2^-10
TC_BOUND_TOL = {1: (2.0 ** -6, 2.0 ** -9), 2: (2.0 ** -9, 2.0 ** -12)}


@pytest.mark.parametrize("precision", TC_PRECISIONS, ids=TC_IDS)
@pytest.mark.parametrize("name", ["au_6deg_40x72", "au_2deg_75x180"])
def test_tc_bounds_track_fp32(name, precision):
    """The tcgen05 contraction's spectral bounds agree with the FP32 CUDA-core
    bounds to the operands' rounding."""
    p32 = gpu_plan(name)
    p16 = gpu_plan(name, precision=precision)
    scan = synth.random_patterns(1001, n_patterns=100)
    u32 = p32.bounds(*to_dev(scan)).cpu().numpy()
    u16 = p16.bounds(*to_dev(scan)).cpu().numpy()
    rel = np.abs(u16 - u32) / np.maximum(np.abs(u32), 1e-30)
    print(f"{TC_IDS[precision - 1]} bound rel err {name}: max {rel.max():.3e} "
          f"mean {rel.mean():.3e}")
    assert np.all(np.isfinite(u16))
    tmax, tmean = TC_BOUND_TOL[precision]
    assert rel.max() < tmax and rel.mean() < tmean
    p32.close()
    p16.close()


@pytest.mark.parametrize("factor", [1e-6, 1.0, 1e6])
def test_fp16_scaling_extreme_intensities(factor):
    """FP16 operands carry a power-of-two scale per pattern: intensities of
    1e6 (FP16 overflows at 65504) or 1e-6 (below its normal range) give the
    bounds of the FP32 path on the same intensities, and the FP32 path's
    winners."""
    import torch
    p32 = gpu_plan("au_2deg_75x180")
    p16 = gpu_plan("au_2deg_75x180", precision=2)
    scan = synth.random_patterns(1003, n_patterns=100)
    rp, qx, qy, I = to_dev(scan)
    Is = I * factor
    u32 = p32.bounds(rp, qx, qy, Is).cpu().numpy()
    u16 = p16.bounds(rp, qx, qy, Is).cpu().numpy()
    assert np.all(np.isfinite(u16))
    rel = np.abs(u16 - u32) / np.maximum(np.abs(u32), 1e-30 * factor)
    assert rel.max() < 2.0 ** -9, rel.max()
    a = p32.match(rp, qx, qy, Is)
    torch.cuda.synchronize()
    ev32 = p32.get_info()["last_evaluated"]
    b = p16.match(rp, qx, qy, Is)
    torch.cuda.synchronize()
    ev = p16.get_info()["last_evaluated"]
    np.testing.assert_allclose(b["score"].cpu().numpy(), a["score"].cpu().numpy(), rtol=1e-5)
    ka = np.stack([a[k].cpu().numpy().astype(np.int64) for k in ("za_idx", "phi3_bin", "mirror")], 1)
    kb = np.stack([b[k].cpu().numpy().astype(np.int64) for k in ("za_idx", "phi3_bin", "mirror")], 1)
    op = oracle_plan("au_2deg_75x180")
    for i in np.nonzero(np.any(ka != kb, axis=1))[0]:
        mt = O.match_pattern(op, *scan.pattern(i))
        assert check_argmax(mt, *ka[i]) and check_argmax(mt, *kb[i]), i
    # the scale keeps the margin small: few axes beyond the FP32 bound's survivors
    print(f"fp16 factor {factor:g}: {ev} axes evaluated, fp32 bound {ev32}")
    assert ev <= 1.5 * ev32 + 20
    p32.close()
    p16.close()


def test_fp32_bounds_dominate_oracle_maxima(c1):
    """U >= max over phi3 and mirror of C for every axis (the pruning bound)."""
    scan = synth.random_patterns(1002, n_patterns=30)
    u = c1.bounds(*to_dev(scan)).cpu().numpy()
    oplan = oracle_plan("au_2deg_75x180")
    for b in range(scan.n_patterns):
        mt = O.match_pattern(oplan, *scan.pattern(b))
        assert np.all(u[b] >= mt.za_scores - 1e-5 * abs(mt.score)), b


@pytest.fixture(scope="module", params=TC_PRECISIONS, ids=TC_IDS)
def c1_tc(request):
    plan = gpu_plan("au_2deg_75x180", precision=request.param)
    yield plan
    plan.close()


@pytest.mark.parametrize("chunk", [0, 48])
def test_match_tc_matches_oracle(c1_tc, chunk):
    """BF16 or FP16 tensor-core bounds + FP32 evaluation of the survivors: the
    oracle's winner (up to ties) and FP32-level scores."""
    scan = synth.random_patterns(1001, n_patterns=100)
    _match_and_compare(c1_tc, oracle_plan("au_2deg_75x180"), scan, chunk=chunk,
                       exhaustive=False)


@pytest.mark.parametrize("precision", TC_PRECISIONS, ids=TC_IDS)
def test_match_tc_two_stage_k_range(precision):
    """A plan whose contraction K range spans two ring stages, the second only
    partly filled (200 shells of 0.0075 1/A: K runs over 176 shells, a stage
    of two K tiles, then one of a single K tile whose second full barrier is
    only arrived on): the oracle's winners (up to ties) and FP32-level scores."""
    plan = gpu_plan("au_6deg_200x72", precision=precision)
    spad = (200 + 15) // 16 * 16
    k_range = spad - plan.get_info()["k0"]
    assert k_range > 128 and k_range % 128 <= 64, k_range
    scan = synth.random_patterns(1007, n_patterns=60)
    _match_and_compare(plan, oracle_plan("au_6deg_200x72"), scan, exhaustive=False)
    plan.close()


@pytest.mark.parametrize("precision", TC_PRECISIONS, ids=TC_IDS)
def test_full_size_tc_equals_fp32(full_scan, precision):
    """The 256x256 scan, 1-degree plan: BF16 or FP16 certified pruning returns
    the FP32 winners (differences only at FP32 ties, checked against the oracle)."""
    import torch
    p32 = gpu_plan("au_1deg_150x360")
    p16 = gpu_plan("au_1deg_150x360", precision=precision)
    a = p32.match(*to_dev(full_scan))
    b = p16.match(*to_dev(full_scan))
    torch.cuda.synchronize()
    ka = np.stack([a[k].cpu().numpy().astype(np.int64) for k in ("za_idx", "phi3_bin", "mirror")], 1)
    kb = np.stack([b[k].cpu().numpy().astype(np.int64) for k in ("za_idx", "phi3_bin", "mirror")], 1)
    diff = np.nonzero(np.any(ka != kb, axis=1))[0]
    assert len(diff) <= 0.001 * len(ka), len(diff)
    np.testing.assert_allclose(a["score"].cpu().numpy(), b["score"].cpu().numpy(), rtol=1e-5)
    op = oracle_plan("au_1deg_150x360")
    for i in diff:          # every difference must be a documented tie in the oracle
        mt = O.match_pattern(op, *full_scan.pattern(i))
        assert check_argmax(mt, *ka[i]) and check_argmax(mt, *kb[i]), i
    ev = p16.get_info()["last_evaluated"] / full_scan.n_patterns
    print(f"{TC_IDS[precision - 1]} axes evaluated per pattern: {ev:.2f}")
    assert ev < 40
    p32.close()
    p16.close()


# ------------------------------------------------ E4M3 operands (experiment)

def test_fp8_bounds_track_fp32():
    """E4M3 operands (FP16 operands times 2^-6) on kind::f8f6f4: bounds within
    their 2^-4-per-operand rounding of the FP32 bounds."""
    p32 = gpu_plan("au_2deg_75x180")
    p8 = gpu_plan("au_2deg_75x180", precision=3)
    scan = synth.random_patterns(1001, n_patterns=100)
    u32 = p32.bounds(*to_dev(scan)).cpu().numpy()
    u8 = p8.bounds(*to_dev(scan)).cpu().numpy()
    rel = np.abs(u8 - u32) / np.maximum(np.abs(u32), 1e-30)
    print(f"fp8 bound rel err: max {rel.max():.3e} mean {rel.mean():.3e}")
    assert np.all(np.isfinite(u8))
    assert rel.max() < 2.0 ** -2 and rel.mean() < 2.0 ** -5
    p32.close()
    p8.close()


def test_fp8_certified_and_rescored_winners():
    """Certified pruning on E4M3 bounds still returns the FP32 winners (with
    many more exact evaluations); rescoring only the top 8 bounds is an
    uncertified experiment whose agreement is reported."""
    import torch
    p32 = gpu_plan("au_2deg_75x180")
    p8 = gpu_plan("au_2deg_75x180", precision=3)
    scan = synth.random_patterns(1001, n_patterns=100)
    a = p32.match(*to_dev(scan))
    torch.cuda.synchronize()
    ev32 = p32.get_info()["last_evaluated"]
    b = p8.match(*to_dev(scan))
    torch.cuda.synchronize()
    ev8 = p8.get_info()["last_evaluated"]
    c = p8.match(*to_dev(scan), rescore_top=8)
    torch.cuda.synchronize()
    keys = ("za_idx", "phi3_bin", "mirror")
    ka = np.stack([a[k].cpu().numpy().astype(np.int64) for k in keys], 1)
    kb = np.stack([b[k].cpu().numpy().astype(np.int64) for k in keys], 1)
    kc = np.stack([c[k].cpu().numpy().astype(np.int64) for k in keys], 1)
    op = oracle_plan("au_2deg_75x180")
    for i in np.nonzero(np.any(ka != kb, axis=1))[0]:
        mt = O.match_pattern(op, *scan.pattern(i))
        assert check_argmax(mt, *ka[i]) and check_argmax(mt, *kb[i]), i
    agree = 0
    for i in range(scan.n_patterns):
        if np.array_equal(kc[i], ka[i]):
            agree += 1
        else:
            agree += check_argmax(O.match_pattern(op, *scan.pattern(i)), *kc[i])
    print(f"fp8 certified: {ev8 / 100:.1f} axes evaluated per pattern (fp32 bound {ev32 / 100:.1f});"
          f" top-8 rescoring agrees on {agree}/100")
    assert agree >= 80
    p32.close()
    p8.close()


# ------------------------------------------------------ CUDA graph capture

def test_match_async_captured_in_cuda_graph():
    """acom_match_async captured into a CUDA graph: replaying it on new
    contents of the same peak buffers gives what a synchronous match of those
    peaks gives, and acom_sync reports the replay's status."""
    import torch
    plan = gpu_plan("au_2deg_75x180", precision=2)
    a = synth.random_patterns(1301, n_patterns=64)
    # a second scan with the same CSR layout: the same peaks rotated in plane
    ang = 0.37
    bx = (np.cos(ang) * a.qx - np.sin(ang) * a.qy).astype(np.float32)
    by = (np.sin(ang) * a.qx + np.cos(ang) * a.qy).astype(np.float32)
    rp, qx, qy, I = to_dev(a)
    plan.match(rp, qx, qy, I)                    # sizes the workspace
    out = plan.alloc_result(a.n_patterns)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        plan.match_async(rp, qx, qy, I, out)
    qx.copy_(torch.from_numpy(bx).cuda())
    qy.copy_(torch.from_numpy(by).cuda())
    g.replay()
    plan.sync()
    ref = plan.match(rp, qx, qy, I)
    torch.cuda.synchronize()
    for k in ("za_idx", "phi3_bin", "mirror", "score", "orient"):
        assert torch.equal(out[k], ref[k]), k
    plan.close()


def test_autotune_trials_and_tile_orders():
    """acom_autotune times twelve schedules (three chunk sizes, two tile
    orders, one CTA or a CTA pair per MMA) and returns the fastest; both tile
    orders of the contraction give bit-identical results."""
    import torch
    plan = gpu_plan("au_2deg_75x180", precision=2)
    scan = synth.random_patterns(1401, n_patterns=200)
    inp = to_dev(scan)
    best, trials = plan.autotune(*inp)
    assert len(trials) == 12 and all(t["ms"] > 0 for t in trials)
    assert sorted({t["cta_pairs"] for t in trials}) == [0, 1]
    assert best["ms"] == min(t["ms"] for t in trials)
    a = plan.match(*inp, tile_order=0)
    b = plan.match(*inp, tile_order=1, chunk=best["chunk"])
    torch.cuda.synchronize()
    for k in ("za_idx", "phi3_bin", "mirror", "score"):
        assert torch.equal(a[k], b[k]), k
    plan.close()


def test_many_peaks_and_radius_ties(c1):
    """Patterns at the 1024-peak limit and at counts that are not multiples
    of the block size (several peaks per thread in the raster's radius sort),
    with every radius present twice (peak pairs at opposite angles): polar
    spectra and match scores against the oracle."""
    rng = np.random.default_rng(77)
    rows = []
    for n in (1024, 777, 257, 2):
        h = n // 2
        r = rng.uniform(0.1, 1.45, h)
        t = rng.uniform(-np.pi, np.pi, h)
        x = np.concatenate([r * np.cos(t), -r * np.cos(t)])
        y = np.concatenate([r * np.sin(t), -r * np.sin(t)])
        i = rng.lognormal(0.0, 1.0, 2 * h)
        perm = rng.permutation(2 * h)
        rows.append((x[perm].astype(np.float32), y[perm].astype(np.float32),
                     i[perm].astype(np.float32)))
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r[0]) for r in rows])
    qx = np.concatenate([r[0] for r in rows])
    qy = np.concatenate([r[1] for r in rows])
    I = np.concatenate([r[2] for r in rows])
    scan = synth.Scan(rp, qx, qy, I, np.tile(np.eye(3), (len(rows), 1, 1)),
                      np.zeros(len(rows), np.int32), (synth.au_fcc(),), "many peaks")
    sp, xn = c1.polar_spectra(*to_dev(scan))
    sp = sp.cpu().numpy()
    oplan = oracle_plan("au_2deg_75x180")
    prm = oplan.params
    r = c1.match(*to_dev(scan))
    sc = r["score"].cpu().numpy()
    za = r["za_idx"].cpu().numpy()
    kk = r["phi3_bin"].cpu().numpy()
    mi = r["mirror"].cpu().numpy()
    for b in range(scan.n_patterns):
        X = O.polar_image(*scan.pattern(b), prm)
        Xh = np.fft.rfft(X, axis=1)
        assert rel_err(sp[b], np.stack([Xh.real, Xh.imag], axis=-1)) < 1e-5, b
        mt = O.match_pattern(oplan, *scan.pattern(b))
        assert math.isclose(sc[b], mt.score, rel_tol=1e-4), b
        assert check_argmax(mt, za[b], kk[b], mi[b], 1e-5), b


@pytest.mark.parametrize("precision", [1, 2, 3], ids=["bf16", "fp16", "fp8"])
def test_cta_pairs_equal_single_cta(precision):
    """The tensor-core contraction on CTA pairs (cta_group::2) computes the
    same dot products in the same order as one CTA per MMA (the default):
    bounds, winners and scores are bitwise equal, on a chunk with an odd
    number of 64-pattern tiles (the last pair's second CTA has no patterns)."""
    import torch
    plan = gpu_plan("au_2deg_75x180", precision=precision)
    scan = synth.random_patterns(1601, n_patterns=300)
    inp = to_dev(scan)
    for chunk in (0, 192):
        a = plan.match(*inp, za_scores=True, chunk=chunk, cta_pairs=1)
        b = plan.match(*inp, za_scores=True, chunk=chunk, cta_pairs=0)
        torch.cuda.synchronize()
        for k in ("za_idx", "phi3_bin", "mirror", "score", "za_scores", "orient"):
            assert torch.equal(a[k], b[k]), (chunk, k)
    plan.close()
