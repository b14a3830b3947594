"""Continuous refinement through the C ABI against the oracle: the
kinematical score, its gradient and Gauss-Newton matrix at given
orientations; the autograd wrapper against finite differences; refined
orientations against the oracle's refinement; and a coarse 3-degree grid
match followed by refinement on the grain scan.

Tolerances: the score within 1e-4 relative of the FP64 oracle, the gradient
and Gauss-Newton matrix within 1e-3 of their largest entry (FP32 sums of
terms of both signs); refined orientations within 0.02 degrees of the
oracle's (FP32 and FP64 trajectories of the same damped ascent)."""

import math

import numpy as np
import pytest

import synth
from oracle import acom_oracle as O

from gpu_common import CONFIGS, LAM, au_refl, gpu_plan, to_dev

pytestmark = pytest.mark.gpu

CONFIGS.setdefault("au_3deg_150x360", (3.0, 150, 0.01, 360))   # 105 axes


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def plan():
    p = gpu_plan("au_6deg_40x72")
    yield p
    p.close()


def _starts(scan, deg, seed, twin_every=0):
    """Truth rotated by ``deg`` about a random axis (every twin_every-th also
    turned into its Friedel twin), rounded to FP32 as the library sees it."""
    rng = np.random.default_rng(seed)
    out = np.empty((scan.n_patterns, 3, 3))
    for b in range(scan.n_patterns):
        w = rng.normal(size=3)
        m0 = scan.truth[b] @ O.so3_exp(w * math.radians(deg) / np.linalg.norm(w))
        if twin_every and b % twin_every == 0:
            m0 = m0 @ np.diag([-1.0, -1.0, 1.0])
        out[b] = m0
    return out.astype(np.float32)


def test_score_gradient_and_gauss_newton_match_oracle(plan):
    import torch
    scan = synth.random_patterns(1101, n_patterns=64)
    m0 = _starts(scan, 1.0, 0)
    r = (np.random.default_rng(1).normal(size=(scan.n_patterns, 3)) * 0.02).astype(np.float32)
    s, g, gn = plan.kinematical_score(*to_dev(scan), torch.from_numpy(m0).cuda(),
                                      r=torch.from_numpy(r).cuda(), rho=0.05)
    s, g, gn = s.cpu().numpy(), g.cpu().numpy(), gn.cpu().numpy()
    refl = au_refl()
    for b in range(scan.n_patterns):
        qx, qy, I = scan.pattern(b)
        So, go = O.kinematical_score_r(r[b].astype(np.float64), m0[b].astype(np.float64), qx, qy,
                                       I, refl, LAM, 0.02, 0.05)
        R = O.so3_exp(r[b].astype(np.float64)) @ m0[b].astype(np.float64).T
        H = O.kinematical_score(R, qx, qy, I, refl, LAM, 0.02, 0.05).H
        assert s[b] == pytest.approx(So, rel=1e-4), b
        np.testing.assert_allclose(g[b], go, rtol=0, atol=1e-3 * np.abs(go).max(), err_msg=str(b))
        Hv = H[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]
        np.testing.assert_allclose(gn[b], Hv, rtol=0, atol=1e-3 * np.abs(Hv).max(), err_msg=str(b))


def test_autograd_gradient_matches_finite_differences(plan):
    """torch.autograd through the hand-written backward against central
    differences of the FP32 score (step 2e-3 rad)."""
    import torch

    from paper_2111_00171_gb300 import acom
    scan = synth.random_patterns(1103, n_patterns=16)
    peaks = to_dev(scan)
    orient = torch.from_numpy(_starts(scan, 0.5, 2)).cuda()
    r0 = torch.from_numpy((np.random.default_rng(3).normal(size=(16, 3)) * 0.01)
                          .astype(np.float32)).cuda()
    r = r0.clone().requires_grad_(True)
    S = acom.kinematical_score(r, plan, peaks, orient, rho=0.05)
    S.sum().backward()
    h = 2e-3
    fd = torch.zeros_like(r0)
    for j in range(3):
        e = torch.zeros_like(r0)
        e[:, j] = h
        sp, _, _ = plan.kinematical_score(*peaks, orient, r=r0 + e, rho=0.05)
        sm, _, _ = plan.kinematical_score(*peaks, orient, r=r0 - e, rho=0.05)
        fd[:, j] = (sp - sm) / (2 * h)
    a, b = r.grad.cpu().numpy(), fd.cpu().numpy()
    for i in range(16):
        np.testing.assert_allclose(a[i], b[i], rtol=0, atol=2e-2 * np.abs(b[i]).max(), err_msg=str(i))


def test_strained_score_and_gradients_match_oracle(plan):
    """acom_kinematical_score_strain at strains of a few 1e-3 against the
    oracle's kinematical_score_strain: the score within 1e-4 relative, dS/dr
    and dS/de within 1e-3 of their largest entry.  At zero strain the strained
    entry gives the plain entry's score and gradient."""
    import torch
    scan = synth.random_patterns(1104, n_patterns=48)
    m0 = _starts(scan, 0.5, 5)
    rng = np.random.default_rng(6)
    r = (rng.normal(size=(scan.n_patterns, 3)) * 0.01).astype(np.float32)
    e = (rng.normal(size=(scan.n_patterns, 6)) * 3e-3).astype(np.float32)
    peaks = to_dev(scan)
    om = torch.from_numpy(m0).cuda()
    rd = torch.from_numpy(r).cuda()
    s, g, _, de = plan.kinematical_score(*peaks, om, r=rd, rho=0.05,
                                         strain=torch.from_numpy(e).cuda())
    s, g, de = s.cpu().numpy(), g.cpu().numpy(), de.cpu().numpy()
    refl = au_refl()
    for b in range(scan.n_patterns):
        qx, qy, I = scan.pattern(b)
        rb = r[b].astype(np.float64)
        R = O.so3_exp(rb) @ m0[b].astype(np.float64).T
        sc, deo = O.kinematical_score_strain(R, e[b].astype(np.float64), qx, qy, I, refl,
                                             LAM, 0.02, 0.05)
        go = O.so3_left_jacobian(rb).T @ sc.grad
        assert s[b] == pytest.approx(sc.S, rel=1e-4), b
        np.testing.assert_allclose(g[b], go, rtol=0, atol=1e-3 * np.abs(go).max(), err_msg=str(b))
        np.testing.assert_allclose(de[b], deo, rtol=0, atol=1e-3 * np.abs(deo).max(),
                                   err_msg=str(b))
    s0, g0, gn0 = plan.kinematical_score(*peaks, om, r=rd, rho=0.05)
    s1, g1, gn1, _ = plan.kinematical_score(*peaks, om, r=rd, rho=0.05,
                                            strain=torch.zeros((scan.n_patterns, 6),
                                                               device="cuda"))
    assert torch.equal(s0, s1) and torch.equal(g0, g1) and torch.equal(gn0, gn1)


def test_strain_autograd_matches_finite_differences(plan):
    """torch.autograd through acom.kinematical_score_strain: dS/de against
    central differences of the FP32 score (step 1e-3 in each component)."""
    import torch

    from paper_2111_00171_gb300 import acom
    scan = synth.random_patterns(1105, n_patterns=16)
    peaks = to_dev(scan)
    orient = torch.from_numpy(_starts(scan, 0.3, 7)).cuda()
    rng = np.random.default_rng(8)
    r = torch.from_numpy((rng.normal(size=(16, 3)) * 0.005).astype(np.float32)).cuda()
    e0 = torch.from_numpy((rng.normal(size=(16, 6)) * 2e-3).astype(np.float32)).cuda()
    e = e0.clone().requires_grad_(True)
    S = acom.kinematical_score_strain(r, e, plan, peaks, orient, rho=0.05)
    S.sum().backward()
    h = 1e-3
    fd = torch.zeros_like(e0)
    for j in range(6):
        d = torch.zeros_like(e0)
        d[:, j] = h
        sp = plan.kinematical_score(*peaks, orient, r=r, rho=0.05, strain=e0 + d)[0]
        sm = plan.kinematical_score(*peaks, orient, r=r, rho=0.05, strain=e0 - d)[0]
        fd[:, j] = (sp - sm) / (2 * h)
    a, b = e.grad.cpu().numpy(), fd.cpu().numpy()
    for i in range(16):
        np.testing.assert_allclose(a[i], b[i], rtol=0, atol=3e-2 * np.abs(b[i]).max(),
                                   err_msg=str(i))


def test_refine_matches_oracle(plan):
    """acom_refine from starts 1.5 degrees off (every third a Friedel twin)
    against the oracle's refine_with_twin from the same FP32 starts."""
    import torch
    scan = synth.random_patterns(1102, n_patterns=48)
    m0 = _starts(scan, 1.5, 4, twin_every=3)
    orient = torch.from_numpy(m0.copy()).cuda()
    _, score, tw = plan.refine(*to_dev(scan), orient)
    mg, score, tw = orient.cpu().numpy().astype(np.float64), score.cpu().numpy(), tw.cpu().numpy()
    refl = au_refl()
    ops = O.proper_point_group("cubic")
    prm = O.RefineParams()
    close = same_twin = 0
    err = []
    for b in range(scan.n_patterns):
        mo, so, two = O.refine_with_twin(m0[b].astype(np.float64), *scan.pattern(b), refl, LAM, prm)
        d = O.misorientation_deg(mg[b], mo, ops)
        close += d < 0.02
        same_twin += bool(tw[b]) == two
        if d < 0.02:
            assert score[b] == pytest.approx(so, rel=1e-3), b
        err.append(O.misorientation_deg(mg[b], scan.truth[b], ops))
    err = np.array(err)
    print(f"refined vs oracle within 0.02 deg: {close}/48, twin choice equal {same_twin}/48; "
          f"vs truth median {np.median(err):.3f} mean {err.mean():.3f} deg")
    assert close >= 44 and same_twin >= 46
    assert np.median(err) < 0.2


def test_coarse_match_then_refine_grain_scan():
    """The grain scan (64x64 corner of the 256x256 recipe) matched on the
    3-degree plan in BF16, then refined: far below the grid's error."""
    import torch
    scan = synth.grain_scan(1002, H=64, W=64)
    coarse = gpu_plan("au_3deg_150x360", precision=1)
    inp = to_dev(scan)
    r = coarse.match(*inp, runner=True)
    grid = r["orient"].cpu().numpy().astype(np.float64)
    orient = r["orient"].contiguous()
    coarse.refine(*inp, orient, orient_alt=r["runner_orient"])
    torch.cuda.synchronize()
    ref = orient.cpu().numpy().astype(np.float64)
    ops = O.proper_point_group("cubic")
    rng = np.random.default_rng(6)
    idx = rng.choice(scan.n_patterns, 400, replace=False)
    e_grid = np.array([O.misorientation_deg(grid[b], scan.truth[b], ops) for b in idx])
    e_ref = np.array([O.misorientation_deg(ref[b], scan.truth[b], ops) for b in idx])
    print(f"3-degree grid: mean {e_grid.mean():.3f} median {np.median(e_grid):.3f}; refined: "
          f"mean {e_ref.mean():.3f} median {np.median(e_ref):.3f} deg")
    assert np.median(e_ref) < 0.2 and e_ref.mean() < e_grid.mean()
    coarse.close()


def test_runner_up_is_outside_the_winners_neighbourhood():
    """The runner-up is the best axis that is neither the winner nor one of
    its grid neighbours (the oracle's maximum over those axes, up to ties
    within 1e-5), its score is the oracle's exact maximum for that axis, and
    its orientation is that axis' grid orientation (up to the crystal's
    symmetry: a symmetric axis has tied maxima)."""
    import torch
    plan = gpu_plan("au_2deg_75x180")
    from gpu_common import oracle_plan
    op = oracle_plan("au_2deg_75x180")
    scan = synth.random_patterns(1104, n_patterns=40)
    r = plan.match(*to_dev(scan), runner=True, za_scores=True)
    torch.cuda.synchronize()
    za, ru = r["za_idx"].cpu().numpy(), r["runner_za"].cpu().numpy()
    rs, ro = r["runner_score"].cpu().numpy(), r["runner_orient"].cpu().numpy()
    nb = O.za_neighbours(op.za, plan.step_deg)
    N = op.params.n_phi
    ops = O.proper_point_group("cubic")
    for b in range(scan.n_patterns):
        assert ru[b] != za[b] and ru[b] not in nb[za[b]], b
        if ru[b] < 0:
            continue
        mt = O.match_pattern(op, *scan.pattern(b))
        assert rs[b] == pytest.approx(mt.za_scores[ru[b]], rel=1e-4), b
        outside = np.setdiff1d(np.arange(len(op.za)), np.append(nb[za[b]], za[b]))
        best_out = mt.za_scores[outside].max()
        assert mt.za_scores[ru[b]] >= best_out * (1 - 1e-5), (b, ru[b], best_out)
        C = np.stack([mt.C[ru[b]], mt.Cm[ru[b]]])
        # the grid orientation of the axis' maximum, or of a bin tied with it
        # within 1e-5 (FP32 scores cannot order those); elementwise under the
        # best symmetry operation (the angle from the trace is ill-conditioned
        # for FP32-stored matrices near identity)
        tied = np.argwhere(C >= C.max() - 1e-5 * abs(C.max()))
        err = min(np.abs(S @ ro[b] - O.orientation_matrix(op.za[ru[b]], -2 * math.pi * k / N,
                                                             int(mir))).max()
                  for mir, k in tied for S in ops)
        assert err < 2e-6, (b, err, len(tied))
    plan.close()
