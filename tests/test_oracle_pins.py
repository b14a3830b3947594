"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formula: each compares it with a closed
form, a brute-force enumeration, an invariant, a value the paper prints
(fixtures in tests/golden/) or the exact result of a special case.
"""

import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import acom_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


AU = _golden("fig1_fcc_au.json")
A_AU = AU["lattice_constant_A"]
LAM = 0.01969


def au_reflections(q_max=1.5, **kw):
    L = np.eye(3) * A_AU
    return O.reflections(L, AU["frac_pos"], [79.0] * 4, [0.25] * 4, q_max, **kw)


def mg_lattice():
    a, c = 3.21, 5.21
    return np.array([[a, 0, 0], [-a / 2, a * math.sqrt(3) / 2, 0], [0, 0, c]])


MG_POS = [[1 / 3, 2 / 3, 1 / 4], [2 / 3, 1 / 3, 3 / 4]]


@pytest.fixture(scope="module")
def c1_plan():
    v0, v1, v2, om = O.cubic_triangle()
    za = O.zone_axis_grid(v0, v1, v2, 2.0, om)
    prm = O.PlanParams(n_shells=75, dq=0.02, n_phi=180, delta=0.08, lam=LAM)
    return O.orientation_plan(au_reflections(), za, prm)


# ---------------------------------------------------------------- Eq. 1 ----

@pytest.mark.parametrize("lattice", [
    np.eye(3) * 4.08,
    mg_lattice(),
    np.array([[3.1, 0.2, -0.1], [0.4, 4.3, 0.3], [-0.2, 0.5, 5.7]]),
])
def test_reciprocal_basis_duality(lattice):
    """a_i* . a_j = delta_ij is the defining property of the reciprocal basis
    without 2 pi."""
    rb = O.reciprocal_basis(lattice)
    np.testing.assert_allclose(rb @ np.asarray(lattice).T, np.eye(3), atol=1e-14)


# ------------------------------------------------------------- Eqs. 2-3 ----

def test_fcc_reflection_set_and_structure_factor_closed_form():
    """fcc: F = 4 f(|g|) when h, k, l are all even or all odd, 0 otherwise.
    Brute force over a box twice as large as needed finds the same set."""
    refl = au_reflections(drop_extinct=False)
    q = np.linalg.norm(refl.g, axis=1)
    f = 79.0 * np.exp(-0.25 * q * q)
    h, k, l = refl.hkl.T
    unmixed = ((h % 2) == (k % 2)) & ((k % 2) == (l % 2))
    np.testing.assert_allclose(refl.F[unmixed].real, 4 * f[unmixed], rtol=1e-12)
    np.testing.assert_allclose(refl.F[unmixed].imag, 0, atol=1e-10)
    np.testing.assert_allclose(np.abs(refl.F[~unmixed]), 0, atol=1e-10)
    # independent enumeration: cubic lattice, |g| = |hkl| / a
    n = 2 * int(1.5 * A_AU) + 2
    brute = set()
    for hh, kk, ll in itertools.product(range(-n, n + 1), repeat=3):
        qq = math.sqrt(hh * hh + kk * kk + ll * ll) / A_AU
        if 0 < qq < 1.5:
            brute.add((hh, kk, ll))
    assert brute == set(map(tuple, refl.hkl.tolist()))
    live = au_reflections()
    assert len(live.F) == int(unmixed.sum()) == 258
    radii = np.unique(np.round(np.linalg.norm(live.g, axis=1), 9))
    assert len(radii) == 13
    assert abs(radii[0] - math.sqrt(3) / A_AU) < 1e-9       # {111}
    assert abs(radii[1] - 2 / A_AU) < 1e-9                  # {200}


def test_hcp_structure_factor_closed_form():
    """hcp basis (1/3,2/3,1/4), (2/3,1/3,3/4): |F|^2 = 0 for h+2k = 0 mod 3
    and l odd; 4 f^2 for h+2k = 0 mod 3, l even; 3 f^2 for h+2k != 0 mod 3,
    l odd; f^2 for h+2k != 0 mod 3, l even."""
    refl = O.reflections(mg_lattice(), MG_POS, [12.0] * 2, [0.3] * 2, 1.5,
                         drop_extinct=False)
    q = np.linalg.norm(refl.g, axis=1)
    f2 = (12.0 * np.exp(-0.3 * q * q)) ** 2
    h, k, l = refl.hkl.T
    m3 = ((h + 2 * k) % 3) == 0
    lodd = (l % 2) != 0
    expect = np.where(m3 & lodd, 0.0, np.where(m3, 4.0, np.where(lodd, 3.0, 1.0)))
    np.testing.assert_allclose(np.abs(refl.F) ** 2, expect * f2, rtol=1e-9,
                               atol=1e-9 * f2.max())
    # with a hexagonal basis the search box must also catch (h, -h, l) rows
    cart = refl.hkl.astype(float) @ O.reciprocal_basis(mg_lattice())
    assert np.all(np.linalg.norm(cart, axis=1) < 1.5)


# ------------------------------------------------- wavelength and Eq. 6 ----

def test_wavelength_textbook_value():
    """Textbook relativistic wavelength lambda = 12.2643 / sqrt(V (1 +
    0.97845e-6 V)) Angstrom; 300 kV gives 0.01969 Angstrom."""
    V = 300e3
    textbook = 12.2643 / math.sqrt(V * (1 + 0.97845e-6 * V))
    assert abs(O.electron_wavelength(300.0) - textbook) < 2e-6
    assert abs(O.electron_wavelength(300.0) - 0.01969) < 5e-6


def test_excitation_error_geometry():
    """s_g = 0 on the Ewald sphere |k + g| = |k|; for a zero-order-Laue-zone
    g (g . k = 0) s_g = -|g|^2 / (2 |k + g|) ~ -lambda |g|^2 / 2."""
    k = O.beam_vector(LAM)
    K = np.linalg.norm(k)
    rng = np.random.default_rng(3)
    for _ in range(10):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        g = -k + K * d                      # on the sphere centred at -k
        assert abs(O.excitation_error(g, k)) < 1e-9
    g = np.array([1.2, -0.3, 0.0])
    s = O.excitation_error(g, k)
    assert abs(s - (-(g @ g) / (2 * math.sqrt(K * K + g @ g)))) < 1e-15
    assert abs(s + LAM * (g @ g) / 2) < 1e-5


# -------------------------------------------------------------- Eq. 10 ----

def test_za_frame_maps_z_to_zone_axis():
    rng = np.random.default_rng(5)
    for _ in range(20):
        w = rng.normal(size=3)
        w /= np.linalg.norm(w)
        R = O.za_frame(w)
        np.testing.assert_allclose(R @ np.array([0, 0, 1.0]), w, atol=1e-14)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
    phi1, theta2 = O.za_angles([0, 0, 1.0])
    assert theta2 == 0.0
    np.testing.assert_allclose(O.za_frame([0, 0, 1.0]), np.eye(3), atol=1e-15)


# --------------------------------------------------------- zone-axis grid --

@pytest.mark.parametrize("step,count", [(3.0, 105), (2.0, 231), (1.0, 903), (0.5, 3486)])
def test_cubic_grid_counts_and_triangle(step, count):
    v0, v1, v2, om = O.cubic_triangle()
    za = O.zone_axis_grid(v0, v1, v2, step, om)
    assert len(za) == count
    np.testing.assert_allclose(np.linalg.norm(za, axis=1), 1, atol=1e-14)
    # standard triangle of m-3m: 0 <= x <= y <= z
    assert np.all(za[:, 0] >= -1e-12)
    assert np.all(za[:, 0] <= za[:, 1] + 1e-12)
    assert np.all(za[:, 1] <= za[:, 2] + 1e-12)
    for v in (v0, v1, v2):
        assert np.min(np.linalg.norm(za - v, axis=1)) < 1e-12


def test_hexagonal_grid_count():
    v0, v1, v2, om = O.hexagonal_triangle()
    za = O.zone_axis_grid(v0, v1, v2, 1.0, om)
    assert len(za) == 1770
    az = np.degrees(np.arctan2(za[:, 1], za[:, 0]))
    ok = np.hypot(za[:, 0], za[:, 1]) < 1e-12
    assert np.all(ok | ((az > -1e-9) & (az < 30 + 1e-9)))
    assert np.all(za[:, 2] >= -1e-12)


# -------------------------------------------------------------------- plan --

def test_plan_normalised(c1_plan):
    """A = 1/||P0||_2 makes every non-empty slice unit-norm."""
    nrm = np.sqrt(np.sum(c1_plan.P ** 2, axis=(1, 2)))
    np.testing.assert_allclose(nrm, 1.0, rtol=1e-12)


def test_plan_fft_is_along_phi3(c1_plan):
    """The plan spectrum's DC term is the sum over phi3 and its N/2 term the
    alternating sum (definition of the DFT along phi3)."""
    P = c1_plan.P
    N = P.shape[2]
    np.testing.assert_allclose(c1_plan.P_hat[..., 0].real, P.sum(axis=2), atol=1e-12)
    alt = (P * ((-1.0) ** np.arange(N))).sum(axis=2)
    np.testing.assert_allclose(c1_plan.P_hat[..., N // 2].real, alt, atol=1e-12)


def test_plan_001_first_row_four_200_spots(c1_plan):
    """Fig. 1f: at [001] the first populated row holds the four {200} spots
    (the {111} points lie far off the Ewald sphere), 4-fold symmetric."""
    gold = _golden("fig1_plan_001_first_row.json")
    prm = c1_plan.params
    z0 = int(np.argmin(np.linalg.norm(c1_plan.za - np.array(gold["zone_axis"]), axis=1)))
    assert np.allclose(c1_plan.za[z0], gold["zone_axis"])
    P = c1_plan.P[z0]
    N = prm.n_phi
    q_s = prm.shells()
    q200 = 2.0 / A_AU
    populated = np.nonzero(P.max(axis=1) > 0)[0]
    assert q_s[populated[0]] > q200 - prm.delta - 1e-12
    s0 = int(np.argmin(np.abs(q_s - q200)))
    row = P[s0]
    peaks = [j for j in range(N) if row[j] > row[(j - 1) % N] and row[j] >= row[(j + 1) % N]]
    assert len(peaks) == gold["n_spots"]
    expect = sorted(int(round(math.degrees(math.atan2(h[1], h[0])) % 360 / 360 * N)) % N
                    for h in gold["first_row_hkl"])
    assert sorted(peaks) == expect
    np.testing.assert_allclose(P, np.roll(P, N // 4, axis=1), atol=1e-12)


# ------------------------------------------------------------ polar image --

def test_polar_image_single_peak_values():
    """One peak on a bin angle: X(s, j0) = q_m^gamma I^(omega/2)
    (1 - |q_m - q_s| / delta) for shells within delta, 0 elsewhere, and the
    angular support at shell s is |dphi| q_s < delta."""
    prm = O.PlanParams(n_shells=40, dq=0.025, n_phi=72, delta=0.08,
                       gamma_pow=1.0, omega=1.0)
    q_s = prm.shells()
    j0 = 9
    ang = 2 * math.pi * j0 / prm.n_phi
    qm, I = 0.53, 4.0
    X = O.polar_image([qm * math.cos(ang)], [qm * math.sin(ang)], [I], prm)
    expect = qm * math.sqrt(I) * np.maximum(1 - np.abs(qm - q_s) / prm.delta, 0)
    np.testing.assert_allclose(X[:, j0], expect, rtol=1e-12, atol=1e-12)
    dphi = np.abs(O.wrap_angle(prm.phis() - ang))
    for s in range(prm.n_shells):
        outside = (dphi * q_s[s] >= prm.delta) | (abs(qm - q_s[s]) >= prm.delta)
        assert np.all(X[s, outside] == 0)
    # omega = 0: intensities are ignored; gamma = 0: radius is ignored
    prm0 = O.PlanParams(n_shells=40, dq=0.025, n_phi=72, delta=0.08,
                        gamma_pow=0.0, omega=0.0)
    X0 = O.polar_image([qm * math.cos(ang)], [qm * math.sin(ang)], [I], prm0)
    np.testing.assert_allclose(X0[:, j0], np.maximum(1 - np.abs(qm - q_s) / 0.08, 0),
                               rtol=1e-12, atol=1e-12)


def test_polar_image_wraps_and_ignores_order():
    prm = O.PlanParams(n_shells=30, dq=0.05, n_phi=36, delta=0.1)
    rng = np.random.default_rng(11)
    q = rng.uniform(0.1, 1.4, 12)
    g = rng.uniform(-math.pi, math.pi, 12)
    I = rng.uniform(0.5, 2, 12)
    qx, qy = q * np.cos(g), q * np.sin(g)
    X = O.polar_image(qx, qy, I, prm)
    p = rng.permutation(12)
    np.testing.assert_allclose(O.polar_image(qx[p], qy[p], I[p], prm), X, atol=1e-12)
    # rotating the peaks by whole bins rolls the image along phi3
    r = 2 * math.pi * 5 / prm.n_phi
    Xr = O.polar_image(q * np.cos(g + r), q * np.sin(g + r), I, prm)
    np.testing.assert_allclose(Xr, np.roll(X, 5, axis=1), atol=1e-9)


# ------------------------------------------------------------ correlation --

@pytest.mark.parametrize("N", [12, 10, 9])
def test_fft_correlation_equals_direct_circular_sum(N):
    rng = np.random.default_rng(N)
    Z, S = 3, 4
    P = rng.normal(size=(Z, S, N))
    X = rng.normal(size=(S, N))
    C, Cm = O.correlogram(np.fft.rfft(P, axis=2), X)
    # brute force written as explicit loops
    Cb = np.zeros((Z, N))
    Cmb = np.zeros((Z, N))
    for z in range(Z):
        for k in range(N):
            for s in range(S):
                for j in range(N):
                    Cb[z, k] += P[z, s, j] * X[s, (j + k) % N]
                    Cmb[z, k] += P[z, s, j] * X[s, (-j - k) % N]
    np.testing.assert_allclose(C, Cb, atol=1e-12)
    np.testing.assert_allclose(Cm, Cmb, atol=1e-12)
    Cd, Cmd = O.direct_correlation(P, X)
    np.testing.assert_allclose(Cd, Cb, atol=1e-12)
    np.testing.assert_allclose(Cmd, Cmb, atol=1e-12)


def test_mirror_correlation_is_correlation_of_mirrored_pattern(c1_plan):
    """Conjugating FFT{X} mirrors the pattern: C_mirror of a pattern equals
    C of its y -> -y mirror image."""
    prm = c1_plan.params
    rng = np.random.default_rng(2)
    q = rng.uniform(0.3, 1.45, 15)
    g = rng.uniform(-math.pi, math.pi, 15)
    I = rng.uniform(1, 5, 15)
    X = O.polar_image(q * np.cos(g), q * np.sin(g), I, prm)
    Xm = O.polar_image(q * np.cos(g), -q * np.sin(g), I, prm)
    C, Cm = O.correlogram(c1_plan.P_hat[:20], X)
    C2, Cm2 = O.correlogram(c1_plan.P_hat[:20], Xm)
    np.testing.assert_allclose(Cm, C2, atol=1e-9 * np.abs(C).max())
    np.testing.assert_allclose(C, Cm2, atol=1e-9 * np.abs(C).max())


def test_self_indexing_is_exact(c1_plan):
    """X := P_z gives C(z, 0) = ||P_z||^2 = 1, the global maximum by
    Cauchy-Schwarz since every ||P_z'|| = 1 (kinematical self-indexing)."""
    rng = np.random.default_rng(7)
    for z in rng.choice(len(c1_plan.za), 6, replace=False):
        X = c1_plan.P[z]
        C, Cm = O.correlogram(c1_plan.P_hat, X)
        assert abs(C[z, 0] - 1.0) < 1e-12
        assert C.max() <= 1.0 + 1e-12 and Cm.max() <= 1.0 + 1e-12
        mt = O.best_match(C, Cm, X)
        assert mt.score == pytest.approx(1.0, abs=1e-12)
        assert abs(mt.score_cos - 1.0) < 1e-12
        # a different winner is allowed only as an exact tie (symmetric slice)
        assert (mt.za, mt.k, mt.mirror) == (z, 0, 0) or abs(mt.score - 1) < 1e-12


def test_noiseless_grid_patterns_recovered(c1_plan):
    """A noiseless pattern generated exactly at a grid zone axis and grid
    phi3 (direct or mirror) scores its maximum there, up to exact ties with
    zero symmetry-reduced misorientation.  The image weights (sqrt of the
    shaped intensity) and the plan weights (|F|, excitation error inside the
    tent) differ, so a grid neighbour may win by a small margin: that is
    allowed only within 1.5 grid steps and 1 % of the score, and the exact
    recoveries must be the large majority."""
    refl = au_reflections()
    ops = O.proper_point_group("cubic")
    rng = np.random.default_rng(1)
    N = c1_plan.params.n_phi
    za = c1_plan.za
    exact = 0
    for z in rng.choice(len(za), 12, replace=False):
        k = int(rng.integers(N))
        mir = int(rng.integers(2))
        m = O.orientation_matrix(za[z], -2 * math.pi * k / N, mir)
        qx, qy, I = O.kinematical_pattern(refl, m, LAM, AU["sigma"], 1e-3)
        mt = O.match_pattern(c1_plan, qx, qy, I)
        at_truth = (mt.Cm if mir else mt.C)[z, k]
        me = O.orientation_matrix(za[mt.za], -2 * math.pi * mt.k / N, mt.mirror)
        mis = O.misorientation_deg(me, m, ops)
        if at_truth >= mt.score * (1 - 1e-12):
            exact += 1
            assert mis < 1e-4
        else:
            assert at_truth >= 0.99 * mt.score
            assert mis < 1.5 * 2.0
    assert exact >= 10


def test_symmetry_equivalent_orientations_score_equally(c1_plan):
    refl = au_reflections()
    ops = O.proper_point_group("cubic")
    rng = np.random.default_rng(4)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    m = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                  [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                  [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
    base = O.match_pattern(c1_plan, *O.kinematical_pattern(refl, m, LAM, 0.02, 1e-3))
    for S in ops[:8]:
        other = O.match_pattern(c1_plan, *O.kinematical_pattern(refl, S @ m, LAM, 0.02, 1e-3))
        assert other.score == pytest.approx(base.score, rel=1e-10)


def test_fig1_zone_axes_inplane_symmetry_and_recovery():
    """Fig. 1g/h: patterns along [001], [011], [111], [113], [135] are
    indexed to their own zone axis, with 4-, 2-, 6-fold and single in-plane
    correlation maxima."""
    gold = _golden("fig1_inplane_symmetry.json")["folds"]
    names = ["001", "011", "111", "113", "135"]
    za = np.array([[int(c) for c in n] for n in names], dtype=float)
    za /= np.linalg.norm(za, axis=1)[:, None]
    prm = O.PlanParams(n_shells=75, dq=0.02, n_phi=360, delta=0.08, lam=LAM)
    refl = au_reflections()
    plan = O.orientation_plan(refl, za, prm)
    N = prm.n_phi
    for i, name in enumerate(names):
        m = O.orientation_matrix(za[i], 0.3, 0)
        qx, qy, I = O.kinematical_pattern(refl, m, LAM, 0.02, 1e-3)
        mt = O.match_pattern(plan, qx, qy, I)
        assert mt.za == i
        C = mt.C[i]
        fold = gold[name]
        if fold > 1:
            np.testing.assert_allclose(C, np.roll(C, N // fold), atol=1e-9 * C.max())
        top = np.sort(C)[::-1]
        n_max = int(np.sum(C >= C.max() * (1 - 1e-9)))
        assert n_max == fold, (name, n_max)


# ------------------------------------------------------------- refinement --

def test_parabolic_offset_exact_on_parabola():
    for x0 in (-0.5, -0.31, 0.0, 0.2, 0.49):
        c = [5.0 - 2.0 * (t - x0) ** 2 for t in (-1, 0, 1)]
        assert O.parabolic_offset(*c) == pytest.approx(x0, abs=1e-14)
    assert O.parabolic_offset(1.0, 1.0, 1.0) == 0.0          # flat: no shift
    assert O.parabolic_offset(0.0, 1.0, 1.5) == 0.5          # clamped


def test_rotation_between_and_refined_axis():
    rng = np.random.default_rng(9)
    for _ in range(10):
        u, v = rng.normal(size=3), rng.normal(size=3)
        u /= np.linalg.norm(u)
        v /= np.linalg.norm(v)
        R = O.rotation_between(u, v)
        np.testing.assert_allclose(R @ u, v, atol=1e-12)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)
        axis = np.cross(u, v)
        np.testing.assert_allclose(R @ axis, axis, atol=1e-12)


def test_refinement_reduces_offgrid_error(c1_plan):
    """A pattern between grid points is refined closer to the truth than
    the grid result, on average."""
    refl = au_reflections()
    ops = O.proper_point_group("cubic")
    rng = np.random.default_rng(12)
    za = c1_plan.za
    nb = O.za_neighbours(za, 2.0)
    grid_err, ref_err = [], []
    N = c1_plan.params.n_phi
    for z in rng.choice(np.arange(30, len(za)), 10, replace=False):
        w = za[z] + 0.012 * rng.normal(size=3)
        w /= np.linalg.norm(w)
        phi3 = -2 * math.pi * (rng.integers(N) + rng.uniform(-0.5, 0.5)) / N
        m = O.orientation_matrix(w, phi3, 0)
        mt = O.match_pattern(c1_plan, *O.kinematical_pattern(refl, m, LAM, 0.02, 1e-3))
        mg = O.orientation_matrix(za[mt.za], -2 * math.pi * mt.k / N, mt.mirror)
        rf = O.refine(mt, za, 2.0, nb)
        grid_err.append(O.misorientation_deg(mg, m, ops, True))
        ref_err.append(O.misorientation_deg(rf.m, m, ops, True))
    assert np.mean(ref_err) < np.mean(grid_err)


# ---------------------------------------------------------- several phases --

@pytest.fixture(scope="module")
def two_phase_plans():
    """fcc Au (cubic triangle) and hcp Mg (hexagonal triangle) plans on 6-degree
    grids with the same shells, bins and tent, so one polar image serves both."""
    prm = O.PlanParams(n_shells=40, dq=0.0375, n_phi=72, delta=0.08, lam=LAM)
    v0, v1, v2, om = O.cubic_triangle()
    au = O.orientation_plan(au_reflections(), O.zone_axis_grid(v0, v1, v2, 6.0, om), prm)
    mg_refl = O.reflections(mg_lattice(), MG_POS, [12.0] * 2, [0.3] * 2, 1.5)
    v0, v1, v2, om = O.hexagonal_triangle()
    mg = O.orientation_plan(mg_refl, O.zone_axis_grid(v0, v1, v2, 6.0, om), prm)
    return (au, mg), (au_reflections(), mg_refl)


def test_multi_phase_self_indexing(two_phase_plans):
    """X := P_z of phase p scores exactly 1 in phase p (Cauchy-Schwarz with
    unit-norm slices) and strictly less in the other phase, whose slices all
    differ from it: the decision is p."""
    plans, _ = two_phase_plans
    rng = np.random.default_rng(11)
    for p in (0, 1):
        for z in rng.choice(len(plans[p].za), 4, replace=False):
            mm = O.match_multi_image(plans, plans[p].P[z])
            assert mm.phase == p
            assert abs(mm.phase_scores[p] - 1.0) < 1e-12
            assert mm.phase_scores[1 - p] < 1.0 - 1e-6
            assert mm.match is mm.matches[p]


def test_multi_phase_scores_are_brute_force_maxima(two_phase_plans):
    """Each phase's score is the maximum over that phase's axes, phi3 bins and
    mirror of the plain circular sums; the decision is the larger one."""
    plans, _ = two_phase_plans
    prm = plans[0].params
    rng = np.random.default_rng(12)
    q = rng.uniform(0.3, 1.4, 20)
    g = rng.uniform(-math.pi, math.pi, 20)
    X = O.polar_image(q * np.cos(g), q * np.sin(g), rng.uniform(1, 5, 20), prm)
    mm = O.match_multi_image(plans, X)
    best = []
    for p, plan in enumerate(plans):
        C, Cm = O.direct_correlation(plan.P, X)
        best.append(max(C.max(), Cm.max()))
        assert mm.phase_scores[p] == pytest.approx(best[p], rel=1e-12)
    assert mm.phase == int(np.argmax(best))


def test_multi_phase_tie_goes_to_lower_phase(two_phase_plans):
    (au, _), _ = two_phase_plans
    mm = O.match_multi_image([au, au], au.P[3])
    assert mm.phase == 0 and mm.phase_scores[0] == mm.phase_scores[1]


def test_multi_phase_noiseless_patterns_get_their_phase(two_phase_plans):
    """Noiseless kinematical patterns of either phase at grid orientations
    are assigned the phase they were generated from."""
    plans, refls = two_phase_plans
    rng = np.random.default_rng(13)
    for p in (0, 1):
        za = plans[p].za
        N = plans[p].params.n_phi
        for z in rng.choice(len(za), 6, replace=False):
            m = O.orientation_matrix(za[z], -2 * math.pi * int(rng.integers(N)) / N,
                                     int(rng.integers(2)))
            qx, qy, I = O.kinematical_pattern(refls[p], m, LAM, 0.02, 1e-3)
            assert O.match_multi(plans, qx, qy, I).phase == p, (p, z)


# ------------------------------------------------- continuous refinement --

def _rand_rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _score_case(seed):
    refl = au_reflections()
    rng = np.random.default_rng(seed)
    m = _rand_rot(rng)
    qx, qy, I = O.kinematical_pattern(refl, m, LAM, AU["sigma"], 1e-3)
    qx = qx + rng.normal(0, 0.005, len(qx))
    qy = qy + rng.normal(0, 0.005, len(qy))
    return refl, m, qx, qy, I * np.exp(0.1 * rng.normal(size=len(I)))


def test_score_gradient_matches_finite_differences():
    """dS/dw for R -> Exp(w) R against central differences of the score."""
    refl, m, qx, qy, I = _score_case(21)
    R = O.so3_exp([0.01, -0.015, 0.02]) @ m.T
    for rho in (0.02, 0.08):
        sc = O.kinematical_score(R, qx, qy, I, refl, LAM, 0.02, rho)
        h = 1e-6
        fd = np.array([(O.kinematical_score(O.so3_exp(h * e) @ R, qx, qy, I, refl, LAM, 0.02, rho).S
                        - O.kinematical_score(O.so3_exp(-h * e) @ R, qx, qy, I, refl, LAM, 0.02,
                                              rho).S) / (2 * h) for e in np.eye(3)])
        np.testing.assert_allclose(sc.grad, fd, rtol=1e-6, atol=1e-7 * np.abs(fd).max())


def test_score_axis_angle_gradient_matches_finite_differences():
    """dS/dr at r != 0, where the left Jacobian of SO(3) enters."""
    refl, m, qx, qy, I = _score_case(22)
    r = np.array([0.2, -0.1, 0.15])
    S, g = O.kinematical_score_r(r, m, qx, qy, I, refl, LAM, 0.02, 0.05)
    h = 1e-6
    fd = np.array([(O.kinematical_score_r(r + h * e, m, qx, qy, I, refl, LAM, 0.02, 0.05)[0]
                    - O.kinematical_score_r(r - h * e, m, qx, qy, I, refl, LAM, 0.02, 0.05)[0])
                   / (2 * h) for e in np.eye(3)])
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-7 * np.abs(fd).max())


def test_strain_score_reduces_to_the_score_at_zero_strain():
    """At e = 0 the strained score, its rotation gradient and Gauss-Newton
    matrix are those of the unstrained score."""
    refl, m, qx, qy, I = _score_case(23)
    R = O.so3_exp([0.01, 0.02, -0.01]) @ m.T
    a = O.kinematical_score(R, qx, qy, I, refl, LAM, 0.02, 0.05)
    b, _ = O.kinematical_score_strain(R, np.zeros(6), qx, qy, I, refl, LAM, 0.02, 0.05)
    assert b.S == pytest.approx(a.S, rel=1e-14)
    np.testing.assert_allclose(b.grad, a.grad, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(b.H, a.H, rtol=1e-12, atol=1e-14)


def test_strain_gradient_matches_finite_differences():
    """dS/de for the six strain components against central differences of
    the score, at zero and at a non-zero strain; the rotation gradient at
    non-zero strain against differences too."""
    refl, m, qx, qy, I = _score_case(24)
    R = O.so3_exp([-0.01, 0.015, 0.01]) @ m.T
    h = 1e-7
    for e0 in (np.zeros(6), np.array([2e-3, -1e-3, 5e-4, -1.5e-3, 1e-3, 3e-3])):
        sc, de = O.kinematical_score_strain(R, e0, qx, qy, I, refl, LAM, 0.02, 0.05)
        fd = np.array([(O.kinematical_score_strain(R, e0 + h * d, qx, qy, I, refl, LAM, 0.02,
                                                   0.05)[0].S
                        - O.kinematical_score_strain(R, e0 - h * d, qx, qy, I, refl, LAM, 0.02,
                                                     0.05)[0].S) / (2 * h) for d in np.eye(6)])
        np.testing.assert_allclose(de, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
        fw = np.array([(O.kinematical_score_strain(O.so3_exp(1e-6 * w) @ R, e0, qx, qy, I, refl,
                                                   LAM, 0.02, 0.05)[0].S
                        - O.kinematical_score_strain(O.so3_exp(-1e-6 * w) @ R, e0, qx, qy, I,
                                                     refl, LAM, 0.02, 0.05)[0].S) / 2e-6
                       for w in np.eye(3)])
        np.testing.assert_allclose(sc.grad, fw, rtol=1e-6, atol=1e-7 * np.abs(fw).max())


def test_strain_of_an_isotropic_scaling_moves_every_spot_radially():
    """e = t I scales every reflection by (1 + t): the strained score at R
    equals the unstrained score of the scaled reflection set."""
    refl, m, qx, qy, I = _score_case(25)
    R = m.T
    t = 4e-3
    sc, _ = O.kinematical_score_strain(R, np.array([t, 0, 0, t, 0, t]), qx, qy, I, refl, LAM, 0.02,
                                       0.05)
    # the scaled set keeps the unstrained amplitudes: scale g, then restore |g|^gamma
    scaled = O.Reflections(g=refl.g * (1 + t), hkl=refl.hkl, F=refl.F / (1 + t))
    ref = O.kinematical_score(R, qx, qy, I, scaled, LAM, 0.02, 0.05)
    assert sc.S == pytest.approx(ref.S, rel=1e-12)


def test_score_single_peak_single_reflection_closed_form():
    """One reflection and one peak: b / ||b|| = 1, so S = a exp(-|d|^2/2rho^2)."""
    g = np.array([[0.5, 0.2, 0.01]])
    refl = O.Reflections(g=g, hkl=np.zeros((1, 3)), F=np.array([7.0 + 0j]))
    R = O.so3_exp([0.1, 0.2, -0.3])
    v = R @ g[0]
    qx, qy, I = np.array([v[0] + 0.01]), np.array([v[1] - 0.02]), np.array([9.0])
    q = math.hypot(qx[0], qy[0])
    sc = O.kinematical_score(R, qx, qy, I, refl, LAM, 0.02, 0.03)
    assert sc.S == pytest.approx(q * 3.0 * math.exp(-(0.01 ** 2 + 0.02 ** 2) / (2 * 0.03 ** 2)),
                                 rel=1e-12)


def test_score_invariant_under_crystal_rotations():
    """R and R S give the same score for every proper rotation S of m-3m: the
    reflection set and |F| are invariant under the point group."""
    refl, m, qx, qy, I = _score_case(23)
    R = m.T
    base = O.kinematical_score(R, qx, qy, I, refl, LAM, 0.02, 0.03).S
    for S in O.proper_point_group("cubic")[:8]:
        assert O.kinematical_score(R @ S, qx, qy, I, refl, LAM, 0.02, 0.03).S == \
            pytest.approx(base, rel=1e-10)


def test_refinement_recovers_noiseless_orientations_and_their_twin():
    """Noiseless patterns at random (off-grid) orientations, started 1.5
    degrees off or from the Friedel twin of such a start: the refinement
    returns the true orientation, and the score picks it over the twin."""
    refl = au_reflections()
    ops = O.proper_point_group("cubic")
    prm = O.RefineParams()
    rng = np.random.default_rng(31)
    close = twin_ok = 0
    for _ in range(8):
        m = _rand_rot(rng)
        qx, qy, I = O.kinematical_pattern(refl, m, LAM, AU["sigma"], 1e-3)
        w = rng.normal(size=3)
        m0 = m @ O.so3_exp(w * math.radians(1.5) / np.linalg.norm(w))
        mr, _, _ = O.refine_with_twin(m0, qx, qy, I, refl, LAM, prm)
        close += O.misorientation_deg(mr, m, ops) < 0.05
        mt, _, chose_twin = O.refine_with_twin(m0 @ np.diag([-1.0, -1.0, 1.0]), qx, qy, I, refl,
                                               LAM, prm)
        twin_ok += chose_twin and O.misorientation_deg(mt, m, ops) < 0.05
    assert close >= 7 and twin_ok >= 7


# ------------------------------------------- several matches per pattern --

def test_delete_peaks_distances():
    """Removed within r_del, intensity times (d - r_del)/(delta - r_del) up to
    delta, unchanged beyond (hand-computed distances to one spot at the
    origin)."""
    spots = np.array([[0.0, 0.0]])
    qx = np.array([0.01, 0.05, 0.06, 0.2])
    qy = np.array([0.0, 0.0, 0.08, 0.0])          # distances 0.01, 0.05, 0.1, 0.2
    I = np.array([1.0, 2.0, 3.0, 4.0])
    x, y, i = O.delete_peaks(qx, qy, I, spots, r_del=0.04, delta=0.08)
    np.testing.assert_allclose(x, [0.05, 0.06, 0.2])
    np.testing.assert_allclose(i, [2.0 * (0.05 - 0.04) / 0.04, 3.0, 4.0])


@pytest.fixture(scope="module")
def au_6deg_plan():
    v0, v1, v2, om = O.cubic_triangle()
    za = O.zone_axis_grid(v0, v1, v2, 6.0, om)
    return O.orientation_plan(au_reflections(), za,
                              O.PlanParams(n_shells=40, dq=0.0375, n_phi=72, delta=0.08, lam=LAM))


def test_two_overlapping_grid_patterns_are_both_found(au_6deg_plan):
    """Peaks of two noiseless patterns at grid orientations, superimposed:
    two rounds of match and deletion return both orientations (up to the
    crystal's symmetry), each with the full pattern's correlation at it."""
    plan = au_6deg_plan
    refl = au_reflections()
    ops = O.proper_point_group("cubic")
    N = plan.params.n_phi
    rng = np.random.default_rng(41)
    found = 0
    for _ in range(4):
        zs = rng.choice(len(plan.za), 2, replace=False)
        ms = [O.orientation_matrix(plan.za[z], -2 * math.pi * int(rng.integers(N)) / N, 0)
              for z in zs]
        pats = [O.kinematical_pattern(refl, m, LAM, AU["sigma"], 1e-3) for m in ms]
        qx, qy, I = (np.concatenate([p[i] for p in pats]) for i in range(3))
        res = O.match_multiple(plan, refl, qx, qy, I, 2, r_del=0.04, lam=LAM, sigma=AU["sigma"])
        assert len(res) == 2
        got = [min(O.misorientation_deg(r.m, m, ops) for m in ms) for r in res]
        found += sum(g < 1e-3 for g in got)
        X = O.polar_image(qx, qy, I, plan.params)
        C, Cm = O.correlogram(plan.P_hat, X)
        for r in res:
            assert r.score == pytest.approx((Cm if r.mirror else C)[r.za, r.k], rel=1e-12)
    assert found >= 7


def test_single_pattern_second_match_is_weak(au_6deg_plan):
    """One noiseless pattern: after its peaks are deleted little or nothing
    is left, so a second match, if any, scores far below the first."""
    plan = au_6deg_plan
    refl = au_reflections()
    N = plan.params.n_phi
    m = O.orientation_matrix(plan.za[5], -2 * math.pi * 7 / N, 0)
    qx, qy, I = O.kinematical_pattern(refl, m, LAM, AU["sigma"], 1e-3)
    res = O.match_multiple(plan, refl, qx, qy, I, 3, r_del=0.04, lam=LAM, sigma=AU["sigma"])
    assert len(res) >= 1
    assert all(r.reduced_score < 0.2 * res[0].reduced_score for r in res[1:])


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("kind,order", [("cubic", 24), ("hexagonal", 12)])
def test_misorientation_metric_closed_forms(kind, order):
    """Reading R13 pinned by closed forms: the proper point groups O and 622
    have 24 and 12 distinct rotations and are closed under products; an
    orientation and any symmetry equivalent of it are 0 apart; a small extra
    rotation about any axis is its own angle apart (every non-identity
    operation of these groups turns by at least 60 degrees, more than twice
    the largest extra rotation tried); the in-plane Friedel twin m Rz(pi) is
    0 apart once reduced over the twin.  Zero
    angles are compared at 1e-4 degrees: the angle comes from acos of the
    trace, which near the identity turns rounding of order 1e-16 into about
    1e-6 degrees."""
    ops = O.proper_point_group(kind)
    assert len(ops) == order
    for S in ops:
        assert abs(np.linalg.det(S) - 1) < 1e-12
        np.testing.assert_allclose(S @ S.T, np.eye(3), atol=1e-12)
    keys = {tuple(np.round(S, 9).ravel()) for S in ops}
    assert len(keys) == order
    for A, B in itertools.product(ops, ops):
        assert tuple(np.round(A @ B, 9).ravel()) in keys
    rng = np.random.default_rng(13)
    for _ in range(6):
        m = _random_rotation(rng)
        for S in ops:
            assert O.misorientation_deg(S @ m, m, ops) < 1e-4
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        theta = math.radians(rng.uniform(0.1, 20.0))
        d = O.misorientation_deg(m @ O.so3_exp(theta * axis), m, ops)
        assert abs(d - math.degrees(theta)) < 1e-6
        assert O.misorientation_deg(m @ O.rot_z(math.pi), m, ops, True) < 1e-4


def test_bench_misorientation_equals_the_oracle_definition():
    """The vectorised metric the benchmark reports (host logic) equals the
    oracle's definition pattern by pattern: the mean misorientation, the
    mean reduced over the Friedel twin and the mean zone-axis tilt."""
    import bench
    rng = np.random.default_rng(21)
    ops = O.proper_point_group("cubic")
    truth = np.stack([_random_rotation(rng) for _ in range(12)])
    est = np.stack([t @ O.so3_exp(rng.normal(scale=0.3, size=3)) for t in truth])
    est[::3] = est[::3] @ O.rot_z(math.pi)          # some Friedel twins
    m, mt, tilt = bench.misorientation(est.astype(np.float32), truth, ops)
    ref = np.mean([O.misorientation_deg(e, t, ops) for e, t in zip(est, truth)])
    ref_t = np.mean([O.misorientation_deg(e, t, ops, True) for e, t in zip(est, truth)])
    ref_z = np.mean([O.za_tilt_error_deg(e, t, ops) for e, t in zip(est, truth)])
    assert abs(m - ref) < 1e-3 and abs(mt - ref_t) < 1e-3 and abs(tilt - ref_z) < 1e-3


# ------------------------------------------- zone-axis tilt error (R13) --

@pytest.mark.parametrize("kind", ["cubic", "hexagonal"])
def test_za_tilt_error_closed_forms(kind):
    """The paper's metric (the angle between estimated and true zone axes)
    against closed forms: tilting the sample by theta about an axis in the
    detector plane moves the beam direction by theta, so it reads theta
    (for theta below half the angle between the true axis and its nearest
    distinct symmetry equivalent, either sign, so that no other equivalent is
    closer); an in-plane rotation leaves the beam direction alone (0); a
    symmetry equivalent and the beam-reversing twin m Ry(pi) read 0."""
    ops = O.proper_point_group(kind)
    rng = np.random.default_rng(31)
    done = 0
    while done < 8:
        m = _random_rotation(rng)
        wt = m[:, 2]
        seps = [math.degrees(math.acos(min(1.0, abs(float(np.dot(S @ wt, wt))))))
                for S in ops]
        seps = [d for d in seps if d > 1e-6]
        if min(seps) < 12.0:
            continue                          # too close to a symmetry element
        a = rng.uniform(0, 2 * math.pi)
        axis = np.array([math.cos(a), math.sin(a), 0.0])
        for theta in (0.05, 0.7, 3.0, 5.5):
            t = O.za_tilt_error_deg(m @ O.so3_exp(math.radians(theta) * axis), m, ops)
            assert abs(t - theta) < 1e-6, (theta, t)
        assert O.za_tilt_error_deg(m @ O.rot_z(rng.uniform(-3, 3)), m, ops) < 1e-5
        for S in ops:
            assert O.za_tilt_error_deg(S @ m, m, ops) < 1e-5
        assert O.za_tilt_error_deg(m @ O.ROT_Y_PI, m, ops) < 1e-5
        done += 1


# ------------------------------------- sub-grid refinement (R14) closed forms --

def _synthetic_match(za_scores, N=12):
    """A match at axis 0, bin 0, direct, whose correlation of axis 0 peaks
    symmetrically at bin 0 (parabola offset 0)."""
    Z = len(za_scores)
    C = np.zeros((Z, N))
    C[:, 0] = za_scores
    C[:, 1] = C[:, -1] = 0.5 * np.asarray(za_scores)
    return O.Match(za=0, k=0, mirror=0, score=float(za_scores[0]), score_cos=0.0,
                   za_scores=np.asarray(za_scores, dtype=np.float64), C=C, Cm=np.zeros_like(C))


def _tilted(u, axis, ang):
    return O.so3_exp(math.radians(ang) * np.asarray(axis, dtype=np.float64)) @ u


def test_refine_neighbour_mean_closed_forms():
    """Reading R14 against closed forms.  (a) Four neighbours placed
    symmetrically about the grid axis with equal scores average to the grid
    axis itself.  (b) One neighbour v at angle alpha from the grid axis u,
    scores a (u) and b (v): the normalised weighted mean a u + b v lies in
    the plane of u and v at atan2(b sin alpha, a + b cos alpha) from u.
    (c) A neighbour scoring just below 0.9 of the best is left out, one just
    above is taken.  (d) An axis outside the grid neighbourhood never counts,
    whatever its score.  In every case the refined orientation is a rotation
    whose beam direction m z is the refined axis."""
    u = np.array([0.3, -0.2, 0.9])
    u /= np.linalg.norm(u)
    ex = np.cross(u, [1.0, 0, 0])
    ex /= np.linalg.norm(ex)
    ey = np.cross(u, ex)
    alpha = 1.7
    # (a)
    za = np.stack([u] + [_tilted(u, d, alpha) for d in (ex, -ex, ey, -ey)])
    rf = O.refine(_synthetic_match([1.0, 0.97, 0.97, 0.97, 0.97]), za, 2.0, [np.arange(5)])
    np.testing.assert_allclose(rf.w, u, atol=1e-12)
    # (b), (c), (d): u, v (tilted toward ey), a far axis with a higher score
    v = _tilted(u, ex, alpha)
    far = _tilted(u, ey, 40.0)
    za = np.stack([u, v, far])
    nb = [np.array([0, 1]), np.array([0, 1]), np.array([2])]
    for b, taken in ((0.95, True), (0.9 * (1 + 1e-9), True), (0.9 * (1 - 1e-9), False)):
        rf = O.refine(_synthetic_match([1.0, b, 5.0]), za, 2.0, nb)
        got = math.degrees(math.acos(min(1.0, float(np.dot(rf.w, u)))))
        a = math.radians(alpha)
        want = math.degrees(math.atan2(b * math.sin(a), 1.0 + b * math.cos(a))) if taken else 0.0
        assert abs(got - want) < 1e-9, (b, got, want)
        assert abs(float(np.dot(rf.w, np.cross(u, v)))) < 1e-12       # in the plane of u, v
        to_v = math.degrees(math.acos(min(1.0, float(np.dot(rf.w, v)))))
        assert abs(to_v - (alpha - want)) < 1e-9                      # between u and v
        np.testing.assert_allclose(rf.m @ np.array([0, 0, 1.0]), rf.w, atol=1e-12)
        np.testing.assert_allclose(rf.m.T @ rf.m, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(rf.m) - 1) < 1e-12
        assert rf.dk == 0.0 and rf.phi3 == 0.0


# ------------------------------------ forward model: shape factor and cut --

def test_shape_factor_gaussian_values():
    """Eq. 8: D(0) = 1, D(sigma) = exp(-1/2), D(sigma sqrt(2 ln 1000)) = 1e-3,
    even in s."""
    for sig in (0.02, 0.0015):
        assert O.shape_factor_gaussian(0.0, sig) == 1.0
        assert math.isclose(O.shape_factor_gaussian(sig, sig), math.exp(-0.5), rel_tol=1e-12)
        c = sig * math.sqrt(2 * math.log(1000.0))
        assert math.isclose(O.shape_factor_gaussian(c, sig), 1e-3, rel_tol=1e-12)
        assert O.shape_factor_gaussian(-c, sig) == O.shape_factor_gaussian(c, sig)


@pytest.mark.parametrize("sigma,shells", [(0.02, None), (0.0015, (4, 8))])
def test_forward_spots_cut_at_001(sigma, shells):
    """The forward pattern of the [001] orientation (m = I) holds exactly the
    reflections with D(s_g) >= 1e-3, i.e. |s_g| <= sigma sqrt(2 ln 1000).
    Closed form at [001]: a zero-order-Laue-zone reflection (g_z = 0, g
    perpendicular to the beam) has |s_g| = |g|^2 / (2 sqrt(1/lambda^2 +
    |g|^2)); every other one has |g_z| >= 1/a and |s_g| far above the cut.
    With sigma = 0.02 the cut keeps the whole zone; with sigma = 0.0015 it
    falls between the {220} and {400} rings (h^2 + k^2 + l^2 = 4 and 8 kept)."""
    refl = au_reflections()
    m = O.orientation_matrix(np.array([0, 0, 1.0]), 0.0, 0)
    np.testing.assert_allclose(m, np.eye(3), atol=1e-15)
    got = O.forward_spots(refl, m, LAM, sigma)
    cut = sigma * math.sqrt(2 * math.log(1000.0))
    hkl2 = (refl.hkl ** 2).sum(axis=1)
    zolz = refl.hkl[:, 2] == 0
    g2 = (refl.g[:, :2] ** 2).sum(axis=1)
    s_abs = g2 / (2 * np.sqrt(1 / LAM ** 2 + g2))
    want = zolz & (s_abs <= cut)
    if shells is not None:
        assert set(hkl2[want]) == set(shells)
    else:
        assert want.sum() == zolz.sum()
    exp_xy = refl.g[want, :2]
    assert len(got) == len(exp_xy)
    order = lambda a: a[np.lexsort((a[:, 1], a[:, 0]))]
    np.testing.assert_allclose(order(np.asarray(got)), order(exp_xy), atol=1e-12)


# --------------- the paper's kinematical accuracy experiment (loose check) --

def test_kinematical_accuracy_trend_with_k_max():
    """"ACOM of Kinematical Calculated Diffraction Patterns": the patterns the
    plan is built from (fcc Au, kinematical, at the grid's zone axes) matched
    against the plan give a mean zone-axis error of about 3 degrees at
    k_max = 1.0, about 0.3 degrees at 1.5 (ten times less), and another 2-3
    times less at 2.0.  A loose check of that trend on the 2-degree grid
    (231 axes, shells of 0.02 up to k_max, 180 bins, peaks above 1e-3 of the
    strongest): the error at 1.0 lies in the degrees regime (1 to 6), at 1.5
    below 0.5 degrees and at least 5 times below that at 1.0, and at 2.0 no
    larger than at 1.5.  Measured: 1.69, 0.068 and 0.024 degrees."""
    ops = O.proper_point_group("cubic")
    v0, v1, v2, om = O.cubic_triangle()
    za = O.zone_axis_grid(v0, v1, v2, 2.0, om)
    mean = {}
    for kmax in (1.0, 1.5, 2.0):
        refl = au_reflections(q_max=kmax)
        S = int(round(kmax / 0.02))
        plan = O.orientation_plan(refl, za, O.PlanParams(S, 0.02, 180, 0.08, lam=LAM))
        err = []
        for z in range(len(za)):
            m = O.orientation_matrix(za[z], 0.0, 0)
            mt = O.match_pattern(plan, *O.kinematical_pattern(refl, m, LAM, 0.02, 1e-3))
            me = O.orientation_matrix(za[mt.za], -2 * math.pi * mt.k / 180, mt.mirror)
            err.append(O.za_tilt_error_deg(me, m, ops))
        mean[kmax] = float(np.mean(err))
    print("mean zone-axis error by k_max:", mean)
    assert 1.0 < mean[1.0] < 6.0
    assert mean[1.5] < 0.5 and mean[1.0] >= 5.0 * mean[1.5]
    assert mean[2.0] <= mean[1.5]


# --------------------------------------- the paper's unique-radius shells --

def test_unique_radii_are_the_fcc_closed_form():
    """The paper's shells for Au at q_max 1.5: |g| = sqrt(n)/a for the n =
    h^2 + k^2 + l^2 < (1.5 a)^2 that fcc allows (h, k, l all even or all
    odd, not all zero): 3, 4, 8, 11, 12, 16, 19, 20, 24, 27, 32, 35, 36."""
    allowed = sorted({h * h + k * k + l * l
                      for h, k, l in itertools.product(range(-7, 8), repeat=3)
                      if (h % 2 == k % 2 == l % 2) and (h, k, l) != (0, 0, 0)
                      and h * h + k * k + l * l < (1.5 * A_AU) ** 2})
    assert allowed == [3, 4, 8, 11, 12, 16, 19, 20, 24, 27, 32, 35, 36]
    r = O.unique_shell_radii(au_reflections())
    np.testing.assert_allclose(r, np.sqrt(allowed) / A_AU, rtol=1e-12)


def test_paper_mode_plan_001_closed_form():
    """The paper's P0 at [001] over the unique radii: the {111} shell is empty
    (every {111} reflection has |g_z| = 1/a, far off the Ewald sphere); the
    {200} shell has the four in-plane spots at 0, 90, 180, 270 degrees, so at
    phi = 0 it equals q_s^gamma |F_200| (1 - |s_200| / delta) with |F_200| =
    4 f(|g|) and |s_200| = |g|^2 / (2 sqrt(1/lambda^2 + |g|^2)) (g
    perpendicular to the beam), and the shell is 4-fold symmetric."""
    refl = au_reflections()
    N, delta = 180, 0.08
    prm = O.paper_params(refl, N, delta)
    P0 = O.plan_slice_unique(refl, np.array([0, 0, 1.0]), prm)
    assert P0.shape == (13, N)
    assert np.all(P0[0] == 0.0)
    q = 2.0 / A_AU
    F = 4 * 79.0 * math.exp(-0.25 * q * q)
    s = q * q / (2 * math.sqrt(1 / LAM ** 2 + q * q))
    assert math.isclose(P0[1, 0], q * F * (1 - s / delta), rel_tol=1e-12)
    np.testing.assert_allclose(P0[1], np.roll(P0[1], N // 4), rtol=1e-12, atol=1e-12)
    assert P0[1, N // 8] == 0.0                       # 45 degrees: between the spots


def test_paper_mode_self_indexing_is_exact():
    """Cauchy-Schwarz holds for the paper's plan too: the image X := P_z
    correlates to exactly 1 with its own slice at phi3 bin 0 and to less with
    every other slice."""
    refl = au_reflections()
    v0, v1, v2, om = O.cubic_triangle()
    za = O.zone_axis_grid(v0, v1, v2, 6.0, om)
    prm = O.paper_params(refl, 72, 0.08)
    plan = O.orientation_plan(refl, za, prm, O.plan_slice_unique)
    for z in (0, len(za) // 2, len(za) - 1):
        mt = O.match_image(plan, plan.P[z])
        assert math.isclose(mt.score, 1.0, rel_tol=1e-12)
        assert mt.za_scores[z] == pytest.approx(1.0, rel=1e-12)
        others = np.delete(mt.za_scores, z)
        assert np.all(others < 1.0 - 1e-9)


def test_uniform_shells_keep_the_papers_argmax_on_grid_patterns():
    """Reading R3: the uniform shells the CUDA path uses against the paper's
    unique radii, on noiseless kinematical patterns at every zone axis of the
    2-degree grid with a random in-plane bin: both shell sets recover the
    generating (axis, bin) for most patterns, pick the same argmax for at
    least 90 % of them, and keep the mean zone-axis error below 0.3 degrees
    (measured: 220 of 231 identical; exact recoveries 213 for the paper's
    shells, 218 for uniform ones; 0.095 and 0.068 degrees)."""
    refl = au_reflections()
    ops = O.proper_point_group("cubic")
    v0, v1, v2, om = O.cubic_triangle()
    za = O.zone_axis_grid(v0, v1, v2, 2.0, om)
    plan_p = O.orientation_plan(refl, za, O.paper_params(refl, 180, 0.08), O.plan_slice_unique)
    plan_u = O.orientation_plan(refl, za, O.PlanParams(75, 0.02, 180, 0.08, lam=LAM))
    rng = np.random.default_rng(1)
    same = exact_p = exact_u = 0
    tilt_p, tilt_u = [], []
    for z in range(len(za)):
        k0 = int(rng.integers(180))
        m = O.orientation_matrix(za[z], -2 * math.pi * k0 / 180, 0)
        pat = O.kinematical_pattern(refl, m, LAM, 0.02, 1e-3)
        a, b = O.match_pattern(plan_p, *pat), O.match_pattern(plan_u, *pat)
        same += (a.za, a.k, a.mirror) == (b.za, b.k, b.mirror)
        exact_p += (a.za, a.k, a.mirror) == (z, k0, 0)
        exact_u += (b.za, b.k, b.mirror) == (z, k0, 0)
        for mt, acc in ((a, tilt_p), (b, tilt_u)):
            me = O.orientation_matrix(za[mt.za], -2 * math.pi * mt.k / 180, mt.mirror)
            acc.append(O.za_tilt_error_deg(me, m, ops))
    print(f"same argmax {same}/{len(za)}, exact paper {exact_p}, exact uniform {exact_u}, "
          f"tilt paper {np.mean(tilt_p):.3f} uniform {np.mean(tilt_u):.3f}")
    assert same >= 0.9 * len(za)
    assert exact_p >= 0.85 * len(za) and exact_u >= 0.85 * len(za)
    assert np.mean(tilt_p) < 0.3 and np.mean(tilt_u) < 0.3
