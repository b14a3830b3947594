"""FP64 CPU oracle for the sparse correlation match of arXiv 2111.00171
("Automated Crystal Orientation Mapping in py4DSTEM using Sparse Correlation
Matching").

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA path is checked against.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library itself
never calls it and has no CPU fallback.  It shares no code, table or constant
generator with the CUDA path.

Every step follows the paper's statement of the method in FP64 NumPy, in the
paper's order and notation; the FFT is a library primitive (numpy.fft), used
only where the paper itself uses a Fourier transform.  Readings of passages
where the paper is silent or ambiguous are marked "reading:" below.

Functions and the passages they follow
--------------------------------------
reciprocal_basis          Eq. 1 (Structure Factor Calculations)
reflections               Eqs. 2-4: lattice points inside q_max, F_hkl
electron_wavelength       relativistic electron wavelength (Calculation of
                          Kinematical Diffraction Patterns; formula not printed)
excitation_error          Eq. 6 with alpha = 0
shape_factor_gaussian     Eq. 8
rot_z, rot_x, euler_zxz   Eq. 10 (the paper's sign convention)
zone_axis_grid            "Generation of an Orientation Plan": SLERP grid
unique_shell_radii, plan_slice_unique
                          the paper's own shells (unique radii |g|, the sum
                          over {g : |g| = q_s}); the CUDA path and the other
                          functions here use uniform shells (reading R3)
za_frame                  inverse of the first two terms of Eq. 10
orientation_plan          P0, A and P = A P0 (Generation of an Orientation
                          Plan), then the FFT along phi3
polar_image               sparse polar image X (Correlation Pattern Matching)
correlogram               C and C_mirror (Correlation Pattern Matching)
direct_correlation        the same correlations as plain circular sums
best_match                maximum over (zone axis, phi3, mirror)
match_multi               several phases: one plan and one match per crystal
                          structure (ACOM Integration); phase decision (reading)
refine                    sub-grid refinement (the paper is silent; reading)
orientation_matrix        Eq. 9/10 composition of the result
kinematical_pattern       forward model (Calculation of Kinematical
                          Diffraction Patterns) used by the oracle's own pins
kinematical_score         continuous correlation of the peaks with the
                          kinematical pattern of an orientation (Eqs. 6, 8;
                          the paper refines on the grid only: reading), its
                          gradient and Gauss-Newton matrix
kinematical_score_strain  the same score with the reciprocal lattice deformed by a
                          small symmetric strain e (g -> (I + e) g, reading),
                          and dS/de beside dS/dw
refine_continuous         gradient ascent of that score from a grid match
refine_with_twin          the same from the match and from its in-plane
                          Friedel twin m Rz(pi), keeping the higher score
forward_spots, delete_peaks, match_multiple
                          several matches per pattern by iterative peak
                          deletion (Matching of Overlapping Diffraction
                          Patterns)
misorientation_deg        symmetry-reduced misorientation (reading)

Parity status: structure factors, plan, image, correlation and best match are
pinned by the tests under ``tests/test_oracle_pins.py`` (closed forms, brute
force, Cauchy-Schwarz self-indexing, grid recovery, symmetry, and the paper's
kinematical accuracy trend with k_max).  The paper fixes no formula for
``refine``, ``misorientation_deg`` or ``za_tilt_error_deg`` (readings): they
are pinned by closed forms instead (exact parabola vertex, Rodrigues
rotation, the neighbour mean's angle and threshold, point-group closure,
symmetry equivalents at zero angle, small rotations and tilts at their own
angle) and by noiseless off-grid patterns refined closer to the truth than
the grid on average.  The forward model's excitation cut (``forward_spots``)
is pinned by the zero-order-Laue-zone closed form at [001]; the paper's
unique-radius shells (``unique_shell_radii``, ``plan_slice_unique``) by the
fcc radius set, the [001] slice and self-indexing.  The strain gradient of
``kinematical_score_strain`` is pinned by central finite differences of the
score itself and by its reduction to ``kinematical_score`` at zero strain.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# --------------------------------------------------------------------------
# Structure factors (Structure Factor Calculations, Eqs. 1-4)
# --------------------------------------------------------------------------


def reciprocal_basis(lattice):
    """Eq. 1: a* = (b x c)/V, b* = (c x a)/V, c* = (a x b)/V, no 2*pi.

    ``lattice`` holds the real-space vectors a, b, c as rows (Angstrom); the
    result holds a*, b*, c* as rows (1/Angstrom).
    """
    a, b, c = (np.asarray(v, dtype=np.float64) for v in lattice)
    V = float(np.dot(a, np.cross(b, c)))
    return np.array([np.cross(b, c) / V, np.cross(c, a) / V, np.cross(a, b) / V])


@dataclass
class Reflections:
    hkl: np.ndarray   # int64 [G, 3], lexicographic (h, k, l) order
    g: np.ndarray     # float64 [G, 3], crystal Cartesian (1/Angstrom)
    F: np.ndarray     # complex128 [G]


def reflections(lattice, frac_pos, ff_A, ff_B, q_max, drop_extinct=True):
    """Eqs. 2-4: every reciprocal lattice point g_hkl = h a* + k b* + l c*
    with 0 < |g| < q_max, and its structure factor

        F_hkl = sum_n f_n(|g|) exp(-2 pi i (h,k,l) . p_n),

    with the single-Gaussian form factor f_n(q) = A_n exp(-B_n q^2) (q = |g|,
    no 2*pi).  The paper sizes the (h,k,l) search box from the shortest
    reciprocal vector; here the box is the rigorous one, |h| <= q_max |a|
    (since h = g . a), which contains every point of the sphere.

    reading: V_g is zero where F vanishes, and "non-zero reciprocal lattice
    points" are those with F != 0: with ``drop_extinct`` the reflections with
    |F| < 1e-9 max|F| are removed (this matters for omega = 0).
    """
    L = np.asarray(lattice, dtype=np.float64)
    rb = reciprocal_basis(L)
    n = [int(math.floor(q_max * np.linalg.norm(L[i]))) for i in range(3)]
    hkl = np.array([(h, k, l)
                    for h in range(-n[0], n[0] + 1)
                    for k in range(-n[1], n[1] + 1)
                    for l in range(-n[2], n[2] + 1)], dtype=np.int64)
    g = hkl.astype(np.float64) @ rb
    q = np.linalg.norm(g, axis=1)
    keep = (q > 0) & (q < q_max)
    hkl, g, q = hkl[keep], g[keep], q[keep]
    p = np.asarray(frac_pos, dtype=np.float64).reshape(-1, 3)
    A = np.asarray(ff_A, dtype=np.float64).reshape(-1)
    B = np.asarray(ff_B, dtype=np.float64).reshape(-1)
    F = np.zeros(len(hkl), dtype=np.complex128)
    for atom in range(len(p)):
        f_n = A[atom] * np.exp(-B[atom] * q * q)
        F += f_n * np.exp(-2j * np.pi * (hkl.astype(np.float64) @ p[atom]))
    if drop_extinct and len(F):
        live = np.abs(F) >= 1e-9 * np.abs(F).max()
        hkl, g, F = hkl[live], g[live], F[live]
    return Reflections(hkl=hkl, g=g, F=F)


# --------------------------------------------------------------------------
# Kinematical diffraction (Calculation of Kinematical Diffraction Patterns)
# --------------------------------------------------------------------------


def electron_wavelength(kV):
    """Relativistically corrected electron wavelength in Angstrom:
    lambda = h / sqrt(2 m0 e V (1 + e V / (2 m0 c^2)))  (CODATA constants)."""
    h = 6.62607015e-34
    m0 = 9.1093837015e-31
    e = 1.602176634e-19
    c = 299792458.0
    V = kV * 1e3
    return h / math.sqrt(2 * m0 * e * V * (1 + e * V / (2 * m0 * c * c))) * 1e10


def beam_vector(lam):
    """reading: the wavevector points along -z (beam antiparallel to the zone
    axis, which is +z after the plan rotation), |k| = 1/lambda."""
    return np.array([0.0, 0.0, -1.0 / lam])


def excitation_error(g, k):
    """Eq. 6 with alpha = 0: s_g = -g.(2k + g) / (2 |k + g|)."""
    g = np.asarray(g, dtype=np.float64)
    return -np.einsum('...i,...i->...', g, 2 * k + g) / (
        2 * np.linalg.norm(k + g, axis=-1))


def shape_factor_gaussian(s, sigma):
    """Eq. 8: D = exp(-s^2 / (2 sigma^2))."""
    return np.exp(-(s * s) / (2 * sigma * sigma))


# --------------------------------------------------------------------------
# Orientations (Generation of an Orientation Plan, Eqs. 9-10)
# --------------------------------------------------------------------------


def rot_z(phi):
    """First (and third) factor of Eq. 10."""
    c, s = math.cos(phi), math.sin(phi)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_x(theta):
    """Middle factor of Eq. 10, with the paper's signs (+S2 above the
    diagonal)."""
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, s], [0.0, -s, c]])


def euler_zxz(phi1, theta2, phi3):
    """Eq. 10: m = Rz(phi1) Rx(theta2) Rz(phi3); d = m d0 (Eq. 9) maps sample
    coordinates to crystal coordinates."""
    return rot_z(phi1) @ rot_x(theta2) @ rot_z(phi3)


def za_angles(w):
    """(phi1, theta2) with Rz(phi1) Rx(theta2) z_hat = w: the third column of
    Rz(phi1) Rx(theta2) is (-S1 S2, C1 S2, C2)."""
    w = np.asarray(w, dtype=np.float64)
    w = w / np.linalg.norm(w)
    theta2 = math.acos(max(-1.0, min(1.0, w[2])))
    phi1 = math.atan2(-w[0], w[1])
    return phi1, theta2


def za_frame(w):
    """The rotation made of the first two terms of Eq. 10 for zone axis w;
    its inverse (transpose) brings crystal vectors into the zone-axis frame."""
    phi1, theta2 = za_angles(w)
    return rot_z(phi1) @ rot_x(theta2)


def slerp(p0, p1, t):
    """Spherical linear interpolation between unit vectors (Shoemake 1985)."""
    p0 = np.asarray(p0, dtype=np.float64)
    p1 = np.asarray(p1, dtype=np.float64)
    om = math.acos(max(-1.0, min(1.0, float(np.dot(p0, p1)))))
    if om < 1e-15:
        return p0.copy()
    return (math.sin((1 - t) * om) * p0 + math.sin(t * om) * p1) / math.sin(om)


def zone_axis_grid(v0, v1, v2, step_deg, solid_angle):
    """Zone-axis grid spanning the three boundary vectors by SLERP
    (Generation of an Orientation Plan).

    reading (the paper gives no point rule): n = floor(sqrt(2 Omega)/step)
    subdivisions, Omega the solid angle of the symmetry-reduced triangle; the
    points are, for i = 0..n and j = 0..i, a = slerp(v0, v1, i/n),
    b = slerp(v0, v2, i/n), w = slerp(a, b, j/i) (w = v0 for i = 0), in that
    (i, j) order.  Returns float64 [Z, 3] unit vectors.
    """
    v0, v1, v2 = (np.asarray(v, dtype=np.float64) / np.linalg.norm(v)
                  for v in (v0, v1, v2))
    n = int(math.floor(math.sqrt(2.0 * solid_angle) / math.radians(step_deg)))
    n = max(n, 1)
    pts = []
    for i in range(n + 1):
        if i == 0:
            pts.append(v0.copy())
            continue
        a = slerp(v0, v1, i / n)
        b = slerp(v0, v2, i / n)
        for j in range(i + 1):
            w = slerp(a, b, j / i)
            pts.append(w / np.linalg.norm(w))
    return np.array(pts)


def cubic_triangle():
    """[001], [011], [111] and the solid angle 4 pi / 48 of the m-3m
    standard triangle (Generation of an Orientation Plan, Fig. 1d)."""
    return (np.array([0.0, 0.0, 1.0]), np.array([0.0, 1.0, 1.0]) / math.sqrt(2),
            np.array([1.0, 1.0, 1.0]) / math.sqrt(3), 4 * math.pi / 48)


def hexagonal_triangle():
    """reading: [0001], the a axis and the direction 30 degrees from it in
    the basal plane bound the 1/24-sphere region of 6/mmm."""
    return (np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0]),
            np.array([math.cos(math.pi / 6), math.sin(math.pi / 6), 0.0]),
            4 * math.pi / 24)


# --------------------------------------------------------------------------
# Orientation plan (Generation of an Orientation Plan)
# --------------------------------------------------------------------------


def wrap_angle(x):
    """mod(x + pi, 2 pi) - pi with floor-mod, as in the plan and image
    expressions."""
    return np.mod(x + np.pi, 2 * np.pi) - np.pi


@dataclass
class PlanParams:
    n_shells: int
    dq: float            # uniform shells q_s = (s + 1) dq
    n_phi: int           # N in-plane bins phi_j = 2 pi j / N
    delta: float         # correlation kernel size
    gamma_pow: float = 1.0
    omega: float = 1.0
    lam: float = 0.01969
    radii: np.ndarray = None   # the paper's shells (unique_shell_radii); None: uniform

    def shells(self):
        if self.radii is not None:
            return np.asarray(self.radii, dtype=np.float64)
        return (np.arange(self.n_shells, dtype=np.float64) + 1.0) * self.dq

    def phis(self):
        return 2 * np.pi * np.arange(self.n_phi, dtype=np.float64) / self.n_phi


@dataclass
class Plan:
    za: np.ndarray        # [Z, 3]
    P: np.ndarray         # [Z, S, N] normalised plan, real
    P_hat: np.ndarray     # [Z, S, N//2+1] FFT along phi3
    A: np.ndarray         # [Z] normalisation
    params: PlanParams


def plan_slice(refl: Reflections, w, prm: PlanParams):
    """P0 for one zone axis w:

        P0(s, j) = sum_g q_s^gamma |V_g|^omega
                   max{1 - (1/delta) sqrt(rho_term + s_g^2
                                          + wrap(phi_j - gamma_g)^2 q_s^2), 0}

    with g' = R^T g (R the first two terms of Eq. 10 for w), s_g from Eq. 6
    at the beam of ``beam_vector``, gamma_g = atan2(g'_y, g'_x).

    reading (uniform shells): the paper sums over {g : |g| = q_s} at the
    unique radii.  With uniform shells q_s = (s+1) dq no g lies on a shell, so
    the radial distance enters the tent exactly as in the image expression:
    rho_term = (rho_g - q_s)^2, rho_g = sqrt(g'_x^2 + g'_y^2), and every g
    contributes to every shell where the tent is positive.
    """
    R = za_frame(w)
    gp = refl.g @ R                      # rows: (R^T g)^T
    k = beam_vector(prm.lam)
    s_g = excitation_error(gp, k)
    rho = np.hypot(gp[:, 0], gp[:, 1])
    gam = np.arctan2(gp[:, 1], gp[:, 0])
    amp = np.abs(refl.F) ** prm.omega
    q_s = prm.shells()
    phi = prm.phis()
    # only reflections whose tent can be positive (|s_g| < delta) contribute
    live = np.abs(s_g) < prm.delta
    P0 = np.zeros((prm.n_shells, prm.n_phi))
    for gi in np.nonzero(live)[0]:
        dphi = wrap_angle(phi[None, :] - gam[gi])                     # [1, N]
        arg = ((rho[gi] - q_s[:, None]) ** 2 + s_g[gi] ** 2
               + dphi ** 2 * q_s[:, None] ** 2)                       # [S, N]
        tent = np.maximum(1.0 - np.sqrt(arg) / prm.delta, 0.0)
        P0 += (q_s[:, None] ** prm.gamma_pow) * amp[gi] * tent
    return P0


def unique_shell_radii(refl: Reflections, rtol=1e-9):
    """The paper's shells (Generation of an Orientation Plan): the distinct
    lengths |g| of the reflections, ascending.  Lengths within ``rtol``
    (relative) of each other are one radius (rounding of the lattice sums).
    reading R2: the extinct reflections are not among them."""
    q = np.sort(np.linalg.norm(refl.g, axis=1))
    out = [q[0]]
    for v in q[1:]:
        if v > out[-1] * (1.0 + rtol):
            out.append(v)
    return np.array(out)


def paper_params(refl: Reflections, n_phi, delta, gamma_pow=1.0, omega=1.0, lam=0.01969):
    """PlanParams whose shells are the paper's unique radii of ``refl``."""
    radii = unique_shell_radii(refl)
    return PlanParams(len(radii), float('nan'), n_phi, delta, gamma_pow, omega, lam, radii)


def plan_slice_unique(refl: Reflections, w, prm: PlanParams, rtol=1e-9):
    """P0 for one zone axis w as the paper prints it (Generation of an
    Orientation Plan), over the unique radii q_s = prm.radii:

        P0(s, j) = sum_{g : |g| = q_s} q_s^gamma |V_g|^omega
                   max{1 - (1/delta) sqrt(s_g^2 + wrap(phi_j - gamma_g)^2 q_s^2), 0}

    g' = R^T g, s_g from Eq. 6, gamma_g = atan2(g'_y, g'_x) as in plan_slice;
    each reflection belongs to the one shell of its own length and has no
    radial term."""
    R = za_frame(w)
    gp = refl.g @ R
    s_g = excitation_error(gp, beam_vector(prm.lam))
    gam = np.arctan2(gp[:, 1], gp[:, 0])
    amp = np.abs(refl.F) ** prm.omega
    qg = np.linalg.norm(refl.g, axis=1)
    q_s = prm.shells()
    phi = prm.phis()
    P0 = np.zeros((len(q_s), prm.n_phi))
    for gi in range(len(qg)):
        on = np.nonzero(np.abs(q_s - qg[gi]) <= rtol * qg[gi])[0]
        if len(on) == 0:
            continue
        s = on[0]
        dphi = wrap_angle(phi - gam[gi])
        tent = np.maximum(1.0 - np.sqrt(s_g[gi] ** 2 + dphi ** 2 * q_s[s] ** 2) / prm.delta, 0.0)
        P0[s] += q_s[s] ** prm.gamma_pow * amp[gi] * tent
    return P0


def orientation_plan(refl: Reflections, za, prm: PlanParams, slice_fn=None):
    """P = A P0 with A = 1/sqrt(sum_{phi3, q_s} P0^2) (A = 0 for an empty
    slice), then the 1D Fourier transform along phi3 (numpy rfft: sum_j
    P_j exp(-2 pi i f j / N)).  P0 per zone axis from ``slice_fn``: plan_slice
    (uniform shells, the default) or plan_slice_unique (the paper's unique
    radii, with prm from paper_params)."""
    slice_fn = plan_slice if slice_fn is None else slice_fn
    za = np.asarray(za, dtype=np.float64)
    Z = len(za)
    P = np.zeros((Z, prm.n_shells, prm.n_phi))
    A = np.zeros(Z)
    for z in range(Z):
        P0 = slice_fn(refl, za[z], prm)
        nrm = math.sqrt(float(np.sum(P0 * P0)))
        A[z] = 1.0 / nrm if nrm > 0 else 0.0
        P[z] = A[z] * P0
    P_hat = np.fft.rfft(P, axis=2)
    return Plan(za=za, P=P, P_hat=P_hat, A=A, params=prm)


# --------------------------------------------------------------------------
# Correlation pattern matching
# --------------------------------------------------------------------------


def polar_image(qx, qy, I, prm: PlanParams):
    """Sparse polar image

        X(phi_j, q_s) = sum_{m : |q_m - q_s| < delta} q_m^gamma I_m^(omega/2)
                        max{1 - (1/delta) sqrt((q_m - q_s)^2
                                     + wrap(phi_j - gamma_m)^2 q_s^2), 0}

    with q_m = sqrt(qx^2 + qy^2), gamma_m = atan2(qy, qx).  Returns [S, N].
    reading: negative intensities weigh 0 for omega > 0; I^0 = 1.
    """
    qx = np.asarray(qx, dtype=np.float64)
    qy = np.asarray(qy, dtype=np.float64)
    I = np.asarray(I, dtype=np.float64)
    q_m = np.hypot(qx, qy)
    g_m = np.arctan2(qy, qx)
    wgt = q_m ** prm.gamma_pow * np.maximum(I, 0.0) ** (prm.omega / 2.0)
    q_s = prm.shells()
    phi = prm.phis()
    X = np.zeros((prm.n_shells, prm.n_phi))
    for m in range(len(q_m)):
        band = np.abs(q_m[m] - q_s) < prm.delta
        if not band.any():
            continue
        qs = q_s[band][:, None]
        dphi = wrap_angle(phi[None, :] - g_m[m])
        arg = (q_m[m] - qs) ** 2 + dphi ** 2 * qs ** 2
        X[band] += wgt[m] * np.maximum(1.0 - np.sqrt(arg) / prm.delta, 0.0)
    return X


def correlogram(P_hat, X):
    """C(z, phi3)   = sum_s IFFT{ FFT{P}^* FFT{X} }
       C_mirror     = sum_s IFFT{ FFT{P}^* FFT{X}^* }
    along phi3 (Correlation Pattern Matching).  ``P_hat`` [Z, S, F] is the
    plan's rfft, X [S, N] the polar image; returns (C, C_mirror) [Z, N]."""
    N = X.shape[-1]
    X_hat = np.fft.rfft(X, axis=-1)                       # [S, F]
    Pc = np.conj(P_hat)
    C = np.fft.irfft(np.einsum('zsf,sf->zf', Pc, X_hat), n=N, axis=-1)
    Cm = np.fft.irfft(np.einsum('zsf,sf->zf', Pc, np.conj(X_hat)), n=N, axis=-1)
    return C, Cm


def direct_correlation(P, X):
    """The same two correlations written as circular sums (no FFT):
       C[z, k]        = sum_s sum_j P[z, s, j] X[s, (j + k) mod N]
       C_mirror[z, k] = sum_s sum_j P[z, s, j] X[s, (-j - k) mod N]."""
    Z, S, N = P.shape
    C = np.zeros((Z, N))
    Cm = np.zeros((Z, N))
    j = np.arange(N)
    for k in range(N):
        C[:, k] = np.einsum('zsj,sj->z', P, X[:, (j + k) % N])
        Cm[:, k] = np.einsum('zsj,sj->z', P, X[:, (-j - k) % N])
    return C, Cm


@dataclass
class Match:
    za: int
    k: int
    mirror: int
    score: float            # raw correlation value at the best (za, k, mirror)
    score_cos: float        # score / ||X||_2 (<= 1 because ||P_z|| = 1)
    za_scores: np.ndarray   # [Z] max over k and mirror
    C: np.ndarray           # [Z, N]
    Cm: np.ndarray          # [Z, N]


def best_match(C, Cm, X=None):
    """For each zone axis the larger of C and C_mirror, maximised over phi3;
    the best zone axis is the global maximum (Correlation Pattern Matching).

    reading (tie rule): exact ties go to the lowest zone-axis index, then the
    direct correlation before the mirror, then the lowest phi3 bin.
    """
    Z, N = C.shape
    stacked = np.stack([C, Cm], axis=1).reshape(Z * 2 * N)   # order (z, mir, k)
    idx = int(np.argmax(stacked))
    z, rem = divmod(idx, 2 * N)
    mir, k = divmod(rem, N)
    score = float(stacked[idx])
    xn = float(np.sqrt(np.sum(X * X))) if X is not None else float('nan')
    return Match(za=z, k=k, mirror=mir, score=score,
                 score_cos=score / xn if xn > 0 else 0.0,
                 za_scores=np.maximum(C.max(axis=1), Cm.max(axis=1)),
                 C=C, Cm=Cm)


def match_image(plan: Plan, X):
    C, Cm = correlogram(plan.P_hat, X)
    return best_match(C, Cm, X)


def match_pattern(plan: Plan, qx, qy, I):
    return match_image(plan, polar_image(qx, qy, I, plan.params))


# --------------------------------------------------------------------------
# Several phases (ACOM Integration)
# --------------------------------------------------------------------------


@dataclass
class MultiMatch:
    phase: int                 # the phase decision
    match: Match               # that phase's best (zone-axis index within the phase)
    phase_scores: np.ndarray   # [n_phases] best raw correlation of each phase
    matches: list              # every phase's Match


def match_multi_image(plans, X):
    """Match a polar image against the plan of every phase (ACOM Integration:
    with several crystal structures, a plan and a correlation match per
    structure).

    reading (phase decision): the phase whose plan gives the highest raw
    correlation.  Every slice of every plan has unit norm, so the scores of
    different phases are comparable; an exact tie goes to the lower phase
    index.  The plans must share shells, bins and image exponents, so one
    polar image serves them all."""
    p0 = plans[0].params
    for p in plans[1:]:
        q = p.params
        assert (q.n_shells, q.dq, q.n_phi, q.delta, q.gamma_pow, q.omega) == \
            (p0.n_shells, p0.dq, p0.n_phi, p0.delta, p0.gamma_pow, p0.omega)
    ms = [match_image(p, X) for p in plans]
    sc = np.array([m.score for m in ms])
    ph = int(np.argmax(sc))        # the first maximum: lower phase on ties
    return MultiMatch(phase=ph, match=ms[ph], phase_scores=sc, matches=ms)


def match_multi(plans, qx, qy, I):
    return match_multi_image(plans, polar_image(qx, qy, I, plans[0].params))


# --------------------------------------------------------------------------
# Sub-grid refinement and the orientation matrix (paper silent; reading)
# --------------------------------------------------------------------------


def parabolic_offset(c_minus, c0, c_plus):
    """Vertex of the parabola through (-1, c-), (0, c0), (1, c+):
    dk = (c- - c+) / (2 (c- - 2 c0 + c+)), clamped to [-1/2, 1/2]; 0 when the
    three points are not concave."""
    den = c_minus - 2.0 * c0 + c_plus
    if not den < 0.0:
        return 0.0
    return float(min(0.5, max(-0.5, (c_minus - c_plus) / (2.0 * den))))


def za_neighbours(za, step_deg):
    """Zone axes within 1.5 grid steps of each other (reading: the grid
    neighbourhood used for refinement).  Returns a list of index arrays."""
    za = np.asarray(za, dtype=np.float64)
    cosang = np.clip(za @ za.T, -1.0, 1.0)
    lim = math.cos(math.radians(1.5 * step_deg))
    return [np.nonzero(cosang[z] >= lim)[0] for z in range(len(za))]


def rotation_between(u, v):
    """Smallest rotation taking unit vector u to unit vector v (Rodrigues)."""
    u = np.asarray(u, dtype=np.float64) / np.linalg.norm(u)
    v = np.asarray(v, dtype=np.float64) / np.linalg.norm(v)
    ax = np.cross(u, v)
    s = np.linalg.norm(ax)
    c = float(np.dot(u, v))
    if s < 1e-15:
        return np.eye(3)
    ax = ax / s
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    return np.eye(3) + s * K + (1 - c) * (K @ K)


ROT_Y_PI = np.diag([-1.0, 1.0, -1.0])


def orientation_matrix(w, phi3, mirror):
    """reading: a direct match at (w, phi3) is m = R(w) Rz(phi3) with R(w) the
    first two terms of Eq. 10; a mirror match is m = R(w) Rz(phi3) Ry(pi)
    (the pattern of m Ry(pi) is the y -> -y mirror of the pattern of m, by
    Friedel's law).  The in-plane angle of bin k is phi3 = -2 pi k / N."""
    m = za_frame(w) @ rot_z(phi3)
    if mirror:
        m = m @ ROT_Y_PI
    return m


@dataclass
class Refined:
    phi3: float
    dk: float
    w: np.ndarray
    m: np.ndarray


def refine(match: Match, za, step_deg, nbrs=None):
    """reading (the paper reports grid results only): phi3 from the parabola
    through the best bin and its two circular neighbours of the chosen
    (direct or mirror) correlation; the zone axis as the score-weighted mean
    of the best zone axis and its grid neighbours whose score is at least
    0.9 of the best, renormalised; the orientation is then tilted by the
    smallest rotation taking the best grid axis to the refined axis."""
    za = np.asarray(za, dtype=np.float64)
    Cz = (match.Cm if match.mirror else match.C)[match.za]
    N = len(Cz)
    k = match.k
    dk = parabolic_offset(Cz[(k - 1) % N], Cz[k], Cz[(k + 1) % N])
    phi3 = -2.0 * math.pi * (k + dk) / N
    if nbrs is None:
        nbrs = za_neighbours(za, step_deg)
    best = match.za_scores[match.za]
    acc = np.zeros(3)
    for z2 in nbrs[match.za]:
        sc = match.za_scores[z2]
        if sc >= 0.9 * best:
            acc += sc * za[z2]
    w_ref = acc / np.linalg.norm(acc) if np.linalg.norm(acc) > 0 else za[match.za]
    m = rotation_between(za[match.za], w_ref) @ orientation_matrix(
        za[match.za], phi3, match.mirror)
    return Refined(phi3=phi3, dk=dk, w=w_ref, m=m)


# --------------------------------------------------------------------------
# Forward model for the oracle's own pins
# --------------------------------------------------------------------------


def kinematical_pattern(refl: Reflections, m, lam, sigma, rel_threshold=0.0):
    """Kinematical pattern of orientation m (Calculation of Kinematical
    Diffraction Patterns): g_lab = m^T g, s_g by Eq. 6, intensity
    |F|^2 D(s_g) with the Gaussian D of Eq. 8, position (g_lab_x, g_lab_y).
    Peaks below ``rel_threshold`` of the strongest are dropped."""
    gl = refl.g @ np.asarray(m, dtype=np.float64)        # rows (m^T g)^T
    s = excitation_error(gl, beam_vector(lam))
    I = np.abs(refl.F) ** 2 * shape_factor_gaussian(s, sigma)
    keep = I > rel_threshold * I.max()
    return gl[keep, 0], gl[keep, 1], I[keep]


# --------------------------------------------------------------------------
# Continuous refinement (reading: the paper stops at the grid and its
# sub-grid refinement; this score makes the orientation a continuous variable)
# --------------------------------------------------------------------------


def so3_exp(w):
    """Rotation by the angle |w| about w / |w| (Rodrigues' formula)."""
    w = np.asarray(w, dtype=np.float64)
    t = float(np.linalg.norm(w))
    K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    if t < 1e-12:
        return np.eye(3) + K
    return np.eye(3) + math.sin(t) / t * K + (1 - math.cos(t)) / (t * t) * (K @ K)


def peak_weights(qx, qy, I, gamma_pow, omega):
    """a_m = q_m^gamma I_m^(omega/2), the weight of a peak in the polar image
    (negative intensities weigh 0 for omega > 0; I^0 = 1)."""
    q = np.hypot(qx, qy)
    I = np.asarray(I, dtype=np.float64)
    Iw = np.where(I > 0, np.abs(I) ** (omega / 2), 0.0) if omega > 0 else np.ones_like(I)
    return q ** gamma_pow * Iw


@dataclass
class Score:
    S: float
    grad: np.ndarray     # [3] dS/dw for R -> Exp(w) R at w = 0
    H: np.ndarray        # [3, 3] Gauss-Newton approximation of -d2S/dw2


def kinematical_score(R, qx, qy, I, refl: Reflections, lam, sigma, rho, gamma_pow=1.0,
                      omega=1.0):
    """Continuous kinematical correlation of a pattern with orientation R
    (crystal to lab, R = m^T):

        S = sum_m sum_g a_m b_g exp(-|p_m - (R g)_xy|^2 / (2 rho^2)) / ||b||

    a_m = q_m^gamma I_m^(omega/2) the peak weight of the polar image, b_g =
    |g|^gamma |F_g|^omega D(s_g)^(omega/2) the same weight for the kinematical
    intensity |F_g|^2 D(s_g) of reflection g (D the Gaussian shape factor of
    Eq. 8, s_g the excitation error of R g by Eq. 6, beam along -z), p_m the
    peak position.  reading: the plan's correlation with its slice normalised
    to unit norm (Generation of an Orientation Plan), the tent replaced by a
    Gaussian of width rho in the detector plane and the excitation error kept
    exact; by Cauchy-Schwarz it is largest where b is proportional to the
    observed weights.

    The gradient is taken for a rotation w applied in the lab frame:
    d(R g)/dw_j = e_j x (R g), so dS/dw = sum_g (R g) x dS/d(R g).  H adds,
    for each product of two Gaussian factors, the outer products of the
    derivatives of their arguments (position: (R g)_x and (R g)_y over rho^2;
    excitation: s_g over sigma_e^2 = 2 sigma^2 / omega), weighted by the
    product, over ||b||."""
    v = refl.g @ np.asarray(R, dtype=np.float64).T            # [G, 3] rows R g
    k = beam_vector(lam)
    kv = k + v
    nkv = np.linalg.norm(kv, axis=1)
    s = excitation_error(v, k)
    ds_dv = -kv * ((nkv + s) / (nkv * nkv))[:, None]          # derivative of Eq. 6
    gn = np.linalg.norm(refl.g, axis=1)
    # D^(omega/2) is a Gaussian in s of variance se2 = 2 sigma^2 / omega
    se2 = 2 * sigma * sigma / omega if omega > 0 else math.inf
    b = gn ** gamma_pow * np.abs(refl.F) ** omega * np.exp(-(s * s) / (2 * se2))
    nb = float(np.sqrt(np.sum(b * b)))
    if nb == 0.0:
        return Score(0.0, np.zeros(3), np.zeros((3, 3)))
    db_dv = (-s / se2 * b)[:, None] * ds_dv                     # [G, 3]
    a = peak_weights(qx, qy, I, gamma_pow, omega)
    p = np.stack([np.asarray(qx, np.float64), np.asarray(qy, np.float64)], axis=1)
    d = p[None, :, :] - v[:, None, :2]                          # [G, M, 2]
    aE = a[None, :] * np.exp(-np.sum(d * d, axis=2) / (2 * rho * rho))
    sE = aE.sum(axis=1)                                         # [G]
    W = b * sE
    C = float(W.sum())
    S = C / nb
    # d(raw sum)/dv, then the quotient rule with d||b||/dv_g = b_g db_g/dv / ||b||
    dC_dv = np.zeros_like(v)
    dC_dv[:, :2] = b[:, None] * np.einsum('gm,gmc->gc', aE, d) / (rho * rho)
    dC_dv += sE[:, None] * db_dv
    dS_dv = dC_dv / nb - (C / nb ** 3) * b[:, None] * db_dv
    grad = np.cross(v, dS_dv).sum(axis=0)
    zero = np.zeros(len(v))
    jx = np.stack([zero, v[:, 2], -v[:, 1]], axis=1)
    jy = np.stack([-v[:, 2], zero, v[:, 0]], axis=1)
    js = np.cross(v, ds_dv)
    H = ((np.einsum('g,gi,gj->ij', W, jx, jx) + np.einsum('g,gi,gj->ij', W, jy, jy)) / (rho * rho)
         + (np.einsum('g,gi,gj->ij', W, js, js) / se2 if omega > 0 else 0.0)) / nb
    return Score(S, grad, H)


def kinematical_score_strain(R, e6, qx, qy, I, refl: Reflections, lam, sigma, rho,
                             gamma_pow=1.0, omega=1.0):
    """kinematical_score with the reciprocal lattice deformed by a small
    symmetric strain e, components e6 = (xx, xy, xz, yy, yz, zz) in the
    crystal frame: each reflection moves to R (I + e) g.  reading: lattice
    strain, which the paper does not treat, moves the spots and changes their
    excitation errors; the amplitudes |g|^gamma |F_g|^omega keep their
    unstrained values (their change with |g| is second order for small e).
    Returns (Score at that strain, dS/de6): with u_g = R^T dS/d(R (I+e) g),
    dS/de_kl = sum_g u_k g_l + u_l g_k for k != l and sum_g u_k g_k on the
    diagonal, g the unstrained vector."""
    e6 = np.asarray(e6, dtype=np.float64)
    E = np.array([[e6[0], e6[1], e6[2]], [e6[1], e6[3], e6[4]], [e6[2], e6[4], e6[5]]])
    R = np.asarray(R, dtype=np.float64)
    g0 = refl.g
    v = g0 @ (np.eye(3) + E) @ R.T                              # rows R (I + e) g
    k = beam_vector(lam)
    kv = k + v
    nkv = np.linalg.norm(kv, axis=1)
    s = excitation_error(v, k)
    ds_dv = -kv * ((nkv + s) / (nkv * nkv))[:, None]
    gn = np.linalg.norm(g0, axis=1)
    se2 = 2 * sigma * sigma / omega if omega > 0 else math.inf
    b = gn ** gamma_pow * np.abs(refl.F) ** omega * np.exp(-(s * s) / (2 * se2))
    nb = float(np.sqrt(np.sum(b * b)))
    if nb == 0.0:
        return Score(0.0, np.zeros(3), np.zeros((3, 3))), np.zeros(6)
    db_dv = (-s / se2 * b)[:, None] * ds_dv
    a = peak_weights(qx, qy, I, gamma_pow, omega)
    p = np.stack([np.asarray(qx, np.float64), np.asarray(qy, np.float64)], axis=1)
    d = p[None, :, :] - v[:, None, :2]
    aE = a[None, :] * np.exp(-np.sum(d * d, axis=2) / (2 * rho * rho))
    sE = aE.sum(axis=1)
    W = b * sE
    C = float(W.sum())
    S = C / nb
    dC_dv = np.zeros_like(v)
    dC_dv[:, :2] = b[:, None] * np.einsum('gm,gmc->gc', aE, d) / (rho * rho)
    dC_dv += sE[:, None] * db_dv
    dS_dv = dC_dv / nb - (C / nb ** 3) * b[:, None] * db_dv
    grad = np.cross(v, dS_dv).sum(axis=0)
    zero = np.zeros(len(v))
    jx = np.stack([zero, v[:, 2], -v[:, 1]], axis=1)
    jy = np.stack([-v[:, 2], zero, v[:, 0]], axis=1)
    js = np.cross(v, ds_dv)
    H = ((np.einsum('g,gi,gj->ij', W, jx, jx) + np.einsum('g,gi,gj->ij', W, jy, jy)) / (rho * rho)
         + (np.einsum('g,gi,gj->ij', W, js, js) / se2 if omega > 0 else 0.0)) / nb
    u = dS_dv @ R                                               # rows R^T dS/dv
    M = u.T @ g0                                                # sum_g u g^T
    de = np.array([M[0, 0], M[0, 1] + M[1, 0], M[0, 2] + M[2, 0], M[1, 1], M[1, 2] + M[2, 1],
                   M[2, 2]])
    return Score(S, grad, H), de


def so3_left_jacobian(r):
    """J with Exp(r + d) = Exp(J d) Exp(r) to first order in d:
    J = I + (1 - cos t)/t^2 [r]x + (t - sin t)/t^3 [r]x^2, t = |r|."""
    r = np.asarray(r, dtype=np.float64)
    t = float(np.linalg.norm(r))
    K = np.array([[0, -r[2], r[1]], [r[2], 0, -r[0]], [-r[1], r[0], 0]])
    if t < 1e-6:
        return np.eye(3) + 0.5 * K + (K @ K) / 6.0
    return np.eye(3) + (1 - math.cos(t)) / t ** 2 * K + (t - math.sin(t)) / t ** 3 * (K @ K)


def kinematical_score_r(r, m0, qx, qy, I, refl: Reflections, lam, sigma, rho, gamma_pow=1.0,
                        omega=1.0):
    """The score at the orientation whose crystal-to-lab rotation is
    Exp(r) m0^T, and its gradient with respect to the axis-angle vector r:
    dS/dr = J(r)^T dS/dw with J the left Jacobian of SO(3)."""
    R = so3_exp(r) @ np.asarray(m0, dtype=np.float64).T
    sc = kinematical_score(R, qx, qy, I, refl, lam, sigma, rho, gamma_pow, omega)
    return sc.S, so3_left_jacobian(r).T @ sc.grad


@dataclass
class RefineParams:
    """reading: 20 Gauss-Newton ascent steps with the position width rho
    shrinking geometrically from rho_start to rho_end; Levenberg-Marquardt
    damping; each rotation step capped.  Chosen on synthetic scans: a wide
    start captures the coarse grid's error, an end several times the peak
    position noise keeps that noise from pulling the in-plane angle, and the
    damping lets 20 steps converge on noiseless patterns."""
    steps: int = 20
    rho_start: float = 0.15
    rho_end: float = 0.03
    sigma: float = 0.02
    damping: float = 0.3
    max_step_deg: float = 1.0

    def rho(self, t):
        if self.steps <= 1:
            return self.rho_end
        return self.rho_start * (self.rho_end / self.rho_start) ** (t / (self.steps - 1))


def refine_step(H, grad, prm: RefineParams):
    """w = (H + damping diag(H))^-1 grad, at most max_step_deg."""
    A = H + prm.damping * np.diag(np.diag(H)) + 1e-12 * max(np.trace(H), 1e-300) * np.eye(3)
    w = np.linalg.solve(A, grad) if np.trace(H) > 0 else np.zeros(3)
    n = float(np.linalg.norm(w))
    cap = math.radians(prm.max_step_deg)
    return w * (cap / n) if n > cap else w


def refine_continuous(m0, qx, qy, I, refl: Reflections, lam, prm: RefineParams,
                      gamma_pow=1.0, omega=1.0):
    """Gradient ascent of kinematical_score from orientation m0; returns the
    refined orientation m (sample to crystal) and the final score."""
    R = np.asarray(m0, dtype=np.float64).T
    for t in range(prm.steps):
        sc = kinematical_score(R, qx, qy, I, refl, lam, prm.sigma, prm.rho(t), gamma_pow, omega)
        R = so3_exp(refine_step(sc.H, sc.grad, prm)) @ R
    sc = kinematical_score(R, qx, qy, I, refl, lam, prm.sigma, prm.rho_end, gamma_pow, omega)
    return R.T, sc.S


def refine_with_twin(m0, qx, qy, I, refl: Reflections, lam, prm: RefineParams, gamma_pow=1.0,
                     omega=1.0):
    """Refine m0 and its in-plane Friedel twin m0 Rz(pi), which a grid match
    cannot tell apart near a zone axis (kinematical intensities of g and -g
    are equal), and keep the one of higher score (ties: m0).  The exact
    excitation errors of the continuous score differ between the two away
    from the zone axis.  Returns (m, score, twin chosen)."""
    ma, sa = refine_continuous(m0, qx, qy, I, refl, lam, prm, gamma_pow, omega)
    mb, sb = refine_continuous(np.asarray(m0, dtype=np.float64) @ np.diag([-1.0, -1.0, 1.0]),
                               qx, qy, I, refl, lam, prm, gamma_pow, omega)
    return (mb, sb, True) if sb > sa else (ma, sa, False)


# --------------------------------------------------------------------------
# Several matches per pattern (Matching of Overlapping Diffraction Patterns)
# --------------------------------------------------------------------------


def forward_spots(refl: Reflections, m, lam, sigma, d_min=1e-3):
    """Detector positions (R g)_xy, R = m^T, of the reflections of the
    forward pattern of orientation m.  reading: a reflection belongs to the
    forward pattern when its Gaussian shape factor D(s_g) (Eq. 8) is at least
    d_min."""
    v = refl.g @ np.asarray(m, dtype=np.float64)
    s = excitation_error(v, beam_vector(lam))
    keep = shape_factor_gaussian(s, sigma) >= d_min
    return v[keep, :2]


def delete_peaks(qx, qy, I, spots, r_del, delta):
    """Peaks within r_del of a forward spot are removed; peaks between r_del
    and the correlation kernel size delta keep (d - r_del) / (delta - r_del)
    of their intensity, d the distance to the nearest spot; the others are
    unchanged."""
    qx = np.asarray(qx, dtype=np.float64)
    qy = np.asarray(qy, dtype=np.float64)
    I = np.asarray(I, dtype=np.float64)
    if len(spots) == 0 or len(qx) == 0:
        return qx, qy, I
    d = np.min(np.hypot(qx[:, None] - spots[None, :, 0], qy[:, None] - spots[None, :, 1]), axis=1)
    keep = d >= r_del
    f = np.where(d < delta, (d - r_del) / (delta - r_del), 1.0)
    return qx[keep], qy[keep], (I * f)[keep]


@dataclass
class MatchN:
    za: int
    k: int
    mirror: int
    score: float          # correlation of the original, full pattern at (za, k, mirror)
    score_cos: float      # the same over ||X|| of the full pattern
    reduced_score: float  # the maximum of the reduced pattern that found it
    m: np.ndarray         # grid orientation
    match: Match = None   # the match of the reduced pattern (its correlogram)


def match_multiple(plan: Plan, refl: Reflections, qx, qy, I, n_matches, r_del, lam, sigma,
                   d_min=1e-3):
    """Up to n_matches orientations: match, compute the forward pattern of the
    match, delete or weaken the peaks it explains, match again.  Stops early
    when no peak is left or the best correlation of what is left is 0 (no
    further orientation).  Each match is reported with the correlation of the
    original full pattern at its (zone axis, phi3 bin, mirror), as the paper
    does, and with the maximum of the reduced pattern that found it.
    reading: the forward pattern is that of the grid orientation of the match."""
    X = polar_image(qx, qy, I, plan.params)
    C, Cm = correlogram(plan.P_hat, X)
    xn = float(np.sqrt(np.sum(X * X)))
    N = plan.params.n_phi
    cur = (np.asarray(qx, np.float64), np.asarray(qy, np.float64), np.asarray(I, np.float64))
    out = []
    for _ in range(n_matches):
        if len(cur[0]) == 0:
            break
        mt = match_pattern(plan, *cur)
        if not mt.score > 0:
            break
        full = float((Cm if mt.mirror else C)[mt.za, mt.k])
        m = orientation_matrix(plan.za[mt.za], -2 * math.pi * mt.k / N, mt.mirror)
        out.append(MatchN(mt.za, mt.k, mt.mirror, full, full / xn if xn > 0 else 0.0,
                          mt.score, m, mt))
        cur = delete_peaks(*cur, forward_spots(refl, m, lam, sigma, d_min), r_del,
                           plan.params.delta)
    return out


# --------------------------------------------------------------------------
# Accuracy metrics (reading)
# --------------------------------------------------------------------------


def proper_point_group(kind):
    """Proper rotations of m-3m (the 24 of O) or 6/mmm (the 12 of 622), as
    3x3 matrices acting on crystal Cartesian coordinates."""
    ops = []
    if kind == 'cubic':
        import itertools
        for perm in itertools.permutations(range(3)):
            for signs in itertools.product((1.0, -1.0), repeat=3):
                M = np.zeros((3, 3))
                for r in range(3):
                    M[r, perm[r]] = signs[r]
                if np.linalg.det(M) > 0:
                    ops.append(M)
    elif kind == 'hexagonal':
        for n in range(6):
            R = rot_z(n * math.pi / 3)
            ops.append(R)
            ops.append(R @ np.diag([1.0, -1.0, -1.0]))    # 2-fold about x
    else:
        raise ValueError(kind)
    return ops


def rotation_angle_deg(R):
    c = (np.trace(R) - 1.0) / 2.0
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))


def misorientation_deg(m_est, m_true, ops, friedel_twin=False):
    """min over proper symmetry operations S of the angle of m_true^T S m_est;
    with ``friedel_twin`` also over m_est Rz(pi)."""
    cands = [np.asarray(m_est)]
    if friedel_twin:
        cands.append(np.asarray(m_est) @ rot_z(math.pi))
    best = 180.0
    for me in cands:
        for S in ops:
            best = min(best, rotation_angle_deg(np.asarray(m_true).T @ S @ me))
    return best


def za_tilt_error_deg(m_est, m_true, ops):
    """Angle between the beam directions m z_hat of the two orientations,
    minimised over the symmetry operations and the sign of the axis (the
    paper's zone-axis tilt error)."""
    we = np.asarray(m_est)[:, 2]
    wt = np.asarray(m_true)[:, 2]
    best = 180.0
    for S in ops:
        c = abs(float(np.dot(S @ we, wt)))
        best = min(best, math.degrees(math.acos(min(1.0, c))))
    return best
