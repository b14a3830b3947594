"""Seeded synthetic inputs for the sparse correlation match.

This module only makes inputs: crystal descriptions, random orientations,
Voronoi grain maps and kinematical Bragg-peak lists in CSR form.  It holds
none of the matching method's arithmetic (no polar image, plan, Fourier
transform or correlation) and imports neither the oracle nor the library;
both sides read the same arrays from here.

The peak lists come from a forward model written here on its own terms:
reflections are selected by the textbook extinction rules of the fcc and hcp
structures (not by evaluating structure-factor phase sums), the excitation
error is the geometric distance |k| - |k + g| from the lattice point to the
Ewald sphere, and the intensity is |F|^2 exp(-s^2 / 2 sigma^2).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ------------------------------------------------------------------ crystals


@dataclass(frozen=True)
class CrystalSpec:
    name: str
    kind: str                     # 'fcc' | 'hcp'
    lattice: np.ndarray           # rows a, b, c (Angstrom)
    frac_pos: np.ndarray          # [n_atoms, 3]
    ff_A: float                   # f(q) = ff_A exp(-ff_B q^2), q in 1/Angstrom
    ff_B: float
    step_region: tuple = field(default=())


def au_fcc(a=4.08):
    """fcc Au, a = 4.08 Angstrom, 4 atoms per cell, f(q) = 79 exp(-0.25 q^2)."""
    return CrystalSpec("Au", "fcc", np.eye(3) * a,
                       np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]]),
                       79.0, 0.25)


def mg_hcp(a=3.21, c=5.21):
    """Mg-like hcp (P6_3/mmc), 2 atoms per cell, f(q) = 12 exp(-0.3 q^2)."""
    L = np.array([[a, 0, 0], [-a / 2, a * math.sqrt(3) / 2, 0], [0, 0, c]])
    return CrystalSpec("Mg", "hcp", L,
                       np.array([[1 / 3, 2 / 3, 1 / 4], [2 / 3, 1 / 3, 3 / 4]]),
                       12.0, 0.3)


def reflection_table(spec: CrystalSpec, q_max):
    """Lattice points 0 < |g| < q_max with non-zero intensity |F|^2 from the
    extinction rules of the structure type.  Returns (g [G,3], F2 [G])."""
    L = np.asarray(spec.lattice, dtype=np.float64)
    recip_rows = np.linalg.inv(L).T
    n = [int(math.ceil(q_max * np.linalg.norm(L[i]))) for i in range(3)]
    h, k, l = np.meshgrid(np.arange(-n[0], n[0] + 1), np.arange(-n[1], n[1] + 1),
                          np.arange(-n[2], n[2] + 1), indexing="ij")
    hkl = np.stack([h.ravel(), k.ravel(), l.ravel()], axis=1)
    g = hkl @ recip_rows
    q = np.linalg.norm(g, axis=1)
    sel = (q > 0) & (q < q_max)
    hkl, g, q = hkl[sel], g[sel], q[sel]
    f2 = (spec.ff_A * np.exp(-spec.ff_B * q * q)) ** 2
    hh, kk, ll = hkl.T
    if spec.kind == "fcc":
        mult = np.where(((hh - kk) % 2 == 0) & ((kk - ll) % 2 == 0), 16.0, 0.0)
    elif spec.kind == "hcp":
        m3 = ((hh + 2 * kk) % 3) == 0
        lodd = (ll % 2) != 0
        mult = np.where(m3 & lodd, 0.0, np.where(m3, 4.0, np.where(lodd, 3.0, 1.0)))
    else:
        raise ValueError(spec.kind)
    keep = mult > 0
    return g[keep], (mult * f2)[keep]


# -------------------------------------------------------------- orientations


def random_rotations(rng, n):
    """Uniform random rotations (normalised 4-D Gaussian quaternions)."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def voronoi_labels(rng, H, W, n_grains):
    """Grain id of every pixel (row-major) of an H x W scan: nearest of
    n_grains seeds uniform in [0, W) x [0, H), pixel centres, ties to the
    lower seed index."""
    seeds = rng.uniform(0, 1, size=(n_grains, 2)) * np.array([W, H])
    yy, xx = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel()], axis=1)
    lab = np.empty(len(pts), dtype=np.int64)
    for i in range(0, len(pts), 8192):
        d = ((pts[i:i + 8192, None, :] - seeds[None, :, :]) ** 2).sum(-1)
        lab[i:i + 8192] = np.argmin(d, axis=1)
    return lab


# ---------------------------------------------------------- forward model


def noiseless_peaks(g, F2, m, lam, sigma):
    """Lab-frame peak list of orientation m (d_crystal = m d_sample): every
    reflection, at (g_lab_x, g_lab_y), g_lab = m^T g, with intensity
    F2 exp(-s^2 / 2 sigma^2), s = |k| - |k + g_lab|, k = (0, 0, -1/lam)."""
    gl = g @ np.asarray(m)
    k = np.array([0.0, 0.0, -1.0 / lam])
    s = (1.0 / lam) - np.linalg.norm(gl + k, axis=1)
    return gl[:, 0], gl[:, 1], F2 * np.exp(-(s * s) / (2 * sigma * sigma))


@dataclass
class Scan:
    row_ptr: np.ndarray      # int64 [B + 1]
    qx: np.ndarray           # float32 [nnz]
    qy: np.ndarray
    I: np.ndarray
    truth: np.ndarray        # float64 [B, 3, 3] true orientation matrices
    phase: np.ndarray        # int32 [B] index into ``crystals``
    crystals: tuple
    recipe: str

    @property
    def n_patterns(self):
        return len(self.row_ptr) - 1

    def pattern(self, b):
        s, e = self.row_ptr[b], self.row_ptr[b + 1]
        return self.qx[s:e], self.qy[s:e], self.I[s:e]

    def subset(self, idx):
        idx = np.asarray(idx)
        counts = self.row_ptr[idx + 1] - self.row_ptr[idx]
        rp = np.zeros(len(idx) + 1, dtype=np.int64)
        np.cumsum(counts, out=rp[1:])
        src = np.concatenate([np.arange(self.row_ptr[b], self.row_ptr[b + 1]) for b in idx]) \
            if len(idx) else np.zeros(0, dtype=np.int64)
        return Scan(rp, self.qx[src], self.qy[src], self.I[src], self.truth[idx],
                    self.phase[idx], self.crystals, self.recipe + f" (subset of {len(idx)})")


def _assemble(lists, counts, rng, pos_noise, int_noise):
    """Top-``counts[b]`` peaks of each pattern's noiseless list, then
    Gaussian position noise and lognormal intensity noise."""
    B = len(lists)
    rp = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    nnz = int(rp[-1])
    qx = np.empty(nnz)
    qy = np.empty(nnz)
    I = np.empty(nnz)
    for b, (x, y, i) in enumerate(lists):
        s, e = rp[b], rp[b + 1]
        qx[s:e], qy[s:e], I[s:e] = x[:e - s], y[:e - s], i[:e - s]
    qx += rng.normal(0.0, pos_noise, nnz)
    qy += rng.normal(0.0, pos_noise, nnz)
    I *= np.exp(int_noise * rng.normal(size=nnz))
    return rp, qx.astype(np.float32), qy.astype(np.float32), I.astype(np.float32)


def _sorted_list(g, F2, m, lam, sigma):
    x, y, i = noiseless_peaks(g, F2, m, lam, sigma)
    o = np.argsort(-i, kind="stable")
    return x[o], y[o], i[o]


def random_patterns(seed, n_patterns=100, crystal=None, q_max=1.5, lam=0.01969,
                    sigma=0.02, rel_threshold=1e-3, max_peaks=40,
                    pos_noise=0.005, int_noise=0.1):
    """Independent patterns at uniformly random orientations: peaks above
    ``rel_threshold`` of the strongest are kept, capped at ``max_peaks`` by
    noiseless intensity, then noised (Gaussian positions, lognormal
    intensities)."""
    rng = np.random.default_rng(seed)
    spec = crystal or au_fcc()
    g, F2 = reflection_table(spec, q_max)
    R = random_rotations(rng, n_patterns)
    lists, counts = [], []
    for b in range(n_patterns):
        x, y, i = _sorted_list(g, F2, R[b], lam, sigma)
        n = min(int(np.sum(i > rel_threshold * i[0])), max_peaks)
        lists.append((x, y, i))
        counts.append(n)
    rp, qx, qy, I = _assemble(lists, np.array(counts), rng, pos_noise, int_noise)
    return Scan(rp, qx, qy, I, R, np.zeros(n_patterns, np.int32), (spec,),
                f"{n_patterns} random {spec.name} patterns, seed {seed}")


def mixed_patterns(seed, n_patterns=100, crystals=None, q_max=1.5, lam=0.01969,
                   sigma=0.02, rel_threshold=1e-3, max_peaks=40,
                   pos_noise=0.005, int_noise=0.1):
    """Independent patterns whose phase is drawn uniformly from ``crystals``
    (50/50 for two), each at a uniformly random orientation, with the peak
    rules of ``random_patterns``."""
    rng = np.random.default_rng(seed)
    specs = tuple(crystals or (au_fcc(), mg_hcp()))
    tables = [reflection_table(s, q_max) for s in specs]
    phase = rng.integers(0, len(specs), n_patterns).astype(np.int32)
    R = random_rotations(rng, n_patterns)
    lists, counts = [], []
    for b in range(n_patterns):
        x, y, i = _sorted_list(*tables[phase[b]], R[b], lam, sigma)
        n = min(int(np.sum(i > rel_threshold * i[0])), max_peaks)
        lists.append((x, y, i))
        counts.append(n)
    rp, qx, qy, I = _assemble(lists, np.array(counts), rng, pos_noise, int_noise)
    names = "/".join(s.name for s in specs)
    return Scan(rp, qx, qy, I, R, phase, specs,
                f"{n_patterns} random patterns of {names}, seed {seed}")


def grain_scan(seed, H=256, W=256, n_grains=200, crystals=None, q_max=1.5,
               lam=0.01969, sigma=0.02, peaks="uniform10-60",
               pos_noise=0.005, int_noise=0.1):
    """H x W scan over a Voronoi map of ``n_grains`` grains, one uniformly
    random orientation (and phase, 50/50 over ``crystals``) per grain.  Each
    pattern keeps its n strongest noiseless peaks, n ~ U{10..60}
    ('uniform10-60') or clip(Poisson(30), 5, 80) ('poisson30'), then noise."""
    rng = np.random.default_rng(seed)
    specs = tuple(crystals or (au_fcc(),))
    tables = [reflection_table(s, q_max) for s in specs]
    lab = voronoi_labels(rng, H, W, n_grains)
    R = random_rotations(rng, n_grains)
    gphase = rng.integers(0, len(specs), n_grains) if len(specs) > 1 else \
        np.zeros(n_grains, dtype=np.int64)
    glist = [_sorted_list(*tables[gphase[i]], R[i], lam, sigma) for i in range(n_grains)]
    B = H * W
    if peaks == "uniform10-60":
        n = rng.integers(10, 61, B)
    elif peaks == "poisson30":
        n = np.clip(rng.poisson(30, B), 5, 80)
    else:
        raise ValueError(peaks)
    avail = np.array([len(glist[i][0]) for i in range(n_grains)])
    n = np.minimum(n, avail[lab])
    rp = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(n, out=rp[1:])
    nnz = int(rp[-1])
    # gather the first n[b] entries of grain lab[b]'s list
    goff = np.zeros(n_grains + 1, dtype=np.int64)
    np.cumsum(avail, out=goff[1:])
    allx = np.concatenate([gl[0] for gl in glist])
    ally = np.concatenate([gl[1] for gl in glist])
    alli = np.concatenate([gl[2] for gl in glist])
    pos = np.arange(nnz) - np.repeat(rp[:-1], n)
    src = np.repeat(goff[lab], n) + pos
    qx = allx[src] + rng.normal(0.0, pos_noise, nnz)
    qy = ally[src] + rng.normal(0.0, pos_noise, nnz)
    I = alli[src] * np.exp(int_noise * rng.normal(size=nnz))
    names = "+".join(s.name for s in specs)
    return Scan(rp, qx.astype(np.float32), qy.astype(np.float32), I.astype(np.float32),
                R[lab], gphase[lab].astype(np.int32), specs,
                f"{H}x{W} {names} scan, {n_grains} Voronoi grains, peaks {peaks}, seed {seed}")
