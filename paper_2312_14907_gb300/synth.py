"""Seeded synthetic inputs for MPBP problems (no model arithmetic here).

This module only draws the inputs of a problem: the object grid, the true
density and displacement fields, the probe, the scattering vectors, the scan
grid, the starting point of a reconstruction and Poisson counts for a given
intensity.  It holds none of the forward model or gradient arithmetic; the
intensities that Poisson counts are drawn from come from whichever
implementation the caller runs (the CUDA forward in the benchmark, the FP64
oracle in the tests).

The paper's own sample, probe and geometry (its Sec. 4 and Table 1) are not
available, so these generators stand in for them with the same structure: a
single-crystal film with a support, a smooth displacement field with
phase-discontinuity lines, a focused complex probe, raster scans with heavy
overlap and low-count Poisson data.
"""
from dataclasses import dataclass, field, replace
import math

import numpy as np

SEED_BASE = 2312149070

# In-plane Bragg peaks [100], [110], [120], [210] of the paper's cubic film
# (Sec. 4), in reciprocal-lattice units, as 3-vectors with l = 0.
PAPER_PEAKS = np.array([[1, 0, 0], [1, 1, 0], [1, 2, 0], [2, 1, 0]], dtype=np.float64)
# Relative magnitudes of those four peaks' objects (Sec. 4), normalised to the first.
PAPER_SCALINGS = np.array([0.004, 0.0035, 0.0021, 0.0010]) / 0.004
AXIS_PEAKS = np.array([[1, 0, 0], [0, 1, 0], [1, 1, 1]], dtype=np.float64)
AXIS_PEAKS[2] /= math.sqrt(3.0)


@dataclass
class ProblemSpec:
    """Sizes and generator settings of one MPBP problem."""
    name: str
    n1: int
    n2: int
    ncomp: int
    npeaks: int
    m: int
    scan_side: int
    step: int
    G: np.ndarray
    seed: int
    bumps: int = 4
    straight: int = 1
    curved: int = 0
    jump: float = 0.5
    bump_amp: float = 0.3
    sigma: float = 6.0
    quad: float = 0.01
    support: int = 0
    alpha_true: np.ndarray = None
    phase_scale: float = 2.0 * math.pi
    probe_per_peak: bool = False
    photons: float = 1e4

    @property
    def nscan(self):
        return self.scan_side * self.scan_side

    @property
    def nframes(self):
        return self.nscan * self.npeaks

    @property
    def offset(self):
        span = (self.scan_side - 1) * self.step + self.m
        return (min(self.n1, self.n2) - span) // 2


def _probe_shape(m):
    # probe width and curvature keep their shape relative to the frame
    return 6.0 * m / 32.0, 0.01 * (32.0 / m) ** 2


def config(k):
    """The five benchmark problems (index 1..5)."""
    if k == 1:
        s, q = _probe_shape(32)
        return ProblemSpec("mpbp-64-m32-d3", 64, 64, 3, 3, 32, 7, 4, AXIS_PEAKS.copy(),
                           SEED_BASE + 1, bumps=4, straight=1, sigma=s, quad=q)
    if k == 2:
        s, q = _probe_shape(64)
        return ProblemSpec("mpbp-256-m64-d3", 256, 256, 3, 3, 64, 31, 6, AXIS_PEAKS.copy(),
                           SEED_BASE + 2, bumps=16, straight=3, sigma=s, quad=q)
    if k == 3:
        s, q = _probe_shape(128)
        return ProblemSpec("mpbp-512-m128-d4", 512, 512, 3, 4, 128, 61, 6, PAPER_PEAKS.copy(),
                           SEED_BASE + 3, bumps=0, straight=3, curved=3, sigma=s, quad=q,
                           alpha_true=PAPER_SCALINGS.copy())
    if k == 5:
        s, q = _probe_shape(128)
        rng = np.random.default_rng(SEED_BASE + 5)
        G = rng.standard_normal((6, 3))
        G /= np.linalg.norm(G, axis=1, keepdims=True)
        return ProblemSpec("mpbp-1024-m128-d6", 1024, 1024, 3, 6, 128, 121, 8, G,
                           SEED_BASE + 5, bumps=32, straight=6, curved=6, sigma=s, quad=q)
    raise ValueError("config index must be 1, 2, 3 or 5 (4 is batched_configs())")


def batched_configs():
    """16 independent problems of uneven sizes (objects 128..512, frames 32/64/128,
    3 or 4 peaks, scan grids 15x15..61x61)."""
    out = []
    for i in range(16):
        n = 16 * round((128 + 384 * i / 15) / 16)
        m = (32, 64, 128)[i % 3]
        while m > n // 2:          # cap at N/2, kept a power of two
            m //= 2
        d = 3 + (i % 2)
        side = 15 + (46 * i) // 15
        step = (n - m) // (side - 1)
        G = AXIS_PEAKS.copy() if d == 3 else PAPER_PEAKS.copy()
        s, q = _probe_shape(m)
        out.append(ProblemSpec("batch%02d-%d-m%d-d%d" % (i, n, m, d), n, n, 3, d, m, side,
                               step, G, SEED_BASE + 4 * 1000 + i, bumps=8, straight=2,
                               curved=1, sigma=s, quad=q))
    return out


def tiny(ncomp=3, npeaks=2, n=12, m=8, side=3, step=2, seed=SEED_BASE + 99):
    """A small problem for finite-difference and brute-force checks."""
    G = (AXIS_PEAKS if npeaks <= 3 else PAPER_PEAKS)[:npeaks, :ncomp].copy()
    if ncomp == 2 and npeaks <= 3:
        G = np.array([[1.0, 0.0], [0.0, 1.0], [0.6, 0.8]])[:npeaks]
    s, q = 1.6 * m / 8, 0.01 * (32.0 / m) ** 2 / 4
    return ProblemSpec("tiny", n, n, ncomp, npeaks, m, side, step, G, seed, bumps=2,
                       straight=1, sigma=s, quad=q)


def scan_positions(spec):
    """Top-left (row, col) of each frame; row-major over the scan grid."""
    o = spec.offset
    r = o + spec.step * np.arange(spec.scan_side)
    rr, cc = np.meshgrid(r, r, indexing="ij")
    return np.stack([rr.ravel(), cc.ravel()], axis=1).astype(np.int32)


def _support_mask(spec):
    n1, n2 = spec.n1, spec.n2
    side = spec.support or int(round(0.75 * min(n1, n2)))
    a0 = (n1 - side) // 2
    a1 = (n2 - side) // 2
    mask = np.zeros((n1, n2), bool)
    mask[a0:a0 + side, a1:a1 + side] = True
    return mask, (a0, a1, side)


def _unit(rng, c):
    v = rng.standard_normal(c)
    return v / np.linalg.norm(v)


def truth(spec):
    """True density rho [n1][n2] and displacement u [C][n1][n2] (lattice units).

    rho = 1 on a centred square support (3/4 of the grid side), 0 outside.
    u = sum of Gaussian bumps (amplitude bump_amp along a random direction,
    width N/16..N/8) + straight step lines (a jump of `jump` times a random unit
    vector on one side of a random line through the support) + curved lines
    (the same jump inside a random disk of radius N/8..N/3)."""
    rng = np.random.default_rng(spec.seed)
    n1, n2, C = spec.n1, spec.n2, spec.ncomp
    mask, (a0, a1, side) = _support_mask(spec)
    rho = mask.astype(np.float64)
    y, x = np.meshgrid(np.arange(n1, dtype=np.float64), np.arange(n2, dtype=np.float64),
                       indexing="ij")
    u = np.zeros((C, n1, n2))
    N = min(n1, n2)
    for _ in range(spec.bumps):
        c0 = a0 + rng.uniform(0, side)
        c1 = a1 + rng.uniform(0, side)
        w = rng.uniform(N / 16, N / 8)
        v = _unit(rng, C)
        g = np.exp(-((y - c0) ** 2 + (x - c1) ** 2) / (2 * w * w))
        u += spec.bump_amp * v[:, None, None] * g[None]
    for _ in range(spec.straight):
        p0 = a0 + rng.uniform(0, side)
        p1 = a1 + rng.uniform(0, side)
        th = rng.uniform(0, math.pi)
        b = spec.jump * _unit(rng, C)
        dist = (y - p0) * math.cos(th) - (x - p1) * math.sin(th)
        u += b[:, None, None] * (dist > 0)[None]
    for _ in range(spec.curved):
        c0 = a0 + rng.uniform(0, side)
        c1 = a1 + rng.uniform(0, side)
        rad = rng.uniform(N / 8, N / 3)
        b = spec.jump * _unit(rng, C)
        u += b[:, None, None] * (((y - c0) ** 2 + (x - c1) ** 2) < rad * rad)[None]
    return rho, u


def alpha_truth(spec):
    if spec.alpha_true is not None:
        return np.asarray(spec.alpha_true, np.float64).copy()
    return np.ones(spec.npeaks)


def probe(spec, asym=0.0):
    """Complex Gaussian probe exp(-|k-c|^2/(2 sigma^2)) exp(i quad |k-c|^2), c = (M/2, M/2),
    unit peak amplitude.  `asym` > 0 stretches it along rows and adds a linear
    phase so that row/column transpositions change the result (test use)."""
    m = spec.m
    k0, k1 = np.meshgrid(np.arange(m, dtype=np.float64), np.arange(m, dtype=np.float64),
                         indexing="ij")
    d0, d1 = k0 - m / 2, k1 - m / 2
    r2 = d0 * d0 / (1.0 + asym) ** 2 + d1 * d1
    p = np.exp(-r2 / (2 * spec.sigma ** 2)) * np.exp(1j * spec.quad * (d0 * d0 + d1 * d1))
    if asym:
        p = p * np.exp(1j * asym * 0.3 * d0)
    if spec.probe_per_peak:
        p = np.stack([p * np.exp(1j * 0.1 * d) for d in range(spec.npeaks)])
    return p.astype(np.complex128)


def random_probe(spec, rng):
    """An unstructured complex probe (for parity tests that must catch index mistakes)."""
    shape = (spec.npeaks, spec.m, spec.m) if spec.probe_per_peak else (spec.m, spec.m)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / 2


def init_state(spec):
    """Reconstruction starting point: rho = 1 everywhere, u = 0, alpha = 1."""
    return (np.ones((spec.n1, spec.n2)), np.zeros((spec.ncomp, spec.n1, spec.n2)),
            np.ones(spec.npeaks))


def photon_scale(I, photons):
    """Factor that makes the brightest frame of intensities I [D][J][M][M] hold
    `photons` expected counts in total."""
    tot = I.reshape(I.shape[0] * I.shape[1], -1).sum(axis=1).max()
    return float(photons / tot) if tot > 0 else 1.0


def poisson_counts(I, seed):
    """Poisson counts with means I (NumPy's PCG64 sampler, seeded)."""
    rng = np.random.default_rng(seed)
    return rng.poisson(np.maximum(I, 0.0)).astype(np.float32)


def template_counts(spec, seed, scan_index=None):
    """Count-like data [D][J][M][M] without any forward model: per peak a fixed
    speckle template (a few Gaussian spots on a weak floor, DC at [0][0]) times
    a seeded per-frame level, rounded.  For tests that only need some data of
    the right shape and range (the loss and gradient are compared for the same
    y on both sides).  scan_index: only those scan positions ([D][len][M][M],
    the same values as the full array's)."""
    rng = np.random.default_rng(seed)
    m = spec.m
    q = np.fft.fftfreq(m) * m
    q0, q1 = np.meshgrid(q, q, indexing="ij")
    tmpl = np.empty((spec.npeaks, m, m), np.float32)
    for d in range(spec.npeaks):
        t = 0.05 + np.zeros((m, m))
        for _ in range(6):
            c0, c1 = rng.normal(0, m / 8, 2)
            w = rng.uniform(1.0, m / 16)
            t += rng.uniform(5, 60) * np.exp(-((q0 - c0) ** 2 + (q1 - c1) ** 2) / (2 * w * w))
        tmpl[d] = t
    level = rng.uniform(0.2, 1.5, (spec.npeaks, spec.nscan)).astype(np.float32)
    if scan_index is not None:
        level = np.ascontiguousarray(level[:, np.asarray(scan_index)])
    return np.ascontiguousarray(np.rint(level[:, :, None, None] * tmpl[:, None, :, :]).astype(np.float32))


def perturbed_state(spec, rng, scale=0.05):
    """A generic state near the truth (for gradient checks away from the optimum)."""
    rho, u = truth(spec)
    rho = rho + scale * rng.standard_normal(rho.shape) + 0.2
    u = u + scale * rng.standard_normal(u.shape)
    alpha = alpha_truth(spec) * (1.0 + scale * rng.standard_normal(spec.npeaks))
    alpha[0] = 1.0
    return rho, u, alpha


def epoch_order(nframes, seed):
    """A seeded shuffle of all D*J frame numbers (Alg. 1, line 1): the random
    order of one epoch of minibatches, drawn here and passed to both the
    GPU path and the oracle as an input."""
    return np.random.default_rng(seed).permutation(nframes).astype(np.int32)


def support_mask(spec, margin=5):
    """The support constraint of the reconstruction: 1 on the object's
    square support grown by `margin` pixels on every side (the paper grows the
    film support by 5 pixels), 0 elsewhere (float32)."""
    _, (a0, a1, side) = _support_mask(spec)
    mask = np.zeros((spec.n1, spec.n2), np.float32)
    mask[max(a0 - margin, 0):a0 + side + margin, max(a1 - margin, 0):a1 + side + margin] = 1.0
    return mask
