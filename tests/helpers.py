"""Shared builders of seeded test cases.

Inputs come from paper_2312_14907_gb300.synth; measured data are Poisson
counts of the FP64 oracle's forward model.  Nothing here calls the CUDA path,
so every expected value in the tests comes from the oracle.
"""
import numpy as np

import oracle
from paper_2312_14907_gb300 import synth


class Case:
    """One problem: geometry, probe, data and a state to evaluate at (all float32
    for the GPU; the oracle reads the same values in double precision)."""

    def __init__(self, spec, scan=None, probe=None, seed=0, state="init", bg=False,
                 photons=None, noise=True):
        self.spec = spec
        self.scan = synth.scan_positions(spec) if scan is None else np.asarray(scan, np.int32)
        rng = np.random.default_rng(spec.seed + 17 * seed)
        self.oracle = oracle.OracleProblem.from_spec(spec, self.scan)
        P = synth.probe(spec) if probe is None else probe
        self.rho_t, self.u_t = synth.truth(spec)
        self.alpha_t = synth.alpha_truth(spec)
        rho_t, u_t = self.rho_t.astype(np.float32), self.u_t.astype(np.float32)
        I = self.oracle.forward(rho_t, u_t, self.alpha_t.astype(np.float32), P.astype(np.complex64))
        scale = synth.photon_scale(I, photons or spec.photons)
        self.probe = (P * np.sqrt(scale)).astype(np.complex64)
        I = I * scale
        self.bg = None
        if bg:
            self.bg = rng.uniform(0.0, 0.05 * I.mean() + 0.1, I.shape).astype(np.float32)
            I = I + self.bg
        self.I_truth = I
        self.y = synth.poisson_counts(I, spec.seed + 1000 + seed) if noise else I.astype(np.float32)
        if state == "init":
            rho, u, alpha = synth.init_state(spec)
        elif state == "truth":
            rho, u, alpha = self.rho_t, self.u_t, self.alpha_t
        else:
            rho, u, alpha = synth.perturbed_state(spec, rng, 0.05)
        self.rho = np.ascontiguousarray(rho, np.float32)
        self.u = np.ascontiguousarray(u, np.float32)
        self.alpha = np.ascontiguousarray(alpha, np.float32)

    def oracle_loss_grad(self, frames=None, rho=None, u=None, alpha=None):
        return self.oracle.loss_grad(self.rho if rho is None else rho, self.u if u is None else u,
                                     self.alpha if alpha is None else alpha, self.probe, self.y,
                                     bg=self.bg, frames=frames)


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    a = a.astype(np.complex128 if np.iscomplexobj(a) else np.float64)
    b = b.astype(np.complex128 if np.iscomplexobj(b) else np.float64)
    nb = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0)


def custom_spec(n, m, side, step, npeaks=3, ncomp=3, seed=0, offset=None, probe_per_peak=False, n2=None):
    """A problem of chosen size (n x n, or n x n2); offset (the first scan
    position) may be negative."""
    G = (synth.AXIS_PEAKS if npeaks <= 3 else synth.PAPER_PEAKS)[:npeaks, :ncomp].copy()
    if ncomp < 3 and npeaks <= 3:
        G = np.array([[1.0, 0.0], [0.0, 1.0], [0.6, 0.8]])[:npeaks, :ncomp]
    sig, quad = 6.0 * m / 32, 0.01 * (32.0 / m) ** 2
    spec = synth.ProblemSpec("custom-%d-m%d" % (n, m), n, n if n2 is None else n2, ncomp, npeaks, m, side, step, G,
                             synth.SEED_BASE + 500 + seed, bumps=6, straight=2, curved=1,
                             sigma=sig, quad=quad, probe_per_peak=probe_per_peak)
    if offset is not None:
        r = offset + step * np.arange(side)
        rr, cc = np.meshgrid(r, r, indexing="ij")
        scan = np.stack([rr.ravel(), cc.ravel()], axis=1).astype(np.int32)
        return spec, scan
    return spec, synth.scan_positions(spec)
