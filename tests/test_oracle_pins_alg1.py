"""Pins of the oracle's Alg. 1 pieces: the per-peak-phase form (Sec. 5, TS),
the auxiliary variables of Eq. 8 and the Adam update.

As in test_oracle_pins.py, none of these re-types a formula: the gradients
are checked against central differences, the phase form against the
displacement form at phases that the displacement field defines, and Adam
against closed forms of gradient sequences whose moments can be summed by
hand (Kingma and Ba's update).
"""
import math

import numpy as np
import pytest

from paper_2312_14907_gb300 import synth


def _tiny(oracle_mod, ncomp=3, npeaks=3, seed=31):
    spec = synth.tiny(ncomp=ncomp, npeaks=npeaks, n=12, m=8, side=3, step=2)
    scan = synth.scan_positions(spec)
    p = oracle_mod.OracleProblem.from_spec(spec, scan)
    rng = np.random.default_rng(seed)
    P = synth.random_probe(spec, rng)
    rho_t, u_t = synth.truth(spec)
    I = p.forward(rho_t + 0.5, u_t, synth.alpha_truth(spec), P)
    y = synth.poisson_counts(I, seed).astype(np.float64)
    rho, u, alpha = synth.perturbed_state(spec, rng, 0.1)
    return spec, p, P, y, np.asarray(rho, float), np.asarray(u, float), np.asarray(alpha, float), rng


def _central(f, x, idx, h):
    x0 = x[idx]
    x[idx] = x0 + h
    fp = f()
    x[idx] = x0 - h
    fm = f()
    x[idx] = x0
    return (fp - fm) / (2 * h)


# --------------------------------------------------------------------------
# per-peak phases (the TS variables)
# --------------------------------------------------------------------------

def test_phase_form_equals_displacement_form_at_its_phases(oracle_mod):
    """phi_m = phase_scale G_m . u makes both forms the same objects (Eq. 3)."""
    spec, p, P, y, rho, u, alpha, _ = _tiny(oracle_mod)
    phi = spec.phase_scale * np.einsum("mc,cij->mij", np.asarray(spec.G), u)
    f_u, gr_u, _, ga_u = p.loss_grad(rho, u, alpha, P, y)
    f_p, gr_p, gphi, ga_p = p.loss_grad_phases(rho, phi, alpha, P, y)
    assert abs(f_p - f_u) <= 1e-12 * abs(f_u)
    np.testing.assert_allclose(gr_p, gr_u, rtol=1e-10, atol=1e-12 * np.abs(gr_u).max())
    np.testing.assert_allclose(ga_p, ga_u, rtol=1e-10)
    # a phase change of 2 pi at one pixel of one peak changes no object
    phi2 = phi.copy()
    phi2[1, 5, 6] += 2 * math.pi
    assert abs(p.loss_grad_phases(rho, phi2, alpha, P, y)[0] - f_p) <= 1e-11 * abs(f_p)


def test_phase_gradient_matches_central_differences(oracle_mod):
    spec, p, P, y, rho, u, alpha, rng = _tiny(oracle_mod, npeaks=2)
    phi = rng.uniform(-3, 3, (spec.npeaks, spec.n1, spec.n2))
    f0, _, gphi, _ = p.loss_grad_phases(rho, phi, alpha, P, y)
    scale = np.abs(gphi).max()
    for _ in range(8):
        idx = (rng.integers(0, spec.npeaks), rng.integers(0, spec.n1), rng.integers(0, spec.n2))
        fd = _central(lambda: p.loss_grad_phases(rho, phi, alpha, P, y)[0], phi, idx, 1e-5)
        assert abs(fd - gphi[idx]) <= 1e-6 * scale, (idx, fd, gphi[idx])


# --------------------------------------------------------------------------
# the auxiliary variables of Eq. 8 and the support mask
# --------------------------------------------------------------------------

def test_log_variables_gradient_matches_central_differences(oracle_mod):
    spec, p, P, y, rho, u, alpha, rng = _tiny(oracle_mod)
    chi = np.log(np.clip(rho, 0.2, None))   # rho is 0 off the object support
    alpha_t = np.log(alpha)
    mask = np.ones((spec.n1, spec.n2))
    mask[:2, :] = 0.0
    mask[:, -3:] = 0.0

    def f():
        return p.loss_grad_log(chi, u, alpha_t, P, y, mask=mask)[0]

    f0, gchi, gu, ga = p.loss_grad_log(chi, u, alpha_t, P, y, mask=mask)
    scale = max(np.abs(gchi).max(), np.abs(gu).max())
    for _ in range(8):
        i, j = rng.integers(2, spec.n1), rng.integers(0, spec.n2 - 3)
        assert abs(_central(f, chi, (i, j), 1e-6) - gchi[i, j]) <= 1e-6 * scale
        c = rng.integers(0, spec.ncomp)
        assert abs(_central(f, u, (c, i, j), 1e-6) - gu[c, i, j]) <= 1e-6 * scale
    for d in range(1, spec.npeaks):
        fd = _central(f, alpha_t, d, 1e-6)
        assert abs(fd - ga[d]) <= 1e-6 * max(abs(ga[d]), 1e-3 * scale)
    # alpha_0 is not a variable; outside the support rho = 0 and chi has no effect
    assert ga[0] == 0.0
    assert np.all(gchi[mask == 0] == 0.0)
    chi2 = chi.copy()
    chi2[mask == 0] += 5.0
    assert p.loss_grad_log(chi2, u, alpha_t, P, y, mask=mask)[0] == f0


# --------------------------------------------------------------------------
# Adam
# --------------------------------------------------------------------------

def test_adam_constant_gradient_steps_by_lr(oracle_mod):
    """With a constant gradient g the bias-corrected moments are g and g^2, so
    every step is lr * g / (|g| + eps) from the first one on."""
    g = np.array([3.0, -0.25, 1e-3, -7e4])
    x = np.zeros(4)
    m, v = np.zeros(4), np.zeros(4)
    lr, eps = 0.01, 1e-8
    for t in range(1, 8):
        x_prev = x.copy()
        oracle_mod.adam_update(x, g, m, v, t, lr, 0.9, 0.999, eps)
        np.testing.assert_allclose(x - x_prev, -lr * g / (np.abs(g) + eps), rtol=1e-12)


def test_adam_alternating_gradient_closed_form(oracle_mod):
    """g_k = (-1)^k g: the first moment sums to
    (1 - b1) g (-1)^t (1 - (-b1)^t) / (1 + b1), the second to (1 - b2^t) g^2."""
    g = np.array([2.0, -0.5])
    b1, b2, lr, eps = 0.9, 0.999, 0.1, 1e-8
    x = np.zeros(2)
    m, v = np.zeros(2), np.zeros(2)
    for t in range(1, 12):
        x_prev = x.copy()
        oracle_mod.adam_update(x, (-1) ** t * g, m, v, t, lr, b1, b2, eps)
        mhat = (1 - b1) * g * (-1) ** t * (1 - (-b1) ** t) / ((1 + b1) * (1 - b1 ** t))
        np.testing.assert_allclose(x - x_prev, -lr * mhat / (np.abs(g) + eps), rtol=1e-11)


def test_adam_epoch_of_minibatches_lowers_the_loss(oracle_mod):
    """One shuffled epoch of Alg. 1 (minibatches of 5 frames) from a perturbed
    start lowers the full loss, and never moves alpha_0 or pixels off the support."""
    spec, p, P, y, rho, u, alpha, rng = _tiny(oracle_mod)
    chi, alpha_t = np.log(np.clip(rho, 0.2, None)), np.log(alpha)
    mask = np.ones((spec.n1, spec.n2))
    mask[0, :] = 0.0
    f0 = p.loss_grad_log(chi, u, alpha_t, P, y, mask=mask)[0]
    chi0 = chi.copy()
    opt = oracle_mod.OracleAdam(p, P, y, mask=mask, lr_u=0.01, lr_chi=0.02, lr_alpha=0.02)
    order = synth.epoch_order(spec.nframes, 7)
    for k in range(0, spec.nframes, 5):
        opt.step(order[k:k + 5], chi, u, alpha_t)
    f1 = p.loss_grad_log(chi, u, alpha_t, P, y, mask=mask)[0]
    assert f1 < f0, (f1, f0)
    assert alpha_t[0] == math.log(alpha[0])
    np.testing.assert_array_equal(chi[0], chi0[0])
    assert opt.t.value == -(-spec.nframes // 5)


def test_illumination_closed_forms(oracle_mod):
    """A constant probe of amplitude c over a scan that tiles the grid once
    gives c^2 per peak everywhere; a single frame gives |P|^2 itself, cut by
    the grid edge; per-peak probes add up."""
    D, m = 2, 4
    G = np.eye(3)[:D]
    scan = np.array([[0, 0], [0, 4], [4, 0], [4, 4]], np.int32)
    p = oracle_mod.OracleProblem(8, 8, 3, D, m, scan, G)
    ill = p.illumination(np.full((m, m), 1.5 + 2.0j))
    np.testing.assert_allclose(ill, D * 6.25 * np.ones((8, 8)), rtol=1e-14)
    rng = np.random.default_rng(9)
    P = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    one = oracle_mod.OracleProblem(6, 7, 3, 1, m, np.array([[3, -1]], np.int32), G[:1])
    ill = one.illumination(P)
    ref = np.zeros((6, 7))
    ref[3:6, 0:3] = np.abs(P[0:3, 1:4]) ** 2
    np.testing.assert_allclose(ill, ref, rtol=1e-14, atol=0)
    pp = oracle_mod.OracleProblem(8, 8, 3, D, m, scan, G, probe_per_peak=True)
    P2 = np.stack([np.full((m, m), 1.0 + 0j), np.full((m, m), 2.0 + 0j)])
    np.testing.assert_allclose(pp.illumination(P2), 5.0 * np.ones((8, 8)), rtol=1e-14)
