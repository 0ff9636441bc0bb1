"""Pins of the oracle's scan positions off the pixel grid.

Eq. 2's shift S_j moves the object laterally by the scan position s_j.  For
s_j = n_j + d_j (n_j integer, |d_j| <= 1/2) the exit wave sampled on the
object's pixels is P(k - d_j) O(n_j + k): the frame keeps the integer window
and takes the probe shifted by d_j, the band-limited interpolation of P
(oracle.probe_shift), as one probe per frame (probe_per_peak = 2).

Each pin checks a closed form, a composition law, a norm identity, the
direction of the shift, or finite differences; none re-types the shift.
"""
import numpy as np
import pytest

from paper_2312_14907_gb300 import synth


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("m", [8, 16])
def test_zero_offset_is_the_identity(oracle_mod, m):
    P = _rand_c(np.random.default_rng(1), (m, m))
    np.testing.assert_allclose(oracle_mod.probe_shift(P, 0.0, 0.0), P, rtol=0, atol=1e-13)


@pytest.mark.parametrize("m", [8, 16])
def test_two_half_pixel_shifts_are_one_pixel_roll(oracle_mod, m):
    """Composition: shifting by 1/2 twice is the circular shift by one pixel,
    P(k - 1): row k takes row k - 1 (the sign of the shift and the axis)."""
    P = _rand_c(np.random.default_rng(2), (m, m))
    h0 = oracle_mod.probe_shift(oracle_mod.probe_shift(P, 0.5, 0.0), 0.5, 0.0)
    np.testing.assert_allclose(h0, np.roll(P, 1, axis=0), rtol=0, atol=1e-12)
    h1 = oracle_mod.probe_shift(oracle_mod.probe_shift(P, 0.0, -0.5), 0.0, -0.5)
    np.testing.assert_allclose(h1, np.roll(P, -1, axis=1), rtol=0, atol=1e-12)
    # shifts along the two axes commute and add
    a = oracle_mod.probe_shift(oracle_mod.probe_shift(P, 0.3, 0.0), 0.0, -0.2)
    b = oracle_mod.probe_shift(P, 0.3, -0.2)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
    c = oracle_mod.probe_shift(oracle_mod.probe_shift(P, 0.3, 0.1), -0.45, 0.25)
    np.testing.assert_allclose(c, oracle_mod.probe_shift(P, -0.15, 0.35), rtol=0, atol=1e-12)


@pytest.mark.parametrize("q0,q1", [(1, 0), (0, 3), (-3, 2), (2, -1)])
def test_fourier_mode_takes_a_phase(oracle_mod, q0, q1):
    """A band-limited mode exp(2 pi i q.k/M) with |q| < M/2 shifted by d is
    the same mode times exp(-2 pi i q.d/M); negative q pins the frequency
    range [-M/2, M/2)."""
    m = 8
    k0, k1 = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    mode = np.exp(2j * np.pi * (q0 * k0 + q1 * k1) / m)
    d0, d1 = 0.37, -0.21
    ref = mode * np.exp(-2j * np.pi * (q0 * d0 + q1 * d1) / m)
    np.testing.assert_allclose(oracle_mod.probe_shift(mode, d0, d1), ref, rtol=0, atol=1e-13)


def test_shift_preserves_the_norm(oracle_mod):
    """Parseval: the shift only changes phases of the spectrum."""
    rng = np.random.default_rng(3)
    for m in (8, 16):
        P = _rand_c(rng, (m, m))
        for d in ((0.5, 0.5), (-0.13, 0.41), (0.5, -0.5)):
            Q = oracle_mod.probe_shift(P, *d)
            assert abs(np.linalg.norm(Q) - np.linalg.norm(P)) <= 1e-12 * np.linalg.norm(P)


def test_smooth_probe_moves_by_the_offset(oracle_mod):
    """A wide Gaussian probe well inside the window: the centroid of |P_d|^2
    sits d pixels further along (the exit wave P(r - s) follows the scan)."""
    m = 32
    k0, k1 = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    P = np.exp(-((k0 - 15.3) ** 2 + (k1 - 16.1) ** 2) / (2 * 3.0 ** 2)) * np.exp(0.02j * (k0 - 16) ** 2)

    def centroid(Z):
        w = np.abs(Z) ** 2
        return np.array([(w * k0).sum(), (w * k1).sum()]) / w.sum()

    for d in ((0.25, 0.0), (0.0, -0.4), (0.5, 0.3)):
        np.testing.assert_allclose(centroid(oracle_mod.probe_shift(P, *d)) - centroid(P), d, atol=2e-6)


def _subpixel_problem(oracle_mod, n=12, m=8, D=2, seed=31):
    scan = np.array([[-2, -1], [0, 3], [3, 0], [4, 4], [1, -3]], np.int32)
    G = np.array([[1.0, 0.0, 0.0], [0.6, 0.8, 0.0]])[:D]
    rng = np.random.default_rng(seed)
    P = _rand_c(rng, (m, m))
    offs = rng.uniform(-0.5, 0.5, (scan.shape[0], 2))
    rho = rng.uniform(0.5, 1.5, (n, n))
    u = rng.standard_normal((3, n, n)) * 0.2
    alpha = np.array([1.0, 0.8])[:D]
    y = rng.poisson(30.0, (D, scan.shape[0], m, m)).astype(float)
    return scan, G, P, offs, rho, u, alpha, y


def test_per_frame_probes_with_zero_offsets_match_the_shared_probe(oracle_mod):
    scan, G, P, offs, rho, u, alpha, y = _subpixel_problem(oracle_mod)
    D, m, n = G.shape[0], P.shape[0], rho.shape[0]
    p1 = oracle_mod.OracleProblem(n, n, 3, D, m, scan, G)
    p2 = oracle_mod.OracleProblem(n, n, 3, D, m, scan, G, probe_per_peak=2)
    Pf = oracle_mod.frame_probes(p2, P, np.zeros_like(offs))
    r1 = p1.loss_grad(rho, u, alpha, P, y)
    r2 = p2.loss_grad(rho, u, alpha, Pf, y)
    assert abs(r1[0] - r2[0]) <= 1e-13 * r1[0]
    for a, b in zip(r1[1:], r2[1:]):
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-12 * np.abs(a).max())
    np.testing.assert_allclose(p2.illumination(Pf), p1.illumination(P), rtol=1e-13)


def test_frame_probes_follow_frame_order(oracle_mod):
    """Frame f = m J + j of a per-frame problem uses probe f: a frame's
    intensity equals the one-probe forward model with that frame's probe."""
    scan, G, P, offs, rho, u, alpha, y = _subpixel_problem(oracle_mod)
    D, m, n, J = G.shape[0], P.shape[0], rho.shape[0], scan.shape[0]
    p2 = oracle_mod.OracleProblem(n, n, 3, D, m, scan, G, probe_per_peak=2)
    Pf = oracle_mod.frame_probes(p2, P, offs)
    I = p2.forward(rho, u, alpha, Pf)
    p1 = oracle_mod.OracleProblem(n, n, 3, D, m, scan, G)
    for f in (0, J - 1, J + 2, 2 * J - 1):
        mpk, j = divmod(f, J)
        I1 = p1.forward(rho, u, alpha, Pf[f])
        np.testing.assert_allclose(I[mpk, j], I1[mpk, j], rtol=1e-12, atol=1e-12 * I1.max())


def test_gradient_fd_with_per_frame_probes(oracle_mod):
    scan, G, P, offs, rho, u, alpha, y = _subpixel_problem(oracle_mod)
    D, m, n = G.shape[0], P.shape[0], rho.shape[0]
    p = oracle_mod.OracleProblem(n, n, 3, D, m, scan, G, probe_per_peak=2)
    Pf = oracle_mod.frame_probes(p, P, offs)
    f0, gr, gu, ga = p.loss_grad(rho, u, alpha, Pf, y)
    h = 1e-5
    for (i, j) in [(0, 0), (5, 6), (11, 3), (2, 9)]:
        for arr, g, idx in ((rho, gr, (i, j)), (u, gu, (2, i, j))):
            arr[idx] += h
            fp = p.loss(rho, u, alpha, Pf, y)
            arr[idx] -= 2 * h
            fm = p.loss(rho, u, alpha, Pf, y)
            arr[idx] += h
            assert abs((fp - fm) / (2 * h) - g[idx]) <= 1e-6 * np.abs(g).max()
    alpha[1] += h
    fp = p.loss(rho, u, alpha, Pf, y)
    alpha[1] -= 2 * h
    fm = p.loss(rho, u, alpha, Pf, y)
    alpha[1] += h
    assert abs((fp - fm) / (2 * h) - ga[1]) <= 1e-6 * abs(ga[1])


def test_half_pixel_scan_of_a_flat_object(oracle_mod):
    """rho = 1, u = 0, alpha = 1 and a frame inside the grid: every frame's
    intensity is |F P_d|^2 = |F P|^2, whatever d (the shift only puts a
    linear phase on the probe's spectrum)."""
    n, m = 16, 8
    scan = np.array([[2, 3], [4, 4]], np.int32)
    G = np.array([[1.0, 0.0, 0.0]])
    rng = np.random.default_rng(5)
    P = _rand_c(rng, (m, m))
    p = oracle_mod.OracleProblem(n, n, 3, 1, m, scan, G, probe_per_peak=2)
    Pf = oracle_mod.frame_probes(p, P, np.array([[0.5, -0.5], [0.23, 0.31]]))
    I = p.forward(np.ones((n, n)), np.zeros((3, n, n)), np.ones(1), Pf)
    ref = np.abs(np.fft.fft2(P)) ** 2
    for j in range(2):
        np.testing.assert_allclose(I[0, j], ref, rtol=1e-10, atol=1e-10 * ref.max())


def test_per_peak_probes_are_shifted_per_frame(oracle_mod):
    """With one probe per peak, frame f = m J + j takes P_m shifted by d_j."""
    scan, G, P, offs, rho, u, alpha, y = _subpixel_problem(oracle_mod)
    D, m, n, J = G.shape[0], P.shape[0], rho.shape[0], scan.shape[0]
    rng = np.random.default_rng(9)
    Pp = _rand_c(rng, (D, m, m))
    p2 = oracle_mod.OracleProblem(n, n, 3, D, m, scan, G, probe_per_peak=2)
    Pf = oracle_mod.frame_probes(p2, Pp, offs)
    assert Pf.shape == (D * J, m, m)
    for mpk in range(D):
        for j in (0, J - 1):
            ref = oracle_mod.probe_shift(Pp[mpk], offs[j, 0], offs[j, 1])
            np.testing.assert_array_equal(Pf[mpk * J + j], ref)
    # and the loss of a per-frame problem is the sum of its frames' losses,
    # each from the one-probe model with that frame's probe
    f_all, *_ = p2.loss_grad(rho, u, alpha, Pf, y)
    p1 = oracle_mod.OracleProblem(n, n, 3, D, m, scan, G)
    tot = 0.0
    for f in range(D * J):
        tot += p1.loss_grad(rho, u, alpha, Pf[f], y, frames=[f])[0]
    assert abs(tot - f_all) <= 1e-12 * f_all
