"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's formulas: each checks a closed form, an
invariance the paper states, a library special case, or finite differences.
"""
import math

import numpy as np
import pytest

from paper_2312_14907_gb300 import synth


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# --------------------------------------------------------------------------
# The far-field transform F of Eq. 2 (direct DFT inside the oracle)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m", [4, 8, 16])
def test_dft_closed_forms(oracle_mod, m):
    # delta at the origin -> all ones
    x = np.zeros((m, m), complex)
    x[0, 0] = 1
    np.testing.assert_allclose(oracle_mod.dft2(x), np.ones((m, m)), atol=1e-13)
    # constant c -> c M^2 delta
    c = 0.7 - 0.2j
    out = oracle_mod.dft2(np.full((m, m), c))
    ref = np.zeros((m, m), complex)
    ref[0, 0] = c * m * m
    np.testing.assert_allclose(out, ref, atol=1e-11 * m * m)
    # integer ramp exp(+2 pi i (a k0 + b k1)/M) -> M^2 at (a, b) only
    a, b = 1, m - 2
    k0, k1 = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    ramp = np.exp(2j * np.pi * (a * k0 + b * k1) / m)
    ref = np.zeros((m, m), complex)
    ref[a, b] = m * m
    np.testing.assert_allclose(oracle_mod.dft2(ramp), ref, atol=1e-11 * m * m)
    # shifted delta -> exp(-2 pi i q.k'/M): fixes the sign of the exponent and
    # which index is the row
    x = np.zeros((m, m), complex)
    x[a, b + 1 - m] = 1
    q0, q1 = k0, k1
    ref = np.exp(-2j * np.pi * (q0 * a + q1 * ((b + 1) % m)) / m)
    np.testing.assert_allclose(oracle_mod.dft2(x), ref, atol=1e-13)
    # the adjoint F^H maps the all-ones array to M^2 delta as well
    ref = np.zeros((m, m), complex)
    ref[0, 0] = m * m
    np.testing.assert_allclose(oracle_mod.dft2(np.ones((m, m)), +1), ref, atol=1e-11 * m * m)


@pytest.mark.parametrize("m", [8, 16, 32])
def test_dft_matches_numpy_fft(oracle_mod, m):
    """Library special case: F is NumPy's fft2 and F^H is M^2 ifft2."""
    rng = np.random.default_rng(7)
    x = _rand_c(rng, (m, m))
    np.testing.assert_allclose(oracle_mod.dft2(x, -1), np.fft.fft2(x), rtol=0, atol=1e-12 * m * m)
    np.testing.assert_allclose(oracle_mod.dft2(x, +1), np.fft.ifft2(x) * m * m, rtol=0,
                               atol=1e-12 * m * m)


@pytest.mark.parametrize("m", [8, 32])
def test_dft_parseval_and_adjoint(oracle_mod, m):
    rng = np.random.default_rng(11)
    x, y = _rand_c(rng, (m, m)), _rand_c(rng, (m, m))
    X = oracle_mod.dft2(x)
    assert abs(np.sum(abs(X) ** 2) - m * m * np.sum(abs(x) ** 2)) <= 1e-13 * m * m * np.sum(abs(x) ** 2)
    lhs = np.vdot(y, X)                      # <y, F x>
    rhs = np.vdot(oracle_mod.dft2(y, +1), x)  # <F^H y, x>
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs) * m


# --------------------------------------------------------------------------
# Eq. 1 / Eq. 3: the effective object
# --------------------------------------------------------------------------

def test_object_build_phase_convention(oracle_mod):
    """phi = 2 pi u.G: a quarter lattice unit along G = [100] is a quarter turn,
    half a unit along [010] is a half turn; alpha and rho scale the magnitude."""
    n = 6
    G = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    p = oracle_mod.OracleProblem(n, n, 3, 2, 4, np.zeros((1, 2)), G)
    rho = np.linspace(0.5, 2.0, n * n).reshape(n, n)
    u = np.zeros((3, n, n))
    u[0] = 0.25
    u[1] = 0.5
    u[2] = 0.123        # no effect: both G have l = 0
    alpha = np.array([1.0, 0.3])
    O = p.object_build(rho, u, alpha)
    np.testing.assert_allclose(O[0], 1j * rho, atol=1e-15)
    np.testing.assert_allclose(O[1], -0.3 * rho, atol=1e-15)


# --------------------------------------------------------------------------
# Eq. 2: forward model
# --------------------------------------------------------------------------

def test_flat_object_gives_probe_spectrum(oracle_mod):
    """rho = 1, u = 0, alpha = 1: every frame inside the grid is |FFT(P)|^2; a
    frame hanging over the edge sees the probe cut by the grid (zero outside)."""
    spec = synth.tiny(npeaks=3, n=16, m=8, side=3, step=3)
    rng = np.random.default_rng(3)
    P = synth.random_probe(spec, rng)
    scan = np.array([[0, 0], [8, 8], [4, 2], [-3, 5], [10, 13]], np.int32)
    p = oracle_mod.OracleProblem(16, 16, 3, 3, 8, scan, spec.G)
    I = p.forward(np.ones((16, 16)), np.zeros((3, 16, 16)), np.ones(3), P)
    full = abs(np.fft.fft2(P)) ** 2
    for d in range(3):
        for j in range(3):
            np.testing.assert_allclose(I[d, j], full, rtol=1e-12, atol=1e-12 * full.max())
        # frame 3 starts at row -3: rows 0..2 of the frame are outside
        Pm = P.copy()
        Pm[:3, :] = 0
        np.testing.assert_allclose(I[d, 3], abs(np.fft.fft2(Pm)) ** 2, atol=1e-11 * full.max())
        # frame 4 starts at (10, 13): only rows 0..5 and columns 0..2 are inside
        Pm = P.copy()
        Pm[:, 3:] = 0
        Pm[6:, :] = 0
        np.testing.assert_allclose(I[d, 4], abs(np.fft.fft2(Pm)) ** 2, atol=1e-11 * full.max())


def test_single_pixel_object_pins_shift_orientation(oracle_mod):
    """A one-pixel object at (r0, r1) seen by a frame with top-left s makes the
    exit wave a delta at k* = (r0 - s0, r1 - s1), so I is flat at |P(k*)|^2."""
    m, n = 8, 20
    rng = np.random.default_rng(5)
    P = _rand_c(rng, (m, m))
    scan = np.array([[3, 9], [9, 3], [12, 12], [0, 0]], np.int32)
    G = np.array([[1.0, 0.0, 0.0]])
    p = oracle_mod.OracleProblem(n, n, 3, 1, m, scan, G)
    rho = np.zeros((n, n))
    r0, r1 = 5, 11
    rho[r0, r1] = 2.0
    I = p.forward(rho, np.zeros((3, n, n)), np.ones(1), P)
    k = (r0 - 3, r1 - 9)
    np.testing.assert_allclose(I[0, 0], np.full((m, m), 4.0 * abs(P[k]) ** 2), rtol=1e-12)
    # the transposed scan position does not contain the pixel
    np.testing.assert_allclose(I[0, 1], 0.0, atol=1e-30)
    np.testing.assert_allclose(I[0, 2], 0.0, atol=1e-30)
    k = (r0, r1)
    assert r1 >= m  # outside frame 3 as well
    np.testing.assert_allclose(I[0, 3], 0.0, atol=1e-30)


def test_background_adds_to_intensity(oracle_mod):
    spec = synth.tiny()
    scan = synth.scan_positions(spec)
    p = oracle_mod.OracleProblem.from_spec(spec, scan)
    rng = np.random.default_rng(8)
    bg = rng.uniform(0, 3, (spec.npeaks, spec.nscan, spec.m, spec.m))
    I = p.forward(*synth.init_state(spec), np.zeros((spec.m, spec.m)), bg=bg)
    np.testing.assert_array_equal(I, bg)
    y = rng.poisson(2.0, bg.shape).astype(float)
    f = p.loss(*synth.init_state(spec), np.zeros((spec.m, spec.m)), y, bg=bg)
    assert abs(f - 0.5 * np.sum((np.sqrt(bg) - np.sqrt(y)) ** 2)) <= 1e-12 * f


# --------------------------------------------------------------------------
# Eq. 4: the loss
# --------------------------------------------------------------------------

def test_constant_probe_constant_patch_closed_form(oracle_mod):
    """P = p0 and O = o0 over the whole frame: Psi = M^2 p0 o0 at q = 0 only, so
    f = 1/2 [ (M^2 |p0 o0| - sqrt(y_0))^2 + sum_{q != 0} y_q ]."""
    m, n = 8, 8
    p0 = 0.3 + 0.4j
    rho0, ph = 1.7, 0.25
    G = np.array([[1.0, 0.0, 0.0]])
    p = oracle_mod.OracleProblem(n, n, 3, 1, m, np.zeros((1, 2), np.int32), G)
    u = np.zeros((3, n, n))
    u[0] = ph
    rng = np.random.default_rng(9)
    y = rng.poisson(5.0, (1, 1, m, m)).astype(float)
    f = p.loss(np.full((n, n), rho0), u, np.array([1.0]), np.full((m, m), p0), y)
    amp = m * m * abs(p0) * rho0
    ref = 0.5 * ((amp - math.sqrt(y[0, 0, 0, 0])) ** 2 + y.sum() - y[0, 0, 0, 0])
    assert abs(f - ref) <= 1e-12 * ref


def _tiny_problem(oracle_mod, ncomp=3, npeaks=2, seed=21, n=12, m=8, side=3, step=2):
    spec = synth.tiny(ncomp=ncomp, npeaks=npeaks, n=n, m=m, side=side, step=step)
    scan = synth.scan_positions(spec)
    p = oracle_mod.OracleProblem.from_spec(spec, scan)
    rng = np.random.default_rng(seed)
    P = synth.random_probe(spec, rng)
    rho_t, u_t = synth.truth(spec)
    I = p.forward(rho_t + 0.5, u_t, synth.alpha_truth(spec), P)
    y = synth.poisson_counts(I, seed).astype(np.float64) + 0.0
    rho, u, alpha = synth.perturbed_state(spec, rng, 0.1)
    alpha[1:] *= 1.1
    return spec, p, P, y, rho, u, alpha


def test_uniform_displacement_is_a_global_phase(oracle_mod):
    spec, p, P, y, rho, u, alpha = _tiny_problem(oracle_mod, npeaks=3)
    I0 = p.forward(rho, u, alpha, P)
    I1 = p.forward(rho, u + np.array([0.37, -1.2, 2.5])[:, None, None], alpha, P)
    np.testing.assert_allclose(I1, I0, rtol=1e-11, atol=1e-11 * I0.max())


def test_lattice_vector_ambiguity_eq6(oracle_mod):
    """Eq. 6b: adding m_d in Z to u.G_d at any pixel changes no object.
    For G = x, y, (1,1,1)/sqrt3, du = (1, 0, -1) gives u.G += (1, 0, 0)."""
    spec, p, P, y, rho, u, alpha = _tiny_problem(oracle_mod, npeaks=3)
    rng = np.random.default_rng(4)
    mask = rng.random(rho.shape) < 0.4
    u2 = u.copy()
    u2[0] += mask * 1.0
    u2[2] -= mask * 1.0
    f0 = p.loss(rho, u, alpha, P, y)
    f1 = p.loss(rho, u2, alpha, P, y)
    assert abs(f1 - f0) <= 1e-12 * f0


def test_single_peak_ambiguity_eq7(oracle_mod):
    """Eq. 6c / Eq. 7: with one peak G, u' = u + m G / |G|^2 for any integer field
    m (all ones, or alternating +5/-5) produces the same diffraction patterns."""
    n, m = 12, 8
    G = np.array([[1.0, 1.0, 0.0]])       # [110]
    spec = synth.tiny(npeaks=1)
    scan = synth.scan_positions(spec)
    p = oracle_mod.OracleProblem(n, n, 3, 1, m, scan, G)
    rng = np.random.default_rng(6)
    P = _rand_c(rng, (m, m))
    rho = rng.uniform(0.5, 1.5, (n, n))
    u = rng.standard_normal((3, n, n)) * 0.3
    I0 = p.forward(rho, u, np.ones(1), P)
    for field in (np.ones((n, n)), 5.0 * (-1.0) ** np.arange(n * n).reshape(n, n)):
        u2 = u + field[None] * (G[0] / (G[0] @ G[0]))[:, None, None]
        I1 = p.forward(rho, u2, np.ones(1), P)
        np.testing.assert_allclose(I1, I0, rtol=1e-10, atol=1e-10 * I0.max())


def test_zero_loss_and_gradient_on_noise_free_data(oracle_mod):
    spec, p, P, y, rho, u, alpha = _tiny_problem(oracle_mod, npeaks=3)
    y0 = p.forward(rho, u, alpha, P)
    f, gr, gu, ga = p.loss_grad(rho, u, alpha, P, y0)
    assert f <= 1e-24 * y0.sum()
    assert np.abs(gr).max() <= 1e-10 and np.abs(gu).max() <= 1e-10 and np.abs(ga).max() <= 1e-10


# --------------------------------------------------------------------------
# The gradient
# --------------------------------------------------------------------------

def _fd_check(p, P, y, rho, u, alpha, rng, npts=6):
    f0, gr, gu, ga = p.loss_grad(rho, u, alpha, P, y)
    worst = 0.0
    n1, n2 = rho.shape

    def central(setter, x0):
        h = 1e-5 * max(1.0, abs(x0))
        setter(x0 + h)
        fp = p.loss(rho, u, alpha, P, y)
        setter(x0 - h)
        fm = p.loss(rho, u, alpha, P, y)
        setter(x0)
        return (fp - fm) / (2 * h)

    scale = max(np.abs(gr).max(), np.abs(gu).max(), np.abs(ga).max())
    for _ in range(npts):
        i, j = rng.integers(0, n1), rng.integers(0, n2)
        x0 = rho[i, j]
        fd = central(lambda v: rho.__setitem__((i, j), v), x0)
        worst = max(worst, abs(fd - gr[i, j]) / scale)
        for c in range(u.shape[0]):
            x0 = u[c, i, j]
            fd = central(lambda v: u.__setitem__((c, i, j), v), x0)
            worst = max(worst, abs(fd - gu[c, i, j]) / scale)
    for d in range(alpha.size):
        fd = central(lambda v: alpha.__setitem__(d, v), alpha[d])
        worst = max(worst, abs(fd - ga[d]) / max(abs(ga[d]), 1e-30 + scale * 1e-3))
    return worst


@pytest.mark.parametrize("ncomp,npeaks", [(3, 2), (3, 3), (2, 2), (3, 4)])
def test_gradient_matches_central_differences(oracle_mod, ncomp, npeaks):
    spec, p, P, y, rho, u, alpha = _tiny_problem(oracle_mod, ncomp=ncomp, npeaks=npeaks)
    worst = _fd_check(p, P, y, rho, u, alpha, np.random.default_rng(ncomp * 10 + npeaks))
    assert worst <= 1e-6, worst


def test_gradient_fd_with_edge_frames_and_per_peak_probe(oracle_mod):
    """Frames hanging over every edge of the grid, one probe per peak, background."""
    n, m, D = 10, 8, 2
    scan = np.array([[-4, -3], [5, 6], [-2, 6], [6, -5], [1, 1]], np.int32)
    G = np.array([[1.0, 0.0, 0.0], [0.6, 0.8, 0.0]])
    p = oracle_mod.OracleProblem(n, n, 3, D, m, scan, G, probe_per_peak=True)
    rng = np.random.default_rng(12)
    P = _rand_c(rng, (D, m, m))
    bg = rng.uniform(0, 1, (D, scan.shape[0], m, m))
    rho = rng.uniform(0.5, 1.5, (n, n))
    u = rng.standard_normal((3, n, n)) * 0.2
    alpha = np.array([1.0, 0.8])
    y = rng.poisson(30.0, bg.shape).astype(float)
    f0, gr, gu, ga = p.loss_grad(rho, u, alpha, P, y, bg=bg)
    h = 1e-5
    for (i, j) in [(0, 0), (9, 9), (0, 9), (4, 5)]:
        rho[i, j] += h
        fp = p.loss(rho, u, alpha, P, y, bg=bg)
        rho[i, j] -= 2 * h
        fm = p.loss(rho, u, alpha, P, y, bg=bg)
        rho[i, j] += h
        assert abs((fp - fm) / (2 * h) - gr[i, j]) <= 1e-6 * np.abs(gr).max()
        u[1, i, j] += h
        fp = p.loss(rho, u, alpha, P, y, bg=bg)
        u[1, i, j] -= 2 * h
        fm = p.loss(rho, u, alpha, P, y, bg=bg)
        u[1, i, j] += h
        assert abs((fp - fm) / (2 * h) - gu[1, i, j]) <= 1e-6 * np.abs(gu).max()


def test_translation_invariance_gives_zero_mean_du(oracle_mod):
    """A uniform shift of u_c multiplies each object by a constant phase, so
    sum_r df/du_c(r) = 0 at every state."""
    spec, p, P, y, rho, u, alpha = _tiny_problem(oracle_mod, npeaks=3)
    f, gr, gu, ga = p.loss_grad(rho, u, alpha, P, y)
    for c in range(3):
        assert abs(gu[c].sum()) <= 1e-10 * np.abs(gu[c]).sum()


def test_homogeneity_identities(oracle_mod):
    """b = 0: f(lambda rho) and f(lambda alpha) scale Psi by lambda, so
    sum rho df/drho = sum_m alpha_m df/dalpha_m = sum (|Psi| - a)|Psi|."""
    spec, p, P, y, rho, u, alpha = _tiny_problem(oracle_mod, npeaks=3)
    f, gr, gu, ga = p.loss_grad(rho, u, alpha, P, y)
    I = p.forward(rho, u, alpha, P)
    ref = np.sum((np.sqrt(I) - np.sqrt(y)) * np.sqrt(I))
    assert abs(np.sum(rho * gr) - ref) <= 1e-10 * abs(ref)
    assert abs(np.sum(alpha * ga) - ref) <= 1e-10 * abs(ref)


def test_in_plane_peaks_give_zero_out_of_plane_gradient(oracle_mod):
    spec, p, P, y, rho, u, alpha = _tiny_problem(oracle_mod, npeaks=4)
    f, gr, gu, ga = p.loss_grad(rho, u, alpha, P, y)
    assert np.abs(gu[2]).max() == 0.0
    assert np.abs(gu[0]).max() > 0


def test_uncovered_pixels_have_zero_gradient(oracle_mod):
    spec = synth.tiny(n=16, m=8, side=2, step=2)
    scan = synth.scan_positions(spec)
    p = oracle_mod.OracleProblem.from_spec(spec, scan)
    rng = np.random.default_rng(2)
    P = synth.random_probe(spec, rng)
    rho, u, alpha = synth.perturbed_state(spec, rng)
    y = rng.poisson(4.0, (spec.npeaks, spec.nscan, 8, 8)).astype(float)
    f, gr, gu, ga = p.loss_grad(rho, u, alpha, P, y)
    covered = np.zeros(rho.shape, bool)
    for s0, s1 in scan:
        covered[max(s0, 0):s0 + 8, max(s1, 0):s1 + 8] = True
    assert not covered.all()
    assert np.all(gr[~covered] == 0) and np.all(gu[:, ~covered] == 0)
    assert np.abs(gr[covered]).min() >= 0 and np.abs(gr[covered]).max() > 0


def test_frame_subsets_add_up(oracle_mod):
    """Eq. 11: the minibatch gradient is a plain sum over its frames."""
    spec, p, P, y, rho, u, alpha = _tiny_problem(oracle_mod, npeaks=3)
    nf = p.nframes
    perm = np.random.default_rng(1).permutation(nf)
    a, b = perm[: nf // 3], perm[nf // 3:]
    fa, gra, gua, gaa = p.loss_grad(rho, u, alpha, P, y, frames=a)
    fb, grb, gub, gab = p.loss_grad(rho, u, alpha, P, y, frames=b)
    f, gr, gu, ga = p.loss_grad(rho, u, alpha, P, y)
    assert abs(fa + fb - f) <= 1e-12 * f
    np.testing.assert_allclose(gra + grb, gr, atol=1e-12 * np.abs(gr).max())
    np.testing.assert_allclose(gua + gub, gu, atol=1e-12 * np.abs(gu).max())
    np.testing.assert_allclose(gaa + gab, ga, atol=1e-12 * np.abs(ga).max())
    f2, _, _, _, fl = p.loss_grad(rho, u, alpha, P, y, frames=perm, frame_loss=True)
    assert abs(fl.sum() - f) <= 1e-12 * f


def test_thread_count_does_not_change_results(oracle_mod):
    spec, p, P, y, rho, u, alpha = _tiny_problem(oracle_mod, npeaks=3)
    r1 = p.loss_grad(rho, u, alpha, P, y, nthreads=1)
    r3 = p.loss_grad(rho, u, alpha, P, y, nthreads=3)
    assert abs(r1[0] - r3[0]) <= 1e-13 * r1[0]
    for a, b in zip(r1[1:], r3[1:]):
        np.testing.assert_allclose(a, b, atol=1e-13 * np.abs(a).max())


# --------------------------------------------------------------------------
# The optimizer iteration (lagged Armijo gradient descent)
# --------------------------------------------------------------------------

def test_step_decreases_loss_with_armijo(oracle_mod):
    spec = synth.tiny(npeaks=3, n=16, m=8, side=4, step=2)
    scan = synth.scan_positions(spec)
    p = oracle_mod.OracleProblem.from_spec(spec, scan)
    P = synth.probe(spec)
    rho_t, u_t = synth.truth(spec)
    y = p.forward(rho_t, u_t, np.ones(3), P)        # noise free
    rho, u, alpha = synth.init_state(spec)
    st = oracle_mod.OracleStepper(p, P, y, t0=0.05, w_alpha=0.0)
    accepted = []
    for _ in range(60):
        f = st.step(rho, u, alpha)
        if st.state.accepted:
            accepted.append(f)
    assert st.state.n_accept + st.state.n_reject == 60
    assert all(b <= a for a, b in zip(accepted, accepted[1:]))
    assert accepted[-1] < accepted[0] / 10
    assert alpha[0] == 1.0


def test_step_bookkeeping_matches_a_replay_of_the_rule(oracle_mod):
    """The lagged-Armijo stepper against a replay of its stated rule, written
    here with the (separately pinned) loss and gradient: on each call
    evaluate f, g at the current point; accept on the first call, or when f
    <= f_prev - c t gn2_prev; on acceptance the point and its gradient become
    the base and t grows (not on the first call), on rejection t shrinks;
    the next point is base - t w g_base with alpha_0 held.  A first step
    length far too long forces rejections, and the rejected trials must lie
    on the line from the base point along the base gradient, each at
    `shrink` times the previous distance."""
    spec = synth.tiny(npeaks=3, n=16, m=8, side=4, step=2)
    scan = synth.scan_positions(spec)
    p = oracle_mod.OracleProblem.from_spec(spec, scan)
    P = synth.probe(spec)
    rho_t, u_t = synth.truth(spec)
    y = p.forward(rho_t, u_t, np.array([1.0, 0.8, 1.3]), P)
    rho, u, alpha = synth.init_state(spec)
    c, grow, shrink, t0, w = 1e-4, 1.25, 0.5, 0.2, (1.0, 0.5, 0.25)
    st = oracle_mod.OracleStepper(p, P, y, c_armijo=c, grow=grow, shrink=shrink, t0=t0,
                                  w_rho=w[0], w_u=w[1], w_alpha=w[2])
    # the replay's own state
    x = [rho.copy(), u.copy(), alpha.copy()]
    base, gbase, f_prev, gn2_prev, t = None, None, None, None, t0
    flags, ts = [], []
    for k in range(16):
        f, gr, gu, ga = p.loss_grad(x[0], x[1], x[2], P, y)
        accept = np.isfinite(f) if k == 0 else (np.isfinite(f) and f <= f_prev - c * t * gn2_prev)
        if accept:
            if k > 0:
                t *= grow
            base = [a.copy() for a in x]
            gbase = [gr.copy(), gu.copy(), ga.copy()]
            f_prev = f
            gn2_prev = w[0] * np.sum(gr * gr) + w[1] * np.sum(gu * gu) + w[2] * np.sum(ga[1:] ** 2)
        else:
            t *= shrink
        prev_trial = [a.copy() for a in x]
        x = [base[0] - t * w[0] * gbase[0], base[1] - t * w[1] * gbase[1],
             np.concatenate([[base[2][0]], base[2][1:] - t * w[2] * gbase[2][1:]])]
        f_lib = st.step(rho, u, alpha)
        assert abs(f_lib - f) <= 1e-12 * abs(f), k
        assert bool(st.state.accepted) == bool(accept), k
        assert abs(st.state.t - t) <= 1e-15 * t, k
        for got, want in zip((rho, u, alpha), x):
            np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * max(1.0, np.abs(want).max()))
        if not accept and k > 0:
            # the rejected trial and the new one lie on one ray from the base point
            for got, old, b in zip((rho, u, alpha), prev_trial, base):
                np.testing.assert_allclose(got - b, shrink * (old - b), rtol=0,
                                           atol=1e-12 * max(1.0, np.abs(old - b).max()))
        flags.append(bool(accept))
        ts.append(st.state.t)
    assert flags[0] and not flags[1], flags           # t0 far too long: the first trial fails
    assert any(flags[2:]) and sum(flags[1:]) >= 3, flags
    assert st.state.n_accept == sum(flags) and st.state.n_reject == len(flags) - sum(flags)
    assert alpha[0] == 1.0
