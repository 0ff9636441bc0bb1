"""Pins of the oracle's phase unwrapper and of the projector Pi_U (Eq. 9-10).

Facts that hold whatever the processing order: a residue-free phase map is
recovered exactly up to one multiple of 2 pi (pinned to the first pixel's
wrapped value), wrapping the output gives back the input on any data,
disconnected mask regions are unwrapped on their own, and Pi_U removes a
lattice-vector jump of the displacement (Eq. 6), is idempotent, and leaves
components outside the span of the G_m and pixels off the mask alone.
"""
import math

import numpy as np

TWO_PI = 2 * math.pi


def _wrap(x):
    return x - TWO_PI * np.floor(x / TWO_PI + 0.5)


def _smooth_phase(rng, n1, n2, amp=15.0, k=6):
    i, j = np.mgrid[0:n1, 0:n2].astype(float)
    phi = np.zeros((n1, n2))
    for _ in range(k):
        ci, cj = rng.uniform(0, n1), rng.uniform(0, n2)
        s = rng.uniform(0.25, 0.45) * min(n1, n2)
        phi += rng.uniform(-amp, amp) * np.exp(-((i - ci) ** 2 + (j - cj) ** 2) / (2 * s * s))
    phi += 0.7 * i - 0.4 * j
    # residue-free: every neighbour difference well inside (-pi, pi)
    assert np.abs(np.diff(phi, axis=0)).max() < 2.0 and np.abs(np.diff(phi, axis=1)).max() < 2.0
    return phi


def test_smooth_map_recovered_up_to_one_multiple_of_2pi(oracle_mod):
    rng = np.random.default_rng(1)
    phi = _smooth_phase(rng, 48, 40)
    w = _wrap(phi)
    out = oracle_mod.unwrap2d(w)
    d = out - phi
    k = np.round(d / TWO_PI)
    assert np.all(k == k.flat[0])
    np.testing.assert_allclose(d, TWO_PI * k, atol=1e-9)
    assert abs(out[0, 0] - w[0, 0]) <= 1e-12


def test_linear_ramp(oracle_mod):
    i, j = np.mgrid[0:20, 0:31].astype(float)
    phi = 2.9 * i - 1.7 * j + 0.3
    out = oracle_mod.unwrap2d(_wrap(phi))
    np.testing.assert_allclose(out, phi, atol=1e-9)


def test_wrapping_the_output_gives_the_input_on_any_data(oracle_mod):
    rng = np.random.default_rng(2)
    w = rng.uniform(-math.pi, math.pi, (30, 27))          # residues everywhere
    out = oracle_mod.unwrap2d(w)
    np.testing.assert_allclose(_wrap(out), w, atol=1e-9)
    assert np.all(np.abs(np.round((out - w) / TWO_PI) * TWO_PI - (out - w)) < 1e-9)


def test_mask_regions_are_unwrapped_on_their_own(oracle_mod):
    rng = np.random.default_rng(3)
    phi = _smooth_phase(rng, 40, 40)
    mask = np.zeros((40, 40))
    mask[2:18, 3:37] = 1.0                                  # region A
    mask[22:38, 5:30] = 1.0                                 # region B, apart from A
    w = _wrap(phi)
    out = oracle_mod.unwrap2d(w, mask)
    off = mask == 0
    np.testing.assert_array_equal(out[off], w[off])
    for sl in (np.s_[2:18, 3:37], np.s_[22:38, 5:30]):
        d = out[sl] - phi[sl]
        k = np.round(d / TWO_PI)
        assert np.all(k == k.flat[0])
        assert abs(out[sl].flat[0] - w[sl].flat[0]) <= 1e-12   # the region's first pixel


def _projector_problem(oracle_mod, ncomp):
    G = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])[:, :ncomp]
    scan = np.zeros((1, 2), np.int32)
    return oracle_mod.OracleProblem(36, 30, ncomp, 2, 8, scan, G)


def test_projector_removes_a_lattice_vector_jump(oracle_mod):
    """Eq. 6: u_x + 1 lattice unit on part of the object changes no phase wrap,
    so the wrapped phases cannot see it; Pi_U, unwrapping them, returns the
    smooth field up to one lattice vector."""
    p = _projector_problem(oracle_mod, 3)
    rng = np.random.default_rng(4)
    u = np.stack([_smooth_phase(rng, 36, 30, amp=8.0) / TWO_PI for _ in range(3)])
    u_jump = u.copy()
    u_jump[0, 10:25, 12:] += 1.0
    out = p.project_u(u_jump)
    for c in range(2):
        d = out[c] - u[c]
        np.testing.assert_allclose(d, np.round(d.flat[0]) * np.ones_like(d), atol=1e-9)
    np.testing.assert_array_equal(out[2], u_jump[2])        # u_z: no G_m has a z part


def test_projector_is_idempotent_and_keeps_pixels_off_the_mask(oracle_mod):
    p = _projector_problem(oracle_mod, 2)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((2, 36, 30)) * 0.8                # phases with residues
    mask = np.ones((36, 30))
    mask[:, :4] = 0.0
    once = p.project_u(u, mask)
    twice = p.project_u(once, mask)
    np.testing.assert_allclose(twice, once, atol=1e-9)
    np.testing.assert_array_equal(once[:, mask == 0], u[:, mask == 0])
    # the correction is a whole number of lattice units in each component here
    d = once - u
    np.testing.assert_allclose(d, np.round(d), atol=1e-9)


def test_reliable_paths_first_confine_a_noisy_patch(oracle_mod):
    """The point of sorting by reliability: a patch of random phases (full of
    residues) is joined last, so away from it the smooth map is recovered
    with a single multiple of 2 pi.  Taking edges in the wrong order, or
    with the second differences unwrapped, lets the patch's errors spread."""
    rng = np.random.default_rng(6)
    phi = _smooth_phase(rng, 48, 48)
    noisy = phi.copy()
    noisy[20:26, 22:28] = rng.uniform(-40, 40, (6, 6))
    out = oracle_mod.unwrap2d(_wrap(noisy))
    far = np.ones_like(phi, bool)
    far[17:29, 19:31] = False
    d = (out - phi)[far]
    k = np.round(d / TWO_PI)
    assert np.all(k == k[0])
    np.testing.assert_allclose(d, TWO_PI * k, atol=1e-9)


def test_projector_with_non_orthogonal_peaks(oracle_mod):
    """Three in-plane peaks (1,0), (0,1), (1,1): a jump of (1, 0) lattice units
    shifts the three phases by 2 pi (1, 0, 1), invisible to wrapping; the
    pseudo-inverse maps the unwrapped phases back to the smooth field."""
    G = np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    p = oracle_mod.OracleProblem(36, 30, 2, 3, 8, np.zeros((1, 2), np.int32), G)
    rng = np.random.default_rng(7)
    u = np.stack([_smooth_phase(rng, 36, 30, amp=5.0) / (2 * TWO_PI) for _ in range(2)])
    u_jump = u.copy()
    u_jump[0, 5:20, 8:22] += 1.0
    out = p.project_u(u_jump)
    for c in range(2):
        d = out[c] - u[c]
        np.testing.assert_allclose(d, d.flat[0] * np.ones_like(d), atol=1e-9)
