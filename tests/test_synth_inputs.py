"""The seeded input recipe (synth.py) against its stated shapes and
distributions: workload sizes and scan offsets, the batched set's frame
count, the probe's shape, the truth's support and displacement features,
the photon scaling, Poisson data and the epoch order.  No model arithmetic
is involved."""
import numpy as np
import pytest

from paper_2312_14907_gb300 import synth


@pytest.mark.parametrize("k,frames,offset", [(1, 147, 4), (2, 2883, 6), (3, 14884, 12), (5, 87846, -32)])
def test_workload_sizes_and_centred_scans(k, frames, offset):
    spec = synth.config(k)
    assert spec.nframes == frames and spec.offset == offset
    scan = synth.scan_positions(spec)
    assert scan.shape == (spec.nscan, 2) and scan.dtype == np.int32
    # row-major raster starting at (offset, offset) with the stated step
    assert tuple(scan[0]) == (offset, offset)
    assert tuple(scan[1]) == (offset, offset + spec.step)
    assert tuple(scan[spec.scan_side]) == (offset + spec.step, offset)
    # centred: the scanned span overhangs both ends of the grid equally (to a pixel)
    last = scan[-1, 0] + spec.m
    assert abs((spec.n1 - last) - offset) <= 1


def test_batched_set():
    specs = synth.batched_configs()
    assert len(specs) == 16
    assert sum(s.nframes for s in specs) == 90844
    for s in specs:
        assert 128 <= s.n1 <= 512 and s.m in (32, 64, 128) and s.m <= s.n1 // 2
        assert s.npeaks in (3, 4) and 15 <= s.scan_side <= 61


def test_probe_shape():
    spec = synth.config(2)
    P = synth.probe(spec)
    m = spec.m
    assert P.shape == (m, m)
    assert np.unravel_index(np.argmax(np.abs(P)), P.shape) == (m // 2, m // 2)
    assert abs(np.abs(P).max() - 1.0) < 1e-12
    # amplitude sigma 6 M / 32 px: at one sigma along a row the amplitude is e^-1/2
    s = int(round(spec.sigma))
    assert abs(spec.sigma - 12.0) < 1e-12
    np.testing.assert_allclose(abs(P[m // 2, m // 2 + s]), np.exp(-0.5), rtol=1e-12)
    # quadratic phase 0.01 (32/M)^2 rad/px^2 about the centre
    np.testing.assert_allclose(np.angle(P[m // 2, m // 2 + 4] / P[m // 2, m // 2]), spec.quad * 16, rtol=1e-12)


def test_truth_support_and_features():
    spec = synth.config(2)
    rho, u = synth.truth(spec)
    n = spec.n1
    side = int(round(0.75 * n))
    a = (n - side) // 2
    assert np.all(rho[a:a + side, a:a + side] == 1.0)
    assert rho.sum() == side * side
    assert u.shape == (spec.ncomp, n, n)
    # bumps of amplitude 0.3 plus jumps of 0.5 lattice units: bounded, with
    # discontinuities (neighbour differences near a jump's size somewhere)
    assert np.abs(u).max() < 0.3 * spec.bumps + 0.5 * (spec.straight + spec.curved) + 1e-9
    d = np.abs(np.diff(u, axis=2)).max()
    assert d > 0.2


def test_photon_scale_and_poisson_counts():
    rng = np.random.default_rng(0)
    I = rng.uniform(0, 1, (3, 5, 8, 8))
    s = synth.photon_scale(I, 1e4)
    totals = (I * s).reshape(15, -1).sum(axis=1)
    assert abs(totals.max() - 1e4) < 1e-6
    y1, y2 = synth.poisson_counts(I * s, 7), synth.poisson_counts(I * s, 7)
    np.testing.assert_array_equal(y1, y2)
    assert y1.dtype == np.float32 and np.all(y1 >= 0) and np.all(y1 == np.round(y1))
    # the sample mean follows the means (many draws: within a few standard errors)
    assert abs(y1.sum() - (I * s).sum()) < 6 * np.sqrt((I * s).sum())


def test_epoch_order_is_a_seeded_permutation():
    a, b = synth.epoch_order(2883, 5), synth.epoch_order(2883, 5)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(np.sort(a), np.arange(2883))
    assert not np.array_equal(a, synth.epoch_order(2883, 6))
