"""GPU phase unwrapping and the projector Pi_U (Eq. 9-10) against the oracle.

For maps without residues the unwrapped result does not depend on the order
in which edges are joined, so the GPU (Boruvka rounds, FP32 reliabilities)
and the oracle (sorted sweep, FP64) must agree element-wise after both pin
each region to its first pixel.  With residues the two may pick different
spanning trees where reliabilities are nearly tied, so there the checks are
the properties every result has: it wraps back to the input, and a noisy
patch stays confined.
"""
import math

import numpy as np
import pytest

from helpers import custom_spec, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TWO_PI = 2 * math.pi


def _wrap(x):
    return x - TWO_PI * np.floor(x / TWO_PI + 0.5)


def _smooth(rng, n1, n2, amp=15.0, k=6):
    i, j = np.mgrid[0:n1, 0:n2].astype(float)
    phi = np.zeros((n1, n2))
    for _ in range(k):
        ci, cj = rng.uniform(0, n1), rng.uniform(0, n2)
        s = rng.uniform(0.25, 0.45) * min(n1, n2)
        phi += rng.uniform(-amp, amp) * np.exp(-((i - ci) ** 2 + (j - cj) ** 2) / (2 * s * s))
    return phi + 0.7 * i - 0.4 * j


def _problem(n, D, G=None):
    from paper_2312_14907_gb300 import mpbp
    spec, scan = custom_spec(n, 16, 2, 8, npeaks=D, ncomp=2 if G is not None else 3, offset=0)
    if G is not None:
        spec.G = np.asarray(G, float)
    return mpbp.Problem.from_spec(spec, scan), spec


def test_unwrap_matches_oracle_on_residue_free_maps():
    import oracle
    rng = np.random.default_rng(1)
    p, spec = _problem(64, 3)
    n = spec.n1
    phi = np.stack([_smooth(rng, n, n) for _ in range(3)])
    w = _wrap(phi).astype(np.float32)
    mask = np.zeros((n, n), np.float32)
    mask[2:30, 3:60] = 1.0
    mask[34:62, 5:50] = 1.0
    for msk in (None, mask):
        got = p.unwrap_phases(torch.from_numpy(w).cuda(),
                              None if msk is None else torch.from_numpy(msk).cuda()).cpu().numpy()
        for m in range(3):
            ref = oracle.unwrap2d(w[m].astype(np.float64), msk)
            assert np.abs(got[m] - ref).max() <= 1e-3, (m, np.abs(got[m] - ref).max())
    p.sync_status()


def test_unwrap_properties_with_residues():
    import oracle
    rng = np.random.default_rng(2)
    p, spec = _problem(64, 3)
    n = spec.n1
    phi = np.stack([_smooth(rng, n, n) for _ in range(3)])
    noisy = phi.copy()
    noisy[:, 26:32, 30:36] = rng.uniform(-40, 40, (3, 6, 6))
    w = _wrap(noisy).astype(np.float32)
    got = p.unwrap_phases(torch.from_numpy(w).cuda()).cpu().numpy()
    d = got - w
    np.testing.assert_allclose(d, TWO_PI * np.round(d / TWO_PI), atol=1e-3)
    far = np.ones((n, n), bool)
    far[23:35, 27:39] = False
    for m in range(3):
        dd = (got[m] - phi[m])[far]
        k = np.round(dd / TWO_PI)
        assert np.all(k == k[0]), m
        ref = oracle.unwrap2d(w[m].astype(np.float64))
        assert np.abs(got[m] - ref)[far].max() <= 1e-3
    p.sync_status()


def test_unwrap_full_size_maps():
    """Three 256 x 256 maps, as many pixels as the bench object: exact
    recovery of residue-free maps up to one multiple of 2 pi each."""
    rng = np.random.default_rng(3)
    p, spec = _problem(256, 3)
    phi = np.stack([_smooth(rng, 256, 256, amp=30.0, k=10) for _ in range(3)])
    w = _wrap(phi).astype(np.float32)
    got = p.unwrap_phases(torch.from_numpy(w).cuda()).cpu().numpy()
    for m in range(3):
        d = got[m] - phi[m]
        k = np.round(d / TWO_PI)
        assert np.all(k == k.flat[0])
        assert np.abs(d - TWO_PI * k).max() <= 2e-3
    p.sync_status()


def test_projector_matches_oracle_and_removes_lattice_jumps():
    import oracle
    G = [[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]]
    p, spec = _problem(48, 3, G=G)
    n = spec.n1
    rng = np.random.default_rng(4)
    u = np.stack([_smooth(rng, n, n, amp=5.0) / (2 * TWO_PI) for _ in range(2)])
    u_jump = u.copy()
    u_jump[0, 8:30, 10:40] += 1.0
    u_jump[1, 20:44, 4:20] -= 1.0
    mask = np.ones((n, n), np.float32)
    mask[:, :3] = 0.0
    ud = torch.from_numpy(u_jump.astype(np.float32)).cuda()
    md = torch.from_numpy(mask).cuda()
    got = p.project_displacement(ud, md).cpu().numpy()
    orc = oracle.OracleProblem(n, n, 2, 3, 16, np.zeros((1, 2), np.int32), np.asarray(G))
    ref = orc.project_u(u_jump.astype(np.float32).astype(np.float64), mask)
    assert np.abs(got - ref).max() <= 1e-4
    inside = mask != 0
    for c in range(2):
        d = (got[c] - u[c])[inside]
        np.testing.assert_allclose(d, np.round(d[0]) * np.ones_like(d), atol=1e-4)
    np.testing.assert_array_equal(got[:, ~inside], u_jump.astype(np.float32)[:, ~inside])
    again = p.project_displacement(torch.from_numpy(got).cuda(), md).cpu().numpy()
    assert np.abs(again - got).max() <= 1e-4
    p.sync_status()


def test_unwrap_barrier_wait_runs_out_and_reports():
    """The unwrapper's grid barriers are bounded: with block 0 never arriving
    (the test hook), the other blocks give up after their time limit, the call
    reports MPBP_ERR_TIMEOUT, and the context then unwraps as the oracle
    does again."""
    import time
    import oracle
    from paper_2312_14907_gb300 import mpbp
    rng = np.random.default_rng(5)
    p, spec = _problem(96, 2)
    n = spec.n1
    phi = np.stack([_smooth(rng, n, n) for _ in range(spec.npeaks)])
    wrapped = torch.from_numpy(_wrap(phi).astype(np.float32)).cuda()
    p.set_test_stall(True)
    t0 = time.time()
    p.unwrap_phases(wrapped)
    with pytest.raises(mpbp.MPBPError) as e:
        p.sync_status()
    assert e.value.status == 5, e.value           # MPBP_ERR_TIMEOUT
    assert time.time() - t0 < 20.0
    p.set_test_stall(False)
    got = p.unwrap_phases(wrapped).cpu().numpy()
    p.sync_status()
    w = _wrap(phi).astype(np.float32)
    for d in range(spec.npeaks):
        ref = oracle.unwrap2d(w[d].astype(np.float64), None)
        assert np.abs(got[d] - ref).max() <= 1e-3, (d, np.abs(got[d] - ref).max())
