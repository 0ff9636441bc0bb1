"""Scan positions off the pixel grid on the GPU against the FP64 oracle.

The GPU forms the shifted probes P(k - d_j) itself (mpbp_set_scan_offsets,
FP32 separable sums with the closed-form interpolation kernel); the oracle
forms them through the DFT in FP64 (oracle.probe_shift).  Tolerances as in
test_gpu_parity: loss 1e-5 relative, gradients 1e-4 relative L2, probes
and intensities 1e-5 relative L2.
"""
import numpy as np
import pytest

import oracle
from helpers import Case, custom_spec, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-5
GRAD_TOL = 1e-4


def _offsets(J, seed):
    d = np.random.default_rng(seed).uniform(-0.5, 0.5, (J, 2))
    d[0] = (0.5, -0.5)        # the ends of the range
    if J > 1:
        d[1] = (0.0, 0.0)     # and an integer position
    return d


def _oracle_frames(case, d):
    spec = case.spec
    p2 = oracle.OracleProblem(spec.n1, spec.n2, spec.ncomp, spec.npeaks, spec.m, case.scan, spec.G,
                              spec.phase_scale, probe_per_peak=2)
    return p2, oracle.frame_probes(p2, case.probe, d)


def _gpu(case, d):
    from paper_2312_14907_gb300 import mpbp
    p = mpbp.Problem.from_spec(case.spec, case.scan)
    p.set_probe(torch.from_numpy(case.probe).cuda())
    p.set_data(torch.from_numpy(case.y).cuda(), None if case.bg is None else torch.from_numpy(case.bg).cuda())
    if d is not None:
        p.set_scan_offsets(d)
    x = tuple(torch.from_numpy(a).cuda() for a in (case.rho, case.u, case.alpha))
    return p, x


def _check(got, ref):
    f, gr, gu, ga = ref
    loss, g_rho, g_u, g_alpha = [t.cpu().numpy() for t in got]
    assert abs(loss[0] - f) <= LOSS_TOL * abs(f), (loss[0], f)
    assert rel_l2(g_rho, gr) <= GRAD_TOL, rel_l2(g_rho, gr)
    for c in range(gu.shape[0]):
        if np.abs(gu[c]).max() > 0:
            assert rel_l2(g_u[c], gu[c]) <= GRAD_TOL, (c, rel_l2(g_u[c], gu[c]))
    assert rel_l2(g_alpha, ga) <= GRAD_TOL, (g_alpha, ga)


@pytest.mark.parametrize("m", [8, 32, 64, 128])
def test_shifted_probes_match_oracle(m):
    from paper_2312_14907_gb300 import mpbp
    rng = np.random.default_rng(m)
    P = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))).astype(np.complex64)
    d = _offsets(9, m)
    got = mpbp.shift_probe(torch.from_numpy(P).cuda(), d).cpu().numpy()
    for i in range(d.shape[0]):
        ref = oracle.probe_shift(P.astype(np.complex128), d[i, 0], d[i, 1])
        assert rel_l2(got[i], ref) <= 1e-5, (i, rel_l2(got[i], ref))
    # an integer position (d = 0) gives the probe itself, exactly
    np.testing.assert_array_equal(got[1], P)


# (n, m, side, step, offset, peaks, comps): the pair (M = 32, 64) and
# M = 128 kernels, frames over every edge; the last with 338 frames, so that
# every block of the M = 128 grid takes two or three frames and reloads its
# probe (one per scan position) while its gradient window slides
SIZES = [
    (64, 32, 6, 7, -3, 3, 3),
    (128, 64, 5, 17, -9, 3, 3),
    (200, 128, 3, 41, -20, 2, 3),
    (256, 128, 13, 10, -6, 2, 3),
]


@pytest.mark.parametrize("n,m,side,step,off,D,C", SIZES)
def test_loss_grad_with_offsets_matches_oracle(n, m, side, step, off, D, C):
    spec, scan = custom_spec(n, m, side, step, npeaks=D, ncomp=C, offset=off)
    case = Case(spec, scan=scan, state="perturbed")
    d = _offsets(scan.shape[0], n)
    p2, Pf = _oracle_frames(case, d)
    p, x = _gpu(case, d)
    _check(p.loss_grad(*x), p2.loss_grad(case.rho, case.u, case.alpha, Pf, case.y))
    # the forward model and the illumination map take the same probes
    I = p.forward(*x).cpu().numpy()
    I_ref = p2.forward(case.rho, case.u, case.alpha, Pf)
    assert rel_l2(I, I_ref) <= 1e-5
    il = p.illumination().cpu().numpy()
    assert rel_l2(il, p2.illumination(Pf)) <= 1e-5
    p.sync_status()


def test_per_peak_probes_with_offsets_and_background():
    spec, scan = custom_spec(128, 64, 4, 21, npeaks=3, offset=-5, probe_per_peak=True)
    case = Case(spec, scan=scan, state="perturbed", bg=True)
    d = _offsets(scan.shape[0], 3)
    p2, Pf = _oracle_frames(case, d)
    assert Pf.shape[0] == spec.npeaks * scan.shape[0]
    p, x = _gpu(case, d)
    _check(p.loss_grad(*x), p2.loss_grad(case.rho, case.u, case.alpha, Pf, case.y, bg=case.bg))
    # a frame subset (the minibatch argument) uses each frame's own probe
    frames = np.array([0, 5, 7, 11, 2], np.int32)
    got = p.loss_grad(*x, frames=torch.from_numpy(frames).cuda())
    _check(got, p2.loss_grad(case.rho, case.u, case.alpha, Pf, case.y, bg=case.bg, frames=frames))
    p.sync_status()


def test_offsets_follow_a_new_probe_and_can_be_cleared():
    spec, scan = custom_spec(96, 32, 5, 15, npeaks=2, offset=-4)
    case = Case(spec, scan=scan, state="perturbed")
    d = _offsets(scan.shape[0], 8)
    p, x = _gpu(case, d)
    # zero offsets: the same probes as the integer positions, so the same
    # loss bit for bit (its sums run in a fixed order); the gradients agree
    # to the rounding of the scatter-add, whose atomic order varies
    p.set_scan_offsets(np.zeros_like(d))
    a = [t.cpu().numpy() for t in p.loss_grad(*x)]
    p.set_scan_offsets(None)
    b = [t.cpu().numpy() for t in p.loss_grad(*x)]
    np.testing.assert_array_equal(a[0], b[0])
    for u, v in zip(a[1:], b[1:]):
        assert rel_l2(u, v) <= 1e-6
    # offsets set before a new probe are applied to that probe
    P2 = (case.probe * np.exp(0.3j)).astype(np.complex64) * 1.1
    p.set_scan_offsets(d)
    p.set_probe(torch.from_numpy(P2).cuda())
    case.probe = P2
    p2, Pf = _oracle_frames(case, d)
    _check(p.loss_grad(*x), p2.loss_grad(case.rho, case.u, case.alpha, Pf, case.y))


def test_host_buffer_call_and_tensor_core_mode_with_offsets():
    from paper_2312_14907_gb300 import mpbp
    spec, scan = custom_spec(128, 64, 5, 17, npeaks=3, offset=-9)
    case = Case(spec, scan=scan, state="perturbed")
    d = _offsets(scan.shape[0], 21)
    p2, Pf = _oracle_frames(case, d)
    ref = p2.loss_grad(case.rho, case.u, case.alpha, Pf, case.y)
    p, x = _gpu(case, d)
    out = p.loss_grad_host(*(torch.from_numpy(a) for a in (case.rho, case.u, case.alpha)),
                           y=torch.from_numpy(case.y))
    _check(out, ref)
    p.set_precision(mpbp.PRECISION_TC_SPLIT16)
    _check(p.loss_grad(*x), ref)
    p.sync_status()


def test_offsets_outside_half_a_pixel_are_rejected():
    from paper_2312_14907_gb300 import mpbp
    spec, scan = custom_spec(64, 32, 3, 10, npeaks=2, offset=0)
    case = Case(spec, scan=scan)
    p, x = _gpu(case, None)
    d = np.zeros((scan.shape[0], 2))
    d[2, 1] = 0.51
    with pytest.raises(mpbp.MPBPError) as e:
        p.set_scan_offsets(d)
    assert e.value.status == 1
    d[2, 1] = np.nan
    with pytest.raises(mpbp.MPBPError):
        p.set_scan_offsets(d)


def test_batched_problems_with_offsets():
    """Persistent launches over several problems: each problem's frames use
    its own shifted probes (every batch schedule)."""
    from paper_2312_14907_gb300 import mpbp
    cases = [Case(*custom_spec(96, 32, 5, 14, npeaks=3, offset=-2, seed=1), state="perturbed"),
             Case(*custom_spec(160, 64, 4, 30, npeaks=2, offset=-5, seed=2), state="perturbed"),
             Case(*custom_spec(200, 128, 2, 60, npeaks=3, offset=-10, seed=3), state="perturbed")]
    offs = [_offsets(c.scan.shape[0], 40 + i) if i != 1 else None for i, c in enumerate(cases)]
    refs = []
    for c, d in zip(cases, offs):
        if d is None:
            refs.append(c.oracle_loss_grad())
        else:
            p2, Pf = _oracle_frames(c, d)
            refs.append(p2.loss_grad(c.rho, c.u, c.alpha, Pf, c.y))
    probs, states = zip(*[_gpu(c, d) for c, d in zip(cases, offs)])
    for mode in (0, 1, 2, 3):
        probs[0].set_batch_schedule(mode, 0)
        outs = mpbp.loss_grad_batched(list(probs), list(states))
        for o, r in zip(outs, refs):
            _check(o, r)
    for p in probs:
        p.sync_status()
