"""Tensor-core DFT precision mode (frame sides 64 and 32) vs the FP64 oracle.

The split-FP16 products keep about 22 bits of each operand and accumulate in
FP32, so the same tolerances as the FFT kernels apply: loss relative error
<= 1e-5, each gradient block relative L2 error <= 1e-4.
"""
import numpy as np
import pytest

from helpers import Case, custom_spec, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-5
GRAD_TOL = 1e-4


def _gpu(case, precision=1):
    from paper_2312_14907_gb300 import mpbp
    p = mpbp.Problem.from_spec(case.spec, case.scan)
    p.set_probe(torch.from_numpy(case.probe).cuda())
    p.set_data(torch.from_numpy(case.y).cuda(),
               None if case.bg is None else torch.from_numpy(case.bg).cuda())
    p.set_precision(precision)
    x = tuple(torch.from_numpy(a).cuda() for a in (case.rho, case.u, case.alpha))
    return p, x


def _check(case, got, frames=None):
    f, gr, gu, ga = case.oracle_loss_grad(frames=frames)
    loss, g_rho, g_u, g_alpha = [t.cpu().numpy() for t in got]
    assert abs(loss[0] - f) <= LOSS_TOL * abs(f), (loss[0], f)
    assert rel_l2(g_rho, gr) <= GRAD_TOL, rel_l2(g_rho, gr)
    for c in range(gu.shape[0]):
        if np.abs(gu[c]).max() > 0:
            assert rel_l2(g_u[c], gu[c]) <= GRAD_TOL, (c, rel_l2(g_u[c], gu[c]))
    assert rel_l2(g_alpha, ga) <= GRAD_TOL, (g_alpha, ga)


# (m, n, scan side, step, offset, peaks, comps): several frames per block,
# ragged edges, scan positions overhanging the grid on every side; at M = 32
# frame counts that leave a group's tile partly empty, and one with more
# frames than the grid's tiles take in one pass (1,600 > 152 x 8); at M = 128
# one with more frames than two per block (338 > 152 x 2)
SIZES = [
    (64, 64, 1, 1, 0, 1, 1),
    (64, 128, 5, 16, -8, 3, 3),
    (64, 150, 7, 15, -20, 4, 2),
    (32, 32, 1, 1, 0, 1, 1),
    (32, 80, 5, 11, -6, 3, 3),
    (32, 96, 7, 13, -9, 2, 2),
    (32, 200, 20, 9, -5, 4, 3),
    (128, 200, 3, 40, -20, 2, 3),
    (128, 256, 13, 10, -6, 2, 3),
]


@pytest.mark.parametrize("m,n,side,step,off,D,C", SIZES)
def test_tc_loss_grad_matches_oracle(m, n, side, step, off, D, C):
    spec, scan = custom_spec(n, m, side, step, npeaks=D, ncomp=C, offset=off)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    assert p.info()["precision"] == 1
    _check(case, p.loss_grad(*x))
    p.sync_status()


@pytest.mark.parametrize("m", [64, 32, 128])
def test_tc_random_probe_per_peak_and_background(m):
    spec, scan = custom_spec(140 * m // 64, m, 4, 22 * m // 64, npeaks=3, offset=-9, probe_per_peak=True)
    rng = np.random.default_rng(5)
    probe = (rng.standard_normal((3, m, m)) + 1j * rng.standard_normal((3, m, m))).astype(np.complex64)
    case = Case(spec, scan=scan, probe=probe, state="perturbed", bg=True)
    p, x = _gpu(case)
    _check(case, p.loss_grad(*x))
    # forward mode keeps the FFT kernel, with its own launch shape
    I = p.forward(*x).cpu().numpy()
    I_ref = case.oracle.forward(case.rho, case.u, case.alpha, case.probe, case.bg)
    assert rel_l2(I, I_ref) <= 1e-5
    p.sync_status()


@pytest.mark.parametrize("m", [64, 32])
def test_tc_frame_subsets_and_bounds(m):
    from paper_2312_14907_gb300 import mpbp
    spec, scan = custom_spec(2 * m, m, 4, 20 * m // 64, npeaks=3, offset=-6)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    frames = np.array([0, 3, 3, 7, 15, 40, 47], np.int32)
    _check(case, p.loss_grad(*x, frames=torch.from_numpy(frames).cuda()), frames=frames)
    loss, g_rho, _, _ = p.loss_grad(*x, frames=torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert loss.item() == 0.0 and float(g_rho.abs().max()) == 0.0
    bad = torch.tensor([1, 48], dtype=torch.int32, device="cuda")
    p.loss_grad(*x, frames=bad)
    with pytest.raises(mpbp.MPBPError) as e:
        p.sync_status()
    assert "BOUNDS" in str(e.value)
    _check(case, p.loss_grad(*x))   # the context stays usable


@pytest.mark.parametrize("k", [2, 1])
def test_tc_agrees_with_fft_path_on_bench_problem(k):
    """The full 256^2, 3-peak, 64x64-frame problem and the 64^2, 32x32-frame
    one: both precision modes in the same context, and the oracle on the whole
    frame set."""
    from paper_2312_14907_gb300 import synth
    case = Case(synth.config(k), state="perturbed", seed=1)
    p, x = _gpu(case, precision=0)
    fft = [t.cpu().numpy() for t in p.loss_grad(*x)]
    p.set_precision(1)
    tc = [t.cpu().numpy() for t in p.loss_grad(*x)]
    assert abs(tc[0][0] - fft[0][0]) <= 1e-5 * abs(fft[0][0])
    for a, b in zip(tc[1:], fft[1:]):
        assert rel_l2(a, b) <= 1e-4
    _check(case, [torch.from_numpy(t) for t in tc])
    p.sync_status()


def test_tc_host_entry_point_and_step():
    spec, scan = custom_spec(160, 64, 5, 22, npeaks=3, offset=-5, seed=3)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    pin = lambda a: torch.from_numpy(a).pin_memory()
    host = [t.numpy() for t in p.loss_grad_host(pin(case.rho), pin(case.u), pin(case.alpha),
                                                  y=pin(case.y))]
    _check(case, [torch.from_numpy(h) for h in host])
    # a few optimizer steps with the tensor-core evaluations lower the loss
    f0 = case.oracle_loss_grad()[0]
    rho, u, alpha = [t.clone() for t in x]
    overlap = (spec.m / spec.step) ** 2 * spec.npeaks
    t0 = 0.5 / (float(np.abs(case.probe).max()) ** 2 * overlap)
    st = p.step_init(t0, w_u=1e-3, w_alpha=1e-3)
    for _ in range(8):
        p.step(rho, u, alpha, st)
    s = p.read_state(st)
    assert s.n_accept >= 1 and s.f_prev < f0, (s.f_prev, f0)
    p.sync_status()


def test_tc_needs_frame_side_32_or_64():
    from paper_2312_14907_gb300 import mpbp
    spec, scan = custom_spec(48, 16, 3, 10, npeaks=2, offset=0)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case, precision=0)
    with pytest.raises(mpbp.MPBPError) as e:
        p.set_precision(1)
    assert "UNSUPPORTED" in str(e.value)
    assert p.info()["precision"] == 0
    _check(case, p.loss_grad(*x))


def test_tc_fullsize_autotune_and_invariants():
    """The autotuner over the schedules (the DFT arithmetic among them); loss
    additivity over a partition of the frames on the full bench problem in
    the tensor-core mode."""
    from paper_2312_14907_gb300 import synth
    case = Case(synth.config(2), state="perturbed", seed=2)
    p, x = _gpu(case)
    p.autotune(*x)                     # the DFT arithmetic is one of its candidates
    assert p.info()["precision"] in (0, 1)
    p.set_precision(1)
    f_all = p.loss_grad(*x)[0].item()
    nf = case.spec.nframes
    half = torch.arange(0, nf, 2, dtype=torch.int32, device="cuda")
    rest = torch.arange(1, nf, 2, dtype=torch.int32, device="cuda")
    fa = p.loss_grad(*x, frames=half)[0].item()
    fb = p.loss_grad(*x, frames=rest)[0].item()
    assert abs(fa + fb - f_all) <= 1e-6 * abs(f_all)
    p.sync_status()


def test_tc_mma_wait_runs_out_and_reports():
    """The tensor-core kernel's waits for its MMAs are bounded: with no MMA
    issued (the test hook), each group's wait gives up after its time limit,
    the call reports MPBP_ERR_TIMEOUT, and the context then computes the
    oracle's result again."""
    import time
    from paper_2312_14907_gb300 import mpbp
    spec, scan = custom_spec(128, 64, 5, 16, npeaks=3, offset=-8)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    p.set_test_stall(True)
    t0 = time.time()
    p.loss_grad(*x)
    with pytest.raises(mpbp.MPBPError) as e:
        p.sync_status()
    assert e.value.status == 5, e.value           # MPBP_ERR_TIMEOUT
    assert time.time() - t0 < 20.0
    p.set_test_stall(False)
    _check(case, p.loss_grad(*x))
    p.sync_status()
