"""CUDA path vs the FP64 oracle, element by element, on seeded inputs.

Tolerances (FP32 kernels against an FP64 definition): loss relative error
<= 1e-5; each gradient block (rho, u, alpha) relative L2 error <= 1e-4;
objects and intensities relative L2 error <= 1e-5.
"""
import numpy as np
import pytest

from helpers import Case, custom_spec, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-5
GRAD_TOL = 1e-4


def _gpu(case):
    from paper_2312_14907_gb300 import mpbp
    p = mpbp.Problem.from_spec(case.spec, case.scan)
    p.set_probe(torch.from_numpy(case.probe).cuda())
    p.set_data(torch.from_numpy(case.y).cuda(),
               None if case.bg is None else torch.from_numpy(case.bg).cuda())
    x = tuple(torch.from_numpy(a).cuda() for a in (case.rho, case.u, case.alpha))
    return p, x


def _check_loss_grad(case, got, frames=None, tol=GRAD_TOL):
    f, gr, gu, ga = case.oracle_loss_grad(frames=frames)
    loss, g_rho, g_u, g_alpha = [t.cpu().numpy() for t in got]
    assert abs(loss[0] - f) <= LOSS_TOL * abs(f), (loss[0], f)
    assert rel_l2(g_rho, gr) <= tol, rel_l2(g_rho, gr)
    for c in range(gu.shape[0]):
        if np.abs(gu[c]).max() > 0:
            assert rel_l2(g_u[c], gu[c]) <= tol, (c, rel_l2(g_u[c], gu[c]))
        else:
            assert np.abs(g_u[c]).max() <= 1e-6 * np.abs(gu).max()
    assert rel_l2(g_alpha, ga) <= tol, (g_alpha, ga)


# (n, m, scan side, step, offset, peaks, comps): several tiles and ragged edges
SIZES = [
    (20, 8, 5, 3, -2, 2, 3),
    (40, 16, 6, 5, -3, 3, 3),
    (64, 32, 7, 4, 4, 3, 3),
    (72, 32, 5, 11, -6, 4, 2),
    (128, 64, 5, 16, -8, 3, 3),
    (200, 128, 3, 40, -20, 2, 3),
]


@pytest.mark.parametrize("n,m,side,step,off,D,C", SIZES)
def test_loss_grad_matches_oracle(n, m, side, step, off, D, C):
    spec, scan = custom_spec(n, m, side, step, npeaks=D, ncomp=C, offset=off)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    _check_loss_grad(case, p.loss_grad(*x))
    p.sync_status()


@pytest.mark.parametrize("m", [8, 16, 32, 64, 128])
def test_forward_and_objects_match_oracle(m):
    n = max(2 * m, 24)
    spec, scan = custom_spec(n, m, 3, m // 2, npeaks=2, offset=-m // 4)
    rng = np.random.default_rng(m)
    probe = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))).astype(np.complex64)
    case = Case(spec, scan=scan, probe=probe, state="perturbed")
    p, x = _gpu(case)
    O = p.object_build(*x).cpu().numpy()
    O_ref = case.oracle.object_build(case.rho, case.u, case.alpha)
    assert rel_l2(O, O_ref) <= 1e-6
    I = p.forward(*x).cpu().numpy()
    I_ref = case.oracle.forward(case.rho, case.u, case.alpha, case.probe)
    for d in range(spec.npeaks):
        for j in range(case.scan.shape[0]):
            assert rel_l2(I[d, j], I_ref[d, j]) <= 1e-5, (d, j)


@pytest.mark.parametrize("m,schedule", [(16, 1), (64, 1), (128, 0), (128, 1)])
def test_random_probe_per_peak_and_background(m, schedule):
    """Unstructured per-peak probes catch transposed or mis-indexed operands
    (and, at M = 128, the reload of the probe held in tensor memory when the
    peak changes); the background enters the intensity of Eq. 2."""
    n = 2 * m + 8
    spec, scan = custom_spec(n, m, 3, m // 2 + 1, npeaks=3, offset=-3, probe_per_peak=True)
    rng = np.random.default_rng(100 + m)
    probe = (rng.standard_normal((3, m, m)) + 1j * rng.standard_normal((3, m, m))).astype(np.complex64)
    case = Case(spec, scan=scan, probe=probe, state="perturbed", bg=True)
    p, x = _gpu(case)
    p.set_fft_schedule(schedule)
    _check_loss_grad(case, p.loss_grad(*x))
    I = p.forward(*x).cpu().numpy()
    I_ref = case.oracle.forward(case.rho, case.u, case.alpha, case.probe, bg=case.bg)
    assert rel_l2(I, I_ref) <= 1e-5


@pytest.mark.parametrize("m", [32, 64, 128])
def test_tile_and_plain_copies_match_oracle(m):
    """Objects whose rows are a multiple of 16 bytes (even n2) reach the FFT
    kernels by TMA tile and bulk copies, odd n2 by cp.async; both layouts,
    with odd and negative scan offsets, against the oracle, through the
    device and the host-buffer entry points."""
    from paper_2312_14907_gb300 import mpbp
    for n2, tiles in ((2 * m + 8, 3), (2 * m + 7, 0)):
        spec, scan = custom_spec(2 * m + 6, m, 3, m // 2 + 1, npeaks=2, offset=-3, n2=n2)
        case = Case(spec, scan=scan, state="perturbed")
        p, x = _gpu(case)
        assert p.info()["tile_copies"] == tiles, (n2, p.info())
        _check_loss_grad(case, p.loss_grad(*x))
        I = p.forward(*x).cpu().numpy()
        I_ref = case.oracle.forward(case.rho, case.u, case.alpha, case.probe)
        assert rel_l2(I, I_ref) <= 1e-5
        p.sync_status()
        # the host-buffer call: the raw-data kernel takes the staged counts
        # by tile copies too (even n2) or by cp.async (odd n2)
        q = mpbp.Problem.from_spec(case.spec, case.scan)
        q.set_probe(torch.from_numpy(case.probe).cuda())
        h = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        got = q.loss_grad_host(h(case.rho), h(case.u), h(case.alpha), y=h(case.y))
        _check_loss_grad(case, got)
        got = q.loss_grad_host(h(case.rho), h(case.u), h(case.alpha), y=h(case.y.astype(np.uint16)))
        _check_loss_grad(case, got)
        q.sync_status()


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("n2,tiles", [(256, 3), (255, 0)])
def test_m128_steady_state_matches_oracle(n2, tiles, schedule):
    """The M = 128 gradient kernel runs one block per SM, so a block takes a
    second frame only when a launch has more than one frame per SM.  338
    frames (13 x 13 scan, 2 peaks) give every block of the 152-block grid two
    or three frames: each prefetches the next frame's inputs while it
    transforms the current one, reuses its buffers and flips its barrier
    phase at least twice.  Element by element against the oracle, through
    the tile-copy path (even n2) and the cp.async path (odd n2), with the
    scan overhanging the grid, under both FFT schedules (radix-2 stages
    across threads by shuffles; three register layouts joined by shared-
    memory exchanges); the same again through a frame list."""
    spec, scan = custom_spec(256, 128, 13, 10, npeaks=2, offset=-6, n2=n2)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    p.set_fft_schedule(schedule)
    assert p.info()["fft_schedule"] == schedule
    info = p.info()
    assert info["tile_copies"] == tiles, info
    assert spec.nframes > 2 * info["frames_grid"], (spec.nframes, info)
    _check_loss_grad(case, p.loss_grad(*x))
    frames = np.random.default_rng(128).permutation(spec.nframes)[:320].astype(np.int32)
    _check_loss_grad(case, p.loss_grad(*x, frames=torch.from_numpy(frames).cuda()), frames=frames)
    p.sync_status()


@pytest.mark.parametrize("n2,tiles,step", [(200, 3, 6), (199, 0, 5)])
def test_m64_steady_state_matches_oracle(n2, tiles, step):
    """The M = 64 gradient kernel runs four blocks per SM (608 blocks): 1,352
    frames (26 x 26 scan, 2 peaks) give every block two or three frames, so
    each prefetches the next frame's inputs, reuses its buffers and flips its
    barrier phase.  Then with one block per SM (about nine frames a block),
    and through a frame list.  Element by element against the oracle, tile
    copies (even n2) and cp.async (odd n2)."""
    spec, scan = custom_spec(170, 64, 26, step, npeaks=2, offset=-6, n2=n2)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    info = p.info()
    assert info["tile_copies"] == tiles, info
    assert spec.nframes > 2 * info["frames_grid"], (spec.nframes, info)
    _check_loss_grad(case, p.loss_grad(*x))
    p.set_schedule(1)
    _check_loss_grad(case, p.loss_grad(*x))
    frames = np.random.default_rng(64).permutation(spec.nframes)[:300].astype(np.int32)
    _check_loss_grad(case, p.loss_grad(*x, frames=torch.from_numpy(frames).cuda()), frames=frames)
    p.sync_status()


@pytest.mark.parametrize("n2", [256, 255])
def test_m128_irregular_scan_matches_oracle(n2):
    """Scan positions off any grid: 173 seeded positions (some repeated, some
    overhanging every edge) and 2 peaks, 346 frames, so that every block of
    the 152-block M = 128 grid takes two or three frames of the column-strip
    order.  A block's gradient window then moves by arbitrary row steps,
    repeats a position (a step of 0), jumps by more than a window, and
    changes column or peak between frames; element by element against the
    oracle, through tile copies (even n2) and cp.async (odd n2)."""
    rng = np.random.default_rng(1701)
    spec, _ = custom_spec(256, 128, 13, 10, npeaks=2, offset=-6, n2=n2)
    pos = np.stack([rng.integers(-40, 200, 150), rng.integers(-40, n2 - 88, 150)], axis=1)
    # a few columns with several rows each: strips whose steps vary
    cols = rng.integers(-20, n2 - 100, 4)
    extra = np.array([[r, c] for c in cols for r in sorted(rng.integers(-30, 180, 5))])
    scan = np.concatenate([pos, extra, pos[:3]]).astype(np.int32)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    assert case.oracle.nframes > 2 * p.info()["frames_grid"]
    _check_loss_grad(case, p.loss_grad(*x))
    p.sync_status()


def test_frame_subset_matches_oracle():
    spec, scan = custom_spec(64, 32, 6, 6, npeaks=3, offset=0)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    frames = np.random.default_rng(3).permutation(case.oracle.nframes)[:37].astype(np.int32)
    got = p.loss_grad(*x, frames=torch.from_numpy(frames).cuda())
    _check_loss_grad(case, got, frames=frames)
    # a frame listed twice counts twice (Eq. 11 is a plain sum)
    frames2 = np.concatenate([frames, frames[:5]]).astype(np.int32)
    got = p.loss_grad(*x, frames=torch.from_numpy(frames2).cuda())
    _check_loss_grad(case, got, frames=frames2)
    # empty minibatch: zero loss and gradient
    loss, g_rho, g_u, g_alpha = p.loss_grad(*x, frames=torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert loss.item() == 0.0 and g_rho.abs().max().item() == 0.0 and g_u.abs().max().item() == 0.0


def test_frame_index_out_of_range_is_reported():
    from paper_2312_14907_gb300 import mpbp
    spec, scan = custom_spec(40, 16, 3, 8, npeaks=2, offset=0)
    case = Case(spec, scan=scan)
    p, x = _gpu(case)
    frames = torch.tensor([0, 5, 10_000, -1], dtype=torch.int32, device="cuda")
    p.loss_grad(*x, frames=frames)
    with pytest.raises(mpbp.MPBPError) as ei:
        p.sync_status()
    assert ei.value.status == 6
    # the skipped slots do not contribute; the context stays usable
    got = p.loss_grad(*x, frames=frames[:2].contiguous())
    _check_loss_grad(case, got, frames=np.array([0, 5], np.int32))
    p.sync_status()


@pytest.mark.parametrize("schedule", [0, 1])
def test_m128_out_of_range_inside_a_block_run(schedule):
    """At M = 128 a block takes a contiguous run of a frame list (exchange
    schedule) or every 152nd entry (shuffle schedule); out-of-range indices in
    the middle of the runs are reported as MPBP_ERR_BOUNDS, leave the valid
    frames' results equal to the oracle's over those frames, and the context
    stays usable."""
    from paper_2312_14907_gb300 import mpbp
    spec, scan = custom_spec(256, 128, 13, 10, npeaks=2, offset=-6)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    p.set_fft_schedule(schedule)
    rng = np.random.default_rng(7)
    good = rng.permutation(spec.nframes)[:320].astype(np.int32)
    bad = good.copy()
    bad[rng.choice(320, 12, replace=False)] = np.array([-1, 10_000] * 6, np.int32)
    got = p.loss_grad(*x, frames=torch.from_numpy(bad).cuda())
    with pytest.raises(mpbp.MPBPError) as ei:
        p.sync_status()
    assert ei.value.status == 6
    valid = bad[(bad >= 0) & (bad < spec.nframes)]
    _check_loss_grad(case, got, frames=valid)
    _check_loss_grad(case, p.loss_grad(*x, frames=torch.from_numpy(good).cuda()), frames=good)
    p.sync_status()


def _check_loss_only(case, got):
    f = case.oracle_loss_grad()[0]
    assert abs(got[0].item() - f) <= LOSS_TOL * abs(f), (got[0].item(), f)


def test_config1_start_and_truth():
    """The 64x64 / M=32 / 3-peak problem: the loss at the reconstruction start
    (rho = 1, u = 0), loss and gradient near the truth, near-zero loss at the
    truth on noise-free data.

    At the flat start the far field of the smooth probe falls below rounding
    noise (in FP64 as well) over most of each frame, and there the factor
    Psi/|Psi| of the gradient has a rounding-determined phase: the gradient is
    not a well-conditioned quantity at that state, so only the loss is compared."""
    from paper_2312_14907_gb300 import synth
    case = Case(synth.config(1), state="init")
    p, x = _gpu(case)
    _check_loss_only(case, p.loss_grad(*x))
    case = Case(synth.config(1), state="perturbed")
    p, x = _gpu(case)
    _check_loss_grad(case, p.loss_grad(*x))
    clean = Case(synth.config(1), state="truth", noise=False)
    p, x = _gpu(clean)
    loss = p.loss_grad(*x)[0].item()
    assert loss <= 1e-9 * float(clean.y.sum())


def test_gpu_invariances():
    """Eq. 6: a uniform displacement and lattice-vector jumps leave the loss unchanged;
    translation invariance makes every df/du_c sum to zero."""
    spec, scan = custom_spec(64, 32, 5, 6, npeaks=3, offset=4)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    rho, u, alpha = x
    f0, _, g_u, _ = p.loss_grad(rho, u, alpha)
    f0 = f0.item()
    f1 = p.loss_grad(rho, (u + torch.tensor([0.3, -0.7, 1.1], device="cuda")[:, None, None]).contiguous(),
                     alpha)[0].item()
    assert abs(f1 - f0) <= 2e-5 * f0
    mask = (torch.rand(u.shape[1:], generator=torch.Generator().manual_seed(1)) < 0.3).cuda()
    u2 = u.clone()
    u2[0] += mask.float()
    u2[2] -= mask.float()
    f2 = p.loss_grad(rho, u2, alpha)[0].item()
    assert abs(f2 - f0) <= 2e-5 * f0
    g = g_u.double()
    for c in range(3):
        assert abs(g[c].sum().item()) <= 1e-4 * g[c].abs().sum().item()


def test_full_bench_problem_matches_oracle():
    """The 256x256 / M=64 / 31x31 scan / 3-peak problem, all 2883 frames, in
    the launch configuration the benchmark times."""
    from paper_2312_14907_gb300 import synth
    case = Case(synth.config(2), state="init")
    p, x = _gpu(case)
    _check_loss_only(case, p.loss_grad(*x))
    case2 = Case(synth.config(2), state="perturbed", seed=1)
    p2, x2 = _gpu(case2)
    _check_loss_grad(case2, p2.loss_grad(*x2))


def test_host_buffer_entry_point_matches_device_path():
    spec, scan = custom_spec(128, 64, 4, 12, npeaks=3, offset=8)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    dev = [t.cpu().numpy() for t in p.loss_grad(*x)]
    pin = lambda a: torch.from_numpy(a).pin_memory()
    host = p.loss_grad_host(pin(case.rho), pin(case.u), pin(case.alpha), y=pin(case.y))
    host = [t.numpy() for t in host]
    assert abs(host[0][0] - dev[0][0]) <= 1e-6 * abs(dev[0][0])
    for a, b in zip(host[1:], dev[1:]):
        assert rel_l2(a, b) <= 1e-5
    _check_loss_grad(case, [torch.from_numpy(h) for h in host])


@pytest.mark.parametrize("m,pinned", [(32, True), (64, False), (128, True), (16, True)])
def test_host_entry_point_paths(m, pinned):
    """Chunks of y copied into staging buffers are read in their natural
    layout by the frame kernel on thread-pair sides (M >= 32), and transposed
    by a separate kernel for M = 16; from page-locked or pageable host memory
    (page-locked outputs are written in place, pageable ones copied back).
    Either way the result matches the device path, and y becomes the
    context's data for later device calls."""
    from paper_2312_14907_gb300 import mpbp
    n = max(3 * m, 48)
    spec, scan = custom_spec(n, m, 5, m // 2, npeaks=2, offset=-m // 8, seed=m)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    dev = [t.cpu().numpy() for t in p.loss_grad(*x)]
    # a second context without data: the host call supplies it
    q = mpbp.Problem.from_spec(case.spec, case.scan)
    q.set_probe(torch.from_numpy(case.probe).cuda())
    host_t = lambda a: torch.from_numpy(np.ascontiguousarray(a))
    wrap = (lambda a: host_t(a).pin_memory()) if pinned else host_t
    out = None
    if pinned:   # page-locked outputs are written by the gradient assembly directly
        out = tuple(torch.full(t.shape, float("nan"), dtype=dt).pin_memory()
                    for t, dt in zip(dev, (torch.float64, torch.float32, torch.float32, torch.float64)))
    host = [t.numpy() for t in q.loss_grad_host(wrap(case.rho), wrap(case.u), wrap(case.alpha),
                                                 y=wrap(case.y), out=out)]
    assert abs(host[0][0] - dev[0][0]) <= 1e-6 * abs(dev[0][0])
    for a, b in zip(host[1:], dev[1:]):
        assert rel_l2(a, b) <= 1e-5
    again = [t.cpu().numpy() for t in q.loss_grad(*x)]   # device call on the data y left behind
    assert abs(again[0][0] - dev[0][0]) <= 1e-6 * abs(dev[0][0])
    for a, b in zip(again[1:], dev[1:]):
        assert rel_l2(a, b) <= 1e-5
    q.sync_status()
    # the same counts as 16-bit integers (read by the frame kernel itself on
    # M = 64 and 128, widened on the device first on M = 16 and 32)
    assert np.all(case.y == np.round(case.y)) and case.y.max() < 65536
    r = mpbp.Problem.from_spec(case.spec, case.scan)
    r.set_probe(torch.from_numpy(case.probe).cuda())
    h16 = [t.numpy() for t in r.loss_grad_host(wrap(case.rho), wrap(case.u), wrap(case.alpha),
                                                y=wrap(case.y.astype(np.uint16)))]
    assert abs(h16[0][0] - dev[0][0]) <= 1e-6 * abs(dev[0][0])
    for a, b in zip(h16[1:], dev[1:]):
        assert rel_l2(a, b) <= 1e-5
    r.sync_status()


def test_autograd_function():
    from paper_2312_14907_gb300 import mpbp
    spec, scan = custom_spec(40, 16, 4, 6, npeaks=2, offset=0)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    rho, u, alpha = [t.clone().requires_grad_(True) for t in x]
    f = mpbp.mpbp_loss(rho, u, alpha, p)
    (2.0 * f).backward()
    ref = p.loss_grad(*x)
    assert abs(f.item() - ref[0].item()) <= 1e-12 * abs(ref[0].item())
    # two evaluations differ only by the order of floating-point atomics
    for g, r in ((rho.grad, ref[1]), (u.grad, ref[2]), (alpha.grad.double(), ref[3])):
        assert (g.double() - 2 * r.double()).abs().max().item() <= 1e-5 * (2 * r).abs().max().item()


def test_batched_matches_single_problems():
    from paper_2312_14907_gb300 import mpbp
    cases = [Case(*custom_spec(40, 16, 4, 6, npeaks=2, offset=0), state="perturbed"),
             Case(*custom_spec(96, 32, 5, 14, npeaks=3, offset=-2, seed=1), state="perturbed"),
             Case(*custom_spec(160, 64, 4, 30, npeaks=4, offset=-5, seed=2), state="perturbed"),
             Case(*custom_spec(200, 128, 2, 60, npeaks=3, offset=-10, seed=3), state="perturbed")]
    probs, states = zip(*[_gpu(c) for c in cases])
    for mode in (0, 1, 2, 3):
        for order in (0, 1):
            probs[0].set_batch_schedule(mode, order)
            outs = mpbp.loss_grad_batched(list(probs), list(states))
            for c, o in zip(cases, outs):
                _check_loss_grad(c, o)
    for p in probs:
        p.sync_status()


@pytest.mark.parametrize("m,schedule", [(64, 1), (128, 0), (128, 1)])
def test_tile_copy_wait_runs_out_and_reports(m, schedule):
    """The frame kernels' waits for their tile copies are bounded: with the
    barrier told to expect bytes that never arrive, each block gives up
    after its time limit, the call reports MPBP_ERR_TIMEOUT, and the context
    computes correctly again afterwards."""
    import time
    from paper_2312_14907_gb300 import mpbp
    spec, scan = custom_spec(2 * m + 8, m, 3, m // 2, npeaks=2, offset=-2)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    p.set_fft_schedule(schedule)
    assert p.info()["tile_copies"] == 3
    p.set_test_stall(True)
    t0 = time.time()
    p.loss_grad(*x)
    with pytest.raises(mpbp.MPBPError) as e:
        p.sync_status()
    assert e.value.status == 5, e.value           # MPBP_ERR_TIMEOUT
    assert time.time() - t0 < 20.0
    p.set_test_stall(False)
    _check_loss_grad(case, p.loss_grad(*x))
    p.sync_status()


def test_batched_tile_copy_wait_runs_out_and_reports():
    """The per-side batched launches take their inputs by tile copies, each
    problem through its own tensor map, with the same bounded wait: with the
    test hook on one problem its copies' barrier waits run out, the call
    reports MPBP_ERR_TIMEOUT for that problem, and the batch then computes
    the oracle's results again."""
    import time
    from paper_2312_14907_gb300 import mpbp
    cases = [Case(*custom_spec(96, 32, 5, 14, npeaks=3, offset=-2, seed=1), state="perturbed"),
             Case(*custom_spec(160, 64, 4, 30, npeaks=4, offset=-5, seed=2), state="perturbed")]
    probs, states = zip(*[_gpu(c) for c in cases])
    probs[0].set_batch_schedule(1, 0)        # one launch per frame side
    probs[1].set_test_stall(True)
    t0 = time.time()
    mpbp.loss_grad_batched(list(probs), list(states))
    with pytest.raises(mpbp.MPBPError) as e:
        probs[1].sync_status()
    assert e.value.status == 5, e.value           # MPBP_ERR_TIMEOUT
    assert time.time() - t0 < 20.0
    probs[1].set_test_stall(False)
    for c, o in zip(cases, mpbp.loss_grad_batched(list(probs), list(states))):
        _check_loss_grad(c, o)
    for p in probs:
        p.sync_status()
