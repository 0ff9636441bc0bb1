"""The deterministic gradient (mpbp_set_deterministic): the gradient windows
of the frame kernels (M = 128 exchange schedule, M = 64 thread pairs) write
back into per-block pieces of column strips, and a second kernel sums the
pieces covering each pixel in a fixed order.  Against the FP64 oracle at
the parity tolerances; bit for bit against itself on repeated calls and
through the captured step; within rounding of the atomic sums; and the calls
it cannot serve are refused.
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


def _check(case, got):
    f, gr, gu, ga = case.oracle_loss_grad()
    loss, g_rho, g_u, g_alpha = [t.cpu().numpy() for t in got]
    assert abs(loss[0] - f) <= LOSS_TOL * abs(f), (loss[0], f)
    assert rel_l2(g_rho, gr) <= GRAD_TOL, rel_l2(g_rho, gr)
    for c in range(gu.shape[0]):
        if np.abs(gu[c]).max() > 0:
            assert rel_l2(g_u[c], gu[c]) <= GRAD_TOL, (c, rel_l2(g_u[c], gu[c]))
    assert rel_l2(g_alpha, ga) <= GRAD_TOL, (g_alpha, ga)


def _same_bits(a, b):
    for s, t in zip(a, b):
        assert torch.equal(s.view(torch.uint8) if s.dtype != torch.uint8 else s,
                           t.view(torch.uint8) if t.dtype != torch.uint8 else t)


def _irregular_scan(n, m, count):
    rng = np.random.default_rng(1701 + m)
    lo, hi = -m // 3, n - 2 * m // 3
    pos = np.stack([rng.integers(lo, hi, count), rng.integers(lo, hi, count)], axis=1)
    cols = rng.integers(lo, hi, 4)
    # strips with several rows each (odd and even steps), and repeats
    extra = np.array([[r, c] for c in cols for r in sorted(rng.integers(lo, hi, 5))])
    return np.concatenate([pos, extra, pos[:3]]).astype(np.int32)


# (m, n, scan side, step, irregular positions): more than two frames a block
# (M = 128: 152 blocks; M = 64: 608)
GEOM = {128: (256, 13, 10, 150), 64: (170, 26, 6, 660)}


@pytest.mark.parametrize("m", [128, 64])
@pytest.mark.parametrize("kind", ["grid", "irregular", "background"])
def test_deterministic_matches_oracle_and_itself(kind, m):
    """Every block takes two or three frames.  Regular scans (strips sliding
    down by an even step), seeded positions off any grid (repeats, odd steps,
    jumps past the window, column and peak changes inside a block's run),
    and a background."""
    n, side, step, count = GEOM[m]
    spec, scan = custom_spec(n, m, side, step, npeaks=2, offset=-6)
    if kind == "irregular":
        scan = _irregular_scan(n, m, count)
    case = Case(spec, scan=scan, state="perturbed", bg=(kind == "background"))
    p, x = _gpu(case)
    atomic = [t.clone() for t in p.loss_grad(*x)]
    p.set_deterministic(True)
    info = p.info()
    assert info["deterministic"] == 1 and info["launches_loss_grad"] == 5
    assert case.oracle.nframes > 2 * info["frames_grid"]
    first = [t.clone() for t in p.loss_grad(*x)]
    _check(case, first)
    for _ in range(3):
        _same_bits(first, p.loss_grad(*x))
    # the atomic sums agree to rounding
    assert abs(first[0].item() - atomic[0].item()) <= 1e-9 * abs(atomic[0].item())
    for a, b in zip(first[1:], atomic[1:]):
        assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= 1e-6
    p.set_deterministic(False)
    assert p.info()["deterministic"] == 0
    p.sync_status()


@pytest.mark.parametrize("m", [128, 64])
def test_deterministic_step_and_captured_replay(m):
    """Eager steps and the captured step's replays from the same state give
    the same bits, run after run."""
    n, side, step, _ = GEOM[m]
    spec, scan = custom_spec(n, m, side, step, npeaks=2, offset=-6)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    p.set_deterministic(True)
    overlap = (spec.m / spec.step) ** 2 * spec.npeaks
    t0 = 1.0 / (spec.m ** 2 * float(np.abs(case.probe).max()) ** 2 * overlap)

    def run(replay):
        rho, u, alpha = [t.clone() for t in x]
        st = p.step_init(t0, w_u=1e-3, w_alpha=1e-3)
        if replay:
            p.step_capture(rho, u, alpha, st)
            for _ in range(4):
                p.step_replay()
        else:
            for _ in range(4):
                p.step(rho, u, alpha, st)
        torch.cuda.synchronize()
        return [rho.clone(), u.clone(), alpha.clone(), st.clone()]

    eager = run(False)
    _same_bits(eager, run(False))
    _same_bits(eager, run(True))
    _same_bits(eager, run(True))
    p.sync_status()


def test_deterministic_plan_follows_the_schedule():
    """At M = 64 the grid follows the resident blocks per SM; each schedule
    gets its own plan, matches the oracle and repeats its own bits."""
    n, side, step, _ = GEOM[64]
    spec, scan = custom_spec(n, 64, side, step, npeaks=2, offset=-6)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    p.set_deterministic(True)
    grids = set()
    for b in (1, 2, 4):
        p.set_schedule(b)
        grids.add(p.info()["frames_grid"])
        first = [t.clone() for t in p.loss_grad(*x)]
        _check(case, first)
        _same_bits(first, p.loss_grad(*x))
    assert len(grids) == 3, grids
    p.sync_status()


def test_deterministic_refusals():
    from paper_2312_14907_gb300 import mpbp
    spec, scan = custom_spec(256, 128, 5, 24, npeaks=2, offset=-6)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    p.set_deterministic(True)

    def refused(fn):
        with pytest.raises(mpbp.MPBPError) as e:
            fn()
        assert e.value.status == 2, e.value          # MPBP_ERR_UNSUPPORTED

    frames = torch.arange(0, 10, dtype=torch.int32, device="cuda")
    refused(lambda: p.loss_grad(*x, frames=frames))
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    refused(lambda: p.loss_grad_host(pin(case.rho), pin(case.u), pin(case.alpha), y=pin(case.y)))
    refused(lambda: p.set_precision(1))
    refused(lambda: p.set_fft_schedule(0))
    refused(lambda: mpbp.loss_grad_batched([p], [x]))
    refused(lambda: p.autotune(*x))
    info = p.info()
    assert info["precision"] == 0 and info["fft_schedule"] == 1 and info["deterministic"] == 1
    _check(case, p.loss_grad(*x))
    # back to the atomic sums: everything is served again
    p.set_deterministic(False)
    got = p.loss_grad(*x, frames=frames)
    f = case.oracle_loss_grad(frames=frames.cpu().numpy())[0]
    assert abs(got[0].item() - f) <= LOSS_TOL * abs(f)
    p.sync_status()
    # frame sides other than 64 and 128, and objects without tile copies
    # (odd n2)
    for sp, sc in (custom_spec(64, 32, 3, 10, npeaks=2, offset=-4), custom_spec(256, 128, 3, 40, npeaks=2, n2=255,
                                                                                offset=-6),
                   custom_spec(150, 64, 3, 20, npeaks=2, n2=149, offset=-4)):
        q, _ = _gpu(Case(sp, scan=sc, state="perturbed"))
        refused(lambda: q.set_deterministic(True))
        assert q.info()["deterministic"] == 0
