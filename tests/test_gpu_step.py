"""The optimizer iteration (A8: lagged-Armijo gradient descent) on the GPU.

Trajectories of an FP32 and an FP64 implementation drift apart, so the oracle
replays the GPU's own iterates: at every step it re-evaluates the loss and
gradient at the point the GPU evaluated, re-takes the accept/reject decision
from the GPU's state, and rebuilds the update from its own gradient.
"""
import numpy as np
import pytest

from helpers import Case, custom_spec, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(case, **kw):
    from paper_2312_14907_gb300 import mpbp
    p = mpbp.Problem.from_spec(case.spec, case.scan)
    p.set_probe(torch.from_numpy(case.probe).cuda())
    p.set_data(torch.from_numpy(case.y).cuda())
    x = [torch.from_numpy(a.copy()).cuda() for a in (case.rho, case.u, case.alpha)]
    return p, x


def _t0(case):
    overlap = (case.spec.m / case.spec.step) ** 2 * case.spec.npeaks
    return 0.5 / (float(np.abs(case.probe).max() ** 2) * overlap)


def test_step_replays_against_oracle():
    spec, scan = custom_spec(64, 32, 6, 6, npeaks=3, offset=1)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _setup(case)
    w = dict(w_rho=1.0, w_u=0.05, w_alpha=0.01)
    st = p.step_init(_t0(case), **w)
    base_x = base_g = None
    n_acc = n_rej = 0
    for k in range(14):
        xk = [t.cpu().numpy().astype(np.float64) for t in x]
        before = p.read_state(st)
        p.step(*x, st)
        after = p.read_state(st)
        x1 = [t.cpu().numpy().astype(np.float64) for t in x]
        f_ref, gr, gu, ga = case.oracle.loss_grad(*xk, case.probe, case.y)
        # loss at the evaluated iterate
        assert abs(after.f_last - f_ref) <= 1e-5 * abs(f_ref), (k, after.f_last, f_ref)
        # the decision, re-taken in FP64 from the GPU's own numbers
        accept = k == 0 or after.f_last <= before.f_prev - before.c_armijo * before.t * before.gn2_prev
        assert bool(after.accepted) == accept, k
        t_exp = before.t * (before.grow if (accept and k > 0) else 1.0) * (1.0 if accept else before.shrink)
        assert abs(after.t - t_exp) <= 1e-15 * t_exp
        if accept:
            n_acc += 1
            base_x, base_g = xk, (gr, gu, ga)
            gn2 = w["w_rho"] * np.sum(gr ** 2) + w["w_u"] * np.sum(gu ** 2) + w["w_alpha"] * np.sum(ga[1:] ** 2)
            assert abs(after.gn2_prev - gn2) <= 2e-4 * gn2
        else:
            n_rej += 1
        # the update from the base point along the oracle's gradient there
        for xb, g, x_new, wb, name in ((base_x[0], base_g[0], x1[0], w["w_rho"], "rho"),
                                        (base_x[1], base_g[1], x1[1], w["w_u"], "u")):
            step = -after.t * wb * g
            err = np.linalg.norm((x_new - xb) - step)
            assert err <= 1e-3 * np.linalg.norm(step) + 1e-6 * np.linalg.norm(xb), (k, name)
        a_exp = base_x[2] - after.t * w["w_alpha"] * base_g[2]
        a_exp[0] = base_x[2][0]
        assert np.allclose(x1[2], a_exp, rtol=1e-5, atol=1e-7)
        assert x1[2][0] == base_x[2][0]
    assert after.n_accept == n_acc and after.n_reject == n_rej and after.k == 14
    # the first trial steps overshoot on this case (the FP64 oracle's own
    # stepper rejects 9 of 14), so both branches of the update are replayed
    assert n_acc >= 3 and n_rej >= 3


def test_step_decreases_loss_on_noise_free_data():
    from paper_2312_14907_gb300 import synth
    case = Case(synth.config(1), state="init", noise=False)
    p, x = _setup(case)
    st = p.step_init(_t0(case) * 4, w_rho=1.0, w_u=0.02, w_alpha=0.0)
    accepted = []
    for _ in range(120):
        p.step(*x, st)
        s = p.read_state(st)
        if s.accepted:
            accepted.append(s.f_last)
    assert all(b <= a for a, b in zip(accepted, accepted[1:]))
    assert accepted[-1] < accepted[0] / 10
    p.sync_status()


def test_step_graph_capture_matches_eager():
    """A captured iteration replays with device-side decisions only."""
    spec, scan = custom_spec(96, 32, 6, 12, npeaks=3, offset=0)
    case = Case(spec, scan=scan, state="perturbed")
    pe, xe = _setup(case)
    ste = pe.step_init(_t0(case), w_rho=1.0, w_u=0.05, w_alpha=0.01)
    pg, xg = _setup(case)
    stg = pg.step_init(_t0(case), w_rho=1.0, w_u=0.05, w_alpha=0.01)
    # warm up outside the capture (workspace already allocated at create)
    pe.step(*xe, ste)
    pg.step(*xg, stg)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            pg.step(*xg, stg)
    for _ in range(8):
        pe.step(*xe, ste)
        g.replay()
    torch.cuda.synchronize()
    a, b = pe.read_state(ste), pg.read_state(stg)
    assert (a.k, a.n_accept, a.n_reject) == (b.k, b.n_accept, b.n_reject)
    assert abs(a.f_last - b.f_last) <= 1e-6 * abs(a.f_last)
    for u, v in zip(xe, xg):
        assert rel_l2(v.cpu().numpy(), u.cpu().numpy()) <= 1e-5
    pg.sync_status()


def test_native_step_capture_and_replay_match_eager():
    """mpbp_step_capture / mpbp_step_replay: the context's own graph of one
    step replays the eager iterations exactly (same decisions, same iterate)."""
    from paper_2312_14907_gb300 import mpbp
    spec, scan = custom_spec(128, 64, 5, 16, npeaks=3, offset=-4)
    case = Case(spec, scan=scan, state="perturbed")
    pe, xe = _setup(case)
    ste = pe.step_init(_t0(case), w_rho=1.0, w_u=0.05, w_alpha=0.01)
    pg, xg = _setup(case)
    stg = pg.step_init(_t0(case), w_rho=1.0, w_u=0.05, w_alpha=0.01)
    with pytest.raises(mpbp.MPBPError):
        pg.step_replay()                      # nothing captured yet
    pg.frames_timing(True)
    with pytest.raises(mpbp.MPBPError):
        pg.step_capture(*xg, stg)             # timing events cannot be captured
    pg.frames_timing(False)
    pg.step_capture(*xg, stg)                 # records, runs nothing
    for _ in range(8):
        pe.step(*xe, ste)
        pg.step_replay()
    torch.cuda.synchronize()
    a, b = pe.read_state(ste), pg.read_state(stg)
    assert (a.k, a.n_accept, a.n_reject) == (b.k, b.n_accept, b.n_reject) and a.k == 8
    assert abs(a.f_last - b.f_last) <= 1e-6 * abs(a.f_last)
    for u, v in zip(xe, xg):
        assert rel_l2(v.cpu().numpy(), u.cpu().numpy()) <= 1e-5
    # an eager evaluation in between leaves the graph usable
    pg.loss_grad(*xg)
    pg.step_replay()
    pe.step(*xe, ste)
    torch.cuda.synchronize()
    assert pg.read_state(stg).k == pe.read_state(ste).k == 9
    pg.sync_status()
