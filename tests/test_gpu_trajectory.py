"""The 512^2, M = 128, 4-peak problem at full size: optimizer iterations
replayed from one captured CUDA graph, and the FP64 oracle replayed at the
GPU's own iterates (the trajectory is the GPU's; at each kept iterate the
loss and gradient must match the oracle's at that same state).

The oracle evaluates a seeded 1/16 of the scan positions (every peak at
each), as a problem of its own, with the same count data on both sides; the
full-size context's step records the loss it evaluated, which must equal a
plain evaluation at the same state."""
import numpy as np
import pytest

from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEEP = (0, 1, 10)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_trajectory_replayed_on_the_oracle(precision):
    """Both DFT arithmetics: FP32 FFTs (0) and the split tensor-core DFTs (1,
    four 64 x 64 sub-transforms per 128 x 128 frame)."""
    import oracle
    from paper_2312_14907_gb300 import mpbp, synth
    spec = synth.config(3)
    scan = synth.scan_positions(spec)
    probe = (synth.probe(spec) * 3.0).astype(np.complex64)
    p = mpbp.Problem.from_spec(spec, scan)
    p.set_probe(torch.from_numpy(probe).cuda())
    yd = torch.from_numpy(synth.template_counts(spec, spec.seed + 80)).cuda()
    p.set_data(yd)
    del yd
    p.set_precision(precision)
    xs = synth.perturbed_state(spec, np.random.default_rng(spec.seed + 81), 0.05)
    x = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda() for a in xs]
    overlap = (spec.m / spec.step) ** 2 * spec.npeaks
    # first step: the inverse Gauss-Newton curvature bound of a density pixel
    # (M^2 max|P|^2 x the frames covering it)
    state = p.step_init(1.0 / (spec.m ** 2 * float(np.abs(probe).max() ** 2) * overlap), w_u=1e-3,
                        w_alpha=1e-3)
    p.step_capture(*x, state)
    snaps, f_rec = {}, {}
    for k in range(max(KEEP) + 1):
        if k in KEEP:
            snaps[k] = [t.cpu().numpy().copy() for t in x]
        p.step_replay()
        torch.cuda.synchronize()
        if k in KEEP:
            f_rec[k] = mpbp.Problem.read_state(state).f_last
    p.sync_status()
    st = mpbp.Problem.read_state(state)
    assert st.n_accept >= 1 and st.k == max(KEEP) + 1
    # the recorded loss of each kept step is the plain evaluation at its state
    q_full = mpbp.Problem.from_spec(spec, scan)
    q_full.set_probe(torch.from_numpy(probe).cuda())
    q_full.set_data(torch.from_numpy(synth.template_counts(spec, spec.seed + 80)).cuda())
    q_full.set_precision(precision)
    for k, a in snaps.items():
        # the loss of a step equals a plain evaluation at its state (the loss
        # alone, on the FFTs, for FP32; the same precision's loss and gradient
        # otherwise)
        if precision == 0:
            f = q_full.loss(*[torch.from_numpy(v).cuda() for v in a]).item()
            assert abs(f - f_rec[k]) <= 1e-9 * abs(f), (k, f, f_rec[k])
        else:
            f = q_full.loss_grad(*[torch.from_numpy(v).cuda() for v in a])[0].item()
            assert abs(f - f_rec[k]) <= 1e-12 * abs(f), (k, f, f_rec[k])
    q_full.close()
    # the oracle at the GPU's iterates, on a seeded 1/16 of the scan positions
    js = np.sort(np.random.default_rng(spec.seed + 82).choice(scan.shape[0], scan.shape[0] // 16, replace=False))
    sub = np.ascontiguousarray(scan[js])
    y = synth.template_counts(spec, spec.seed + 80, scan_index=js)
    orc = oracle.OracleProblem.from_spec(spec, sub)
    q = mpbp.Problem(spec.n1, spec.n2, spec.ncomp, spec.npeaks, spec.m, sub, spec.G, spec.phase_scale)
    q.set_probe(torch.from_numpy(probe).cuda())
    q.set_data(torch.from_numpy(y).cuda())
    q.set_precision(precision)
    for k, a in snaps.items():
        xk = [torch.from_numpy(v).cuda() for v in a]
        got = [t.cpu().numpy() for t in q.loss_grad(*xk)]
        f, gr, gu, ga = orc.loss_grad(*a, probe, y)
        # the bound of a gradient block: 1e-4, or for the split tensor-core DFTs
        # (error stated per result rather than bounded) 20 times the FP32 FFTs'
        # error at the same state where that is larger -- the u gradient is
        # assembled from Im(E_m acc_m), a difference of larger terms, and some
        # states amplify every path's rounding by that factor
        ref32 = None
        if precision == 1:
            q.set_precision(0)
            ref32 = [t.cpu().numpy() for t in q.loss_grad(*xk)]
            q.set_precision(1)

        def bound(i, c=None):
            if ref32 is None:
                return 1e-4
            e32 = rel_l2(ref32[i] if c is None else ref32[i][c], (gr, gu, ga)[i - 1] if c is None else gu[c])
            return max(1e-4, 20 * e32)
        assert abs(got[0][0] - f) <= 1e-5 * abs(f), (k, got[0][0], f)
        assert rel_l2(got[1], gr) <= bound(1), (k, rel_l2(got[1], gr))
        for c in range(3):
            if np.abs(gu[c]).max() > 0:
                assert rel_l2(got[2][c], gu[c]) <= bound(2, c), (k, c, rel_l2(got[2][c], gu[c]), bound(2, c))
        assert rel_l2(got[3], ga) <= bound(3), k
    q.sync_status()
