"""The loss without its gradient (mpbp_loss: the fused frame kernel stopped
after the amplitude residual) against the FP64 oracle, and the autograd
function in both of its forms -- gradients saved in forward, or the fused
pass rerun in backward (recompute=True) -- against the oracle and each other."""
import numpy as np
import pytest

from helpers import Case, custom_spec, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gpu(case):
    from paper_2312_14907_gb300 import mpbp
    p = mpbp.Problem.from_spec(case.spec, case.scan)
    p.set_probe(torch.from_numpy(case.probe).cuda())
    p.set_data(torch.from_numpy(case.y).cuda())
    return p, [torch.from_numpy(a).cuda() for a in (case.rho, case.u, case.alpha)]


# (n, m, scan side, step, offset, n2): tile copies (even n2) and cp.async (odd
# n2), every frame side; the M = 128 case has more frames than two per block
@pytest.mark.parametrize("n,m,side,step,off,n2", [
    (24, 8, 4, 5, -2, None), (40, 16, 5, 6, -3, 41), (80, 32, 6, 9, -4, None), (80, 32, 6, 9, -4, 79),
    (150, 64, 6, 17, -5, None), (150, 64, 6, 17, -5, 151), (256, 128, 13, 10, -6, None),
    (256, 128, 13, 10, -6, 255)])
def test_loss_only_matches_oracle(n, m, side, step, off, n2):
    spec, scan = custom_spec(n, m, side, step, npeaks=2, offset=off, n2=n2)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    f = case.oracle_loss_grad()[0]
    got = p.loss(*x).item()
    assert abs(got - f) <= 1e-5 * abs(f), (got, f)
    # the same frames' loss through the gradient path
    full = p.loss_grad(*x)[0].item()
    assert abs(got - full) <= 1e-9 * abs(full)
    frames = np.random.default_rng(m).permutation(spec.nframes)[: max(1, spec.nframes // 3)].astype(np.int32)
    got_s = p.loss(*x, frames=torch.from_numpy(frames).cuda()).item()
    f_s = case.oracle_loss_grad(frames=frames)[0]
    assert abs(got_s - f_s) <= 1e-5 * abs(f_s)
    p.sync_status()


@pytest.mark.parametrize("m", [32, 128])
def test_autograd_recompute_matches_oracle_and_saved_form(m):
    from paper_2312_14907_gb300 import mpbp
    spec, scan = custom_spec(3 * m, m, 5, m // 2, npeaks=3, offset=-3)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    f_o, gr_o, gu_o, ga_o = case.oracle_loss_grad()
    grads = {}
    for recompute in (False, True):
        rho, u, alpha = [t.clone().requires_grad_(True) for t in x]
        f = mpbp.mpbp_loss(rho, u, alpha, p, recompute=recompute)
        assert abs(f.item() - f_o) <= 1e-5 * abs(f_o)
        (3.0 * f).backward()
        grads[recompute] = [t.grad.detach().double().cpu().numpy() / 3.0 for t in (rho, u, alpha)]
        assert rel_l2(grads[recompute][0], gr_o) <= 1e-4
        assert rel_l2(grads[recompute][1], gu_o) <= 1e-4
        assert rel_l2(grads[recompute][2], ga_o) <= 1e-4
    # the two forms agree up to the order of the floating-point atomics
    for a, b in zip(grads[False], grads[True]):
        assert rel_l2(a, b) <= 1e-5
    p.sync_status()
