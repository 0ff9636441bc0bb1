"""The allocation-free entry point (mpbp_loss_grad_noalloc) against the
context entry point (mpbp_loss_grad), on two calls in a row.

It serves callers that cannot allocate device memory; it works in a fixed
scratch array that keeps the previous call's contents, so the second call
checks that everything that must start from zero is cleared.  This file runs
last so that a failure here leaves every other test already run."""
import numpy as np
import pytest

from helpers import Case, custom_spec, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matches_context_entry_point_twice():
    from paper_2312_14907_gb300 import mpbp
    spec, scan = custom_spec(96, 32, 6, 12, npeaks=3, offset=-4)
    case = Case(spec, scan=scan, state="perturbed")
    p = mpbp.Problem.from_spec(spec, scan)
    probe = torch.from_numpy(case.probe).cuda()
    y = torch.from_numpy(case.y).cuda()
    p.set_probe(probe)
    p.set_data(y)
    x = [torch.from_numpy(a).cuda() for a in (case.rho, case.u, case.alpha)]
    ref = [t.cpu().numpy() for t in p.loss_grad(*x)]
    for call in range(2):
        out = (torch.full((1,), np.nan, dtype=torch.float64, device="cuda"),
               torch.full(p.shapes["rho"], np.nan, dtype=torch.float32, device="cuda"),
               torch.full(p.shapes["u"], np.nan, dtype=torch.float32, device="cuda"),
               torch.full((spec.npeaks,), np.nan, dtype=torch.float64, device="cuda"))
        got = [t.cpu().numpy() for t in mpbp.loss_grad_noalloc(p, probe, y, *x, out)]
        assert abs(got[0][0] - ref[0][0]) <= 1e-5 * abs(ref[0][0]), call
        assert rel_l2(got[1], ref[1]) <= 1e-4, call
        assert rel_l2(got[2], ref[2]) <= 1e-4, call
        assert rel_l2(got[3], ref[3]) <= 1e-4, call


def test_noalloc_rejects_problems_beyond_its_scratch():
    from paper_2312_14907_gb300 import mpbp, synth
    spec = synth.config(2)             # about 50 MB of scratch: more than the array holds
    scan = synth.scan_positions(spec)
    p = mpbp.Problem.from_spec(spec, scan)
    dev = "cuda"
    probe = torch.zeros((spec.m, spec.m), dtype=torch.complex64, device=dev)
    y = torch.zeros(p.shapes["frames"], dtype=torch.float32, device=dev)
    x = [torch.zeros(p.shapes[k], dtype=torch.float32, device=dev) for k in ("rho", "u", "alpha")]
    out = (torch.zeros(1, dtype=torch.float64, device=dev), torch.zeros(p.shapes["rho"], device=dev),
           torch.zeros(p.shapes["u"], device=dev), torch.zeros(spec.npeaks, dtype=torch.float64, device=dev))
    with pytest.raises(mpbp.MPBPError) as ei:
        mpbp.loss_grad_noalloc(p, probe, y, *x, out)
    assert ei.value.status == 2
