"""The allocation-free entry point (mpbp_loss_grad_noalloc), for callers
that cannot allocate device memory, against the FP64 oracle and against the
context entry point (mpbp_loss_grad).

It works in one fixed scratch array that keeps the previous call's contents.
The calls below change the geometry between calls (frame side, probe per
peak, grid size), so that the second evaluation of a problem runs over
scratch laid out for another one: anything that must start from zero and is
not cleared shows up as a mismatch.  This file runs last so that a failure
here leaves every other test already run."""
import numpy as np
import pytest

from helpers import Case, custom_spec, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-5
GRAD_TOL = 1e-4


def _problem(kind):
    from paper_2312_14907_gb300 import mpbp
    if kind == "a":
        spec, scan = custom_spec(96, 32, 6, 12, npeaks=3, offset=-4)
        probe = None
    else:
        spec, scan = custom_spec(136, 64, 4, 22, npeaks=3, offset=-5, probe_per_peak=True, n2=120)
        rng = np.random.default_rng(41)
        probe = (rng.standard_normal((3, 64, 64)) + 1j * rng.standard_normal((3, 64, 64))).astype(np.complex64)
    case = Case(spec, scan=scan, probe=probe, state="perturbed")
    p = mpbp.Problem.from_spec(spec, scan)
    dev = {"probe": torch.from_numpy(case.probe).cuda(), "y": torch.from_numpy(case.y).cuda()}
    dev["x"] = [torch.from_numpy(a).cuda() for a in (case.rho, case.u, case.alpha)]
    return case, p, dev


def _outs(p):
    return (torch.full((1,), np.nan, dtype=torch.float64, device="cuda"),
            torch.full(p.shapes["rho"], np.nan, dtype=torch.float32, device="cuda"),
            torch.full(p.shapes["u"], np.nan, dtype=torch.float32, device="cuda"),
            torch.full((p.npeaks,), np.nan, dtype=torch.float64, device="cuda"))


def _close(got, ref):
    assert abs(got[0][0] - ref[0]) <= LOSS_TOL * abs(ref[0]), (got[0][0], ref[0])
    assert rel_l2(got[1], ref[1]) <= GRAD_TOL
    for c in range(ref[2].shape[0]):
        if np.abs(ref[2][c]).max() > 0:
            assert rel_l2(got[2][c], ref[2][c]) <= GRAD_TOL, c
    assert rel_l2(got[3], ref[3]) <= GRAD_TOL


def test_noalloc_matches_oracle_and_context_across_geometries():
    from paper_2312_14907_gb300 import mpbp
    a_case, a_p, a_dev = _problem("a")
    b_case, b_p, b_dev = _problem("b")
    a_ref = a_case.oracle_loss_grad()
    b_ref = b_case.oracle_loss_grad()
    # the context entry point on problem a, for the call-to-call comparison
    a_p.set_probe(a_dev["probe"])
    a_p.set_data(a_dev["y"])
    a_ctx = [t.cpu().numpy() for t in a_p.loss_grad(*a_dev["x"])]
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for kind in ("a", "b", "a", "a"):
        case, p, dv, ref = (a_case, a_p, a_dev, a_ref) if kind == "a" else (b_case, b_p, b_dev, b_ref)
        out = mpbp.loss_grad_noalloc(p, dv["probe"], dv["y"], *dv["x"], _outs(p), dev_err=err)
        mpbp.noalloc_check(err)
        assert err.item() == 0
        got = [t.cpu().numpy() for t in out]
        _close(got, ref)
        if kind == "a":
            _close(got, a_ctx)


def test_noalloc_reports_a_nonfinite_loss_and_recovers():
    from paper_2312_14907_gb300 import mpbp
    case, p, dv = _problem("a")
    rho, u, alpha = dv["x"]
    bad = alpha.clone()
    bad[1] = float("nan")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    mpbp.loss_grad_noalloc(p, dv["probe"], dv["y"], rho, u, bad, _outs(p), dev_err=err)
    with pytest.raises(mpbp.MPBPError) as ei:
        mpbp.noalloc_check(err)
    assert ei.value.status == 4
    out = mpbp.loss_grad_noalloc(p, dv["probe"], dv["y"], rho, u, alpha, _outs(p), dev_err=err)
    mpbp.noalloc_check(err)
    _close([t.cpu().numpy() for t in out], case.oracle_loss_grad())


def test_noalloc_binding_rejects_bad_tensors():
    from paper_2312_14907_gb300 import mpbp
    case, p, dv = _problem("a")
    rho, u, alpha = dv["x"]
    cases = [
        dict(probe=dv["probe"].cpu()),                               # host memory
        dict(probe=dv["probe"].to(torch.complex128)),                # wrong dtype
        dict(y=dv["y"][:, :-1].contiguous()),                        # too few frames
        dict(rho=rho.t()),                                           # not contiguous
    ]
    for bad in cases:
        args = dict(probe=dv["probe"], y=dv["y"], rho=rho, u=u, alpha=alpha)
        args.update(bad)
        with pytest.raises((TypeError, ValueError)):
            mpbp.loss_grad_noalloc(p, args["probe"], args["y"], args["rho"], args["u"], args["alpha"], _outs(p))
    out = list(_outs(p))
    out[0] = torch.zeros(1, dtype=torch.float32, device="cuda")       # loss must be float64
    with pytest.raises(TypeError):
        mpbp.loss_grad_noalloc(p, dv["probe"], dv["y"], rho, u, alpha, tuple(out))


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
