"""The unfused comparison path that bench.py times beside the library (plain
PyTorch ops, FP32): on the CPU it must compute the same loss and gradient as
the FP64 oracle, so that the comparison is between equal computations."""
import numpy as np
import pytest

from helpers import Case, custom_spec, rel_l2

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("m,off,per_peak", [(16, -3, False), (32, 2, True)])
def test_unfused_path_matches_oracle(m, off, per_peak):
    import bench
    spec, scan = custom_spec(2 * m + 10, m, 3, m // 2 + 1, npeaks=3, offset=off, probe_per_peak=per_peak)
    rng = np.random.default_rng(m)
    probe = None
    if per_peak:
        probe = (rng.standard_normal((3, m, m)) + 1j * rng.standard_normal((3, m, m))).astype(np.complex64)
    case = Case(spec, scan=scan, probe=probe, state="perturbed")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a))
    amp = t(np.sqrt(case.y).astype(np.float32))
    G = torch.tensor(np.asarray(spec.G), dtype=torch.float32)
    f, gr, gu, ga = bench.torch_loss_grad(torch, t(case.rho), t(case.u), t(case.alpha), t(case.probe), amp,
                                          t(np.asarray(case.scan, np.int64)), G, spec.phase_scale, m)
    f_o, gr_o, gu_o, ga_o = case.oracle_loss_grad()
    assert abs(float(f) - f_o) <= 1e-5 * abs(f_o)
    assert rel_l2(gr.numpy(), gr_o) <= 1e-4
    assert rel_l2(gu.numpy(), gu_o) <= 1e-4
    assert rel_l2(ga.numpy(), ga_o) <= 1e-4
