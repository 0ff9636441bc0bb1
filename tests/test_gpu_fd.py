"""GPU gradient against central finite differences of the FP64 loss at 64
seeded pixels of the 256^2, 3-peak, 31x31-scan, 64x64-frame problem.

The loss of Eq. 4 at a perturbed state is differenced in rho at each pixel
(and in u_x at the first 16), over the frames whose patch covers the pixel
(the other frames do not depend on it), with the FP64 oracle, so that the
difference quotient is limited only by its O(h^2) truncation.  Both precision
modes of the GPU gradient (FP32 FFTs; split-FP16 tensor-core DFTs) are
compared with it at 1e-4 relative L2 over the sampled pixels.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NPIX = 64   # pixels whose rho derivative is differenced
NU = 16     # of which the first NU also in u_x


def _covering_frames(spec, scan, i, j):
    out = []
    for m in range(spec.npeaks):
        for k, (sx, sy) in enumerate(scan):
            if sx <= i < sx + spec.m and sy <= j < sy + spec.m:
                out.append(m * scan.shape[0] + k)
    return np.array(out, np.int32)


@pytest.fixture(scope="module")
def fd_case():
    import oracle
    from paper_2312_14907_gb300 import synth
    spec = synth.config(2)
    scan = synth.scan_positions(spec)
    rng = np.random.default_rng(spec.seed + 64)
    probe = (synth.probe(spec) * 3.0).astype(np.complex64)
    y = synth.template_counts(spec, spec.seed + 65)
    rho, u, alpha = [np.ascontiguousarray(a, np.float32) for a in synth.perturbed_state(spec, rng, 0.05)]
    # pixels inside the scanned area
    lo = max(int(scan.min()), 0)
    hi = min(int(scan.max()) + spec.m, spec.n1)
    pix = rng.integers(lo, hi, size=(NPIX, 2))
    orc = oracle.OracleProblem.from_spec(spec, scan)
    r64, u64, a64 = rho.astype(np.float64), u.astype(np.float64), alpha.astype(np.float64)
    h = 1e-4
    fd_rho, fd_u = np.empty(NPIX), np.empty(NU)
    for n, (i, j) in enumerate(pix):
        fr = _covering_frames(spec, scan, i, j)

        def f(rr, uu):
            return orc.loss_grad(rr, uu, a64, probe, y, frames=fr)[0]

        rp, rm = r64.copy(), r64.copy()
        rp[i, j] += h
        rm[i, j] -= h
        fd_rho[n] = (f(rp, u64) - f(rm, u64)) / (2 * h)
        if n < NU:
            up, um = u64.copy(), u64.copy()
            up[0, i, j] += h
            um[0, i, j] -= h
            fd_u[n] = (f(r64, up) - f(r64, um)) / (2 * h)
    return spec, scan, probe, y, (rho, u, alpha), pix, fd_rho, fd_u


@pytest.mark.parametrize("precision", [0, 1])
def test_gradient_matches_central_differences_at_64_pixels(fd_case, precision):
    from paper_2312_14907_gb300 import mpbp
    spec, scan, probe, y, x, pix, fd_rho, fd_u = fd_case
    p = mpbp.Problem.from_spec(spec, scan)
    p.set_probe(torch.from_numpy(probe).cuda())
    p.set_data(torch.from_numpy(y).cuda())
    p.set_precision(precision)
    _, g_rho, g_u, _ = [t.cpu().numpy() for t in p.loss_grad(*[torch.from_numpy(a).cuda() for a in x])]
    p.sync_status()
    got_rho = g_rho[pix[:, 0], pix[:, 1]]
    got_u = g_u[0, pix[:NU, 0], pix[:NU, 1]]
    for got, fd in ((got_rho, fd_rho), (got_u, fd_u)):
        assert np.abs(fd).max() > 0
        rel = np.linalg.norm(got - fd) / np.linalg.norm(fd)
        assert rel <= 1e-4, rel
        assert np.abs(got - fd).max() <= 1e-3 * np.abs(fd).max()
