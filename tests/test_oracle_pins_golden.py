"""Pins that use the values the paper prints for its simulated data set
(Sec. 4; fixture tests/golden/sec4_numerical_experiment.txt).

The closed form: with noise-free data made at peak scalings alpha_t and the
same density and displacement, sqrt(I) - sqrt(y) = (alpha_m - alpha_t,m)|Psi'|
frame by frame (Psi' the far field at alpha = 1), so the loss of Eq. 4 is
1/2 sum_m (alpha_m - alpha_t,m)^2 sum |Psi'|^2 and, by Parseval for the
unnormalised DFT,
    df/dalpha_m = (alpha_m - alpha_t,m) M^2 sum_j sum_k |P_m(k)|^2 rho(s_j + k)^2
(rho = 0 outside the grid).  The right-hand side is summed here directly,
without the oracle's transforms.
"""
import os

import numpy as np

from paper_2312_14907_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sec4_numerical_experiment.txt")


def _golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].split()
            if line:
                out.setdefault(line[0], []).append([float(v) for v in line[1:]])
    return out


def test_inputs_follow_the_printed_experiment():
    g = _golden()
    np.testing.assert_array_equal(np.array(g["peak"]), synth.PAPER_PEAKS)
    s = np.array(g["scaling"]).ravel()
    np.testing.assert_allclose(synth.PAPER_SCALINGS, s / s[0], rtol=1e-15)
    np.testing.assert_allclose(synth.PAPER_SCALINGS, [1.0, 0.875, 0.525, 0.25], rtol=1e-15)
    spec = synth.config(3)          # the 4-peak workload: the paper's peaks, scan step and scalings
    assert spec.npeaks == 4 and spec.step == int(g["scan_step"][0][0])
    np.testing.assert_array_equal(spec.G[:, :3], synth.PAPER_PEAKS)
    np.testing.assert_allclose(synth.alpha_truth(spec), s / s[0], rtol=1e-15)


def test_alpha_gradient_closed_form_at_the_printed_scalings(oracle_mod):
    g = _golden()
    s = np.array(g["scaling"]).ravel()
    alpha_t = s / s[0]
    n, m, D = 16, 8, 4
    rng = np.random.default_rng(41)
    scan = np.array([[r, c] for r in (-2, 3, 8) for c in (-1, 4, 9)], np.int32)
    p = oracle_mod.OracleProblem(n, n, 3, D, m, scan, synth.PAPER_PEAKS)
    P = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    rho = rng.uniform(0.3, 1.5, (n, n))
    u = rng.standard_normal((3, n, n)) * 0.4
    y = p.forward(rho, u, alpha_t, P)                   # noise free, no background
    alpha = np.ones(D)
    f, gr, gu, ga = p.loss_grad(rho, u, alpha, P, y)
    P2 = np.abs(P) ** 2
    ref = np.zeros(D)
    energy = 0.0
    for s0, s1 in scan:
        for k0 in range(m):
            for k1 in range(m):
                r0, r1 = s0 + k0, s1 + k1
                if 0 <= r0 < n and 0 <= r1 < n:
                    energy += P2[k0, k1] * rho[r0, r1] ** 2
    energy *= m * m                                     # sum_q |Psi'|^2 of one peak, all frames
    ref = (alpha - alpha_t) * energy
    np.testing.assert_allclose(ga, ref, rtol=1e-10, atol=1e-10 * energy)
    assert ga[0] == 0.0 or abs(ga[0]) <= 1e-10 * energy   # the reference peak: alpha_t = 1
    assert np.all(ga[1:] > 0)                           # lowering alpha_m toward alpha_t lowers f
    # and the loss itself: 1/2 sum_m (alpha_m - alpha_t,m)^2 times the same energy
    assert abs(f - 0.5 * np.sum((alpha - alpha_t) ** 2) * energy) <= 1e-10 * f
