"""The paper's minibatch optimizer (Alg. 1 without its projector line) and
the per-peak-phase form (Sec. 5) on the GPU, against the FP64 oracle.

Adam normalises every step by the gradient's running RMS, so a gradient
element that sits at the FP32 rounding level can move by up to a step in
either direction on one side and not the other.  The replay therefore starts
each oracle step from the GPU's own state (variables and moments), and
compares: the minibatch loss (<= 1e-5), the new moments (relative L2 <= 1e-4,
the gradient tolerance), the update wherever the gradient element is at least
1e-3 of the block's largest (<= 1e-2 step sizes), and everywhere Adam's bound
on one step, (1 - b1) / sqrt(1 - b2) step sizes.
"""
import math

import numpy as np
import pytest

from helpers import Case, custom_spec, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LR = dict(lr_u=0.01, lr_chi=0.1, lr_alpha=0.1)


def _problem(case, mask=None):
    from paper_2312_14907_gb300 import mpbp
    p = mpbp.Problem.from_spec(case.spec, case.scan)
    p.set_probe(torch.from_numpy(case.probe).cuda())
    p.set_data(torch.from_numpy(case.y).cuda())
    return p


def _case():
    spec, scan = custom_spec(96, 32, 6, 12, npeaks=3, offset=0, seed=4)
    return Case(spec, scan=scan, state="perturbed", seed=4)


def _log_state(case):
    chi = np.log(np.clip(case.rho, 0.2, None)).astype(np.float32)
    return chi, case.u.astype(np.float32).copy(), np.log(case.alpha).astype(np.float32)


def _mask(spec):
    m = np.ones((spec.n1, spec.n2), np.float32)
    m[:4, :] = 0.0
    m[:, -5:] = 0.0
    return m


def test_phase_form_matches_oracle():
    case = _case()
    rng = np.random.default_rng(8)
    phi = rng.uniform(-3, 3, (case.spec.npeaks, case.spec.n1, case.spec.n2)).astype(np.float32)
    p = _problem(case)
    rho, alpha = [torch.from_numpy(a).cuda() for a in (case.rho, case.alpha)]
    for frames in (None, np.array([0, 5, 5, 17, 40, 101], np.int32)):
        fd = None if frames is None else torch.from_numpy(frames).cuda()
        got = [t.cpu().numpy() for t in p.loss_grad_phases(rho, torch.from_numpy(phi).cuda(), alpha, frames=fd)]
        f, gr, gphi, ga = case.oracle.loss_grad_phases(case.rho, phi, case.alpha, case.probe, case.y,
                                                       frames=frames)
        assert abs(got[0][0] - f) <= 1e-5 * abs(f)
        assert rel_l2(got[1], gr) <= 1e-4
        for m in range(case.spec.npeaks):
            assert rel_l2(got[2][m], gphi[m]) <= 1e-4, m
        assert rel_l2(got[3], ga) <= 1e-4
    # at the phases a displacement field defines, the two forms agree
    phi_u = (case.spec.phase_scale * np.einsum("mc,cij->mij", np.asarray(case.spec.G), case.u)).astype(np.float32)
    a = [t.cpu().numpy() for t in p.loss_grad_phases(rho, torch.from_numpy(phi_u).cuda(), alpha)]
    b = [t.cpu().numpy() for t in p.loss_grad(rho, torch.from_numpy(case.u).cuda(), alpha)]
    assert abs(a[0][0] - b[0][0]) <= 1e-5 * abs(b[0][0])
    assert rel_l2(a[1], b[1]) <= 1e-4
    p.sync_status()


def test_adam_minibatch_steps_replay_against_oracle():
    import oracle
    from paper_2312_14907_gb300 import synth
    case = _case()
    spec = case.spec
    mask = _mask(spec)
    p = _problem(case)
    st = p.adam_init(**LR)
    chi0, u0, at0 = _log_state(case)
    chi, u, at = [torch.from_numpy(a.copy()).cuda() for a in (chi0, u0, at0)]
    md = torch.from_numpy(mask).cuda()
    order = synth.epoch_order(spec.nframes, 11)
    b = 12   # 8 minibatches of the 108 frames
    b1, b2 = 0.9, 0.999
    bound = (1 - b1) / math.sqrt(1 - b2) * 1.001
    for k in range(8):
        fr = order[k * b:(k + 1) * b]
        x_prev = [t.cpu().numpy().astype(np.float64) for t in (chi, u, at)]
        mo_prev = [t.cpu().numpy().astype(np.float64) for t in p.adam_get_state()]
        t_prev = p.read_adam_state(st).t
        p.adam_step(torch.from_numpy(fr).cuda(), chi, u, at, st, mask=md)
        x_gpu = [t.cpu().numpy().astype(np.float64) for t in (chi, u, at)]
        mo_gpu = [t.cpu().numpy().astype(np.float64) for t in p.adam_get_state()]
        s_gpu = p.read_adam_state(st)
        assert s_gpu.t == t_prev + 1
        # the oracle's step from the GPU's state
        opt = oracle.OracleAdam(case.oracle, case.probe, case.y, mask=mask, **LR)
        for dst, src in zip((opt.m_chi, opt.v_chi, opt.m_u, opt.v_u, opt.m_a, opt.v_a), mo_prev):
            dst[...] = src.reshape(dst.shape)
        opt.t.value = t_prev
        x_orc = [a.copy() for a in x_prev]
        f_orc = opt.step(fr, *x_orc)
        _, g_chi, g_u, g_a = case.oracle.loss_grad_log(*x_prev, case.probe, case.y, mask=mask, frames=fr)
        assert abs(s_gpu.f_last - f_orc) <= 1e-5 * abs(f_orc), (k, s_gpu.f_last, f_orc)
        for a, o in zip(mo_gpu, (opt.m_chi, opt.v_chi, opt.m_u, opt.v_u, opt.m_a, opt.v_a)):
            if np.abs(o).max() > 0:
                assert rel_l2(a.reshape(o.shape), o) <= 1e-4, k
        for name, xp, xg, xo, g, lr in (("chi", x_prev[0], x_gpu[0], x_orc[0], g_chi, LR["lr_chi"]),
                                        ("u", x_prev[1], x_gpu[1], x_orc[1], g_u, LR["lr_u"]),
                                        ("alpha_t", x_prev[2][1:], x_gpu[2][1:], x_orc[2][1:], g_a[1:],
                                         LR["lr_alpha"])):
            dg, do = xg - xp, xo - xp
            assert np.abs(dg).max() <= bound * lr + 1e-6, (k, name)
            det = np.abs(g) >= 1e-3 * np.abs(g).max()
            assert det.mean() > 0.2 or name == "alpha_t", (k, name, det.mean())
            assert np.abs(dg - do)[det].max() <= 1e-2 * lr, (k, name)
        # alpha_0 and the pixels off the support never move
        assert x_gpu[2][0] == at0[0]
        np.testing.assert_array_equal(x_gpu[0][mask == 0], chi0[mask == 0])
    p.sync_status()


def test_adam_epoch_lowers_the_loss_and_resumes_from_a_checkpoint():
    from paper_2312_14907_gb300 import synth
    case = _case()
    spec = case.spec
    mask = _mask(spec)
    md = torch.from_numpy(mask).cuda()
    p = _problem(case)
    st = p.adam_init(lr_u=0.005, lr_chi=0.02, lr_alpha=0.02)
    chi0, u0, at0 = _log_state(case)
    chi, u, at = [torch.from_numpy(a.copy()).cuda() for a in (chi0, u0, at0)]

    def full_loss(c, uu, a):
        rho = md * torch.exp(c)
        alpha = torch.exp(a)
        alpha[0] = 1.0
        return p.loss_grad(rho.contiguous(), uu, alpha.contiguous())[0].item()

    f0 = full_loss(chi, u, at)
    order = torch.from_numpy(synth.epoch_order(spec.nframes, 3)).cuda()
    for k in range(0, spec.nframes, 25):
        p.adam_step(order[k:k + 25].contiguous(), chi, u, at, st, mask=md)
    assert full_loss(chi, u, at) < f0
    assert p.read_adam_state(st).t == -(-spec.nframes // 25)
    # checkpoint: variables, state, moments; resume in a fresh context
    q = _problem(case)
    st_q = q.adam_init(lr_u=0.005, lr_chi=0.02, lr_alpha=0.02)
    st_q.copy_(st)
    q.adam_set_state(p.adam_get_state())
    chi_q, u_q, at_q = chi.clone(), u.clone(), at.clone()
    nxt = order[:25].contiguous()
    p.adam_step(nxt, chi, u, at, st, mask=md)
    q.adam_step(nxt, chi_q, u_q, at_q, st_q, mask=md)
    torch.cuda.synchronize()
    for a, b in ((chi, chi_q), (u, u_q), (at, at_q)):
        assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= 1e-6
    assert p.read_adam_state(st).t == q.read_adam_state(st_q).t
    p.sync_status()
    q.sync_status()


def test_concurrent_unwrapped_iteration_lowers_the_loss():
    """Alg. 1 with its projector line (the paper's C-UW): an Adam step, then
    Pi_U on u inside the support; one shuffled epoch lowers the full loss,
    and the projected field is a fixed point of Pi_U."""
    from paper_2312_14907_gb300 import synth
    case = _case()
    spec = case.spec
    mask = _mask(spec)
    md = torch.from_numpy(mask).cuda()
    p = _problem(case)
    st = p.adam_init(lr_u=0.005, lr_chi=0.02, lr_alpha=0.02)
    chi0, u0, at0 = _log_state(case)
    chi, u, at = [torch.from_numpy(a.copy()).cuda() for a in (chi0, u0, at0)]

    def full_loss():
        rho = (md * torch.exp(chi)).contiguous()
        alpha = torch.exp(at)
        alpha[0] = 1.0
        return p.loss_grad(rho, u, alpha.contiguous())[0].item()

    f0 = full_loss()
    order = torch.from_numpy(synth.epoch_order(spec.nframes, 5)).cuda()
    for k in range(0, spec.nframes, 25):
        p.adam_step(order[k:k + 25].contiguous(), chi, u, at, st, mask=md)
        p.project_displacement(u, md)
    assert full_loss() < f0
    again = p.project_displacement(u.clone(), md)
    assert rel_l2(again.cpu().numpy(), u.cpu().numpy()) <= 1e-6
    p.sync_status()


def test_illumination_map_matches_oracle():
    """The map behind the final threshold, with frames cut by the grid edge
    and one probe per peak."""
    spec, scan = custom_spec(90, 32, 5, 16, npeaks=3, offset=-9, probe_per_peak=True)
    rng = np.random.default_rng(12)
    probe = (rng.standard_normal((3, 32, 32)) + 1j * rng.standard_normal((3, 32, 32))).astype(np.complex64)
    case = Case(spec, scan=scan, probe=probe, state="perturbed")
    p = _problem(case)
    got = p.illumination().cpu().numpy()
    ref = case.oracle.illumination(case.probe)
    assert rel_l2(got, ref) <= 1e-6
    assert np.all(got[ref == 0] == 0)
    p.sync_status()
