"""FP64 CPU oracle for the MPBP loss and gradient (arXiv 2312.14907).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it; the product path never imports it.

The arithmetic lives in ``mpbp_oracle.c`` (plain C, double precision, direct
DFT, one OpenMP loop over frames); this module compiles it with gcc and calls
it through ctypes with NumPy arrays.  It shares no code with the CUDA path.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpbp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile liboracle.so with gcc (-O2, IEEE arithmetic, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Problem(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int), ("ncomp", ctypes.c_int),
                ("npeaks", ctypes.c_int), ("m", ctypes.c_int), ("nscan", ctypes.c_int),
                ("G", ctypes.POINTER(ctypes.c_double)), ("scan", ctypes.POINTER(ctypes.c_int)),
                ("phase_scale", ctypes.c_double), ("probe_per_peak", ctypes.c_int)]


class StepParams(ctypes.Structure):
    _fields_ = [("c_armijo", ctypes.c_double), ("grow", ctypes.c_double),
                ("shrink", ctypes.c_double), ("t0", ctypes.c_double),
                ("w_rho", ctypes.c_double), ("w_u", ctypes.c_double),
                ("w_alpha", ctypes.c_double)]


class AdamParams(ctypes.Structure):
    _fields_ = [("lr_u", ctypes.c_double), ("lr_chi", ctypes.c_double),
                ("lr_alpha", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("eps", ctypes.c_double)]


class StepState(ctypes.Structure):
    _fields_ = [("f_prev", ctypes.c_double), ("gn2_prev", ctypes.c_double),
                ("t", ctypes.c_double), ("f_last", ctypes.c_double),
                ("k", ctypes.c_int), ("accepted", ctypes.c_int),
                ("n_accept", ctypes.c_int), ("n_reject", ctypes.c_int)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        pp = ctypes.POINTER(Problem)
        lib.oracle_dft2.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int]
        lib.oracle_dft2.restype = None
        lib.oracle_object_build.argtypes = [pp, dp, dp, dp, dp]
        lib.oracle_object_build.restype = None
        lib.oracle_forward.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        lib.oracle_forward.restype = None
        lib.oracle_loss_grad.argtypes = [pp, dp, dp, dp, dp, dp, dp, ip, ctypes.c_int,
                                         dp, dp, dp, dp, ctypes.c_int]
        lib.oracle_loss_grad.restype = ctypes.c_double
        lib.oracle_step.argtypes = [pp, dp, dp, dp, ctypes.POINTER(StepParams),
                                    ctypes.POINTER(StepState), dp, dp, dp, dp, dp, dp,
                                    dp, dp, dp, ctypes.c_int]
        lib.oracle_step.restype = None
        lib.oracle_loss_grad_phases.argtypes = [pp, dp, dp, dp, dp, dp, dp, ip, ctypes.c_int,
                                                dp, dp, dp, ctypes.c_int]
        lib.oracle_loss_grad_phases.restype = ctypes.c_double
        lib.oracle_loss_grad_log.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, ip, ctypes.c_int,
                                             dp, dp, dp, ctypes.c_int]
        lib.oracle_loss_grad_log.restype = ctypes.c_double
        lib.oracle_adam_update.argtypes = [ctypes.c_long, dp, dp, dp, dp, ctypes.c_long,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double]
        lib.oracle_adam_update.restype = None
        lib.oracle_adam_step.argtypes = [pp, dp, dp, dp, ip, ctypes.c_int, dp,
                                         ctypes.POINTER(AdamParams), ctypes.POINTER(ctypes.c_long),
                                         dp, dp, dp, dp, dp, dp, dp, dp, dp, ctypes.c_int]
        lib.oracle_adam_step.restype = ctypes.c_double
        lib.oracle_unwrap2d.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.oracle_unwrap2d.restype = None
        lib.oracle_project_u.argtypes = [pp, dp, dp, dp]
        lib.oracle_project_u.restype = None
        lib.oracle_illumination.argtypes = [pp, dp, dp]
        lib.oracle_illumination.restype = None
        lib.oracle_probe_shift.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp]
        lib.oracle_probe_shift.restype = None
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _d(a):
    """Contiguous float64 copy (complex arrays become interleaved pairs)."""
    a = np.asarray(a)
    if np.iscomplexobj(a):
        a = np.ascontiguousarray(a, dtype=np.complex128).view(np.float64)
    return np.ascontiguousarray(a, dtype=np.float64)


def _c(a):
    """Contiguous complex128 array viewed as interleaved float64 pairs."""
    return np.ascontiguousarray(a, dtype=np.complex128).view(np.float64)


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def max_threads():
    return _load().oracle_max_threads()


def _frames(frames):
    if frames is None:
        return None, 0
    fr = np.ascontiguousarray(frames, dtype=np.int32)
    return fr, fr.size


def _iptr(fr):
    return None if fr is None else fr.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def adam_update(x, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of x (float64, in place) with gradient g at step t >= 1;
    m and v (float64, in place) are the moments (see oracle_adam_update)."""
    lib = _load()
    for a in (x, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _d(g)
    lib.oracle_adam_update(x.size, _ptr(x), _ptr(g), _ptr(m), _ptr(v), int(t), float(lr),
                           float(beta1), float(beta2), float(eps))


def unwrap2d(wrapped, mask=None):
    """Reliability-sorted 2-D phase unwrapping of wrapped [n1][n2] (see
    oracle_unwrap2d); mask nonzero = inside."""
    lib = _load()
    w = _d(wrapped)
    out = np.empty_like(w)
    lib.oracle_unwrap2d(w.shape[0], w.shape[1], _ptr(w), _ptr(None if mask is None else _d(mask)), _ptr(out))
    return out


def dft2(x, sign=-1):
    """Direct unnormalised 2-D DFT of a square complex array; sign -1 = F, +1 = F^H."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.complex128)
    m = x.shape[0]
    assert x.shape == (m, m)
    out = np.empty_like(x)
    lib.oracle_dft2(m, _ptr(x.view(np.float64)), _ptr(out.view(np.float64)), int(sign))
    return out


def probe_shift(P, d0, d1):
    """P(k - d) for a probe [M][M] and a real offset d = (d0, d1): the
    band-limited interpolation through the DFT (see oracle_probe_shift)."""
    lib = _load()
    P = np.ascontiguousarray(P, dtype=np.complex128)
    m = P.shape[0]
    assert P.shape == (m, m)
    out = np.empty_like(P)
    lib.oracle_probe_shift(m, _ptr(P.view(np.float64)), float(d0), float(d1), _ptr(out.view(np.float64)))
    return out


def frame_probes(problem, probe, offsets):
    """One probe per frame [D*J][M][M] for scan positions off the pixel grid:
    frame (m, j) takes probe P_m (or the shared P) shifted by offsets[j]
    (the fractional part d_j of s_j = n_j + d_j; the integer part is the
    problem's scan).  Use with a problem made with probe_per_peak=2."""
    probe = np.asarray(probe, dtype=np.complex128)
    offsets = np.asarray(offsets, dtype=np.float64).reshape(problem.nscan, 2)
    D, J, m = problem.npeaks, problem.nscan, problem.m
    per_peak = probe.ndim == 3 and probe.shape[0] == D and D > 1
    out = np.empty((D * J, m, m), np.complex128)
    for mpk in range(D):
        P = probe[mpk] if per_peak else probe.reshape(-1, m, m)[0]
        for j in range(J):
            out[mpk * J + j] = probe_shift(P, offsets[j, 0], offsets[j, 1])
    return out


class OracleProblem:
    """Geometry of one MPBP problem (see mpbp_oracle.c for the layouts)."""

    def __init__(self, n1, n2, ncomp, npeaks, m, scan, G, phase_scale=2 * np.pi,
                 probe_per_peak=False):
        self.G = _d(G).reshape(npeaks, ncomp)
        self.scan = np.ascontiguousarray(scan, dtype=np.int32).reshape(-1, 2)
        self.shape = (n1, n2)
        self.ncomp, self.npeaks, self.m = ncomp, npeaks, m
        self.nscan = self.scan.shape[0]
        self.phase_scale = float(phase_scale)
        # False / 0: one probe; True / 1: one per peak; 2: one per frame
        self.probe_per_peak = int(probe_per_peak)
        self.c = Problem(n1, n2, ncomp, npeaks, m, self.nscan,
                         _ptr(self.G), self.scan.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                         self.phase_scale, int(probe_per_peak))

    @classmethod
    def from_spec(cls, spec, scan):
        return cls(spec.n1, spec.n2, spec.ncomp, spec.npeaks, spec.m, scan, spec.G,
                   spec.phase_scale, spec.probe_per_peak)

    @property
    def nframes(self):
        return self.npeaks * self.nscan

    def object_build(self, rho, u, alpha):
        lib = _load()
        n1, n2 = self.shape
        rho, u, alpha = _d(rho), _d(u), _d(alpha)
        out = np.empty((self.npeaks, n1, n2), np.complex128)
        lib.oracle_object_build(ctypes.byref(self.c), _ptr(rho), _ptr(u), _ptr(alpha),
                                _ptr(out.view(np.float64)))
        return out

    def forward(self, rho, u, alpha, probe, bg=None):
        lib = _load()
        rho, u, alpha, probe = _d(rho), _d(u), _d(alpha), _c(probe)
        bg = None if bg is None else _d(bg)
        out = np.empty((self.npeaks, self.nscan, self.m, self.m), np.float64)
        lib.oracle_forward(ctypes.byref(self.c), _ptr(rho), _ptr(u), _ptr(alpha),
                           _ptr(probe), _ptr(bg), _ptr(out))
        return out

    def loss_grad(self, rho, u, alpha, probe, y, bg=None, frames=None, nthreads=0,
                  frame_loss=False):
        """Returns (loss, g_rho, g_u, g_alpha[, per-frame losses])."""
        lib = _load()
        n1, n2 = self.shape
        rho, u, alpha, probe, y = _d(rho), _d(u), _d(alpha), _c(probe), _d(y)
        bg = None if bg is None else _d(bg)
        g_rho = np.empty((n1, n2))
        g_u = np.empty((self.ncomp, n1, n2))
        g_alpha = np.empty(self.npeaks)
        fr = None
        nfr = 0
        if frames is not None:
            fr = np.ascontiguousarray(frames, dtype=np.int32)
            nfr = fr.size
        fl = np.empty(nfr if fr is not None else self.nframes) if frame_loss else None
        loss = lib.oracle_loss_grad(
            ctypes.byref(self.c), _ptr(rho), _ptr(u), _ptr(alpha), _ptr(probe), _ptr(bg),
            _ptr(y), None if fr is None else fr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            nfr, _ptr(g_rho), _ptr(g_u), _ptr(g_alpha), _ptr(fl), int(nthreads))
        if frame_loss:
            return loss, g_rho, g_u, g_alpha, fl
        return loss, g_rho, g_u, g_alpha

    def loss(self, rho, u, alpha, probe, y, bg=None, nthreads=0):
        return self.loss_grad(rho, u, alpha, probe, y, bg=bg, nthreads=nthreads)[0]

    def illumination(self, probe):
        """sum over frames of |P(r - s_j)|^2 on the object grid (oracle_illumination)."""
        lib = _load()
        out = np.empty(self.shape)
        lib.oracle_illumination(ctypes.byref(self.c), _ptr(_c(probe)), _ptr(out))
        return out

    def project_u(self, u, mask=None):
        """Pi_U of Eq. 10 (see oracle_project_u); returns the projected u."""
        lib = _load()
        u = _d(u)
        out = np.empty_like(u)
        lib.oracle_project_u(ctypes.byref(self.c), _ptr(u), _ptr(None if mask is None else _d(mask)), _ptr(out))
        return out

    def loss_grad_phases(self, rho, phi, alpha, probe, y, bg=None, frames=None, nthreads=0):
        """Per-peak-phase form: phi [D][n1][n2]; returns (loss, g_rho, g_phi, g_alpha)."""
        lib = _load()
        n1, n2 = self.shape
        rho, phi, alpha, probe, y = _d(rho), _d(phi), _d(alpha), _c(probe), _d(y)
        bg = None if bg is None else _d(bg)
        g_rho, g_phi, g_alpha = np.empty((n1, n2)), np.empty((self.npeaks, n1, n2)), np.empty(self.npeaks)
        fr, nfr = _frames(frames)
        loss = lib.oracle_loss_grad_phases(ctypes.byref(self.c), _ptr(rho), _ptr(phi), _ptr(alpha),
                                           _ptr(probe), _ptr(bg), _ptr(y), _iptr(fr), nfr,
                                           _ptr(g_rho), _ptr(g_phi), _ptr(g_alpha), int(nthreads))
        return loss, g_rho, g_phi, g_alpha

    def loss_grad_log(self, chi, u, alpha_t, probe, y, mask=None, bg=None, frames=None, nthreads=0):
        """Eq. 8 variables: rho = mask e^chi, alpha = (1, e^alpha_t[1:]); returns
        (loss, g_chi, g_u, g_alpha_t)."""
        lib = _load()
        n1, n2 = self.shape
        chi, u, alpha_t, probe, y = _d(chi), _d(u), _d(alpha_t), _c(probe), _d(y)
        mask = None if mask is None else _d(mask)
        bg = None if bg is None else _d(bg)
        g_chi, g_u, g_a = np.empty((n1, n2)), np.empty((self.ncomp, n1, n2)), np.empty(self.npeaks)
        fr, nfr = _frames(frames)
        loss = lib.oracle_loss_grad_log(ctypes.byref(self.c), _ptr(chi), _ptr(u), _ptr(alpha_t),
                                        _ptr(mask), _ptr(probe), _ptr(bg), _ptr(y), _iptr(fr), nfr,
                                        _ptr(g_chi), _ptr(g_u), _ptr(g_a), int(nthreads))
        return loss, g_chi, g_u, g_a


class OracleAdam:
    """Alg. 1 without the projector: minibatch Adam in the Eq. 8 variables
    (see oracle_adam_step).  Holds the moments and the step count."""

    def __init__(self, problem, probe, y, mask=None, bg=None, lr_u=0.01, lr_chi=0.1,
                 lr_alpha=0.1, beta1=0.9, beta2=0.999, eps=1e-8, nthreads=0):
        self.p = problem
        self.probe, self.y = _c(probe), _d(y)
        self.mask = None if mask is None else _d(mask)
        self.bg = None if bg is None else _d(bg)
        self.params = AdamParams(lr_u, lr_chi, lr_alpha, beta1, beta2, eps)
        n1, n2 = problem.shape
        self.m_chi, self.v_chi = np.zeros((n1, n2)), np.zeros((n1, n2))
        self.m_u, self.v_u = np.zeros((problem.ncomp, n1, n2)), np.zeros((problem.ncomp, n1, n2))
        self.m_a, self.v_a = np.zeros(problem.npeaks), np.zeros(problem.npeaks)
        self.t = ctypes.c_long(0)
        self.nthreads = nthreads

    def step(self, frames, chi, u, alpha_t):
        """Updates chi, u, alpha_t (float64, in place) from the listed frames;
        returns the minibatch loss before the update."""
        lib = _load()
        for a in (chi, u, alpha_t):
            assert a.dtype == np.float64 and a.flags.c_contiguous
        fr, nfr = _frames(frames)
        return lib.oracle_adam_step(ctypes.byref(self.p.c), _ptr(self.probe), _ptr(self.bg),
                                    _ptr(self.y), _iptr(fr), nfr, _ptr(self.mask),
                                    ctypes.byref(self.params), ctypes.byref(self.t),
                                    _ptr(chi), _ptr(u), _ptr(alpha_t), _ptr(self.m_chi),
                                    _ptr(self.v_chi), _ptr(self.m_u), _ptr(self.v_u),
                                    _ptr(self.m_a), _ptr(self.v_a), int(self.nthreads))


class OracleStepper:
    """Lagged-Armijo gradient descent in FP64 (see oracle_step in mpbp_oracle.c)."""

    def __init__(self, problem, probe, y, bg=None, c_armijo=1e-4, grow=1.25, shrink=0.5,
                 t0=1.0, w_rho=1.0, w_u=1.0, w_alpha=1.0, nthreads=0):
        self.p = problem
        self.probe, self.y = _c(probe), _d(y)
        self.bg = None if bg is None else _d(bg)
        self.params = StepParams(c_armijo, grow, shrink, t0, w_rho, w_u, w_alpha)
        self.state = StepState(0.0, 0.0, t0, 0.0, 0, 0, 0, 0)
        n1, n2 = problem.shape
        self.rho_prev = np.zeros((n1, n2))
        self.u_prev = np.zeros((problem.ncomp, n1, n2))
        self.alpha_prev = np.zeros(problem.npeaks)
        self.grho_prev = np.zeros((n1, n2))
        self.gu_prev = np.zeros((problem.ncomp, n1, n2))
        self.galpha_prev = np.zeros(problem.npeaks)
        self.nthreads = nthreads

    def step(self, rho, u, alpha):
        """Updates rho, u, alpha (float64 arrays) in place; returns the loss evaluated."""
        lib = _load()
        for a in (rho, u, alpha):
            assert a.dtype == np.float64 and a.flags.c_contiguous
        lib.oracle_step(ctypes.byref(self.p.c), _ptr(self.probe), _ptr(self.bg), _ptr(self.y),
                        ctypes.byref(self.params), ctypes.byref(self.state),
                        _ptr(rho), _ptr(u), _ptr(alpha), _ptr(self.rho_prev), _ptr(self.u_prev),
                        _ptr(self.alpha_prev), _ptr(self.grho_prev), _ptr(self.gu_prev),
                        _ptr(self.galpha_prev), int(self.nthreads))
        return self.state.f_last
