"""Python binding of the MPBP C ABI (include/mpbp.h).

Argument marshalling only: every step of the loss and gradient runs in the
CUDA kernels of libmpbp.so.  PyTorch supplies device memory and the current
stream.  There is no CPU fallback: without the library or a GPU every call
raises.
"""
import ctypes
import math
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libmpbp.so")
_lib = None

STATUS = {0: "MPBP_OK", 1: "MPBP_ERR_INVALID_ARG", 2: "MPBP_ERR_UNSUPPORTED", 3: "MPBP_ERR_CUDA",
          4: "MPBP_ERR_NONFINITE", 5: "MPBP_ERR_TIMEOUT", 6: "MPBP_ERR_BOUNDS", 7: "MPBP_ERR_OOM",
          8: "MPBP_ERR_NO_DATA"}


class MPBPError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__("%s%s" % (STATUS.get(status, status), (": " + msg) if msg else ""))


class _Problem(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int32), ("n2", ctypes.c_int32), ("ncomp", ctypes.c_int32),
                ("npeaks", ctypes.c_int32), ("m", ctypes.c_int32), ("nscan", ctypes.c_int32),
                ("G", ctypes.POINTER(ctypes.c_double)), ("scan", ctypes.POINTER(ctypes.c_int32)),
                ("probe_per_peak", ctypes.c_int32), ("phase_scale", ctypes.c_double)]


class StepParams(ctypes.Structure):
    _fields_ = [("c_armijo", ctypes.c_double), ("grow", ctypes.c_double),
                ("shrink", ctypes.c_double), ("t0", ctypes.c_double), ("w_rho", ctypes.c_double),
                ("w_u", ctypes.c_double), ("w_alpha", ctypes.c_double)]


class AdamParams(ctypes.Structure):
    _fields_ = [("lr_u", ctypes.c_double), ("lr_chi", ctypes.c_double),
                ("lr_alpha", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("eps", ctypes.c_double)]


class AdamState(ctypes.Structure):
    _fields_ = [("lr_u", ctypes.c_double), ("lr_chi", ctypes.c_double),
                ("lr_alpha", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("f_last", ctypes.c_double), ("bc1", ctypes.c_double),
                ("bc2", ctypes.c_double), ("t", ctypes.c_int64)]


class StepState(ctypes.Structure):
    _fields_ = [("f_prev", ctypes.c_double), ("gn2_prev", ctypes.c_double),
                ("t", ctypes.c_double), ("f_last", ctypes.c_double), ("k", ctypes.c_int32),
                ("accepted", ctypes.c_int32), ("n_accept", ctypes.c_int32),
                ("n_reject", ctypes.c_int32), ("c_armijo", ctypes.c_double),
                ("grow", ctypes.c_double), ("shrink", ctypes.c_double), ("w_rho", ctypes.c_double),
                ("w_u", ctypes.c_double), ("w_alpha", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("workspace_bytes", ctypes.c_int64), ("frames_grid", ctypes.c_int32),
                ("frames_block", ctypes.c_int32), ("frames_smem", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("num_sms", ctypes.c_int32),
                ("launches_loss_grad", ctypes.c_int32), ("launches_step", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("tile_copies", ctypes.c_int32),
                ("fft_schedule", ctypes.c_int32),
                ("deterministic", ctypes.c_int32)]


EXPORTS = ["mpbp_status_string", "mpbp_create", "mpbp_destroy", "mpbp_last_error",
           "mpbp_get_info", "mpbp_set_probe", "mpbp_set_data", "mpbp_object_build",
           "mpbp_forward", "mpbp_loss_grad", "mpbp_loss_grad_host", "mpbp_step_init",
           "mpbp_step", "mpbp_loss_grad_batched", "mpbp_set_schedule", "mpbp_sync_status",
           "mpbp_frames_timing", "mpbp_frames_timing_read", "mpbp_loss_grad_noalloc",
           "mpbp_set_batch_schedule", "mpbp_autotune", "mpbp_autotune_batched",
           "mpbp_set_precision", "mpbp_step_capture", "mpbp_step_replay",
           "mpbp_adam_init", "mpbp_adam_step", "mpbp_adam_get_state", "mpbp_adam_set_state",
           "mpbp_loss_grad_phases", "mpbp_unwrap_phases", "mpbp_project_displacement",
           "mpbp_illumination", "mpbp_set_test_stall", "mpbp_loss_grad_host_counts16",
           "mpbp_set_scan_offsets", "mpbp_shift_probe", "mpbp_loss", "mpbp_set_fft_schedule",
           "mpbp_set_deterministic"]

FFT_SHUFFLE = 0           # M = 128: radix-2 stages across threads by warp shuffles
FFT_EXCHANGE = 1          # M = 128: three register layouts joined by shared-memory exchanges
PRECISION_FP32 = 0        # FFTs on the CUDA cores
PRECISION_TC_SPLIT16 = 1  # dense DFT matrices on the tensor cores, split FP16


def library_path():
    return _LIB_PATH


def load(build_if_missing=True):
    """Loads libmpbp.so (building it with nvcc first if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        if not build_if_missing:
            raise MPBPError(3, "libmpbp.so is not built")
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(_LIB_PATH)
    V, I32, D, P = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.POINTER
    st = ctypes.c_int
    lib.mpbp_status_string.argtypes = [st]
    lib.mpbp_status_string.restype = ctypes.c_char_p
    lib.mpbp_create.argtypes = [P(_Problem), P(V)]
    lib.mpbp_create.restype = st
    lib.mpbp_destroy.argtypes = [V]
    lib.mpbp_destroy.restype = None
    lib.mpbp_last_error.argtypes = [V]
    lib.mpbp_last_error.restype = ctypes.c_char_p
    lib.mpbp_get_info.argtypes = [V, P(Info)]
    lib.mpbp_get_info.restype = st
    lib.mpbp_set_probe.argtypes = [V, V, V]
    lib.mpbp_set_probe.restype = st
    lib.mpbp_set_data.argtypes = [V, V, V, V]
    lib.mpbp_set_data.restype = st
    lib.mpbp_object_build.argtypes = [V, V, V, V, V, V]
    lib.mpbp_object_build.restype = st
    lib.mpbp_forward.argtypes = [V, V, V, V, V, V]
    lib.mpbp_forward.restype = st
    lib.mpbp_loss_grad.argtypes = [V, V, V, V, V, I32, V, V, V, V, V]
    lib.mpbp_loss_grad.restype = st
    lib.mpbp_loss.argtypes = [V, V, V, V, V, I32, V, V]
    lib.mpbp_loss.restype = st
    lib.mpbp_loss_grad_host.argtypes = [V, V, V, V, V, V, V, V, V, V]
    lib.mpbp_loss_grad_host.restype = st
    lib.mpbp_loss_grad_host_counts16.argtypes = [V, V, V, V, V, V, V, V, V, V]
    lib.mpbp_loss_grad_host_counts16.restype = st
    lib.mpbp_step_init.argtypes = [V, P(StepParams), V, V]
    lib.mpbp_step_init.restype = st
    lib.mpbp_step.argtypes = [V, V, V, V, V, V]
    lib.mpbp_step.restype = st
    lib.mpbp_loss_grad_batched.argtypes = [I32, V, V, V, V, V, V, V, V, V]
    lib.mpbp_loss_grad_batched.restype = st
    lib.mpbp_set_schedule.argtypes = [V, I32]
    lib.mpbp_set_schedule.restype = st
    lib.mpbp_set_fft_schedule.argtypes = [V, I32]
    lib.mpbp_set_fft_schedule.restype = st
    lib.mpbp_set_deterministic.argtypes = [V, I32]
    lib.mpbp_set_deterministic.restype = st
    lib.mpbp_set_precision.argtypes = [V, I32]
    lib.mpbp_set_precision.restype = st
    lib.mpbp_adam_init.argtypes = [V, P(AdamParams), V, V]
    lib.mpbp_adam_init.restype = st
    lib.mpbp_adam_step.argtypes = [V, V, I32, V, V, V, V, V, V]
    lib.mpbp_adam_step.restype = st
    lib.mpbp_adam_get_state.argtypes = [V, V, V, V, V, V, V, V]
    lib.mpbp_adam_get_state.restype = st
    lib.mpbp_adam_set_state.argtypes = [V, V, V, V, V, V, V, V]
    lib.mpbp_adam_set_state.restype = st
    lib.mpbp_loss_grad_phases.argtypes = [V, V, V, V, V, I32, V, V, V, V, V]
    lib.mpbp_loss_grad_phases.restype = st
    lib.mpbp_illumination.argtypes = [V, V, V]
    lib.mpbp_illumination.restype = st
    lib.mpbp_unwrap_phases.argtypes = [V, V, V, V, V]
    lib.mpbp_unwrap_phases.restype = st
    lib.mpbp_project_displacement.argtypes = [V, V, V, V]
    lib.mpbp_project_displacement.restype = st
    lib.mpbp_step_capture.argtypes = [V, V, V, V, V]
    lib.mpbp_step_capture.restype = st
    lib.mpbp_step_replay.argtypes = [V, V]
    lib.mpbp_step_replay.restype = st
    lib.mpbp_set_batch_schedule.argtypes = [V, I32, I32]
    lib.mpbp_set_batch_schedule.restype = st
    lib.mpbp_autotune.argtypes = [V, V, V, V, V, V, V, ctypes.c_char_p, V]
    lib.mpbp_autotune.restype = st
    lib.mpbp_autotune_batched.argtypes = [I32, V, V, V, V, V, V, V, ctypes.c_char_p, V]
    lib.mpbp_autotune_batched.restype = st
    lib.mpbp_sync_status.argtypes = [V, V]
    lib.mpbp_sync_status.restype = st
    lib.mpbp_frames_timing.argtypes = [V, I32]
    lib.mpbp_frames_timing.restype = st
    lib.mpbp_set_test_stall.argtypes = [V, I32]
    lib.mpbp_set_test_stall.restype = st
    lib.mpbp_frames_timing_read.argtypes = [V, P(D), P(I32)]
    lib.mpbp_frames_timing_read.restype = st
    lib.mpbp_loss_grad_noalloc.argtypes = [P(_Problem), V, V, V, V, V, V, V, V, V, V, V]
    lib.mpbp_loss_grad_noalloc.restype = st
    lib.mpbp_set_scan_offsets.argtypes = [V, V, V]
    lib.mpbp_set_scan_offsets.restype = st
    lib.mpbp_shift_probe.argtypes = [V, I32, V, I32, V, V]
    lib.mpbp_shift_probe.restype = st
    _lib = lib
    return lib


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _p(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _dev(t, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


def _host(t, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("%s must be a CPU tensor" % name)
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError("%s must be a contiguous %s tensor of shape %s" % (name, dtype, tuple(shape)))
    return t


class Problem:
    """One MPBP problem on the current CUDA device (wraps an mpbp_ctx)."""

    def __init__(self, n1, n2, ncomp, npeaks, m, scan, G, phase_scale=2 * math.pi,
                 probe_per_peak=False):
        self._lib = load()
        self.n1, self.n2, self.ncomp, self.npeaks, self.m = int(n1), int(n2), int(ncomp), int(npeaks), int(m)
        self._scan = np.ascontiguousarray(scan, dtype=np.int32).reshape(-1, 2)
        self._G = np.ascontiguousarray(G, dtype=np.float64).reshape(self.npeaks, self.ncomp)
        self.nscan = self._scan.shape[0]
        self.phase_scale = float(phase_scale)
        self.probe_per_peak = bool(probe_per_peak)
        pr = _Problem(self.n1, self.n2, self.ncomp, self.npeaks, self.m, self.nscan,
                      self._G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      self._scan.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                      int(self.probe_per_peak), self.phase_scale)
        h = ctypes.c_void_p()
        s = self._lib.mpbp_create(ctypes.byref(pr), ctypes.byref(h))
        if s != 0:
            raise MPBPError(s, "mpbp_create")
        self._h = h
        self.device = torch.cuda.current_device()

    @classmethod
    def from_spec(cls, spec, scan):
        return cls(spec.n1, spec.n2, spec.ncomp, spec.npeaks, spec.m, scan, spec.G,
                   spec.phase_scale, spec.probe_per_peak)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mpbp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # shapes
    @property
    def nframes(self):
        return self.npeaks * self.nscan

    @property
    def shapes(self):
        return {"rho": (self.n1, self.n2), "u": (self.ncomp, self.n1, self.n2),
                "alpha": (self.npeaks,), "frames": (self.npeaks, self.nscan, self.m, self.m)}

    def _check(self, s, what):
        if s != 0:
            raise MPBPError(s, "%s: %s" % (what, self._lib.mpbp_last_error(self._h).decode()))

    def _state(self, rho, u, alpha):
        sh = self.shapes
        _dev(rho, torch.float32, sh["rho"], "rho")
        _dev(u, torch.float32, sh["u"], "u")
        _dev(alpha, torch.float32, sh["alpha"], "alpha")

    def info(self):
        inf = Info()
        self._check(self._lib.mpbp_get_info(self._h, ctypes.byref(inf)), "mpbp_get_info")
        return {k: getattr(inf, k) for k, _ in Info._fields_}

    def set_precision(self, mode):
        """DFT arithmetic of the gradient evaluations: PRECISION_FP32 (FFTs) or
        PRECISION_TC_SPLIT16 (tensor cores, frame sides 32, 64 and 128)."""
        self._check(self._lib.mpbp_set_precision(self._h, int(mode)), "mpbp_set_precision")

    def set_fft_schedule(self, schedule):
        """FFT schedule of the M = 128 gradient kernel: FFT_SHUFFLE or FFT_EXCHANGE."""
        self._check(self._lib.mpbp_set_fft_schedule(self._h, int(schedule)), "mpbp_set_fft_schedule")

    def set_deterministic(self, on=True):
        """Bitwise-reproducible gradient sums (mpbp_set_deterministic; frame
        sides 64 and 128, every frame of the context per evaluation)."""
        self._check(self._lib.mpbp_set_deterministic(self._h, 1 if on else 0), "mpbp_set_deterministic")

    def set_schedule(self, blocks_per_sm):
        self._check(self._lib.mpbp_set_schedule(self._h, int(blocks_per_sm)), "mpbp_set_schedule")

    def autotune(self, rho, u, alpha, cache_path=None):
        """Pick the fastest frame-kernel schedule on this data (mpbp_autotune)."""
        self._state(rho, u, alpha)
        loss, g_rho, g_u, _ = self.loss_grad(rho, u, alpha)
        cp = None if cache_path is None else os.fsencode(cache_path)
        self._check(self._lib.mpbp_autotune(self._h, _p(rho), _p(u), _p(alpha), _p(loss), _p(g_rho),
                                            _p(g_u), cp, _stream()), "mpbp_autotune")
        return self.info()["blocks_per_sm"]

    def set_batch_schedule(self, mode, order=0):
        """Schedule of batched calls led by this problem (see mpbp_set_batch_schedule)."""
        self._check(self._lib.mpbp_set_batch_schedule(self._h, int(mode), int(order)),
                    "mpbp_set_batch_schedule")

    def set_probe(self, probe):
        shape = (self.npeaks, self.m, self.m) if self.probe_per_peak else (self.m, self.m)
        _dev(probe, torch.complex64, shape, "probe")
        self._probe = probe
        self._check(self._lib.mpbp_set_probe(self._h, _p(probe), _stream()), "mpbp_set_probe")

    def set_scan_offsets(self, d):
        """Scan positions off the pixel grid: d [J][2] (row, column) offsets in
        [-1/2, 1/2] added to the integer scan (mpbp_set_scan_offsets), or None."""
        if d is None:
            self._check(self._lib.mpbp_set_scan_offsets(self._h, None, _stream()), "mpbp_set_scan_offsets")
            return
        d = np.ascontiguousarray(d, dtype=np.float64)
        if d.shape != (self.nscan, 2):
            raise MPBPError(1, "scan offsets: expected shape (%d, 2), got %s" % (self.nscan, d.shape))
        self._offsets = d
        self._check(self._lib.mpbp_set_scan_offsets(self._h, d.ctypes.data, _stream()),
                    "mpbp_set_scan_offsets")

    def set_data(self, y, bg=None):
        _dev(y, torch.float32, self.shapes["frames"], "y")
        if bg is not None:
            _dev(bg, torch.float32, self.shapes["frames"], "bg")
        self._check(self._lib.mpbp_set_data(self._h, _p(y), _p(bg), _stream()), "mpbp_set_data")

    def object_build(self, rho, u, alpha, out=None):
        self._state(rho, u, alpha)
        if out is None:
            out = torch.empty((self.npeaks, self.n1, self.n2), dtype=torch.complex64, device=rho.device)
        self._check(self._lib.mpbp_object_build(self._h, _p(rho), _p(u), _p(alpha), _p(out),
                                                _stream()), "mpbp_object_build")
        return out

    def forward(self, rho, u, alpha, out=None):
        self._state(rho, u, alpha)
        if out is None:
            out = torch.empty(self.shapes["frames"], dtype=torch.float32, device=rho.device)
        self._check(self._lib.mpbp_forward(self._h, _p(rho), _p(u), _p(alpha), _p(out), _stream()),
                    "mpbp_forward")
        return out

    def loss_grad(self, rho, u, alpha, frames=None, out=None):
        """Returns (loss [1] float64, g_rho, g_u, g_alpha [D] float64), all on the device."""
        self._state(rho, u, alpha)
        dev = rho.device
        if out is None:
            out = (torch.empty(1, dtype=torch.float64, device=dev),
                   torch.empty(self.shapes["rho"], dtype=torch.float32, device=dev),
                   torch.empty(self.shapes["u"], dtype=torch.float32, device=dev),
                   torch.empty(self.npeaks, dtype=torch.float64, device=dev))
        loss, g_rho, g_u, g_alpha = out
        nfr = 0
        if frames is not None:
            if not (frames.is_cuda and frames.dtype == torch.int32 and frames.dim() == 1
                    and frames.is_contiguous()):
                raise TypeError("frames must be a contiguous int32 CUDA vector")
            nfr = frames.numel()
            if nfr == 0:
                # an empty list still needs a non-null pointer (NULL means all frames)
                frames = torch.zeros(1, dtype=torch.int32, device=dev)
        self._check(self._lib.mpbp_loss_grad(self._h, _p(rho), _p(u), _p(alpha), _p(frames), nfr,
                                             _p(loss), _p(g_rho), _p(g_u), _p(g_alpha), _stream()),
                    "mpbp_loss_grad")
        return loss, g_rho, g_u, g_alpha

    def loss(self, rho, u, alpha, frames=None, out=None):
        """Eq. 4 alone (mpbp_loss): returns loss [1] float64 on the device."""
        self._state(rho, u, alpha)
        if out is None:
            out = torch.empty(1, dtype=torch.float64, device=rho.device)
        frames, nfr = self._frames_arg(frames, rho.device)
        self._check(self._lib.mpbp_loss(self._h, _p(rho), _p(u), _p(alpha), _p(frames), nfr, _p(out),
                                        _stream()), "mpbp_loss")
        return out

    def _frames_arg(self, frames, dev):
        nfr = 0
        if frames is not None:
            if not (frames.is_cuda and frames.dtype == torch.int32 and frames.dim() == 1
                    and frames.is_contiguous()):
                raise TypeError("frames must be a contiguous int32 CUDA vector")
            nfr = frames.numel()
            if nfr == 0:
                frames = torch.zeros(1, dtype=torch.int32, device=dev)
        return frames, nfr

    def loss_grad_phases(self, rho, phi, alpha, frames=None):
        """Per-peak-phase form: phi [D][n1][n2] in place of u; returns
        (loss [1] float64, g_rho, g_phi [D][n1][n2], g_alpha [D] float64)."""
        sh = self.shapes
        _dev(rho, torch.float32, sh["rho"], "rho")
        _dev(phi, torch.float32, (self.npeaks,) + tuple(sh["rho"]), "phi")
        _dev(alpha, torch.float32, sh["alpha"], "alpha")
        dev = rho.device
        loss = torch.empty(1, dtype=torch.float64, device=dev)
        g_rho = torch.empty(sh["rho"], dtype=torch.float32, device=dev)
        g_phi = torch.empty_like(phi)
        g_alpha = torch.empty(self.npeaks, dtype=torch.float64, device=dev)
        frames, nfr = self._frames_arg(frames, dev)
        self._check(self._lib.mpbp_loss_grad_phases(self._h, _p(rho), _p(phi), _p(alpha), _p(frames),
                                                    nfr, _p(loss), _p(g_rho), _p(g_phi), _p(g_alpha),
                                                    _stream()), "mpbp_loss_grad_phases")
        return loss, g_rho, g_phi, g_alpha

    def illumination(self):
        """sum over frames of |P_m(r - s_j)|^2 on the object grid (mpbp_illumination)."""
        out = torch.empty(self.shapes["rho"], dtype=torch.float32, device="cuda")
        self._check(self._lib.mpbp_illumination(self._h, _p(out), _stream()), "mpbp_illumination")
        return out

    def unwrap_phases(self, wrapped, mask=None, out=None):
        """2-D unwrapping of D phase maps [D][n1][n2] (mpbp_unwrap_phases)."""
        shp = (self.npeaks,) + tuple(self.shapes["rho"])
        _dev(wrapped, torch.float32, shp, "wrapped")
        if mask is not None:
            _dev(mask, torch.float32, self.shapes["rho"], "mask")
        if out is None:
            out = torch.empty_like(wrapped)
        self._check(self._lib.mpbp_unwrap_phases(self._h, _p(wrapped), _p(mask), _p(out), _stream()),
                    "mpbp_unwrap_phases")
        return out

    def project_displacement(self, u, mask=None):
        """Pi_U of Eq. 10 on u, in place (mpbp_project_displacement)."""
        _dev(u, torch.float32, self.shapes["u"], "u")
        if mask is not None:
            _dev(mask, torch.float32, self.shapes["rho"], "mask")
        self._check(self._lib.mpbp_project_displacement(self._h, _p(u), _p(mask), _stream()),
                    "mpbp_project_displacement")
        return u

    def adam_init(self, lr_u=0.01, lr_chi=0.1, lr_alpha=0.1, beta1=0.9, beta2=0.999, eps=1e-8,
                  state=None):
        """Alg. 1's Adam (mpbp_adam_init); returns the device state buffer."""
        prm = AdamParams(lr_u, lr_chi, lr_alpha, beta1, beta2, eps)
        if state is None:
            state = torch.zeros(ctypes.sizeof(AdamState), dtype=torch.uint8, device="cuda")
        self._check(self._lib.mpbp_adam_init(self._h, ctypes.byref(prm), _p(state), _stream()),
                    "mpbp_adam_init")
        return state

    def adam_step(self, frames, chi, u, alpha_t, state, mask=None):
        """One minibatch iteration of Alg. 1 on chi, u, alpha_t (updated in place)."""
        sh = self.shapes
        _dev(chi, torch.float32, sh["rho"], "chi")
        _dev(u, torch.float32, sh["u"], "u")
        _dev(alpha_t, torch.float32, sh["alpha"], "alpha_t")
        if mask is not None:
            _dev(mask, torch.float32, sh["rho"], "mask")
        frames, nfr = self._frames_arg(frames, chi.device)
        self._check(self._lib.mpbp_adam_step(self._h, _p(frames), nfr, _p(chi), _p(u), _p(alpha_t),
                                              _p(mask), _p(state), _stream()), "mpbp_adam_step")

    def adam_get_state(self):
        """(m_chi, v_chi, m_u, v_u, m_alpha, v_alpha) device copies of the moments."""
        sh, dev = self.shapes, "cuda"
        out = (torch.empty(sh["rho"], device=dev), torch.empty(sh["rho"], device=dev),
               torch.empty(sh["u"], device=dev), torch.empty(sh["u"], device=dev),
               torch.empty(self.npeaks, dtype=torch.float64, device=dev),
               torch.empty(self.npeaks, dtype=torch.float64, device=dev))
        self._check(self._lib.mpbp_adam_get_state(self._h, *[_p(t) for t in out], _stream()),
                    "mpbp_adam_get_state")
        return out

    def adam_set_state(self, moments):
        """Loads moments shaped as adam_get_state's (device tensors)."""
        ms = [t.contiguous() for t in moments]
        self._check(self._lib.mpbp_adam_set_state(self._h, *[_p(t) for t in ms], _stream()),
                    "mpbp_adam_set_state")

    @staticmethod
    def read_adam_state(state):
        return AdamState.from_buffer_copy(state.cpu().numpy().tobytes())

    def loss_grad_host(self, rho, u, alpha, y=None, out=None):
        """Host-buffer variant (copies in, evaluates, copies out, synchronises).
        y: float32 counts, or uint16 photon counts (mpbp_loss_grad_host_counts16)."""
        sh = self.shapes
        _host(rho, torch.float32, sh["rho"], "rho")
        _host(u, torch.float32, sh["u"], "u")
        _host(alpha, torch.float32, sh["alpha"], "alpha")
        counts16 = y is not None and y.dtype == torch.uint16
        if y is not None:
            _host(y, torch.uint16 if counts16 else torch.float32, sh["frames"], "y")
        if out is None:
            out = (torch.empty(1, dtype=torch.float64), torch.empty(sh["rho"], dtype=torch.float32),
                   torch.empty(sh["u"], dtype=torch.float32), torch.empty(self.npeaks, dtype=torch.float64))
        loss, g_rho, g_u, g_alpha = out
        fn = self._lib.mpbp_loss_grad_host_counts16 if counts16 else self._lib.mpbp_loss_grad_host
        self._check(fn(self._h, _p(y), _p(rho), _p(u), _p(alpha), _p(loss), _p(g_rho), _p(g_u), _p(g_alpha),
                       _stream()), "mpbp_loss_grad_host")
        return loss, g_rho, g_u, g_alpha

    def step_init(self, t0, c_armijo=1e-4, grow=1.25, shrink=0.5, w_rho=1.0, w_u=1.0, w_alpha=1.0,
                  state=None):
        prm = StepParams(c_armijo, grow, shrink, t0, w_rho, w_u, w_alpha)
        if state is None:
            state = torch.zeros(ctypes.sizeof(StepState), dtype=torch.uint8, device="cuda")
        self._check(self._lib.mpbp_step_init(self._h, ctypes.byref(prm), _p(state), _stream()),
                    "mpbp_step_init")
        return state

    def step(self, rho, u, alpha, state):
        self._state(rho, u, alpha)
        self._check(self._lib.mpbp_step(self._h, _p(rho), _p(u), _p(alpha), _p(state), _stream()),
                    "mpbp_step")

    def step_capture(self, rho, u, alpha, state):
        """Records one step on these tensors as a CUDA graph (mpbp_step_capture)."""
        self._state(rho, u, alpha)
        self._check(self._lib.mpbp_step_capture(self._h, _p(rho), _p(u), _p(alpha), _p(state)),
                    "mpbp_step_capture")
        self._captured = (rho, u, alpha, state)   # keep the baked-in buffers alive

    def step_replay(self):
        """Launches the captured step on the current stream (mpbp_step_replay)."""
        self._check(self._lib.mpbp_step_replay(self._h, _stream()), "mpbp_step_replay")

    @staticmethod
    def read_state(state):
        raw = state.cpu().numpy().tobytes()
        return StepState.from_buffer_copy(raw)

    def set_test_stall(self, on=True):
        """Test hook: the tile-copy waits of the frame kernels run out (MPBP_ERR_TIMEOUT)."""
        self._check(self._lib.mpbp_set_test_stall(self._h, int(bool(on))), "mpbp_set_test_stall")

    def frames_timing(self, enable=True):
        self._check(self._lib.mpbp_frames_timing(self._h, int(bool(enable))), "mpbp_frames_timing")

    def frames_timing_read(self):
        """(total milliseconds, launches) of the fused frame kernel since the last read."""
        ms, n = ctypes.c_double(), ctypes.c_int32()
        self._check(self._lib.mpbp_frames_timing_read(self._h, ctypes.byref(ms), ctypes.byref(n)),
                    "mpbp_frames_timing_read")
        return ms.value, n.value

    def sync_status(self):
        s = self._lib.mpbp_sync_status(self._h, _stream())
        if s != 0:
            raise MPBPError(s, self._lib.mpbp_last_error(self._h).decode())


def shift_probe(probe, d):
    """P(k - d_i) for one probe (cuda complex64 [M][M]) and offsets d [n][2]
    in [-1/2, 1/2] (mpbp_shift_probe); returns cuda complex64 [n][M][M]."""
    lib = load()
    m = probe.shape[0]
    _dev(probe, torch.complex64, (m, m), "probe")
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 2)
    out = torch.empty((d.shape[0], m, m), dtype=torch.complex64, device=probe.device)
    s = lib.mpbp_shift_probe(_p(probe), m, d.ctypes.data, d.shape[0], _p(out), _stream())
    if s != 0:
        raise MPBPError(s, "mpbp_shift_probe")
    return out


def loss_grad_batched(problems, states, outs=None):
    """Loss and gradient of several problems in one call.  states: list of
    (rho, u, alpha) device tensors; returns a list of (loss, g_rho, g_u, g_alpha)."""
    lib = load()
    n = len(problems)
    if outs is None:
        outs = []
        for p, (rho, u, alpha) in zip(problems, states):
            dev = rho.device
            outs.append((torch.empty(1, dtype=torch.float64, device=dev),
                         torch.empty(p.shapes["rho"], dtype=torch.float32, device=dev),
                         torch.empty(p.shapes["u"], dtype=torch.float32, device=dev),
                         torch.empty(p.npeaks, dtype=torch.float64, device=dev)))
    for p, (rho, u, alpha) in zip(problems, states):
        p._state(rho, u, alpha)
    arr = lambda xs: (ctypes.c_void_p * n)(*[x.data_ptr() if isinstance(x, torch.Tensor) else x for x in xs])
    ctxs = (ctypes.c_void_p * n)(*[p._h.value for p in problems])
    s = lib.mpbp_loss_grad_batched(n, ctxs, arr([s[0] for s in states]), arr([s[1] for s in states]),
                                   arr([s[2] for s in states]), arr([o[0] for o in outs]),
                                   arr([o[1] for o in outs]), arr([o[2] for o in outs]),
                                   arr([o[3] for o in outs]), _stream())
    if s != 0:
        raise MPBPError(s, "mpbp_loss_grad_batched")
    return outs


DEVERR_BOUNDS, DEVERR_NONFINITE, DEVERR_TIMEOUT = 1, 2, 4   # device error bits (MPBP_DEVERR_*)


def loss_grad_noalloc(spec_problem, probe, y, rho, u, alpha, out, dev_err=None):
    """mpbp_loss_grad_noalloc: the loss and gradient computed in the library's
    fixed device scratch array, for callers that cannot allocate device
    memory.  `spec_problem` is a Problem (only its geometry is used); every
    tensor, including the outputs in `out` = (loss [1] float64, g_rho, g_u,
    g_alpha [D] float64) and the optional error word `dev_err` ([1] int32,
    read it with noalloc_check), must already be on the current device.
    Shapes, dtypes, contiguity and the device are checked here, so that no
    wrong pointer reaches the kernels."""
    lib = load()
    p = spec_problem
    sh = p.shapes
    dev = torch.cuda.current_device()
    probe_shape = (p.npeaks, p.m, p.m) if p.probe_per_peak else (p.m, p.m)
    loss, g_rho, g_u, g_alpha = out
    checks = [(probe, torch.complex64, probe_shape, "probe"), (y, torch.float32, sh["frames"], "y"),
              (rho, torch.float32, sh["rho"], "rho"), (u, torch.float32, sh["u"], "u"),
              (alpha, torch.float32, sh["alpha"], "alpha"), (loss, torch.float64, (1,), "loss"),
              (g_rho, torch.float32, sh["rho"], "g_rho"), (g_u, torch.float32, sh["u"], "g_u")]
    if g_alpha is not None:
        checks.append((g_alpha, torch.float64, (p.npeaks,), "g_alpha"))
    if dev_err is not None:
        checks.append((dev_err, torch.int32, (1,), "dev_err"))
    for t, dtype, shape, name in checks:
        _dev(t, dtype, shape, name)
        if t.device.index != dev:
            raise ValueError("%s is on cuda:%d, the current device is cuda:%d" % (name, t.device.index, dev))
    pr = _Problem(p.n1, p.n2, p.ncomp, p.npeaks, p.m, p.nscan,
                  p._G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                  p._scan.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                  int(p.probe_per_peak), p.phase_scale)
    s = lib.mpbp_loss_grad_noalloc(ctypes.byref(pr), _p(probe), _p(y), _p(rho), _p(u), _p(alpha),
                                   _p(loss), _p(g_rho), _p(g_u), _p(g_alpha), _p(dev_err), _stream())
    if s != 0:
        raise MPBPError(s, "mpbp_loss_grad_noalloc")
    return out


def noalloc_check(dev_err):
    """Waits for the current stream, then raises MPBPError for the device
    error bits a loss_grad_noalloc call left in `dev_err` (no-op if 0)."""
    torch.cuda.current_stream().synchronize()
    bits = int(dev_err.item())
    if bits & DEVERR_TIMEOUT:
        raise MPBPError(5, "a bounded wait on the GPU ran out")
    if bits & DEVERR_BOUNDS:
        raise MPBPError(6, "a frame index out of range")
    if bits & DEVERR_NONFINITE:
        raise MPBPError(4, "the loss is not finite")


def autotune_batched(problems, states, cache_path=None):
    """Pick the fastest schedule for loss_grad_batched on these problems."""
    lib = load()
    n = len(problems)
    outs = loss_grad_batched(problems, states)
    arr = lambda xs: (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    ctxs = (ctypes.c_void_p * n)(*[p._h.value for p in problems])
    cp = None if cache_path is None else os.fsencode(cache_path)
    s = lib.mpbp_autotune_batched(n, ctxs, arr([s[0] for s in states]), arr([s[1] for s in states]),
                                  arr([s[2] for s in states]), arr([o[0] for o in outs]),
                                  arr([o[1] for o in outs]), arr([o[2] for o in outs]), cp, _stream())
    if s != 0:
        raise MPBPError(s, "mpbp_autotune_batched")


class MPBPLoss(torch.autograd.Function):
    """f(rho, u, alpha) of Eq. 4 with the hand-written adjoint as its backward.

    Default: forward runs the fused loss+gradient pass once and keeps only
    the object-sized gradients; backward scales them by the incoming
    gradient.  recompute=True: forward runs the loss alone (no adjoint, no
    scatter) and keeps only the inputs; backward reruns the fused pass, which
    recomputes the exit waves and far fields on chip.  Exit waves are never
    stored either way."""

    @staticmethod
    def forward(ctx, rho, u, alpha, problem, recompute=False):
        x = (rho.detach().contiguous(), u.detach().contiguous(), alpha.detach().contiguous())
        ctx.problem = problem
        ctx.recompute = bool(recompute)
        if recompute:
            loss = problem.loss(*x)
            ctx.save_for_backward(*x)
        else:
            loss, g_rho, g_u, g_alpha = problem.loss_grad(*x)
            ctx.save_for_backward(g_rho, g_u, g_alpha)
        return loss[0]

    @staticmethod
    def backward(ctx, grad_out):
        if ctx.recompute:
            _, g_rho, g_u, g_alpha = ctx.problem.loss_grad(*ctx.saved_tensors)
        else:
            g_rho, g_u, g_alpha = ctx.saved_tensors
        go = grad_out.to(torch.float32)
        return go * g_rho, go * g_u, (grad_out * g_alpha).to(torch.float32), None, None


def mpbp_loss(rho, u, alpha, problem, recompute=False):
    return MPBPLoss.apply(rho, u, alpha, problem, recompute)
