"""Throughput of the MPBP loss+gradient hot path on GB300.

One step = one optimizer iteration of the whole hot path on the 1024x1024-
object, 6-peak, 121x121-scan, 128x128-frame problem (87,846 frames, 5.76 GB of
amplitudes): object synthesis, the fused per-frame kernel (patch gather,
probe, 2-D FFT, amplitude residual, adjoint FFT, scatter-add), gradient
assembly, FP64 reductions, the lagged Armijo decision and the update.  The
metric is frames per second.  The 256x256, 64x64-frame problem's numbers
(both precision modes, the paper's minibatch Adam iteration) are reported
beside it under "workload_256".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  N > 1 (under torchrun) runs independent replicas of the
problem, one per rank (weak scaling; the problem has no data-path exchange
between replicas).  `--impl reference` times the FP64 CPU oracle on the host
cores on the same workload instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2312_14907_gb300 import synth  # noqa: E402

HEADLINE = 5          # the 1024^2, M = 128, 6-peak, 121x121-scan problem
SECONDARY = 2         # the 256^2, M = 64, 3-peak, 31x31-scan problem
METRIC = "frames/s for MPBP loss+gradient (fwd+adjoint), % of HBM roofline, 1 GB300"
UNIT = "frames/s"


def flops_per_frame(m):
    """Algorithmic FP32 flops of one frame: two unnormalised 2-D FFTs counted
    as 5 n log2 n with n = M^2, plus 24 flops per pixel of pointwise work
    (probe product 6, residual and loss 10, adjoint probe product 6, the
    accumulate 2)."""
    n = m * m
    return 2 * 5 * n * math.log2(n) + 24 * n


def hbm_bytes_per_frame(spec):
    """Algorithmic DRAM bytes per frame: the FP32 amplitude stream (4 M^2) plus
    the object-sized reads and writes amortised over the frames of one step
    (rho and u read, their gradients written: 2 (1 + C) 4 N^2 / (J D))."""
    return 4 * spec.m ** 2 + 2 * (1 + spec.ncomp) * 4 * spec.n1 * spec.n2 / spec.nframes


def peaks(num_sms=152):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    out = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback", "sm_max_mhz": 2070.0}
    try:
        with open(path) as f:
            d = json.load(f)
        out.update({"hbm_gbs": float(d["hbm_gbs"]), "src": "measured",
                    "bf16_tflops": float(d.get("bf16_tflops", 1900.0)),
                    "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0))})
    except Exception:
        pass
    # plain FP32 pipe: SMs x 128 lanes x 2 flops (FMA) x max SM clock
    out["fp32_tflops"] = num_sms * 128 * 2 * out["sm_max_mhz"] * 1e6 / 1e12
    return out


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs(spec, scan, prob, torch):
    """Synthetic data of the problem on the device: the true object, a unit
    probe, the CUDA forward model for the intensities, the photon scaling
    (the brightest frame holds `spec.photons` expected counts) and Poisson
    counts drawn on the device by a seeded generator.  Returns the scaled
    probe (host complex64) and the counts (device float32)."""
    P = synth.probe(spec).astype(np.complex64)
    rho_t, u_t = synth.truth(spec)
    xt = [torch.from_numpy(a.astype(np.float32)).cuda() for a in (rho_t, u_t, synth.alpha_truth(spec))]
    prob.set_probe(torch.from_numpy(P).cuda())
    I = prob.forward(*xt)
    tot = I.reshape(spec.nframes, -1).sum(dim=1, dtype=torch.float64).max().item()
    scale = float(spec.photons / tot) if tot > 0 else 1.0
    probe = (P * np.sqrt(scale)).astype(np.complex64)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(spec.seed + 1000)
    I.mul_(scale)
    y = torch.poisson(I, generator=gen)
    del I
    return probe, y


def torch_loss_grad(torch, rho, u, alpha, probe, amp, scan, G, phase_scale, m):
    """The same loss and gradient written as plain per-kernel PyTorch ops in
    FP32 / complex64 -- object synthesis, patch gather with zero padding,
    probe product, torch.fft.fft2, amplitude residual and loss, the gradient
    by autograd: the unfused comparison path (not used by the library).
    amp: sqrt(y) [D][J][M][M]; probe [M][M] or [D][M][M]."""
    rho = rho.detach().clone().requires_grad_(True)
    u = u.detach().clone().requires_grad_(True)
    alpha = alpha.detach().clone().requires_grad_(True)
    phi = phase_scale * torch.einsum("mc,cij->mij", G, u)
    O = (alpha[:, None, None] * rho[None]) * torch.polar(torch.ones_like(phi), phi)
    D, n1, n2 = O.shape
    Op = O.new_zeros(D, n1 + 2 * m, n2 + 2 * m)
    Op[:, m:m + n1, m:m + n2] = O
    k = torch.arange(m, device=rho.device)
    rows = (scan[:, 0:1] + m + k)[:, :, None]
    cols = (scan[:, 1:2] + m + k)[:, None, :]
    patches = Op[:, rows, cols]                                    # [D][J][M][M]
    P = probe if probe.dim() == 2 else probe[:, None]
    Psi = torch.fft.fft2(P * patches)
    r = torch.sqrt(Psi.real * Psi.real + Psi.imag * Psi.imag) - amp
    loss = 0.5 * (r * r).sum()
    loss.backward()
    return loss.detach(), rho.grad, u.grad, alpha.grad


def unfused_comparison(torch, prob, spec, scan, probe, y, x, flush, stream, n=10):
    """Times torch_loss_grad against the library's loss and gradient on the
    same state and data (L2 flushed between evaluations, CUDA events)."""
    dev = x[0].device
    amp = torch.sqrt(y) if isinstance(y, torch.Tensor) else torch.from_numpy(np.sqrt(y).astype(np.float32)).to(dev)
    G = torch.tensor(np.asarray(spec.G), dtype=torch.float32, device=dev)
    sc = torch.from_numpy(np.asarray(scan, np.int64)).to(dev)
    pr = torch.from_numpy(probe).to(dev)
    call = lambda: torch_loss_grad(torch, x[0], x[1], x[2], pr, amp, sc, G, spec.phase_scale, spec.m)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(n):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    t_torch = timed(call)
    out = prob.loss_grad(*x)
    t_fused = timed(lambda: prob.loss_grad(*x, out=out))
    ref = [t.double() for t in call()]
    got = [t.double() for t in prob.loss_grad(*x)]
    rel = lambda a_, b_: float(torch.linalg.vector_norm(a_ - b_) / torch.linalg.vector_norm(b_))
    return {"path": "plain per-kernel PyTorch FP32 (einsum, polar, gather, torch.fft.fft2, autograd)",
            "ms_per_eval": t_torch, "value": spec.nframes / (t_torch / 1e3), "unit": UNIT,
            "fused_ms_per_eval": t_fused, "speedup": t_torch / t_fused,
            "unfused_vs_fused": {"loss_rel_err": abs(float(ref[0]) - float(got[0][0])) / abs(float(got[0][0])),
                                 "g_rho_rel_l2": rel(ref[1], got[1]), "g_u_rel_l2": rel(ref[2], got[2]),
                                 "g_alpha_rel_l2": rel(ref[3], got[3])}}


def workload_config(spec):
    """The workload's description, the same in both arms' JSON lines."""
    return {"workload": spec.name, "object": [spec.n1, spec.n2], "frame": spec.m,
            "peaks": spec.npeaks, "scan": [spec.scan_side, spec.scan_side],
            "scan_step": spec.step, "frames_per_step": spec.nframes}


def event_pairs(torch, n):
    return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]


def setup_problem(torch, mpbp, k):
    """Context, data and starting state of workload k, and the lagged-Armijo
    first step length."""
    spec = synth.config(k)
    scan = synth.scan_positions(spec)
    prob = mpbp.Problem.from_spec(spec, scan)
    probe, yd = make_inputs(spec, scan, prob, torch)
    prob.set_probe(torch.from_numpy(probe).cuda())
    prob.set_data(yd)
    rho0, u0, a0 = synth.init_state(spec)
    x = [torch.from_numpy(a.astype(np.float32)).cuda() for a in (rho0, u0, a0)]
    # first step length: the inverse of the Gauss-Newton curvature bound of a
    # pixel's density, M^2 (the unnormalised DFT, Parseval) x max|P|^2 x the
    # frames of all peaks that cover a pixel
    overlap = (spec.m / spec.step) ** 2 * spec.npeaks
    t0 = 1.0 / (spec.m ** 2 * float(np.abs(probe).max() ** 2) * overlap)
    return spec, scan, prob, probe, yd, x, t0


def time_steps(torch, prob, x, t0, steps, warmup, flush, stream, world=1, dist=None, clocks=None):
    """Optimizer steps of one problem: `warmup` eager steps, then `steps`
    replays of the step captured as a CUDA graph, each bracketed by CUDA
    events on the launching stream with L2 flushed before it (outside the
    events).  Then the same steps launched eagerly with the fused frame
    kernel's launches timed by events on their own stream.  Returns
    (per-step ms list of the replays, eager ms per step, frame-kernel ms per
    launch, wall seconds of the timed replays)."""
    state = prob.step_init(t0, w_rho=1.0, w_u=1e-3, w_alpha=1e-3)
    for _ in range(warmup):
        prob.step(*x, state)
    torch.cuda.synchronize()
    prob.sync_status()
    prob.step_capture(*x, state)
    for _ in range(2):
        prob.step_replay()
    torch.cuda.synchronize()
    evs = event_pairs(torch, steps)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ctx = clocks if clocks is not None else _NullCtx()
    with ctx:
        wall0 = time.perf_counter()
        for k in range(steps):
            flush.zero_()                       # evict L2 between timed steps (not timed)
            evs[k][0].record(stream)
            prob.step_replay()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    prob.sync_status()
    n_e = max(3, min(steps, 20))
    eve = event_pairs(torch, n_e)
    prob.frames_timing(True)
    torch.cuda.synchronize()
    for k in range(n_e):
        flush.zero_()
        eve[k][0].record(stream)
        prob.step(*x, state)
        eve[k][1].record(stream)
    torch.cuda.synchronize()
    prob.frames_timing(False)
    eager_ms = sum(a.elapsed_time(b) for a, b in eve) / n_e
    kern_ms, kern_n = prob.frames_timing_read()
    prob.sync_status()
    return step_ms, eager_ms, kern_ms / max(kern_n, 1), wall


class _NullCtx:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def time_evals(torch, prob, x, n, flush, stream, warmup=2):
    """Median-free mean of n loss+gradient evaluations (CUDA events, L2
    flushed between) and the fused frame kernel's mean launch time."""
    for _ in range(warmup):
        prob.loss_grad(*x)
    evs = event_pairs(torch, n)
    prob.frames_timing(True)
    torch.cuda.synchronize()
    for k in range(n):
        flush.zero_()
        evs[k][0].record(stream)
        prob.loss_grad(*x)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    prob.frames_timing(False)
    kms, kn = prob.frames_timing_read()
    prob.sync_status()
    return sum(a.elapsed_time(b) for a, b in evs) / n, kms / max(kn, 1)


def traffic_record(name, rev):
    """DRAM bytes per launch of a kernel from its committed ncu record, or None
    when the record is missing or was taken at another source revision."""
    tr_path = os.path.join(ROOT, "profiles", name)
    try:
        with open(tr_path) as f:
            tr = json.load(f)
        if tr.get("kernel_rev") == rev:
            return tr
    except Exception:
        pass
    return None


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2312_14907_gb300 import mpbp, replicas

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    num_sms = torch.cuda.get_device_properties(local).multi_processor_count
    pk = peaks(num_sms)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2
    stream = torch.cuda.current_stream()

    # ---- the headline: graph-replayed optimizer steps on the 1024^2 problem
    spec, scan, prob, probe, yd, x, t0 = setup_problem(torch, mpbp, HEADLINE)
    info = prob.info()
    clk = ClockSampler(local)
    step_ms, eager_ms, kavg_ms, wall = time_steps(torch, prob, x, t0, args.steps, args.warmup, flush, stream,
                                                  world, dist, clocks=clk)
    tot_ms = replicas.max_over_ranks(sum(step_ms), device="cuda")

    # end to end through the host-buffer C-ABI call: H2D of the step's data and
    # state from pinned memory, evaluation, D2H of loss and gradients
    rho0, u0, a0 = synth.init_state(spec)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    yh = torch.empty(yd.shape, dtype=torch.float32).pin_memory()
    yh.copy_(yd)
    rh, uh, ah = pin(rho0.astype(np.float32)), pin(u0.astype(np.float32)), pin(a0.astype(np.float32))
    outs = (torch.empty(1, dtype=torch.float64).pin_memory(),
            torch.empty(spec.n1, spec.n2, dtype=torch.float32).pin_memory(),
            torch.empty(spec.ncomp, spec.n1, spec.n2, dtype=torch.float32).pin_memory(),
            torch.empty(spec.npeaks, dtype=torch.float64).pin_memory())
    n_e2e = max(3, min(args.steps, 10))

    call_ms = {}

    def e2e_rate(yhost, key):
        for _ in range(2):
            prob.loss_grad_host(rh, uh, ah, y=yhost, out=outs)
        if world > 1:
            dist.barrier()
        ts = []
        for _ in range(n_e2e):
            flush.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            prob.loss_grad_host(rh, uh, ah, y=yhost, out=outs)
            ts.append(time.perf_counter() - t1)
        call_ms[key] = {"min": min(ts) * 1e3, "median": statistics.median(ts) * 1e3, "max": max(ts) * 1e3,
                        "calls": [round(t * 1e3, 2) for t in ts]}
        return replicas.max_over_ranks(sum(ts), device="cuda")

    e2e_s = e2e_rate(yh, "f32")
    # the host link's own rate in this run: the same bytes of y as one plain
    # copy from pinned memory into the (identical) device data tensor
    link_ts = []
    for _ in range(3):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        yd.copy_(yh, non_blocking=True)
        torch.cuda.synchronize()
        link_ts.append(time.perf_counter() - t1)
    link_gbs = yh.numel() * 4 / min(link_ts) / 1e9
    h2d = yh.numel() * 4 + rh.numel() * 4 + uh.numel() * 4 + ah.numel() * 4
    d2h = 8 + outs[1].numel() * 4 + outs[2].numel() * 4 + outs[3].numel() * 8
    # the same call with the photon counts as 16-bit integers (exact: the
    # data are Poisson counts below 65536)
    assert bool((yd == torch.round(yd)).all()) and float(yd.max()) < 32768
    yh16 = yd.to(torch.int16).view(torch.uint16).cpu().pin_memory()
    del yh
    e2e16_s = e2e_rate(yh16, "u16")
    del yh16
    h2d16 = spec.nframes * spec.m ** 2 * 2 + rh.numel() * 4 + uh.numel() * 4 + ah.numel() * 4
    e2e_frames = spec.nframes * n_e2e * world

    value = replicas.whole_job_rate(spec.nframes, args.steps, world, tot_ms)
    fl = flops_per_frame(spec.m) * spec.nframes
    achieved_tf = fl / (kavg_ms / 1e3) / 1e12
    bpf = hbm_bytes_per_frame(spec)
    rev = kernel_revision(spec.m)
    tr = traffic_record("frames_m%d_traffic.json" % spec.m, rev)
    traffic = None
    if tr is not None and tr.get("workload") == spec.name:
        traffic = tr["bytes_per_launch"]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tot_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded truth object, Gaussian probe with quadratic phase, CUDA forward "
                "model, Poisson counts at 1e4 photons in the brightest frame drawn on the device)",
        "config": dict(workload_config(spec), **{
            "l2": "flushed between timed steps (256 MB write, outside the timed region); the "
                  "step's 5.76 GB of amplitudes exceed L2 as well",
            "parallelism": "replicas" if world > 1 else "single"}),
        "step": {"what": "object synthesis + fused frame kernel + gradient assembly + FP64 "
                         "reductions + lagged-Armijo update, replayed as the context's CUDA graph "
                         "(mpbp_step_capture / mpbp_step_replay)",
                 "eager_ms_per_step": eager_ms},
        "iterations_per_s": args.steps * world / (tot_ms / 1e3),
        "hbm_roofline": {"bytes_per_frame": bpf, "achieved_gbs": value * bpf / 1e9 / world,
                         "peak_gbs": pk["hbm_gbs"], "frac": value * bpf / 1e9 / world / pk["hbm_gbs"],
                         "peak_src": pk["src"]},
        "roofline": {"bound": "alu", "kernel": ("frames_x3<tile copies, probe in TMEM> (fused per-frame kernel, "
                                                "shared-memory exchange FFT schedule)"
                                                if info["fft_schedule"] == mpbp.FFT_EXCHANGE else
                                                "frames_t4<128, tile copies, probe in TMEM> (fused per-frame "
                                                "kernel, shuffle FFT schedule)"),
                     "achieved": achieved_tf, "peak": pk["fp32_tflops"], "unit": "TFLOP/s",
                     "frac": achieved_tf / pk["fp32_tflops"], "traffic": traffic,
                     "traffic_src": (tr or {}).get("src"),
                     "kernel_ms": kavg_ms, "kernel_share_of_step": kavg_ms / eager_ms,
                     "flops_per_frame": flops_per_frame(spec.m), "frames_per_launch": spec.nframes,
                     "algorithmic_bytes_per_launch": bpf * spec.nframes,
                     "peak_src": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz (max SM clock)" % (num_sms,
                                                                                        pk["sm_max_mhz"]),
                     "hbm_frac": (spec.nframes * 4 * spec.m ** 2 / (kavg_ms / 1e3) / 1e9) / pk["hbm_gbs"]},
        "e2e": {"value": e2e_frames / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "call": "mpbp_loss_grad_host (host y, rho, u, alpha in; loss and gradients out)",
                "link_h2d_gbs": link_gbs,
                "frac_of_link": (h2d * n_e2e / e2e_s / 1e9) / link_gbs,
                "link_src": "one pinned copy of the same y bytes in this run (torch copy_, best of 3)",
                "ms_per_call": call_ms["f32"]},
        "e2e_counts16": {"value": e2e_frames / e2e16_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d16),
                         "d2h_bytes_per_step": int(d2h),
                         "call": "mpbp_loss_grad_host_counts16 (y as 16-bit photon counts; otherwise as e2e)",
                         "ms_per_call": call_ms["u16"]},
        "gpu_launches": info["launches_step"] * args.steps,
        "clocks": clk.summary(),
        "wall_s": wall,
    }
    # the two FFT schedules of the M = 128 kernel on the same state (loss and
    # gradient evaluations, CUDA events, L2 flushed between)
    sched = {}
    for name, sc in (("exchange", mpbp.FFT_EXCHANGE), ("shuffle", mpbp.FFT_SHUFFLE)):
        prob.set_fft_schedule(sc)
        e_ms, k_ms = time_evals(torch, prob, [t.clone() for t in x], max(3, min(args.steps, 10)), flush, stream)
        sched[name] = {"ms_per_eval": e_ms, "kernel_ms": k_ms,
                       "kernel_frac_fp32": fl / (k_ms / 1e3) / 1e12 / pk["fp32_tflops"]}
    prob.set_fft_schedule(info["fft_schedule"])
    line["fft_schedules"] = dict(sched, timed_step=("exchange" if info["fft_schedule"] == mpbp.FFT_EXCHANGE
                                                    else "shuffle"),
                                 what="columns 32 x 4 and rows 8 x 16 through shared-memory exchanges, or "
                                      "radix-2 stages across threads by warp shuffles")
    # the deterministic gradient (mpbp_set_deterministic) on the same state:
    # time per evaluation, and whether repeated evaluations give the same bits
    prob.set_deterministic(True)
    d_ms, dk_ms = time_evals(torch, prob, [t.clone() for t in x], max(3, min(args.steps, 10)), flush, stream)
    r1 = [t.clone() for t in prob.loss_grad(*x)]
    r2 = prob.loss_grad(*x)
    same = all(torch.equal(a.contiguous().view(torch.uint8), b.contiguous().view(torch.uint8)) for a, b in zip(r1, r2))
    prob.set_deterministic(False)
    line["deterministic"] = {"ms_per_eval": d_ms, "frames_and_sum_ms": dk_ms,
                             "atomic_ms_per_eval": sched["exchange"]["ms_per_eval"],
                             "value": spec.nframes / (d_ms / 1e3), "unit": UNIT, "bitwise_repeat": same,
                             "what": "gradient windows written back into per-block pieces of column strips, "
                                     "summed per pixel in a fixed order (frames_and_sum_ms: the pieces' clearing, "
                                     "the frame kernel and the sum)"}
    # scan positions off the pixel grid (not the headline): seeded offsets in
    # [-1/2, 1/2] per scan position, one shifted probe per position; loss and
    # gradient evaluations on the same state, CUDA events, L2 flushed between
    d_off = np.random.default_rng(spec.seed + 77).uniform(-0.5, 0.5, (scan.shape[0], 2))
    torch.cuda.synchronize()
    ts0 = time.perf_counter()
    prob.set_scan_offsets(d_off)
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - ts0)
    xs = [t.clone() for t in x]
    sp_ms, sk_ms = time_evals(torch, prob, xs, max(3, min(args.steps, 10)), flush, stream)
    prob.set_scan_offsets(None)
    line["subpixel_scan"] = {
        "what": "loss + gradient with seeded scan offsets in [-1/2, 1/2] (one shifted probe per scan position)",
        "ms_per_eval": sp_ms, "value": spec.nframes / (sp_ms / 1e3), "unit": UNIT,
        "kernel_ms": sk_ms, "probe_setup_ms": setup_ms}
    # the unfused comparison path on the same data and state
    line["unfused_torch"] = unfused_comparison(torch, prob, spec, scan, probe, yd, x, flush, stream, n=5)
    del yd
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(torch, mpbp, spec, scan, probe, budget_s=args.cpu_budget)
    prob.close()
    torch.cuda.empty_cache()

    # ---- the 512^2 / M = 128 / 4-peak problem: 200 graph-captured iterations
    line["workload_512_iterations"] = iterations_block(torch, mpbp, args, flush, stream, rank)
    # ---- the 16 problems of uneven sizes in one batched call
    line["batched_16"] = batched_block(torch, mpbp, flush, stream)
    # ---- the 256^2 / M = 64 problem: its step, both precision modes, Alg. 1
    line["workload_256"] = secondary_block(torch, mpbp, args, flush, stream, pk)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def batched_block(torch, mpbp, flush, stream, n=5):
    """The 16 independent problems of uneven sizes (objects 128..512, frame
    sides 32/64/128, 3 or 4 peaks, 90,844 frames) evaluated by one
    mpbp_loss_grad_batched call under each batch schedule (mode 0: one
    persistent launch for every frame side; 1: one per side; 2: as 1, M = 128
    problems on their own; 3: one launch per problem), CUDA events, L2
    flushed between calls; then the schedule mpbp_autotune_batched picks."""
    specs = synth.batched_configs()
    probs, states = [], []
    for spec in specs:
        scan = synth.scan_positions(spec)
        pr = mpbp.Problem.from_spec(spec, scan)
        probe, yd = make_inputs(spec, scan, pr, torch)
        pr.set_probe(torch.from_numpy(probe).cuda())
        pr.set_data(yd)
        del yd
        probs.append(pr)
        states.append([torch.from_numpy(a.astype(np.float32)).cuda() for a in synth.init_state(spec)])
    nframes = sum(sp.nframes for sp in specs)
    outs = mpbp.loss_grad_batched(probs, states)
    res = {"problems": len(specs), "frames": nframes, "modes": {}}
    for mode in (0, 1, 2, 3):
        probs[0].set_batch_schedule(mode, 0)
        for _ in range(2):
            mpbp.loss_grad_batched(probs, states, outs)
        evs = event_pairs(torch, n)
        torch.cuda.synchronize()
        for k in range(n):
            flush.zero_()
            evs[k][0].record(stream)
            mpbp.loss_grad_batched(probs, states, outs)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / n
        res["modes"][str(mode)] = {"ms_per_eval": ms, "value": nframes / (ms / 1e3), "unit": UNIT}
    mpbp.autotune_batched(probs, states)
    torch.cuda.synchronize()
    for pr in probs:
        pr.sync_status()
    res["what"] = ("one mpbp_loss_grad_batched call over all 16 problems; mode 0: one persistent launch for "
                   "every frame side, 1: one per side, 2: as 1 with M = 128 problems on their own, 3: one "
                   "launch per problem (the single-problem kernels)")
    for pr in probs:
        pr.close()
    return res


SNAPSHOTS = (0, 1, 10, 199)   # iterates whose states are replayed on the oracle


def iterations_block(torch, mpbp, args, flush, stream, rank, iters=200):
    """The 512^2, M = 128, 4-peak problem: `iters` optimizer iterations (GD +
    lagged Armijo) replayed from one captured CUDA graph, timed as a whole
    (CUDA events, L2 flushed before), in each DFT arithmetic (FP32 FFTs; the
    split tensor-core DFTs); then the same trajectory again, untimed, keeping
    the states at SNAPSHOTS, whose loss and gradient on a seeded 1/16 of the
    scan positions are compared with the FP64 oracle's at the same states
    (rank 0, unless --no-cpu-baseline)."""
    spec, scan, prob, probe, yd, x, t0 = setup_problem(torch, mpbp, 3)
    del yd
    # a generic start (a seeded 5% perturbation of the true object): at the
    # flat start the far field of most pixels is below rounding and the
    # gradient is not well conditioned, so no parity is defined there
    xp = synth.perturbed_state(spec, np.random.default_rng(spec.seed + 6), 0.05)
    x0 = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda() for a in xp]
    out = {"config": workload_config(spec), "iterations": iters,
           "what": "GD + lagged-Armijo steps replayed from one captured CUDA graph, from a seeded 5% "
                   "perturbation of the true object"}
    state = None
    for name, prec in (("fp32_fft", mpbp.PRECISION_FP32), ("tc_split16", mpbp.PRECISION_TC_SPLIT16)):
        prob.set_precision(prec)
        for t, t_init in zip(x, x0):
            t.copy_(t_init)
        state = prob.step_init(t0, w_rho=1.0, w_u=1e-3, w_alpha=1e-3, state=state)
        prob.step_capture(*x, state)
        prob.step_replay()                      # warm-up (iterate 0 -> 1)
        torch.cuda.synchronize()
        for t, t_init in zip(x, x0):
            t.copy_(t_init)
        state = prob.step_init(t0, w_rho=1.0, w_u=1e-3, w_alpha=1e-3, state=state)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(iters):
            prob.step_replay()
        e1.record(stream)
        torch.cuda.synchronize()
        prob.sync_status()
        ms = e0.elapsed_time(e1)
        st = mpbp.Problem.read_state(state)
        res = {"ms_total": ms, "ms_per_iteration": ms / iters, "value": spec.nframes * iters / (ms / 1e3),
               "unit": UNIT, "accepted": st.n_accept, "rejected": st.n_reject, "loss_last": st.f_last}
        # the trajectory again with its snapshots
        for t, t_init in zip(x, x0):
            t.copy_(t_init)
        state = prob.step_init(t0, w_rho=1.0, w_u=1e-3, w_alpha=1e-3, state=state)
        snaps = {}
        for k in range(iters):
            if k in SNAPSHOTS:
                snaps[k] = [t.cpu().numpy().copy() for t in x]
            prob.step_replay()
            if k == 0:
                torch.cuda.synchronize()
                res["loss_first"] = mpbp.Problem.read_state(state).f_last
        torch.cuda.synchronize()
        prob.sync_status()
        if rank == 0 and not args.no_cpu_baseline:
            res["vs_oracle"] = trajectory_vs_oracle(torch, mpbp, spec, scan, probe, snaps, prec)
        out[name] = res
    prob.set_precision(mpbp.PRECISION_FP32)
    prob.close()
    return out


def trajectory_vs_oracle(torch, mpbp, spec, scan, probe, snaps, precision=0):
    """Loss and gradient of the GPU (in the given DFT arithmetic) and of the
    FP64 oracle at the GPU's own iterates, on a seeded 1/16 of the scan
    positions (every peak) with count data that do not come from the CUDA path
    (synth.template_counts)."""
    import oracle
    sub_scan, js = sample_subproblem(spec, scan, max(1, scan.shape[0] // 16), spec.seed + 18)
    y = synth.template_counts(spec, spec.seed + 19, scan_index=js)
    orc = oracle.OracleProblem.from_spec(spec, sub_scan)
    q = mpbp.Problem(spec.n1, spec.n2, spec.ncomp, spec.npeaks, spec.m, sub_scan, spec.G, spec.phase_scale,
                     spec.probe_per_peak)
    q.set_probe(torch.from_numpy(probe).cuda())
    q.set_data(torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda())
    q.set_precision(precision)

    def rel(a, b):
        a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    res = {"sample": "%d of %d scan positions x %d peaks" % (len(js), scan.shape[0], spec.npeaks),
           "tolerance": {"loss": 1e-5, "gradients": 1e-4}}
    for k, xs in sorted(snaps.items()):
        got = [t.cpu().numpy() for t in q.loss_grad(*[torch.from_numpy(a).cuda() for a in xs])]
        ref = orc.loss_grad(*xs, probe, y)
        res["iterate_%d" % k] = {"loss_rel_err": abs(float(got[0][0]) - ref[0]) / abs(ref[0]),
                                 "g_rho_rel_l2": rel(got[1], ref[1]), "g_u_rel_l2": rel(got[2], ref[2]),
                                 "g_alpha_rel_l2": rel(got[3], ref[3])}
    q.sync_status()
    q.close()
    return res


def secondary_block(torch, mpbp, args, flush, stream, pk):
    """The 256^2, M = 64, 3-peak problem (not the headline): graph-replayed
    steps and the frame kernel's roofline, the tensor-core precision mode,
    and the paper's own minibatch Adam iteration (Alg. 1) with and without
    the projector."""
    spec, scan, prob, probe, yd, x, t0 = setup_problem(torch, mpbp, SECONDARY)
    steps = max(5, min(args.steps, 20))
    # (the steps move x away from the flat start, where the gradient is ill
    # conditioned, before the unfused comparison below)
    step_ms, eager_ms, kavg_ms, _ = time_steps(torch, prob, x, t0, steps, args.warmup, flush, stream)
    ms = sum(step_ms) / len(step_ms)
    achieved = flops_per_frame(spec.m) * spec.nframes / (kavg_ms / 1e3) / 1e12
    rev = kernel_revision(spec.m)
    tr = traffic_record("frames_m%d_traffic.json" % spec.m, rev)
    out = {"config": workload_config(spec), "ms_per_step": ms, "value": spec.nframes / (ms / 1e3),
           "unit": UNIT, "eager_ms_per_step": eager_ms, "iterations_per_s": 1e3 / ms,
           "roofline": {"bound": "alu", "kernel": "frames_t2<64, tile copies, probe in TMEM>", "kernel_ms": kavg_ms,
                        "achieved": achieved, "peak": pk["fp32_tflops"], "unit": "TFLOP/s",
                        "frac": achieved / pk["fp32_tflops"],
                        "traffic": tr["bytes_per_launch"] if tr else None}}
    # the deterministic gradient (mpbp_set_deterministic) on the same state
    xd = [t.clone() for t in x]
    a_ms, _ = time_evals(torch, prob, xd, steps, flush, stream)
    prob.set_deterministic(True)
    d_ms, _ = time_evals(torch, prob, xd, steps, flush, stream)
    r1 = [t.clone() for t in prob.loss_grad(*xd)]
    r2 = prob.loss_grad(*xd)
    same = all(torch.equal(a.contiguous().view(torch.uint8), b.contiguous().view(torch.uint8)) for a, b in zip(r1, r2))
    prob.set_deterministic(False)
    out["deterministic"] = {"ms_per_eval": d_ms, "atomic_ms_per_eval": a_ms, "value": spec.nframes / (d_ms / 1e3),
                            "unit": UNIT, "bitwise_repeat": same}
    # the tensor-core precision mode on the same steps
    prob.set_precision(mpbp.PRECISION_TC_SPLIT16)
    xs = [t.clone() for t in x]
    tc_ms, tc_eager, tk_avg, _ = time_steps(torch, prob, xs, t0, steps, args.warmup, flush, stream)
    prob.set_precision(mpbp.PRECISION_FP32)
    tc_step = sum(tc_ms) / len(tc_ms)
    tc_flops = 4 * 3 * 2 * 128 * 64 * 128   # 4 passes x 3 split products, M=128 N=64 K=128
    out["alt_precision"] = {
        "mode": "tc_split16 (DFT matrices on tcgen05 tensor cores, split-FP16 operands, FP32 accumulation)",
        "ms_per_step": tc_step, "value": spec.nframes / (tc_step / 1e3), "unit": UNIT,
        "kernel": "frames_tc64", "kernel_ms": tk_avg,
        "tensor_tflops": tc_flops * spec.nframes / (tk_avg / 1e3) / 1e12,
        "tensor_flops_per_frame": tc_flops,
        "tensor_peak_tflops": pk["bf16_tflops"], "peak_src": pk["src"] + " (dense bf16 = fp16 rate)"}
    out["alg1"] = alg1_block(torch, prob, spec, x, flush, stream)
    out["alt_precision_m32"] = tc_m32_block(torch, mpbp, flush, stream, pk)
    out["unfused_torch"] = unfused_comparison(torch, prob, spec, scan, probe, yd, x, flush, stream)
    prob.close()
    return out


def tc_m32_block(torch, mpbp, flush, stream, pk, n=10):
    """Frame side 32 in both precision modes: loss and gradient evaluations of
    the 512^2, 4-peak, 61 x 61-scan problem of the batched set (14,884 frames
    of 32 x 32), FP32 FFTs against the tensor-core DFTs (four frames per
    64 x 64 tile), CUDA events, L2 flushed between calls."""
    spec = synth.batched_configs()[15]
    scan = synth.scan_positions(spec)
    prob = mpbp.Problem.from_spec(spec, scan)
    probe, yd = make_inputs(spec, scan, prob, torch)
    prob.set_probe(torch.from_numpy(probe).cuda())
    prob.set_data(yd)
    del yd
    xp = synth.perturbed_state(spec, np.random.default_rng(spec.seed + 6), 0.05)
    x = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda() for a in xp]
    out = {"config": workload_config(spec)}
    res = {}
    for name, mode in (("fp32_fft", mpbp.PRECISION_FP32), ("tc_split16", mpbp.PRECISION_TC_SPLIT16)):
        prob.set_precision(mode)
        ms, kms = time_evals(torch, prob, x, n, flush, stream)
        res[name] = [t.cpu().numpy() for t in prob.loss_grad(*x)]
        out[name] = {"ms_per_eval": ms, "kernel_ms": kms, "value": spec.nframes / (ms / 1e3), "unit": UNIT}
    tc_flops = 4 * 3 * 2 * 128 * 64 * 128 / 4   # per 32 x 32 frame: a quarter of a 64 x 64 tile's passes
    out["tc_split16"]["tensor_tflops"] = tc_flops * spec.nframes / (out["tc_split16"]["kernel_ms"] / 1e3) / 1e12
    out["tc_split16"]["tensor_peak_tflops"] = pk["bf16_tflops"]

    def rel(a, b):
        a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    a, b = res["tc_split16"], res["fp32_fft"]
    out["tc_vs_fft"] = {"loss_rel_err": abs(float(a[0][0]) - float(b[0][0])) / abs(float(b[0][0])),
                        "g_rho_rel_l2": rel(a[1], b[1]), "g_u_rel_l2": rel(a[2], b[2]),
                        "g_alpha_rel_l2": rel(a[3], b[3])}
    prob.close()
    return out


def alg1_block(torch, prob, spec, x, flush, stream):
    """The paper's own iteration (Alg. 1 without its projector): minibatches
    of 50 frames from a seeded shuffle per epoch, Adam in the Eq. 8 variables
    with the paper's step sizes, inside the support mask; eagerly, as one
    CUDA graph per epoch, and with the projector Pi_U after every step."""
    mask = torch.from_numpy(synth.support_mask(spec)).cuda()
    chi = torch.log(torch.clamp(x[0], min=0.2)).contiguous()
    ua = x[1].clone()
    at = torch.log(x[2]).contiguous()
    ast = prob.adam_init(lr_u=0.01, lr_chi=0.1, lr_alpha=0.1)
    bsz = 50
    epochs = [torch.from_numpy(synth.epoch_order(spec.nframes, spec.seed + 100 + e)).cuda() for e in range(3)]
    batches = [[ep[k:k + bsz].contiguous() for k in range(0, spec.nframes, bsz)] for ep in epochs]
    for fr in batches[0]:                    # warm-up epoch
        prob.adam_step(fr, chi, ua, at, ast, mask=mask)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    e0.record(stream)
    for ep in batches[1:]:
        for fr in ep:
            prob.adam_step(fr, chi, ua, at, ast, mask=mask)
    e1.record(stream)
    torch.cuda.synchronize()
    prob.sync_status()
    ep_ms = e0.elapsed_time(e1) / (len(batches) - 1)
    # the same epochs as one CUDA graph each: the epoch's shuffled order is
    # copied into a fixed device buffer whose minibatch slices the captured
    # calls read (the copy is inside the timed region)
    order_buf = torch.empty_like(epochs[0])
    order_buf.copy_(epochs[0])
    gsl = [order_buf[k:k + bsz] for k in range(0, spec.nframes, bsz)]
    gs = torch.cuda.Stream()
    gs.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(gs):
        with torch.cuda.graph(graph, stream=gs):
            for fr in gsl:
                prob.adam_step(fr, chi, ua, at, ast, mask=mask)
    torch.cuda.synchronize()
    graph.replay()                           # warm-up epoch
    torch.cuda.synchronize()
    e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    e4.record(stream)
    for ep in epochs[1:]:
        order_buf.copy_(ep)
        graph.replay()
    e5.record(stream)
    torch.cuda.synchronize()
    prob.sync_status()
    gep_ms = e4.elapsed_time(e5) / (len(epochs) - 1)
    # with the projector line: Pi_U on u after every Adam step (C-UW)
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    prob.project_displacement(ua, mask)      # workspace set-up outside the timing
    torch.cuda.synchronize()
    e2.record(stream)
    for fr in batches[1]:
        prob.adam_step(fr, chi, ua, at, ast, mask=mask)
        prob.project_displacement(ua, mask)
    e3.record(stream)
    torch.cuda.synchronize()
    prob.sync_status()
    cuw_ms = e2.elapsed_time(e3)
    return {
        "iteration": "Alg. 1 minus the projector: minibatch of %d frames, Adam (0.01 u, 0.1 chi, 0.1 alpha)" % bsz,
        "ms_per_epoch": ep_ms, "minibatches_per_epoch": len(batches[0]),
        "ms_per_minibatch": ep_ms / len(batches[0]), "value": spec.nframes / (ep_ms / 1e3), "unit": UNIT,
        "launches_per_minibatch": 5,
        "graph": {"ms_per_epoch": gep_ms, "ms_per_minibatch": gep_ms / len(batches[0]),
                  "value": spec.nframes / (gep_ms / 1e3), "unit": UNIT,
                  "note": "each epoch one CUDA graph replay (minibatch slices of a fixed order buffer)"},
        "with_projector": {"ms_per_epoch": cuw_ms, "ms_per_minibatch": cuw_ms / len(batches[1]),
                           "projector_ms": (cuw_ms - ep_ms) / len(batches[1]),
                           "value": spec.nframes / (cuw_ms / 1e3), "unit": UNIT}}


KERNEL_SOURCES = {
    64: ("frames.cuh", "bulk.cuh", "frames_inst.cuh", "fft_reg.cuh", "fft_pair.cuh", "frames_m64.cu",
         "mpbp_internal.h"),
    128: ("frames.cuh", "frames_t4.cuh", "frames_x3.cuh", "tmem.cuh", "bulk.cuh", "frames_inst.cuh",
          "fft_reg.cuh", "fft_pair.cuh", "fft_quad.cuh", "frames_m128.cu", "mpbp_internal.h"),
}


def kernel_revision(m):
    """Hash of the sources of the fused kernel of frame side m (a committed
    ncu traffic figure taken at another revision is dropped)."""
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2312_14907_gb300", "csrc")
    for name in KERNEL_SOURCES[m]:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def sample_subproblem(spec, scan, count, seed):
    """A seeded sample of `count` scan positions of the problem (all peaks at
    each): the sub-problem's scan table and the positions' indices."""
    rng = np.random.default_rng(seed)
    js = np.sort(rng.choice(scan.shape[0], min(count, scan.shape[0]), replace=False))
    return np.ascontiguousarray(scan[js]), js


def cpu_baseline(torch, mpbp, spec, scan, probe, budget_s=15.0):
    """The FP64 oracle, as it stands, on the host cores, timed on a seeded
    1/16 of the problem's scan positions (every peak at each: 1/16 of the
    frames; whole loss+gradient evaluations of that sub-problem, repeated
    until about `budget_s` seconds), reported in frames per second.  Beside
    it the error of the GPU's loss and gradient against the oracle on the same
    sub-problem, with count data that do not come from the CUDA path
    (synth.template_counts) at a seeded perturbed state."""
    import oracle
    sub_scan, js = sample_subproblem(spec, scan, max(1, scan.shape[0] // 16), spec.seed + 16)
    p = oracle.OracleProblem.from_spec(spec, sub_scan)
    y = synth.template_counts(spec, spec.seed + 17, scan_index=js)
    rho, u, alpha = synth.perturbed_state(spec, np.random.default_rng(spec.seed + 5), 0.05)
    n, t = 0, 0.0
    ref = None
    while (t < budget_s and n < 50) or n == 0:
        t1 = time.perf_counter()
        ref = p.loss_grad(rho, u, alpha, probe, y)
        t += time.perf_counter() - t1
        n += 1
    nf = spec.npeaks * len(js)
    out = {"value": n * nf / t, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
           "sample": "%d loss+gradient evaluation(s) of a seeded 1/16 of the scan positions (%d of %d "
                     "frames, every peak), %.1f s; frames/s extrapolates linearly to the workload"
                     % (n, nf, spec.nframes, t)}
    # the GPU on the same sub-problem, data and state
    q = mpbp.Problem(spec.n1, spec.n2, spec.ncomp, spec.npeaks, spec.m, sub_scan, spec.G, spec.phase_scale,
                     spec.probe_per_peak)
    q.set_probe(torch.from_numpy(probe).cuda())
    q.set_data(torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda())
    got = [t_.cpu().numpy() for t_ in q.loss_grad(*[torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
                                                    for a in (rho, u, alpha)])]
    q.sync_status()
    q.close()

    def rel(a, b):
        a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    out["gpu_vs_oracle"] = {"state": "seeded 5% perturbation of the true object; count data from "
                                     "synth.template_counts; the sub-problem above",
                            "tolerance": {"loss": 1e-5, "gradients": 1e-4},
                            "fp32_fft": {"loss_rel_err": abs(float(got[0][0]) - ref[0]) / abs(ref[0]),
                                         "g_rho_rel_l2": rel(got[1], ref[1]), "g_u_rel_l2": rel(got[2], ref[2]),
                                         "g_alpha_rel_l2": rel(got[3], ref[3])}}
    return out


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores,
    on the headline workload.  Each step is one loss+gradient evaluation of a
    seeded sample of `--ref-frames` frames, drawn from a pool of scan
    positions whose data are Poisson counts of the oracle's own forward model
    at the true object (photon scaling over the pool)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    spec = synth.config(HEADLINE)
    scan = synth.scan_positions(spec)
    pool = max(16, -(-args.ref_frames // spec.npeaks) * 2)
    sub_scan, js = sample_subproblem(spec, scan, pool, spec.seed + 31)
    P = synth.probe(spec)
    p = oracle.OracleProblem.from_spec(spec, sub_scan)
    rho_t, u_t = synth.truth(spec)
    I = p.forward(rho_t, u_t, synth.alpha_truth(spec), P)
    scale = synth.photon_scale(I, spec.photons)
    probe = P * np.sqrt(scale)
    y = synth.poisson_counts(I * scale, spec.seed + 1000)
    rho0, u0, a0 = synth.init_state(spec)
    nsample = min(p.nframes, args.ref_frames)
    rng = np.random.default_rng(7)
    for _ in range(args.warmup):
        p.loss_grad(rho0, u0, a0, probe, y, frames=rng.choice(p.nframes, nsample, replace=False))
    t = 0.0
    for _ in range(args.steps):
        fr = rng.choice(p.nframes, nsample, replace=False)
        t1 = time.perf_counter()
        p.loss_grad(rho0, u0, a0, probe, y, frames=fr)
        t += time.perf_counter() - t1
    value = nsample * args.steps / t
    cfg = dict(workload_config(spec), l2="host cores: no GPU cache involved", parallelism="single")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (the GPU arm's generator: true object, probe, forward model -- here the "
                    "oracle's -- and Poisson counts at 1e4 photons in the brightest frame)",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                             "kind": "oracle",
                             "sample": "%d seeded frames per step, from %d scan positions x %d peaks of the "
                                       "workload's %d frames" % (nsample, len(js), spec.npeaks, spec.nframes)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_drive(args):
    """Profiling driver: set up workload `--drive K` (1, 2, 3 or 5) with
    synthetic data and run `--drive-evals` loss+gradient evaluations, then
    `--drive-steps` optimizer steps (and `--drive-projector` calls of the
    projector Pi_U), without timing (for `ncu` captures of the kernels)."""
    import torch
    from paper_2312_14907_gb300 import mpbp
    spec = synth.config(args.drive)
    scan = synth.scan_positions(spec)
    prob = mpbp.Problem.from_spec(spec, scan)
    probe, yd = make_inputs(spec, scan, prob, torch)
    prob.set_probe(torch.from_numpy(probe).cuda())
    prob.set_data(yd)
    del yd
    x = [torch.from_numpy(a.astype(np.float32)).cuda() for a in synth.init_state(spec)]
    prob.set_precision(args.drive_precision)
    if args.drive_deterministic:
        prob.set_deterministic(True)
    for _ in range(args.drive_evals):
        prob.loss_grad(*x)
    if args.drive_projector:
        mask = torch.from_numpy(synth.support_mask(spec)).cuda()
        ud = x[1] + torch.from_numpy(synth.truth(spec)[1].astype(np.float32)).cuda() * 3.0
        for _ in range(args.drive_projector):
            prob.project_displacement(ud, mask)
    if args.drive_steps:
        overlap = (spec.m / spec.step) ** 2 * spec.npeaks
        t0 = 1.0 / (spec.m ** 2 * float(np.abs(probe).max() ** 2) * overlap)
        state = prob.step_init(t0, w_rho=1.0, w_u=1e-3, w_alpha=1e-3)
        for _ in range(args.drive_steps):
            prob.step(*x, state)
    torch.cuda.synchronize()
    prob.sync_status()
    print("drove %s: %d evaluations, %d steps, %d projector calls" % (spec.name, args.drive_evals,
                                                                       args.drive_steps, args.drive_projector))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-frames", type=int, default=120)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--drive", type=int, default=0,
                    help="profiling driver: run workload 1, 2, 3 or 5 untimed")
    ap.add_argument("--drive-evals", type=int, default=4)
    ap.add_argument("--drive-steps", type=int, default=0)
    ap.add_argument("--drive-projector", type=int, default=0,
                    help="profiling driver: projector calls (Pi_U on the displacement)")
    ap.add_argument("--drive-deterministic", action="store_true",
                    help="profiling driver: the deterministic gradient (mpbp_set_deterministic)")
    ap.add_argument("--drive-precision", type=int, default=0,
                    help="profiling driver: 0 = FP32 FFT kernels, 1 = tensor-core DFTs (M = 64)")
    args = ap.parse_args()
    if args.drive:
        run_drive(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
