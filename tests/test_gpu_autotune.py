"""The autotuner: it picks a valid schedule, remembers it in its JSON-lines
cache, and the tuned schedules still produce the oracle's loss and gradient."""
import json

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


def _check(case, got):
    f, gr, gu, ga = case.oracle_loss_grad()
    loss, g_rho, g_u, g_alpha = [t.cpu().numpy() for t in got]
    assert abs(loss[0] - f) <= 1e-5 * abs(f)
    assert rel_l2(g_rho, gr) <= 1e-4 and rel_l2(g_u, gu) <= 1e-4 and rel_l2(g_alpha, ga) <= 1e-4


def test_single_problem_autotune_and_cache(tmp_path):
    spec, scan = custom_spec(128, 64, 6, 12, npeaks=3, offset=2)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    cache = tmp_path / "tune.jsonl"
    b = p.autotune(*x, cache_path=str(cache))
    assert 1 <= b <= p.info()["blocks_per_sm"] or b >= 1
    lines = [json.loads(l) for l in cache.read_text().splitlines()]
    assert len(lines) == 1 and lines[0]["blocks_per_sm"] == b and "|single|m64|d3|" in lines[0]["key"]
    # the DFT arithmetic is a candidate at M = 64 (FP32 FFTs or tensor cores)
    assert lines[0]["precision"] in (0, 1) and p.info()["precision"] == lines[0]["precision"]
    _check(case, p.loss_grad(*x))
    # a second problem of the same shape reads the cache instead of tuning
    p2, x2 = _gpu(case)
    assert p2.autotune(*x2, cache_path=str(cache)) == b
    assert len(cache.read_text().splitlines()) == 1
    p.sync_status()


def test_m128_autotune_covers_both_fft_schedules(tmp_path):
    """At frame side 128 the autotuner also chooses between the two FFT
    schedules (shuffles across threads; shared-memory exchanges) and caches
    the choice; the chosen schedule still computes the oracle's result."""
    spec, scan = custom_spec(256, 128, 6, 24, npeaks=2, offset=-4)
    case = Case(spec, scan=scan, state="perturbed")
    p, x = _gpu(case)
    cache = tmp_path / "tune.jsonl"
    p.autotune(*x, cache_path=str(cache))
    line = json.loads(cache.read_text().splitlines()[0])
    assert line["fft_schedule"] in (0, 1) and line["blocks_per_sm"] >= 1
    assert p.info()["fft_schedule"] == line["fft_schedule"]
    _check(case, p.loss_grad(*x))
    p2, x2 = _gpu(case)
    p2.set_fft_schedule(1 - line["fft_schedule"])
    p2.autotune(*x2, cache_path=str(cache))          # from the cache
    assert p2.info()["fft_schedule"] == line["fft_schedule"]
    p.sync_status()


def test_batched_autotune_picks_a_working_schedule(tmp_path):
    from paper_2312_14907_gb300 import mpbp
    cases = [Case(*custom_spec(96, 32, 5, 14, npeaks=3, offset=-2, seed=1), state="perturbed"),
             Case(*custom_spec(160, 64, 4, 30, npeaks=4, offset=-5, seed=2), state="perturbed"),
             Case(*custom_spec(200, 128, 2, 60, npeaks=3, offset=-10, seed=3), state="perturbed")]
    probs, states = zip(*[_gpu(c) for c in cases])
    cache = tmp_path / "tune.jsonl"
    mpbp.autotune_batched(list(probs), list(states), cache_path=str(cache))
    line = json.loads(cache.read_text().splitlines()[0])
    assert 0 <= line["mode"] <= 3 and 0 <= line["order"] <= 1
    outs = mpbp.loss_grad_batched(list(probs), list(states))
    for c, o in zip(cases, outs):
        _check(c, o)
    for p in probs:
        p.sync_status()
