"""The serving loop (continuous batching of Algorithm 3 solves, admission by device
footprint): results against the single-problem solve, alone-vs-mix equality, admission
under a tight budget, and the host-side error paths of the request API."""
import numpy as np
import pytest

from helpers import rel_l2, to_dev, to_host
from paper_1805_02158_gb300 import red, synth

pytestmark = pytest.mark.gpu

GIB = 1 << 30


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def requests():
    """A mix of tasks, sizes and PSFs (deblurring and x3 super-resolution)."""
    return [
        synth.make_deblur(0, 64, 64, synth.uniform_psf(9), 2 ** 0.5),
        synth.deblur_gauss256(1, 128),
        synth.sr_x3(2, 96),
        synth.make_deblur(3, 96, 128, synth.gaussian_psf(7, 1.2), 2.0),
        synth.make_deblur(4, 64, 64, synth.uniform_psf(9), 2 ** 0.5),
    ]


def serve(probs, budget=4 * GIB, slots=8, calls=40, tol=0.0):
    S = red.Server(budget, slots)
    outs, tickets = [], []
    for p in probs:
        out = np.zeros((p.height, p.width), np.float32)
        cfg = red.config_for(p, ve="rre", ve_k=5)
        tickets.append(S.submit(cfg, np.ascontiguousarray(p.y32), out, calls, tol))
        outs.append(out)
    stats = []
    for t in tickets:
        st, s = S.wait(t, 120000)
        assert st in (red.RED_OK, red.RED_ENOT_CONVERGED), red.status_string(st)
        stats.append(s)
    S.close()
    return outs, stats


def test_server_matches_single_problem_solve():
    torch = torch_cuda()
    probs = requests()
    outs, stats = serve(probs, calls=40)
    for p, out, s in zip(probs, outs, stats):
        P = red.Problem(red.config_for(p, ve="rre", ve_k=5), to_dev(p.y))
        ref = torch.empty((p.height, p.width), device="cuda")
        d = P.solve(to_dev(p.x0), ref, 40)
        assert s["fp_calls"] == d["fp_calls"] == 40
        assert s["ve_steps"] == d["ve_steps"]
        assert rel_l2(out, to_host(ref)) <= 1e-4


def test_server_alone_equals_mix():
    probs = requests()
    alone, _ = serve([probs[2]], calls=30)
    mix, _ = serve(probs, calls=30)
    assert np.array_equal(alone[0], mix[2])
    alone0, _ = serve([probs[0]], calls=30)
    assert np.array_equal(alone0[0], mix[0])


def test_server_ve_stop_tol_per_request():
    """Requests that end extrapolation by their own criterion (red_config::ve_stop_tol, the
    additional-iterations remark of Sec. III-C) share the server with requests of the same
    problem that do not, and with other problems: each matches the single-problem solve
    with its own setting, extrapolation count included, and the one that ended early made
    fewer extrapolations (three, ending at FP step 16 or 17 of 40)."""
    torch = torch_cuda()
    p = synth.deblur_small(7)
    jobs = [(p, 2.6e-3), (p, 0.0)] + [(q, 0.0) for q in requests()[1:3]]
    S = red.Server(4 * GIB, 8)
    outs, tickets = [], []
    for q, t in jobs:
        out = np.zeros((q.height, q.width), np.float32)
        cfg = red.config_for(q, ve="rre", ve_k=5, ve_stop_tol=t)
        tickets.append(S.submit(cfg, np.ascontiguousarray(q.y32), out, 40, 0.0))
        outs.append(out)
    stats = []
    for tk in tickets:
        st, s = S.wait(tk, 120000)
        assert st == red.RED_OK, red.status_string(st)
        stats.append(s)
    S.close()
    for (q, t), out, s in zip(jobs, outs, stats):
        P = red.Problem(red.config_for(q, ve="rre", ve_k=5, ve_stop_tol=t), to_dev(q.y))
        ref = torch.empty((q.height, q.width), device="cuda")
        d = P.solve(to_dev(q.x0), ref, 40)
        assert s["fp_calls"] == d["fp_calls"] == 40
        assert s["ve_steps"] == d["ve_steps"]
        assert rel_l2(out, to_host(ref)) <= 1e-4
    assert stats[0]["ve_steps"] == 3 < stats[1]["ve_steps"]


def test_server_groups_of_different_sizes_run_concurrently():
    """Requests of both tasks in several size classes (separate groups, streams and
    shared-memory footprints) all complete, and one of them equals its solve alone."""
    probs = [synth.sr_x3(40, 96), synth.sr_x3(41, 384), synth.deblur_gauss256(42, 128),
             synth.deblur_gauss256(43, 384), synth.sr_x3(44, 96), synth.deblur_gauss256(45, 768)]
    mix, stats = serve(probs, calls=20)
    assert all(s["fp_calls"] == 20 for s in stats)
    alone, _ = serve([probs[1]], calls=20)
    assert np.array_equal(alone[0], mix[1])
    for p, out in zip(probs, mix):
        assert np.isfinite(out).all()


def test_server_admission_under_tight_budget():
    """Budget for one 128x128 problem: requests of distinct shapes run one after the
    other (idle problems are freed to make room) and give the same results."""
    probs = [synth.deblur_gauss256(10, 128), synth.make_deblur(11, 128, 96, synth.uniform_psf(9), 2.0),
             synth.deblur_gauss256(12, 96)]
    fp = max(red.footprint(red.config_for(p, ve="rre", ve_k=5)) for p in probs)
    tight, _ = serve(probs, budget=fp + fp // 2, slots=4, calls=25)
    roomy, _ = serve(probs, budget=4 * GIB, slots=4, calls=25)
    for a, b in zip(tight, roomy):
        assert np.array_equal(a, b)


def test_server_tolerance_and_request_errors():
    p = synth.deblur_gauss256(20, 128)
    cfg = red.config_for(p, ve="rre", ve_k=5)
    fp = red.footprint(cfg)
    S = red.Server(4 * GIB, 2)
    # footprint above the budget, and an unsupported size, are refused at submission
    small = red.Server(fp // 2, 2)
    with pytest.raises(red.RedError) as e:
        small.submit(cfg, np.ascontiguousarray(p.y32), np.zeros((128, 128), np.float32), 10)
    assert e.value.status == red.RED_ENOMEM
    small.close()
    bad = red.make_config(task="deblur", height=100, width=100, psf=synth.uniform_psf(9))
    with pytest.raises(red.RedError) as e:
        S.submit(bad, np.zeros((100, 100), np.float32), np.zeros((100, 100), np.float32), 10)
    assert e.value.status in (red.RED_EINVAL, red.RED_EUNSUPPORTED)
    # a converging request stops before its budget; a zero-wait on a long one times out
    out = np.zeros((128, 128), np.float32)
    t1 = S.submit(cfg, np.ascontiguousarray(p.y32), out, 300, 1e-3)
    big = synth.deblur_gauss256(21, 512)
    out2 = np.zeros((512, 512), np.float32)
    t2 = S.submit(red.config_for(big, ve="rre", ve_k=5), np.ascontiguousarray(big.y32), out2, 300, 0.0)
    st, s = S.wait(t2, 0)
    assert st == red.RED_ETIMEOUT and s is None
    st, s = S.wait(t1, 120000)
    assert st == red.RED_OK and s["converged"] == 1 and s["fp_calls"] < 300
    assert s["rel_change"] < 1e-3
    st, s = S.wait(t2, 120000)
    assert st == red.RED_OK and s["fp_calls"] == 300
    st, s = S.poll(t2)
    assert st == red.RED_OK
    with pytest.raises(red.RedError):
        S.poll(12345)
    assert np.isfinite(out2).all() and float(np.abs(out2).max()) > 0
    S.close()


def test_server_shutdown_with_pending_requests():
    p = synth.deblur_gauss256(30, 256)
    cfg = red.config_for(p, ve="rre", ve_k=5)
    S = red.Server(4 * GIB, 1)
    outs = [np.zeros((256, 256), np.float32) for _ in range(4)]
    for o in outs:
        S.submit(cfg, np.ascontiguousarray(p.y32), o, 200, 0.0)
    S.close()   # drains the admitted request, fails the waiting ones, returns
