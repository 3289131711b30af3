"""Host logic of bench.py's call-count studies (Table I's criterion and the (m, kappa) grid
of Fig. 4), run on the CPU against a fake binding whose solves approach the ground truth
at a known rate, so that the calls each variant needs are known in closed form."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class FakeTensor:
    def __init__(self, a):
        self.a = np.array(a, dtype=np.float32)

    def cuda(self):
        return self

    def cpu(self):
        return self

    def numpy(self):
        return self.a


class FakeTorch:
    @staticmethod
    def from_numpy(a):
        return FakeTensor(a)

    @staticmethod
    def empty_like(x):
        return FakeTensor(np.zeros_like(x.a))


def speed(cfg):
    """Error after c calls is 64 / (c * speed): plain FP 1, extrapolation 2 + m/5 + kappa/10
    (MPE), and half of that for RRE and SVD-MPE."""
    if cfg["ve"] == "none":
        return 1.0
    s = 2.0 + cfg["ve_m"] / 5 + (cfg["ve_k"] - 1) / 10
    return s if cfg["ve"] == "mpe" else s / 2


class FakeRed:
    def __init__(self):
        self.truth = {}
        self.solves = 0

    def config_for(self, p, ve="rre", ve_k=5, ve_m=0):
        return {"ve": ve, "ve_k": ve_k, "ve_m": ve_m, "id": id(p)}

    def Problem(self, cfg, y):   # noqa: N802 (mirrors the binding's class)
        red = self

        class P:
            def __init__(self):
                self.cfg = cfg

            def objective(self, o):
                return float(np.mean((o.a - red.truth[cfg["id"]]) ** 2))
        return P()

    def Batch(self, Ps):   # noqa: N802
        red = self

        class B:
            def solve(self, x0s, outs, calls, tol):
                # error 64 / (calls * speed); fixed-point residual 1 / (calls * speed)
                red.solves += 1
                stats = []
                for P, o in zip(Ps, outs):
                    t = red.truth[P.cfg["id"]]
                    o.a = (t + 64.0 / (max(calls, 1) * speed(P.cfg))).astype(np.float32)
                    stats.append({"rel_change": 1.0 / (max(calls, 1) * speed(P.cfg)),
                                  "fp_calls": calls})
                return stats
        return B()


def problems(n):
    from paper_1805_02158_gb300 import synth
    return [synth.make_sr(s, 48, 48, synth.gaussian_psf(7, 1.6), 3, 5.0) for s in range(n)]


def register(fake, probs):
    for p in probs:
        fake.truth[id(p)] = p.x_true.astype(np.float32)


def test_ve_vs_fp_study_counts_calls_in_steps_of_five():
    fake = FakeRed()
    probs = problems(2)
    register(fake, probs)
    out = bench.ve_vs_fp_study(probs, None, FakeTorch, fake, (("rre", 5), ("mpe", 5)))
    # plain FP's error after 200 calls is 64/200; MPE (speed 2.4) reaches it at 200/2.4
    # -> 85 calls (first multiple of 5 above 83.3); RRE (speed 1.2) at 170
    mpe, rre = out["variants"]["mpe_k5"], out["variants"]["rre_k5"]
    assert mpe["calls_to_fp200_cost"] == [85, 85] and mpe["calls_to_fp200_psnr"] == [85, 85]
    assert rre["calls_to_fp200_cost"] == [170, 170] and rre["cost_reached"] == 2
    assert out["rre_calls_to_fp200_cost_mean"] == 170.0
    # the residual criterion: plain FP's residual after 200 calls is 1/200, reached at the
    # same budgets; the traces hold the mean residual at 5, 25, 45, ... calls
    assert mpe["calls_to_fp200_residual"] == [85, 85] and rre["residual_reached"] == 2
    assert out["rre_calls_to_fp200_residual_mean"] == 170.0
    np.testing.assert_allclose(out["fp_residual_every20_calls_mean"],
                               [1.0 / c for c in range(5, 201, 20)])
    np.testing.assert_allclose(mpe["residual_every20_calls_mean"],
                               [1.0 / (2.4 * c) for c in range(5, 201, 20)])


def test_m_kappa_sweep_grid_and_best_pair(monkeypatch):
    fake = FakeRed()
    from paper_1805_02158_gb300 import synth
    made = {}

    def sr_x3(seed, side=256):
        if seed not in made:
            made[seed] = synth.make_sr(seed, 48, 48, synth.gaussian_psf(7, 1.6), 3, 5.0)
            register(fake, [made[seed]])
        return made[seed]
    monkeypatch.setattr(synth, "sr_x3", sr_x3)
    out = bench.mk_sweep_study(FakeTorch, fake, seeds=(0, 1), methods=("mpe", "rre"),
                               ms=(0, 10), kappas=(3, 10))
    assert set(out["grid"]) == {f"{v}_m{m}_kappa{k}" for v in ("mpe", "rre")
                                for m in (0, 10) for k in (3, 10)}
    for key, row in out["grid"].items():
        method, m, kappa = key.split("_")
        s = speed({"ve": method, "ve_m": int(m[1:]), "ve_k": int(kappa[5:]) + 1})
        need = int(np.ceil(200 / s / 5 - 1e-9) * 5)
        reach = need if need <= 200 else None
        assert row["calls_to_fp200_cost"] == [reach, reach], key
        # objective after 200 calls relative to plain FP's: (1/s)^2
        np.testing.assert_allclose(row["objective_at_200_over_fp"], [1 / s ** 2] * 2, rtol=1e-4)
    # the fastest pair of each method is the largest m and kappa of the grid
    assert (out["best_pair"]["mpe"]["m"], out["best_pair"]["mpe"]["kappa"]) == (10, 10)
    assert (out["best_pair"]["rre"]["m"], out["best_pair"]["rre"]["kappa"]) == (10, 10)
    # the slowest pair (RRE, m = 0, kappa = 3: speed 1.15) still reaches it, at 175 calls
    assert out["grid"]["rre_m0_kappa3"]["calls_to_fp200_cost"] == [175, 175]


def test_clock_sampler_starts_sampling_before_the_timed_region(tmp_path, monkeypatch):
    """The sampler returns from start() only once nvidia-smi has written its first sample
    (its start-up stays out of the timed steps), and stop() reads the median clock and the
    active throttle reasons from the samples. A fake nvidia-smi on PATH stands in for the
    real one: it starts after 0.3 s, then writes one line every 50 ms."""
    import stat
    import time
    fake = tmp_path / "bin" / "nvidia-smi"
    fake.parent.mkdir()
    fake.write_text("#!/bin/sh\nsleep 0.3\n"
                    "while true; do\n"
                    "  echo '0, 1965, 2070, 900.1, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "  sleep 0.05\n"
                    "done\n")
    fake.chmod(fake.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(fake.parent) + os.pathsep + os.environ.get("PATH", ""))
    monkeypatch.setenv("RED_CLOCKS_DIR", str(tmp_path / "clocks"))
    s = bench.ClockSampler(0)
    t0 = time.time()
    s.start()
    assert time.time() - t0 >= 0.25
    assert os.path.getsize(s.path) > 0
    time.sleep(0.2)
    c = s.stop()
    assert c["sm_mhz"] == 1965.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] >= 2
