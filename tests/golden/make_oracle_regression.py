"""Writes tests/golden/oracle_regression.json: fingerprints of small solves of the FP64
oracle (Algorithm 3 around Eq. (7); SD-MPE; frozen-gamma cycling) on seeded synthetic
problems. The stored values come only from oracle/ and the input generators; the test
tests/test_oracle_regression.py recomputes them, so any change to the oracle's arithmetic
shows up there and has to be justified by the paper passage it follows.

Usage: python tests/golden/make_oracle_regression.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import fp, red, sd  # noqa: E402
from paper_1805_02158_gb300 import synth  # noqa: E402

SAMPLES = [(0, 0), (3, 5), (7, 11), (15, 2), (9, 14)]


def cases():
    """(name, problem, baseline map factory, method, m, kappa, calls, freeze_after)."""
    deb = synth.make_deblur(11, 16, 16, synth.uniform_psf(5), np.sqrt(2.0))
    srp = synth.make_sr(12, 24, 24, synth.gaussian_psf(7, 1.6), 3, 5.0)

    def fp_map(p):
        return fp.FPOperator(p.y, p.psf, (p.height, p.width), p.scale, p.sigma, p.alpha)

    def sd_map(p):
        return sd.SDOperator(p.y, p.psf, (p.height, p.width), p.scale, p.sigma, p.alpha)

    return [
        ("deblur16_fp", deb, fp_map, "none", 0, 4, 12, None),
        ("deblur16_rre_k4", deb, fp_map, "rre", 0, 4, 12, None),
        ("deblur16_mpe_m2_k3", deb, fp_map, "mpe", 2, 3, 14, None),
        ("deblur16_svdmpe_k4", deb, fp_map, "svdmpe", 0, 4, 12, None),
        ("sr24_rre_k4", srp, fp_map, "rre", 0, 4, 11, None),
        ("deblur16_sd_mpe_k8", deb, sd_map, "mpe", 0, 8, 20, None),
        ("deblur16_rre_frozen", deb, fp_map, "rre", 0, 3, 14, 1),
    ]


def fingerprint(name, p, make, method, m, kappa, calls, freeze_after):
    x, st = red.solve(make(p), p.x0, method, m=m, kappa=kappa, max_calls=calls,
                      freeze_after=freeze_after)
    return {"name": name, "method": method, "m": m, "kappa": kappa, "calls": calls,
            "freeze_after": freeze_after, "fp_calls": st["fp_calls"],
            "ve_steps": st["ve_steps"], "frozen_steps": st["frozen_steps"],
            "sum": float(x.sum()), "sum_sq": float((x * x).sum()),
            "samples": [float(x[i % x.shape[0], j % x.shape[1]]) for i, j in SAMPLES],
            "first_gamma": [float(g) for g in st["gammas"][0]] if st["gammas"] else None}


def compute():
    return [fingerprint(*c) for c in cases()]


if __name__ == "__main__":
    out = {"_source": "written by tests/golden/make_oracle_regression.py from oracle/ only",
           "cases": compute()}
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(f"wrote {len(out['cases'])} cases")
