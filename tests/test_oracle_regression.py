"""The FP64 oracle against the fingerprints stored in tests/golden/oracle_regression.json
(written by tests/golden/make_oracle_regression.py from oracle/ only): a change to the
oracle's arithmetic changes these values and has to name the paper passage that justifies
it. Tolerance 1e-9 relative: FFT and BLAS rounding may differ between machines, never by
more than a few units in the 15th digit per operation."""
import json
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_oracle_regression as gen  # noqa: E402

STORED = {c["name"]: c for c in json.load(open(os.path.join(HERE, "golden", "oracle_regression.json")))["cases"]}


@pytest.mark.parametrize("case", gen.cases(), ids=lambda c: c[0])
def test_oracle_matches_stored_fingerprint(case):
    got = gen.fingerprint(*case)
    ref = STORED[got["name"]]
    for key in ("method", "m", "kappa", "calls", "freeze_after", "fp_calls", "ve_steps",
                "frozen_steps"):
        assert got[key] == ref[key], key
    assert got["sum"] == pytest.approx(ref["sum"], rel=1e-9)
    assert got["sum_sq"] == pytest.approx(ref["sum_sq"], rel=1e-9)
    assert got["samples"] == pytest.approx(ref["samples"], rel=1e-9, abs=1e-9)
    if ref["first_gamma"] is None:
        assert got["first_gamma"] is None
    else:
        assert got["first_gamma"] == pytest.approx(ref["first_gamma"], rel=1e-7, abs=1e-9)
