"""The packed-FP32 NLM kernel (k_nlm_x2, selected by RED_NLM_F32X2=1) against the scalar
kernel and the FP64 oracle. Each kernel runs in its own process (the switch is read once per process) on
the same seeded images, through red_denoise and through a short batched solve; the two
must agree bit for bit (same operations in the same order), and the packed one must meet
the NLM parity bars against the oracle (max |diff| <= 2e-3 on [0, 255], rel. L2 <= 1e-5)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from helpers import f32, rel_l2

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1805_02158_gb300 import red, synth
out = sys.argv[2]
shapes = [(8, 8), (48, 72), (64, 64), (144, 192), (256, 256)]
res = {}
for i, (h, w) in enumerate(shapes):
    psf = synth.uniform_psf(3) if h == 8 else synth.uniform_psf(9)
    p = synth.make_deblur(i, h, w, psf, 2 ** 0.5)
    y = torch.from_numpy(p.y.astype(np.float32)).cuda()
    P = red.Problem(red.config_for(p), y)
    f = torch.empty_like(y)
    P.denoise(y, f)
    np.save(f"{out}/f_{h}x{w}.npy", f.cpu().numpy())
probs = [synth.deblur_gauss256(s, 256) for s in range(3)]
ys = [torch.from_numpy(q.y.astype(np.float32)).cuda() for q in probs]
B = red.Batch([red.Problem(red.config_for(q, ve="rre", ve_k=5), y) for q, y in zip(probs, ys)])
outs = [torch.empty_like(y) for y in ys]
B.solve([y.clone() for y in ys], outs, 12, 0.0)
for s, o in enumerate(outs):
    np.save(f"{out}/solve_{s}.npy", o.cpu().numpy())
print(json.dumps({"ok": True}))
"""


def run_child(tmp, packed):
    env = dict(os.environ)
    env.pop("RED_NLM_F32X2", None)
    # one tuning cache for both processes: the same launch shapes (the Fourier paths agree
    # only to rounding, so a different autotuned choice would break bit equality)
    env["RED_TUNE_CACHE"] = str(tmp.parent / "tune_cache.txt")
    if packed:
        env["RED_NLM_F32X2"] = "1"
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(tmp)], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]


def test_packed_nlm_equals_scalar_and_meets_parity(tmp_path):
    from oracle.nlm import nlm
    from paper_1805_02158_gb300 import synth
    a, b = tmp_path / "scalar", tmp_path / "packed"
    a.mkdir()
    b.mkdir()
    run_child(a, False)
    run_child(b, True)
    names = sorted(os.listdir(a))
    assert names == sorted(os.listdir(b)) and len(names) == 8
    for n in names:
        assert np.array_equal(np.load(a / n), np.load(b / n)), n
    for i, (h, w) in enumerate([(8, 8), (48, 72), (64, 64)]):
        psf = synth.uniform_psf(3) if h == 8 else synth.uniform_psf(9)
        p = synth.make_deblur(i, h, w, psf, 2 ** 0.5)
        ref = nlm(f32(p.y))
        got = np.load(b / f"f_{h}x{w}.npy").astype(np.float64)
        assert np.abs(got - ref).max() <= 2e-3
        assert rel_l2(got, ref) <= 1e-5
