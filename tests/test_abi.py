"""The C-ABI library builds, loads and exports every entry point include/red.h declares;
host-side validation and accounting work without a GPU (no compute is launched here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1805_02158_gb300 import build, red, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return red.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "red.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(red_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(red._SIGS), "binding and header disagree"


def test_config_default_matches_paper_settings(lib):
    c = red.Config()
    lib.red_config_default(ctypes.byref(c))
    assert (c.nlm_patch, c.nlm_search, c.nlm_h) == (5, 11, 10.0)
    assert (c.ve, c.ve_k, c.ve_m, c.cg_iters) == (red.VE_RRE, 5, 0, 20)
    assert abs(c.alpha - 0.02) < 1e-15 and abs(c.sigma - 2 ** 0.5) < 1e-15


def test_status_strings(lib):
    for st in range(9):
        assert red.status_string(st)


def test_footprint_is_host_side_and_grows_with_size(lib):
    small = red.footprint(red.make_config(height=64, width=64, psf=synth.uniform_psf(9)))
    big = red.footprint(red.make_config(height=256, width=256, psf=synth.uniform_psf(9)))
    assert big > 15 * small
    n = 256 * 256
    # iterate history (k + 2 slots) + denoiser output + spectra dominate
    assert big >= (5 + 2) * n * 4 + n * 4


@pytest.mark.parametrize("kw,status", [
    (dict(height=100, width=64), red.RED_EINVAL),          # not 2^a 3^b
    (dict(height=64, width=27), red.RED_EINVAL),           # odd width
    (dict(height=4, width=64), red.RED_EINVAL),            # too small
    (dict(sigma=0.0), red.RED_EINVAL),
    (dict(ve_k=13), red.RED_EINVAL),
    (dict(task="sr", scale=1), red.RED_EINVAL),
    (dict(ve=7), red.RED_EINVAL),                          # no such method
    (dict(storage=5), red.RED_EINVAL),                     # no such storage type
    (dict(ve_k=0), red.RED_EINVAL),                        # no U column
    (dict(ve_m=65), red.RED_EINVAL),                       # lead-in above 64
    (dict(ve_m=-1), red.RED_EINVAL),
    (dict(cg_iters=1001), red.RED_EINVAL),
    (dict(alpha=0.0), red.RED_EINVAL),                     # Eq. (4) needs alpha > 0
    (dict(nlm_h=0.0), red.RED_EINVAL),
    (dict(psf=np.ones((4, 4)) / 16), red.RED_EINVAL),      # even PSF: no centre tap
    (dict(height=8, width=8, psf=synth.uniform_psf(9)), red.RED_EINVAL),   # PSF > image
    (dict(height=4096, width=4096), red.RED_EINVAL),       # above the 2048 side limit
    (dict(baseline=5), red.RED_EINVAL),                    # no such baseline map
    (dict(baseline="sd", sd_mu=-1.0), red.RED_EINVAL),     # negative SD step size
    (dict(ve_freeze=-1), red.RED_EINVAL),
    (dict(ve="none", ve_freeze=1), red.RED_EINVAL),        # nothing to freeze
    (dict(ve_k=1, ve_m=0, ve_freeze=1), red.RED_EINVAL),   # a frozen cycle of 0 steps
    (dict(ve_stop_tol=-1e-3), red.RED_EINVAL),
    (dict(ve_stop_tol=float("nan")), red.RED_EINVAL),
    (dict(ve="none", ve_stop_tol=1e-3), red.RED_EINVAL),   # no extrapolation to end
    (dict(ve_freeze=2, ve_stop_tol=1e-3), red.RED_EINVAL), # frozen cycles keep no last iterate
])
def test_invalid_configs_rejected_before_any_gpu_work(lib, kw, status):
    base = dict(height=64, width=64, psf=synth.uniform_psf(9))
    base.update(kw)
    cfg = red.make_config(**base)
    out = ctypes.c_size_t()
    st = lib.red_problem_footprint(ctypes.byref(cfg), ctypes.byref(out))
    assert st == status
    assert red.lib().red_last_error()


def test_16_bit_storage_footprints(lib):
    """BF16 and FP16 histories take half the ring bytes of FP32 (k + 2 slots of 64 x 64)."""
    sizes = {}
    for st in ("f32", "bf16", "f16"):
        cfg = red.make_config(height=64, width=64, psf=synth.uniform_psf(9), storage=st)
        out = ctypes.c_size_t()
        assert lib.red_problem_footprint(ctypes.byref(cfg), ctypes.byref(out)) == red.RED_OK
        sizes[st] = out.value
    assert sizes["bf16"] == sizes["f16"] == sizes["f32"] - 7 * 64 * 64 * 2


@pytest.mark.parametrize("kw", [dict(baseline="sd"), dict(baseline="sd", sd_mu=1.5),
                                dict(ve_freeze=2), dict(baseline="sd", ve="mpe", ve_k=9),
                                dict(storage="f16", ve_freeze=1, ve_k=2),
                                dict(ve_stop_tol=1e-3), dict(baseline="sd", ve="mpe", ve_stop_tol=2e-3)])
def test_sd_and_frozen_configs_accepted(lib, kw):
    cfg = red.make_config(height=64, width=64, psf=synth.uniform_psf(9), **kw)
    out = ctypes.c_size_t()
    assert lib.red_problem_footprint(ctypes.byref(cfg), ctypes.byref(out)) == red.RED_OK


STRUCT_PROBE = r"""
#include <stddef.h>
#include <stdio.h>
#include "red.h"
#define F(T, f) printf(#T " " #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("red_config sizeof %zu\n", sizeof(red_config));
  printf("red_stats sizeof %zu\n", sizeof(red_stats));
  %FIELDS%
  return 0;
}
"""


def test_struct_layout_matches_binding(tmp_path):
    """Every field of red_config and red_stats sits at the same offset in the C header
    (compiled with gcc) and in the ctypes binding, and the sizes agree."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lines = []
    for T, cls in (("red_config", red.Config), ("red_stats", red.Stats)):
        lines += [f"F({T}, {name})" for name, _ in cls._fields_]
    src = tmp_path / "probe.c"
    src.write_text(STRUCT_PROBE.replace("%FIELDS%", "\n  ".join(lines)))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n"):
        if line.strip():
            T, f, v = line.split()
            got[(T, f)] = int(v)
    assert got[("red_config", "sizeof")] == ctypes.sizeof(red.Config)
    assert got[("red_stats", "sizeof")] == ctypes.sizeof(red.Stats)
    for T, cls in (("red_config", red.Config), ("red_stats", red.Stats)):
        for name, _ in cls._fields_:
            assert got[(T, name)] == getattr(cls, name).offset, (T, name)


def test_svdmpe_config_accepted(lib):
    cfg = red.make_config(height=64, width=64, psf=synth.uniform_psf(9), ve="svdmpe")
    out = ctypes.c_size_t()
    assert lib.red_problem_footprint(ctypes.byref(cfg), ctypes.byref(out)) == red.RED_OK
    assert out.value > 0


def test_unsupported_patch_size(lib):
    cfg = red.make_config(height=64, width=64, psf=synth.uniform_psf(9))
    cfg.nlm_patch = 7
    out = ctypes.c_size_t()
    assert lib.red_problem_footprint(ctypes.byref(cfg), ctypes.byref(out)) == red.RED_EUNSUPPORTED
