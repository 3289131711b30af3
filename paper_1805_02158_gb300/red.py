"""Thin ctypes binding of libred (include/red.h): same entry points, argument marshalling
only. Every computation runs in the CUDA library; there is no fallback. Importing this
module does not load the library; the first call does, and fails loudly if it is missing.

Tensors passed in must be contiguous float32 CUDA tensors (device pointers) unless a
function says host; streams default to torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libred.so")

RED_OK = 0
RED_EINVAL = 1
RED_ENOMEM = 2
RED_ECUDA = 3
RED_EVE_BREAKDOWN = 4
RED_ENOT_CONVERGED = 5
RED_ETIMEOUT = 6
RED_EBUSY = 7
RED_EUNSUPPORTED = 8

DEBLUR, SR = 0, 1
VE_NONE, VE_MPE, VE_RRE, VE_SVDMPE = 0, 1, 2, 3
F32, BF16, F16 = 0, 1, 2
PHASE_NLM, PHASE_FFT, PHASE_CG, PHASE_GRAM, PHASE_VESOLVE, PHASE_COMBINE = range(6)
VE_NAMES = {"none": VE_NONE, "mpe": VE_MPE, "rre": VE_RRE, "svdmpe": VE_SVDMPE}
STORAGE_NAMES = {"f32": F32, "bf16": BF16, "f16": F16}
BASE_FP, BASE_SD = 0, 1
BASELINE_NAMES = {"fp": BASE_FP, "sd": BASE_SD}


class Config(ctypes.Structure):
    _fields_ = [
        ("task", ctypes.c_int), ("height", ctypes.c_int), ("width", ctypes.c_int),
        ("scale", ctypes.c_int), ("psf", ctypes.POINTER(ctypes.c_float)),
        ("psf_h", ctypes.c_int), ("psf_w", ctypes.c_int),
        ("sigma", ctypes.c_double), ("alpha", ctypes.c_double),
        ("nlm_patch", ctypes.c_int), ("nlm_search", ctypes.c_int), ("nlm_h", ctypes.c_double),
        ("ve", ctypes.c_int), ("ve_k", ctypes.c_int), ("ve_m", ctypes.c_int),
        ("cg_iters", ctypes.c_int), ("storage", ctypes.c_int),
        ("baseline", ctypes.c_int), ("sd_mu", ctypes.c_double), ("ve_freeze", ctypes.c_int),
        ("ve_stop_tol", ctypes.c_double),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("fp_calls", ctypes.c_int), ("ve_steps", ctypes.c_int), ("ve_breakdowns", ctypes.c_int),
        ("converged", ctypes.c_int), ("rel_change", ctypes.c_double),
        ("sum_abs_gamma", ctypes.c_double), ("ms_total", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RedError(RuntimeError):
    def __init__(self, status, where, message):
        super().__init__(f"{where}: {status_string(status)} ({status}): {message}")
        self.status = status


_lib = None

_SIGS = {
    "red_config_default": (None, [ctypes.POINTER(Config)]),
    "red_create_problem": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "red_set_observation": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "red_destroy_problem": (ctypes.c_int, [ctypes.c_void_p]),
    "red_fp_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "red_denoise": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "red_ve_extrapolate": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "red_ve_extrapolate_static": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                                 ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                                 ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "red_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_void_p, ctypes.POINTER(Stats), ctypes.c_void_p]),
    "red_objective": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                     ctypes.c_void_p]),
    "red_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "red_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "red_batch_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                       ctypes.c_double, ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(Stats), ctypes.c_void_p]),
    "red_batch_solve_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Stats),
                                            ctypes.c_void_p]),
    "red_batch_set_phase_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "red_batch_phase_ms": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int)]),
    "red_batch_describe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]),
    "red_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "red_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Config), ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)]),
    "red_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(Stats)]),
    "red_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(Stats)]),
    "red_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "red_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "red_last_error": (ctypes.c_char_p, []),
    "red_problem_footprint": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_size_t)]),
    "red_kernel_launches": (ctypes.c_uint64, []),
    "red_measure_peaks": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_void_p]),
}


def lib():
    """Loads libred.so (built in-tree by paper_1805_02158_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libred.so not found at {LIB_PATH}: build it first "
                               "(python -m paper_1805_02158_gb300.build; needs nvcc for sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def measure_peaks(stream=None):
    """Measured FP32-FMA, EX2, FP64-FMA and packed f32x2-FMA throughputs (lane operations / s,
    whole device)."""
    a, b, c, d = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().red_measure_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                   ctypes.byref(d), _stream_ptr(stream)), "red_measure_peaks")
    return {"fp32_fma": a.value, "ex2": b.value, "fp64_fma": c.value, "fp32x2_fma": d.value}


def status_string(st: int) -> str:
    return lib().red_status_string(st).decode()


def _check(st: int, where: str, ok=(RED_OK,)):
    if st not in ok:
        raise RedError(st, where, lib().red_last_error().decode())
    return st


def kernel_launches() -> int:
    return int(lib().red_kernel_launches())


# ---------------------------------------------------------------------------------------
# tensor helpers
# ---------------------------------------------------------------------------------------

def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dptr(t, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("expected a contiguous float32 tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def make_config(task="deblur", height=64, width=64, scale=1, psf=None, sigma=2 ** 0.5,
                alpha=0.02, nlm_h=10.0, ve="rre", ve_k=5, ve_m=0, cg_iters=20,
                storage="f32", baseline="fp", sd_mu=0.0, ve_freeze=0, ve_stop_tol=0.0):
    """Builds a red_config; `psf` is a 2-D float array (kept referenced by the config).
    ve_stop_tol > 0 ends extrapolation at the first FP step whose relative change is below
    it; plain baseline steps follow."""
    import numpy as np
    c = Config()
    lib().red_config_default(ctypes.byref(c))
    psf = np.ascontiguousarray(np.asarray(psf, dtype=np.float32))
    c.task = DEBLUR if task in ("deblur", DEBLUR) else SR
    c.height, c.width, c.scale = int(height), int(width), int(scale)
    c.psf = psf.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    c.psf_h, c.psf_w = psf.shape
    c.sigma, c.alpha, c.nlm_h = float(sigma), float(alpha), float(nlm_h)
    c.ve = VE_NAMES[ve] if isinstance(ve, str) else int(ve)
    c.ve_k, c.ve_m, c.cg_iters = int(ve_k), int(ve_m), int(cg_iters)
    c.storage = STORAGE_NAMES[storage] if isinstance(storage, str) else int(storage)
    c.baseline = BASELINE_NAMES[baseline] if isinstance(baseline, str) else int(baseline)
    c.sd_mu, c.ve_freeze = float(sd_mu), int(ve_freeze)
    c.ve_stop_tol = float(ve_stop_tol)
    c._psf_keepalive = psf
    return c


def config_for(problem, **kw):
    """red_config for a synthetic problem (paper_1805_02158_gb300.synth.Problem)."""
    return make_config(task=problem.task, height=problem.height, width=problem.width,
                       scale=problem.scale, psf=problem.psf, sigma=problem.sigma,
                       alpha=problem.alpha, nlm_h=problem.nlm_h, **kw)


def footprint(cfg: Config) -> int:
    out = ctypes.c_size_t()
    _check(lib().red_problem_footprint(ctypes.byref(cfg), ctypes.byref(out)), "red_problem_footprint")
    return int(out.value)


def ve_extrapolate_static(xs, x_out, method="rre", stream=None):
    """red_ve_extrapolate_static: extrapolates device float32 vectors xs (x_m .. x_{m+kappa+1},
    same number of elements) into x_out without a problem handle and without allocating.
    Returns (status, gamma), gamma None on breakdown."""
    n = xs[0].numel()
    for t in list(xs) + [x_out]:
        if t.numel() != n:
            raise ValueError("all vectors must have the same number of elements")
    arr = (ctypes.c_void_p * len(xs))(*[_dptr(x).value for x in xs])
    gam = (ctypes.c_double * 16)()
    m = VE_NAMES[method]
    st = _check(lib().red_ve_extrapolate_static(arr, len(xs), n, m, _dptr(x_out), gam,
                                                _stream_ptr(stream)),
                "red_ve_extrapolate_static", ok=(RED_OK, RED_EVE_BREAKDOWN))
    if st == RED_EVE_BREAKDOWN:
        return st, None
    return st, [gam[i] for i in range(len(xs) - 1)]


class Problem:
    """A red_problem handle. `y` is a CUDA float32 tensor (LR size for SR)."""

    def __init__(self, cfg: Config, y, stream=None):
        self.cfg = cfg
        self.shape = (cfg.height, cfg.width)
        h = ctypes.c_void_p()
        _check(lib().red_create_problem(ctypes.byref(cfg), _dptr(y), _stream_ptr(stream),
                                        ctypes.byref(h)), "red_create_problem")
        self.handle = h

    def close(self):
        if self.handle:
            lib().red_destroy_problem(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_observation(self, y, stream=None):
        _check(lib().red_set_observation(self.handle, _dptr(y), 0, _stream_ptr(stream)),
               "red_set_observation")

    def fp_step(self, x_in, x_out, stream=None):
        _check(lib().red_fp_step(self.handle, _dptr(x_in, self.shape), _dptr(x_out, self.shape),
                                 _stream_ptr(stream)), "red_fp_step")

    def denoise(self, x, f_out, stream=None):
        _check(lib().red_denoise(self.handle, _dptr(x, self.shape), _dptr(f_out, self.shape),
                                 _stream_ptr(stream)), "red_denoise")

    def ve_extrapolate(self, xs, x_out, stream=None):
        """Returns (status, gamma) with gamma a list of kappa + 1 weights (None on breakdown)."""
        arr = (ctypes.c_void_p * len(xs))(*[_dptr(x, self.shape).value for x in xs])
        gam = (ctypes.c_double * 16)()
        st = _check(lib().red_ve_extrapolate(self.handle, arr, len(xs), _dptr(x_out, self.shape),
                                             gam, _stream_ptr(stream)), "red_ve_extrapolate",
                    ok=(RED_OK, RED_EVE_BREAKDOWN))
        if st == RED_EVE_BREAKDOWN:
            return st, None
        return st, [gam[i] for i in range(len(xs) - 1)]

    def solve(self, x0, x_out, max_fp_calls, rel_tol=0.0, stream=None):
        s = Stats()
        st = _check(lib().red_solve(self.handle, _dptr(x0, self.shape), int(max_fp_calls),
                                    float(rel_tol), _dptr(x_out, self.shape), ctypes.byref(s),
                                    _stream_ptr(stream)), "red_solve", ok=(RED_OK, RED_ENOT_CONVERGED))
        d = s.as_dict()
        d["status"] = st
        return d

    def objective(self, x, stream=None) -> float:
        e = ctypes.c_double()
        _check(lib().red_objective(self.handle, _dptr(x, self.shape), ctypes.byref(e),
                                   _stream_ptr(stream)), "red_objective")
        return float(e.value)


class Batch:
    """A red_batch over Problem objects (kept referenced)."""

    def __init__(self, problems):
        self.problems = list(problems)
        arr = (ctypes.c_void_p * len(self.problems))(*[p.handle.value for p in self.problems])
        h = ctypes.c_void_p()
        _check(lib().red_batch_create(arr, len(self.problems), ctypes.byref(h)), "red_batch_create")
        self.handle = h

    def close(self):
        if self.handle:
            lib().red_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, x0s, x_outs, max_fp_calls, rel_tol=0.0, stream=None):
        n = len(self.problems)
        a = (ctypes.c_void_p * n)(*[_dptr(x, p.shape).value for x, p in zip(x0s, self.problems)])
        b = (ctypes.c_void_p * n)(*[_dptr(x, p.shape).value for x, p in zip(x_outs, self.problems)])
        stats = (Stats * n)()
        st = _check(lib().red_batch_solve(self.handle, a, int(max_fp_calls), float(rel_tol), b, stats,
                                          _stream_ptr(stream)), "red_batch_solve",
                    ok=(RED_OK, RED_ENOT_CONVERGED))
        out = [s.as_dict() for s in stats]
        for d in out:
            d["status"] = st
        return out

    def describe(self):
        """The launch shapes the autotuner chose (dict)."""
        import json
        buf = ctypes.create_string_buffer(1024)
        _check(lib().red_batch_describe(self.handle, buf, 1024), "red_batch_describe")
        return json.loads(buf.value.decode())

    def set_phase_timing(self, enable=True):
        _check(lib().red_batch_set_phase_timing(self.handle, int(bool(enable))),
               "red_batch_set_phase_timing")

    def phase_ms(self, phase):
        """(mean ms of one launch of `phase` in the last cycle, launches averaged)."""
        ms = ctypes.c_double()
        n = ctypes.c_int()
        _check(lib().red_batch_phase_ms(self.handle, int(phase), ctypes.byref(ms), ctypes.byref(n)),
               "red_batch_phase_ms")
        return float(ms.value), int(n.value)

    def solve_host(self, y_hosts, x0_hosts, x_out_hosts, max_fp_calls, rel_tol=0.0, stream=None):
        """Host float32 buffers (C-contiguous numpy arrays or contiguous CPU tensors, pinned
        for asynchronous copies), one per problem: y (the observation, LR-sized for SR) or
        None to keep each problem's current y, x0 and x_out (HR-sized); copies run inside."""
        import numpy as np
        n = len(self.problems)

        def ptrs(xs, sizes, what):
            if len(xs) != n:
                raise ValueError(f"{what}: {len(xs)} buffers for {n} problems")
            out = []
            for x, want in zip(xs, sizes):
                if hasattr(x, "data_ptr"):
                    import torch
                    if (x.dtype != torch.float32 or not x.is_contiguous() or x.is_cuda
                            or x.numel() != want):
                        raise TypeError(f"{what}: expected contiguous float32 CPU tensors of "
                                        f"{want} elements")
                    out.append(x.data_ptr())
                else:
                    if not (isinstance(x, np.ndarray) and x.dtype == np.float32
                            and x.flags.c_contiguous and x.size == want):
                        raise TypeError(f"{what}: expected C-contiguous float32 arrays of "
                                        f"{want} elements")
                    out.append(x.ctypes.data)
            return (ctypes.c_void_p * n)(*out)

        hr = [P.cfg.height * P.cfg.width for P in self.problems]
        lr = [(P.cfg.height // P.cfg.scale) * (P.cfg.width // P.cfg.scale) for P in self.problems]
        ya = ptrs(y_hosts, lr, "y") if y_hosts is not None else None
        stats = (Stats * n)()
        st = _check(lib().red_batch_solve_host(self.handle, ya, ptrs(x0_hosts, hr, "x0"),
                                               int(max_fp_calls), float(rel_tol),
                                               ptrs(x_out_hosts, hr, "x_out"), stats,
                                               _stream_ptr(stream)), "red_batch_solve_host",
                    ok=(RED_OK, RED_ENOT_CONVERGED))
        return [s.as_dict() for s in stats]


class Server:
    """A red_server: requests (config + host observation) solved by a scheduler thread
    with continuous batching. Host buffers of pending requests are kept referenced."""

    def __init__(self, hbm_budget_bytes, max_slots):
        h = ctypes.c_void_p()
        _check(lib().red_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)),
               "red_server_create")
        self.handle = h
        self._keep = {}

    def submit(self, cfg, y_host, x_out_host, max_fp_calls, rel_tol=0.0):
        """y_host / x_out_host: C-contiguous float32 numpy arrays. Returns the ticket."""
        import numpy as np
        for a in (y_host, x_out_host):
            if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous):
                raise TypeError("expected C-contiguous float32 numpy arrays")
        t = ctypes.c_uint64()
        _check(lib().red_submit(self.handle, ctypes.byref(cfg), ctypes.c_void_p(y_host.ctypes.data),
                                ctypes.c_void_p(x_out_host.ctypes.data), int(max_fp_calls),
                                float(rel_tol), ctypes.byref(t)), "red_submit")
        self._keep[t.value] = (cfg, y_host, x_out_host)
        return t.value

    def poll(self, ticket):
        """(status, stats dict or None while RED_EBUSY)."""
        s = Stats()
        st = lib().red_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(s))
        if st == RED_EBUSY:
            return st, None
        if st == RED_EINVAL:
            _check(st, "red_poll")
        return st, s.as_dict()

    def wait(self, ticket, timeout_ms=-1):
        """(status, stats dict or None on RED_ETIMEOUT)."""
        s = Stats()
        st = lib().red_wait(self.handle, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(s))
        if st == RED_ETIMEOUT:
            return st, None
        if st == RED_EINVAL:
            _check(st, "red_wait")
        self._keep.pop(ticket, None)
        return st, s.as_dict()

    def close(self):
        if self.handle:
            lib().red_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
