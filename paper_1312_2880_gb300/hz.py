"""Python binding of the C ABI in ``include/hz.h``: argument marshalling only.

Every step of the solver runs in ``libhz.so``; this module only converts between torch/numpy
arrays and the library's pointers. It raises if the library is missing: there is no fallback.
Device arrays are ``torch.complex128`` CUDA tensors of shape ``(n+1, n+1)`` indexed ``[j, i]``.
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, byref, c_double, c_int, c_size_t, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhz.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "hz.h")

HZ_OK, HZ_EINVAL, HZ_ENOMEM, HZ_ECUDA, HZ_ENOTSETUP, HZ_EBREAKDOWN, HZ_EMAXIT, HZ_ENONFINITE, HZ_ETIMEOUT = range(9)
VARIANTS = {"hyb": 0, "sl": 1, "hlm": 2, "sl_plain": 3}
PRECISIONS = {"fp64": 0, "fp32": 1}
OPS = {"L": 0, "M": 1}
SMOOTHERS = {0: "gs", 1: "kaczmarz", 2: "direct", 3: "jacobi", 4: "sor"}
GS_SMOOTHERS = {"gs": 0, "jacobi": 3, "sor": 4}


class HzError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("levels", c_int), ("variant", c_int), ("precision", c_int), ("nu_gs", c_int),
                ("nu_kacz", c_int), ("guard", c_int), ("k_ref", c_double), ("batch", c_int),
                ("pass_variant", c_int), ("coarse_tail", c_int), ("kacz_form", c_int),
                ("gs_smoother", c_int), ("omega", c_double), ("kacz_rule", c_int)]


class LevelInfo(ctypes.Structure):
    _fields_ = [("n", c_int), ("H", c_double), ("relax_op", c_int), ("smoother", c_int), ("resid_op", c_int),
                ("nu", c_int), ("pass_down", c_int), ("pass_up", c_int), ("in_tail", c_int),
                ("kacz_form", c_int)]


class KernelTime(ctypes.Structure):
    _fields_ = [("kernel", c_int), ("level", c_int), ("ms", ctypes.c_float)]


class RayInfo(ctypes.Structure):
    _fields_ = [("m", c_int), ("nc", c_int), ("unknowns", c_int), ("kH", c_double), ("bytes", c_size_t),
                ("setup_ms", c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", c_double), ("relres_true", c_double), ("history_len", c_int), ("status", c_int),
                ("restarts", c_int)]


_LIB = None


def header_functions() -> list[str]:
    """Names of the functions ``include/hz.h`` declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hz_[a-z0-9_]+)\s*\(", txt)))


def lib() -> ctypes.CDLL:
    """Load ``libhz.so`` (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1312_2880_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    dp = POINTER(c_double)
    sig = {
        "hz_default_opts": (None, [POINTER(Opts)]),
        "hz_create_problem": (c_int, [c_int, dp, c_double, c_int, POINTER(c_void_p)]),
        "hz_set_stream": (c_int, [P, c_void_p]),
        "hz_footprint_bytes": (c_size_t, [c_int, POINTER(Opts)]),
        "hz_setup_hierarchy": (c_int, [P, POINTER(Opts), c_void_p, c_size_t]),
        "hz_describe_hierarchy": (c_int, [P, POINTER(Opts), POINTER(LevelInfo), c_int]),
        "hz_num_levels": (c_int, [P]),
        "hz_get_level_info": (c_int, [P, c_int, POINTER(LevelInfo)]),
        "hz_vcycle": (c_int, [P, c_void_p, c_void_p]),
        "hz_solve": (c_int, [P, c_void_p, c_void_p, c_double, c_int, dp, c_int, POINTER(SolveInfo)]),
        "hz_solve_host": (c_int, [P, c_void_p, c_void_p, c_double, c_int, dp, c_int, POINTER(SolveInfo)]),
        "hz_solve_batch": (c_int, [P, c_void_p, c_void_p, c_double, c_int, POINTER(SolveInfo)]),
        "hz_solve_start": (c_int, [P, c_void_p, c_void_p, c_double, c_int]),
        "hz_solve_poll": (c_int, [P, POINTER(c_int)]),
        "hz_solve_finish": (c_int, [P, dp, c_int, POINTER(SolveInfo)]),
        "hz_apply": (c_int, [P, c_int, c_void_p, c_void_p]),
        "hz_level_presmooth": (c_int, [P, c_int, c_void_p, c_void_p, c_void_p]),
        "hz_level_postsmooth": (c_int, [P, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
        "hz_level_sweeps": (c_int, [P, c_int, c_void_p, c_void_p, c_int, c_int]),
        "hz_coarse_solve": (c_int, [P, c_void_p, c_void_p]),
        "hz_profile_iteration": (c_int, [P, c_void_p, c_void_p, c_int, POINTER(KernelTime), c_int]),
        "hz_profile_graph": (c_int, [P, c_void_p, c_void_p, c_int, POINTER(KernelTime), c_int]),
        "hz_krylov_scalars": (c_int, [P, c_int, POINTER(c_double)]),
        "hz_set_stall_detection": (c_int, [P, c_double, c_double, c_int]),
        "hz_kernel_name": (ctypes.c_char_p, [c_int]),
        "hz_last_error": (ctypes.c_char_p, [P]),
        "hz_status_string": (ctypes.c_char_p, [c_int]),
        "hz_destroy": (None, [P]),
        "hz_apply_dot_noalloc": (c_int, [c_int, c_void_p, c_double, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
        "hz_group_create": (c_int, [POINTER(c_void_p), c_int, POINTER(c_void_p)]),
        "hz_group_solve": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_void_p), c_double, c_int, POINTER(SolveInfo)]),
        "hz_group_last_error": (ctypes.c_char_p, [c_void_p]),
        "hz_group_destroy": (None, [c_void_p]),
        "hz_measure_fp64_rate": (c_int, [c_int, c_void_p, dp, dp]),
        "hz_ray_footprint_bytes": (c_size_t, [c_int, c_double, c_int]),
        "hz_ray_create": (c_int, [P, c_double, c_int, c_void_p, c_size_t, POINTER(c_void_p)]),
        "hz_cycle_scratch_bytes": (c_size_t, [c_int]),
        "hz_ray_spacing": (c_int, [c_int, c_double]),
        "hz_ray_get_info": (c_int, [c_void_p, POINTER(RayInfo)]),
        "hz_ray_restrict": (c_int, [c_void_p, c_void_p, c_void_p]),
        "hz_ray_coarse_solve": (c_int, [c_void_p, c_void_p, c_void_p]),
        "hz_ray_blocks": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
        "hz_ray_correct": (c_int, [c_void_p, c_void_p, c_void_p]),
        "hz_ray_destroy": (None, [c_void_p]),
        "hz_cycle_solve": (c_int, [P, c_void_p, c_void_p, c_void_p, c_double, c_int, c_void_p, c_size_t, dp, c_int,
                                   POINTER(SolveInfo)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def measure_fp64_rate(iters=(1 << 10, 1 << 12, 1 << 14)) -> dict:
    """FP64 FMA throughput of the current device in TFLOP/s (hz_measure_fp64_rate), on torch's
    current stream: the best over the given chain lengths (short launches see the burst clock, as
    the solver's sub-millisecond Krylov kernels do)."""
    import torch

    best = None
    for it in ([iters] if isinstance(iters, int) else iters):
        tf, ms = c_double(), c_double()
        st = lib().hz_measure_fp64_rate(int(it), c_void_p(torch.cuda.current_stream().cuda_stream), byref(tf),
                                        byref(ms))
        if st != HZ_OK:
            raise HzError(st, "hz_measure_fp64_rate failed")
        if best is None or tf.value > best["tflops"]:
            best = {"tflops": tf.value, "ms": ms.value, "iters": int(it)}
    return best


def _ptr(t) -> c_void_p:
    import torch

    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() and t.dtype == torch.complex128, (
        "expected a contiguous complex128 CUDA tensor")
    return c_void_p(t.data_ptr())


KACZ_FORMS = {"auto": -1, "colour": 0, "level": 1, "tile": 2, "cluster": 3, "grid": 4}
KACZ_RULES = {"band": 0, "bins": 1}


def make_opts(variant="hyb", precision="fp64", levels=0, nu_gs=1, nu_kacz=4, guard=True, k_ref=0.0, batch=1,
              pass_variant=-1, coarse_tail=True, kacz_form="auto", gs_smoother="gs", omega=0.0,
              kacz_rule="band") -> Opts:
    """pass_variant: -1 = fused-pass form picked per level by the tile autotuner at setup; 0 = shared-
    memory tiles; 1..8 = register streaming with 2**v rows per warp (FP32 form).
    kacz_form: kernel form of the Kaczmarz levels below the finest (one of KACZ_FORMS); a form that
    does not apply to a level falls back to the default.
    gs_smoother: "gs" (red-black Gauss-Seidel), "jacobi" (damped) or "sor" (red-black, over-relaxed)
    on the levels the rules give Gauss-Seidel; omega: their factor (0 = 0.8 Jacobi, 1 SOR).
    kacz_rule: "band" (every level with some node's k(x) H in [0.625 sqrt 2, 2 sqrt 2) relaxes by
    Kaczmarz) or "bins" (only the level whose k_ref H is in the kH ~ 1.25 bin)."""
    o = Opts()
    lib().hz_default_opts(byref(o))
    o.levels, o.variant, o.precision = levels, VARIANTS[variant], PRECISIONS[precision]
    o.nu_gs, o.nu_kacz, o.guard, o.k_ref, o.batch = nu_gs, nu_kacz, int(bool(guard)), float(k_ref), int(batch)
    o.pass_variant = int(pass_variant)
    o.coarse_tail = int(bool(coarse_tail))
    o.kacz_form = KACZ_FORMS[kacz_form]
    o.gs_smoother = GS_SMOOTHERS[gs_smoother]
    o.omega = float(omega)
    o.kacz_rule = KACZ_RULES[kacz_rule]
    return o


def footprint_bytes(n: int, **opts) -> int:
    return int(lib().hz_footprint_bytes(n, byref(make_opts(**opts))))


def _level_dict(li: LevelInfo) -> dict:
    inv = {v: k for k, v in OPS.items()}
    return {"n": li.n, "H": li.H, "relax_op": inv[li.relax_op], "smoother": SMOOTHERS[li.smoother],
            "resid_op": inv[li.resid_op], "nu": li.nu, "pass_down": li.pass_down, "pass_up": li.pass_up,
            "in_tail": bool(li.in_tail),
            "kacz_form": {v: k for k, v in KACZ_FORMS.items()}.get(li.kacz_form) if li.kacz_form >= 0 else None}


def describe_hierarchy(n: int, kfield, beta: float = 0.5, **opts) -> list:
    """Level schedule the library builds for this medium and these options, computed on the host
    (no GPU needed)."""
    L = lib()
    k = np.ascontiguousarray(kfield, dtype=np.float64)
    h = c_void_p()
    st = L.hz_create_problem(int(n), k.ctypes.data_as(POINTER(c_double)), float(beta), 0, byref(h))
    if st != HZ_OK:
        raise HzError(st, "hz_create_problem failed")
    try:
        out = (LevelInfo * 32)()
        cnt = L.hz_describe_hierarchy(h, byref(make_opts(**opts)), out, 32)
        if cnt < 0:
            raise HzError(HZ_EINVAL, "invalid hierarchy options")
        return [_level_dict(out[i]) for i in range(cnt)]
    finally:
        L.hz_destroy(h)


class Problem:
    """One Helmholtz problem (grid, medium, hierarchy) resident on the current CUDA device.

    Device memory is a single ``torch.uint8`` arena of :func:`footprint_bytes` bytes; work is
    ordered on torch's current stream.
    """

    def __init__(self, n: int, kfield, beta: float = 0.5, *, variant="hyb", precision="fp64", levels=0, nu_gs=1,
                 nu_kacz=4, guard=True, k_ref=0.0, batch=1, arena=None, pass_variant=-1, coarse_tail=True,
                 kacz_form="auto", gs_smoother="gs", omega=0.0, kacz_rule="band"):
        import torch

        L = lib()
        self.n = int(n)
        k = np.ascontiguousarray(kfield, dtype=np.float64)
        if k.shape != (n + 1, n + 1):
            raise ValueError("kfield must have shape (n+1, n+1)")
        h = c_void_p()
        st = L.hz_create_problem(self.n, k.ctypes.data_as(POINTER(c_double)), float(beta), 0, byref(h))
        if st != HZ_OK:
            raise HzError(st, "hz_create_problem failed")
        self._h = h
        self.opts = make_opts(variant, precision, levels, nu_gs, nu_kacz, guard, k_ref, batch, pass_variant,
                              coarse_tail, kacz_form, gs_smoother, omega, kacz_rule)
        self.batch = int(batch)
        self.precision = precision
        self.bytes = int(L.hz_footprint_bytes(self.n, byref(self.opts)))
        if self.bytes == 0:
            raise HzError(HZ_EINVAL, "invalid grid/level combination")
        self.arena = arena if arena is not None else torch.empty(self.bytes, dtype=torch.uint8, device="cuda")
        self._stream()
        self._check(L.hz_setup_hierarchy(h, byref(self.opts), c_void_p(self.arena.data_ptr()), self.bytes))

    # ------------------------------------------------------------------ plumbing
    def _stream(self):
        import torch

        lib().hz_set_stream(self._h, c_void_p(torch.cuda.current_stream().cuda_stream))

    def _check(self, st: int, ok=(HZ_OK,)):
        if st not in ok:
            raise HzError(st, lib().hz_last_error(self._h).decode())
        return st

    def _empty(self, level: int = 0):
        import torch

        m = (self.n >> level) + 1
        return torch.empty((m, m), dtype=torch.complex128, device="cuda")

    def close(self):
        if getattr(self, "_h", None):
            lib().hz_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ queries
    @property
    def num_levels(self) -> int:
        return int(lib().hz_num_levels(self._h))

    def level_info(self, level: int) -> dict:
        li = LevelInfo()
        self._check(lib().hz_get_level_info(self._h, level, byref(li)))
        return _level_dict(li)

    def schedule(self) -> list:
        return [self.level_info(l) for l in range(self.num_levels)]

    # ------------------------------------------------------------------ solver
    def solve(self, rhs, tol: float = 1e-6, maxit: int = 1000, x=None, history_cap: int = 4096,
              allow_fail: bool = False):
        """Bi-CGSTAB solve of L^h x = rhs on the device. Returns (x, info dict, history ndarray)."""
        self._stream()
        x = self._empty() if x is None else x
        hist = np.zeros(max(1, history_cap), dtype=np.float64)
        info = SolveInfo()
        st = lib().hz_solve(self._h, _ptr(rhs), _ptr(x), tol, maxit, hist.ctypes.data_as(POINTER(c_double)),
                            history_cap, byref(info))
        ok = (HZ_OK, HZ_EMAXIT, HZ_EBREAKDOWN, HZ_ENONFINITE) if allow_fail else (HZ_OK,)
        self._check(st, ok)
        d = {"iterations": info.iterations, "relres_true": info.relres_true, "status": st,
             "restarts": info.restarts}
        return x, d, hist[: info.history_len].copy()

    def cycle_solve(self, rhs, ray=None, tol: float = 1e-7, maxc: int = 100, x=None, history_cap: int = 1024,
                    allow_fail: bool = False):
        """Table 7's stand-alone solver (hz_cycle_solve): V-cycle, then the ray correction of ``ray``
        (a :class:`Ray` of this problem, or None) per cycle. Returns (x, info dict, history ndarray)."""
        import torch

        self._stream()
        x = self._empty() if x is None else x
        nb = int(lib().hz_cycle_scratch_bytes(self.n))
        if getattr(self, "_cycle_scratch", None) is None or self._cycle_scratch.numel() < nb:
            self._cycle_scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
        hist = np.zeros(max(1, history_cap), dtype=np.float64)
        info = SolveInfo()
        st = lib().hz_cycle_solve(self._h, ray._h if ray is not None else None, _ptr(rhs), _ptr(x), tol, maxc,
                                  c_void_p(self._cycle_scratch.data_ptr()), nb,
                                  hist.ctypes.data_as(POINTER(c_double)), history_cap, byref(info))
        self._check(st, (HZ_OK, HZ_EMAXIT, HZ_ENONFINITE) if allow_fail else (HZ_OK,))
        d = {"cycles": int(info.iterations), "relres_true": info.relres_true, "status": st}
        return x, d, hist[: info.history_len].copy()

    def solve_batch(self, rhs, tol: float = 1e-6, maxit: int = 1000, x=None, allow_fail: bool = False):
        """All `batch` right-hand sides at once: rhs is a (batch, n+1, n+1) complex128 CUDA tensor.
        Returns (x, list of info dicts)."""
        import torch

        self._stream()
        m = self.n + 1
        assert tuple(rhs.shape) == (self.batch, m, m)
        x = torch.empty_like(rhs) if x is None else x
        infos = (SolveInfo * self.batch)()
        st = lib().hz_solve_batch(self._h, _ptr(rhs), _ptr(x), tol, maxit, infos)
        ok = (HZ_OK, HZ_EMAXIT, HZ_EBREAKDOWN, HZ_ENONFINITE) if allow_fail else (HZ_OK,)
        self._check(st, ok)
        return x, [{"iterations": i.iterations, "relres_true": i.relres_true, "status": i.status,
                    "restarts": i.restarts} for i in infos]

    # ---- non-blocking solve (serving)
    def solve_start(self, rhs, x, tol: float = 1e-6, maxit: int = 1000):
        """Queue a solve and return at once; keep `rhs` and `x` alive until :meth:`solve_finish`."""
        self._stream()
        self._pending = (rhs, x)
        self._check(lib().hz_solve_start(self._h, _ptr(rhs), _ptr(x), tol, maxit))

    def solve_poll(self) -> bool:
        """True once the solve in flight has stopped; never waits."""
        done = c_int(0)
        self._check(lib().hz_solve_poll(self._h, byref(done)))
        return bool(done.value)

    def solve_finish(self, history_cap: int = 4096, allow_fail: bool = False):
        """Wait for the solve in flight; returns (x, info dict, history)."""
        self._stream()
        hist = np.zeros(max(1, history_cap), dtype=np.float64)
        info = SolveInfo()
        st = lib().hz_solve_finish(self._h, hist.ctypes.data_as(POINTER(c_double)), history_cap, byref(info))
        ok = (HZ_OK, HZ_EMAXIT, HZ_EBREAKDOWN, HZ_ENONFINITE) if allow_fail else (HZ_OK,)
        self._check(st, ok)
        x = self._pending[1]
        self._pending = None
        return x, {"iterations": info.iterations, "relres_true": info.relres_true, "status": st,
                   "restarts": info.restarts}, hist[: info.history_len].copy()

    def solve_host(self, rhs: np.ndarray, tol: float = 1e-6, maxit: int = 1000, history_cap: int = 4096,
                   out: np.ndarray | None = None):
        """As :meth:`solve` with host (numpy complex128) input and output."""
        self._stream()
        rhs = np.ascontiguousarray(rhs, dtype=np.complex128)
        x = np.empty_like(rhs) if out is None else out
        hist = np.zeros(max(1, history_cap), dtype=np.float64)
        info = SolveInfo()
        st = lib().hz_solve_host(self._h, c_void_p(rhs.ctypes.data), c_void_p(x.ctypes.data), tol, maxit,
                                 hist.ctypes.data_as(POINTER(c_double)), history_cap, byref(info))
        self._check(st)
        return x, {"iterations": info.iterations, "relres_true": info.relres_true, "status": st,
                   "restarts": info.restarts}, hist[: info.history_len].copy()

    def profile_iteration(self, rhs, iterations: int = 1, x=None, graph: bool = False) -> list:
        """Per-launch device times (ms) of `iterations` Bi-CGSTAB iterations: [(kernel, level, ms)].
        graph=True: measured inside one CUDA graph replay (hz_profile_graph), as in a solve."""
        self._stream()
        x = self._empty() if x is None else x
        cap = 4096
        out = (KernelTime * cap)()
        fn = lib().hz_profile_graph if graph else lib().hz_profile_iteration
        cnt = fn(self._h, _ptr(rhs), _ptr(x), iterations, out, cap)
        if cnt < 0:
            raise HzError(HZ_ECUDA, lib().hz_last_error(self._h).decode())
        return [(lib().hz_kernel_name(out[q].kernel).decode(), out[q].level, float(out[q].ms)) for q in range(min(cnt, cap))]

    def set_stall_detection(self, cos2: float = 1e-12, step2: float = 1e-8, max_restarts: int = 16):
        """Near-breakdown thresholds of the following solves (hz_set_stall_detection)."""
        self._check(lib().hz_set_stall_detection(self._h, float(cos2), float(step2), int(max_restarts)))

    def krylov_scalars(self, instance: int = 0) -> dict:
        """Bi-CGSTAB scalars of an instance after the last solve (diagnostics)."""
        out = (c_double * 17)()
        if lib().hz_krylov_scalars(self._h, instance, out) != 17:
            raise HzError(HZ_ECUDA, lib().hz_last_error(self._h).decode())
        v = list(out)
        return {"rho": complex(v[0], v[1]), "alpha": complex(v[2], v[3]), "omega": complex(v[4], v[5]),
                "beta": complex(v[6], v[7]), "rr": v[8], "ss": v[9], "tt": v[10], "bnorm2": v[11],
                "it": int(v[12]), "done": int(v[13]), "min_cos2": v[14], "shadow_restarts": int(v[15]),
                "min_step2": v[16]}

    def vcycle(self, r):
        self._stream()
        z = self._empty()
        self._check(lib().hz_vcycle(self._h, _ptr(r), _ptr(z)))
        return z

    def apply(self, u, op: str = "L"):
        self._stream()
        v = self._empty()
        self._check(lib().hz_apply(self._h, OPS[op], _ptr(u), _ptr(v)))
        return v

    def level_presmooth(self, level: int, f):
        self._stream()
        u, fc = self._empty(level), self._empty(level + 1)
        self._check(lib().hz_level_presmooth(self._h, level, _ptr(f), _ptr(u), _ptr(fc)))
        return u, fc

    def level_postsmooth(self, level: int, f, u_pre, ec):
        self._stream()
        u = self._empty(level)
        self._check(lib().hz_level_postsmooth(self._h, level, _ptr(f), _ptr(u_pre), _ptr(ec), _ptr(u)))
        return u

    def level_sweeps(self, level: int, f, u, sweeps: int = 1, post: bool = False):
        self._stream()
        out = u.clone()
        self._check(lib().hz_level_sweeps(self._h, level, _ptr(f), _ptr(out), sweeps, int(post)))
        return out

    def coarse_solve(self, f):
        self._stream()
        u = self._empty(self.num_levels - 1)
        self._check(lib().hz_coarse_solve(self._h, _ptr(f), _ptr(u)))
        return u


def ray_spacing(n: int, k_ref: float) -> int:
    """The ray grid factor of the kH <= 2.5 rule (hz_ray_spacing; host only)."""
    return int(lib().hz_ray_spacing(int(n), float(k_ref)))


class Ray:
    """Ray correction of a :class:`Problem` (hz_ray_create): the Galerkin plane-wave coarse problem of
    Sec. 6 on the ray grid of factor ``m`` (0 = the kH <= 2.5 rule)."""

    def __init__(self, problem: Problem, k_ref: float, m: int = 0, arena=None):
        import torch

        problem._stream()
        nb = int(lib().hz_ray_footprint_bytes(problem.n, float(k_ref), int(m)))
        if nb == 0:
            raise HzError(HZ_EINVAL, "invalid ray grid factor for this grid")
        self.arena = arena if arena is not None else torch.empty(nb, dtype=torch.uint8, device="cuda")
        h = c_void_p()
        problem._check(lib().hz_ray_create(problem._h, float(k_ref), int(m), c_void_p(self.arena.data_ptr()), nb,
                                           byref(h)))
        self._h = h
        self.problem = problem
        info = RayInfo()
        problem._check(lib().hz_ray_get_info(h, byref(info)))
        self.m, self.nc, self.unknowns = info.m, info.nc, info.unknowns
        self.kH, self.bytes, self.setup_ms = info.kH, int(info.bytes), info.setup_ms

    def _vec(self):
        import torch

        return torch.empty(self.unknowns, dtype=torch.complex128, device="cuda")

    def restrict(self, r):
        """P^H r: a complex128 CUDA vector of 8 (nc+1)^2 entries ordered 8 C + j."""
        self.problem._stream()
        g = self._vec()
        self.problem._check(lib().hz_ray_restrict(self._h, _ptr(r), _ptr(g)))
        return g

    def coarse_solve(self, g):
        self.problem._stream()
        z = self._vec()
        self.problem._check(lib().hz_ray_coarse_solve(self._h, _ptr(g), _ptr(z)))
        return z

    def blocks(self):
        """The assembled (lower, diag, upper) blocks of P^H A P: (nc+1, Bs, Bs) complex128 CUDA tensors."""
        import torch

        self.problem._stream()
        Bs = 8 * (self.nc + 1)
        out = [torch.empty((self.nc + 1, Bs, Bs), dtype=torch.complex128, device="cuda") for _ in range(3)]
        self.problem._check(lib().hz_ray_blocks(self._h, *[_ptr(t) for t in out]))
        return tuple(out)

    def correct(self, r, x):
        """x += P (P^H A P)^{-1} P^H r, in place on x."""
        self.problem._stream()
        self.problem._check(lib().hz_ray_correct(self._h, _ptr(r), _ptr(x)))
        return x

    def close(self):
        if getattr(self, "_h", None):
            lib().hz_ray_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Several set-up (batched) problems solved together: one CUDA graph per iteration of all."""

    def __init__(self, problems):
        self.problems = list(problems)
        arr = (c_void_p * len(self.problems))(*[p._h.value for p in self.problems])
        h = c_void_p()
        st = lib().hz_group_create(arr, len(self.problems), byref(h))
        if st != HZ_OK:
            raise HzError(st, "hz_group_create failed")
        self._h = h

    def solve(self, rhs_list, tol: float = 1e-6, maxit: int = 1000, allow_fail: bool = False):
        """rhs_list[i]: (batch_i, n_i+1, n_i+1) complex128 CUDA tensor. Returns (x list, infos)."""
        import torch

        for p in self.problems:
            p._stream()
        xs = [torch.empty_like(r) for r in rhs_list]
        rp = (c_void_p * len(xs))(*[_ptr(r).value for r in rhs_list])
        xp = (c_void_p * len(xs))(*[_ptr(x).value for x in xs])
        total = sum(p.batch for p in self.problems)
        infos = (SolveInfo * total)()
        st = lib().hz_group_solve(self._h, rp, xp, tol, maxit, infos)
        ok = (HZ_OK, HZ_EMAXIT, HZ_EBREAKDOWN, HZ_ENONFINITE) if allow_fail else (HZ_OK,)
        if st not in ok:
            raise HzError(st, lib().hz_group_last_error(self._h).decode())
        torch.cuda.synchronize()
        return xs, [{"iterations": i.iterations, "relres_true": i.relres_true, "status": i.status} for i in infos]

    def close(self):
        if getattr(self, "_h", None):
            lib().hz_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
