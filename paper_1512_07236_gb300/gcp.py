"""Thin ctypes binding over libgcp (include/gcp.h).

Argument marshalling only: every step of the purification runs in the
CUDA kernels behind the C ABI.  PyTorch supplies device memory and the
current stream.  There is no CPU fallback: a missing library or GPU raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgcp.so")

# gcp_status
OK, ERR_INVALID_ARG, ERR_NOT_CONVERGED, ERR_ILL_CONDITIONED, ERR_NO_GAP, ERR_NONFINITE, \
    ERR_TIMEOUT, ERR_CUDA, ERR_UNSUPPORTED, ERR_NO_CHECKPOINT = range(10)
# gcp_dtype
F64, F32 = 0, 1
# gcp_precision
PRECISIONS = {"fp64": 0, "fp16x3": 1, "bf16x3": 2, "mixed_fp16": 3, "mixed_bf16": 4,
              "mixed_auto": 5, "fp32": 6}
STOPS = {"idem_fro": 0, "trace": 1}
GUESSES = {"canonical": 0, "hpcp+": 1, "hole": 2}
METHODS = {"hpcp": 0, "pmcp": 1}
HISTORY_FIELDS = 8
EXPORTS = ("gcp_default_options", "gcp_status_string", "gcp_create", "gcp_destroy",
           "gcp_last_error", "gcp_init_guess", "gcp_step", "gcp_solve", "gcp_get_history",
           "gcp_solve_batched", "gcp_backward", "gcp_time_kernels", "gcp_solve_noalloc",
           "gcp_debug_timeout", "gcp_set_batched_order", "gcp_batched_order")


class Options(C.Structure):
    _fields_ = [("prec", C.c_int), ("stop", C.c_int), ("tol", C.c_double),
                ("max_iter", C.c_int), ("fixed_iters", C.c_int), ("ckpt_every", C.c_int),
                ("history_cap", C.c_int), ("use_graph", C.c_int), ("stream", C.c_void_p),
                ("refine", C.c_int), ("guess", C.c_int), ("method", C.c_int),
                ("refine_iters", C.c_int), ("check_symmetry", C.c_int), ("sym_tol", C.c_double)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("iters_lowp", C.c_int),
                ("iters_fp64", C.c_int), ("trace", C.c_double), ("energy", C.c_double),
                ("idem_fro", C.c_double), ("trace_ddbar", C.c_double), ("c_last", C.c_double),
                ("mu", C.c_double), ("beta2", C.c_double), ("hmin", C.c_double),
                ("hmax", C.c_double), ("alpha", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GCPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libgcp.so and declare its prototypes (no GPU needed to load)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libgcp.so not built ({path}); run __graft_entry__.build()")
        lib = C.CDLL(path)
        vp, ip, dp = C.c_void_p, C.c_int, C.c_double
        lib.gcp_default_options.argtypes = [C.POINTER(Options)]
        lib.gcp_default_options.restype = None
        lib.gcp_status_string.argtypes = [ip]
        lib.gcp_status_string.restype = C.c_char_p
        lib.gcp_create.argtypes = [C.POINTER(vp)]
        lib.gcp_destroy.argtypes = [vp]
        lib.gcp_last_error.argtypes = [vp]
        lib.gcp_last_error.restype = C.c_char_p
        lib.gcp_init_guess.argtypes = [vp, vp, ip, ip, ip, ip, vp, ip, ip, C.POINTER(dp),
                                       C.POINTER(Options)]
        lib.gcp_step.argtypes = [vp, vp, ip, ip, ip, ip, C.POINTER(dp), C.POINTER(Options)]
        lib.gcp_solve.argtypes = [vp, vp, ip, ip, ip, ip, vp, ip, ip, C.POINTER(Result),
                                  C.POINTER(Options)]
        lib.gcp_get_history.argtypes = [vp, C.POINTER(dp), ip, C.POINTER(ip)]
        lib.gcp_solve_batched.argtypes = [vp, ip, C.POINTER(vp), C.POINTER(ip), C.POINTER(ip),
                                          C.POINTER(ip), ip, C.POINTER(vp), ip,
                                          C.POINTER(Result), C.POINTER(Options)]
        lib.gcp_backward.argtypes = [vp, vp, ip, ip, ip, ip, vp, dp, vp, C.POINTER(Options)]
        lib.gcp_time_kernels.argtypes = [vp, ip, ip, ip, ip, C.POINTER(dp), C.POINTER(Options)]
        lib.gcp_solve_noalloc.argtypes = [vp, ip, ip, ip, ip, vp, ip, ip, C.POINTER(Result),
                                          C.POINTER(Options), C.c_char_p, ip]
        lib.gcp_debug_timeout.argtypes = [vp, ip, dp, C.POINTER(Options)]
        lib.gcp_set_batched_order.argtypes = [vp, ip]
        lib.gcp_batched_order.argtypes = [vp, C.POINTER(ip), C.POINTER(dp)]
        for name in ("gcp_create", "gcp_destroy", "gcp_init_guess", "gcp_step", "gcp_solve",
                     "gcp_get_history", "gcp_solve_batched", "gcp_backward", "gcp_time_kernels",
                     "gcp_solve_noalloc", "gcp_debug_timeout", "gcp_set_batched_order",
                     "gcp_batched_order"):
            getattr(lib, name).restype = C.c_int
        _lib = lib
        return lib


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype}; use float32 or float64")


def _check_matrix(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dim() != 2 or t.shape[0] != t.shape[1]:
        raise ValueError(f"{name} must be square")
    if t.stride(1) != 1 or t.stride(0) < t.shape[1]:
        raise ValueError(f"{name} must be row-major with unit column stride")


def make_options(prec="fp64", stop="idem_fro", tol=1e-12, max_iter=100, fixed_iters=0,
                 ckpt_every=8, history_cap=0, use_graph=True, stream=None,
                 refine="slices", guess="canonical", method="hpcp", refine_iters=0,
                 check_symmetry=False, sym_tol=0.0) -> Options:
    lib = load_library()
    o = Options()
    lib.gcp_default_options(C.byref(o))
    o.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    o.stop = STOPS[stop] if isinstance(stop, str) else int(stop)
    o.tol = float(tol)
    o.max_iter = int(max_iter)
    o.fixed_iters = int(fixed_iters)
    o.ckpt_every = int(ckpt_every)
    o.history_cap = int(history_cap)
    o.use_graph = 1 if use_graph else 0
    o.refine = {"slices": 0, "fp64": 1}[refine] if isinstance(refine, str) else int(refine)
    o.guess = GUESSES[guess] if isinstance(guess, str) else int(guess)
    o.method = METHODS[method] if isinstance(method, str) else int(method)
    o.refine_iters = int(refine_iters)
    o.check_symmetry = 1 if check_symmetry else 0
    o.sym_tol = float(sym_tol)
    if stream is None:
        stream = torch.cuda.current_stream()
    o.stream = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    return o


class Solver:
    """Owns one libgcp handle (workspace, graphs).  Not thread-safe."""

    def __init__(self):
        if not torch.cuda.is_available():
            raise RuntimeError("libgcp needs a CUDA GPU (no CPU fallback)")
        self.lib = load_library()
        h = C.c_void_p()
        self._check(self.lib.gcp_create(C.byref(h)), h)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.gcp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, h=None, allow=()):
        if st != OK and st not in allow:
            msg = self.lib.gcp_last_error(h if h is not None else self.h)
            raise GCPError(st, f"{self.lib.gcp_status_string(st).decode()}: "
                               f"{msg.decode() if msg else ''}")
        return st

    # -- entry points ------------------------------------------------------
    def init_guess(self, H: torch.Tensor, N: int, out_dtype=None, **opts):
        _check_matrix(H, "H")
        M = H.shape[0]
        D0 = torch.empty((M, M), dtype=out_dtype or H.dtype, device=H.device)
        info = (C.c_double * 5)()
        o = make_options(**opts)
        st = self.lib.gcp_init_guess(self.h, C.c_void_p(H.data_ptr()), M, int(N), H.stride(0),
                                     _dtype_code(H), C.c_void_p(D0.data_ptr()), D0.stride(0),
                                     _dtype_code(D0), info, C.byref(o))
        self._check(st, allow=(ERR_NO_GAP,))
        return D0, dict(mu=info[0], beta2=info[1], hmin=info[2], hmax=info[3], theta=info[4],
                        status=st)

    def step(self, D: torch.Tensor, N: int, **opts):
        """One step of Eq. hpcp3 in place; returns (T1, T2, T3, R, c, applied)."""
        _check_matrix(D, "D")
        out = (C.c_double * 6)()
        o = make_options(**opts)
        self._check(self.lib.gcp_step(self.h, C.c_void_p(D.data_ptr()), D.shape[0], int(N),
                                      D.stride(0), _dtype_code(D), out, C.byref(o)))
        return tuple(out)

    def solve(self, H: torch.Tensor, N: int, out=None, out_dtype=None, raise_on_error=False,
              **opts):
        """Returns (D, info dict).  info['status'] holds the gcp_status."""
        _check_matrix(H, "H")
        M = H.shape[0]
        if out is None:
            dt = out_dtype or (torch.float64 if opts.get("prec", "fp64") in (
                "fp64", 0, "mixed_fp16", "mixed_bf16", "mixed_auto", 3, 4, 5) else torch.float32)
            out = torch.empty((M, M), dtype=dt, device=H.device)
        _check_matrix(out, "out")
        res = Result()
        o = make_options(**opts)
        st = self.lib.gcp_solve(self.h, C.c_void_p(H.data_ptr()), M, int(N), H.stride(0),
                                _dtype_code(H), C.c_void_p(out.data_ptr()), out.stride(0),
                                _dtype_code(out), C.byref(res), C.byref(o))
        allow = () if raise_on_error else (ERR_NOT_CONVERGED, ERR_ILL_CONDITIONED, ERR_NO_GAP)
        self._check(st, allow=allow)
        info = res.as_dict()
        info["status_code"] = st
        return out, info

    def solve_batched(self, Hs, Ns, outs=None, out_dtype=None, raise_on_error=False, **opts):
        """Independent solves of uneven size in one call.  Hs: list of square
        CUDA tensors (same dtype), Ns: list of ints.  Returns (Ds, infos)."""
        B = len(Hs)
        if B == 0 or len(Ns) != B:
            raise ValueError("need one N per H")
        for k, H in enumerate(Hs):
            _check_matrix(H, f"H[{k}]")
            if H.dtype != Hs[0].dtype:
                raise TypeError("all H must share a dtype")
        if outs is None:
            dt = out_dtype or (torch.float64 if opts.get("prec", "fp64") in (
                "fp64", 0, "mixed_fp16", "mixed_bf16", "mixed_auto", 3, 4, 5) else torch.float32)
            outs = [torch.empty((H.shape[0], H.shape[0]), dtype=dt, device=H.device) for H in Hs]
        for k, D in enumerate(outs):
            _check_matrix(D, f"out[{k}]")
            if D.stride(0) != D.shape[0]:
                raise ValueError("batched outputs must be dense (leading dimension M)")
        Hp = (C.c_void_p * B)(*[H.data_ptr() for H in Hs])
        Dp = (C.c_void_p * B)(*[D.data_ptr() for D in outs])
        Mv = (C.c_int * B)(*[H.shape[0] for H in Hs])
        Nv = (C.c_int * B)(*[int(n) for n in Ns])
        Lv = (C.c_int * B)(*[H.stride(0) for H in Hs])
        res = (Result * B)()
        o = make_options(**opts)
        st = self.lib.gcp_solve_batched(self.h, B, Hp, Mv, Nv, Lv, _dtype_code(Hs[0]), Dp,
                                        _dtype_code(outs[0]), res, C.byref(o))
        allow = () if raise_on_error else (ERR_NOT_CONVERGED, ERR_ILL_CONDITIONED, ERR_NO_GAP)
        self._check(st, allow=allow)
        infos = []
        for r in res:
            d = r.as_dict()
            infos.append(d)
        return outs, infos

    def backward(self, H, N, fixed_iters, G_D=None, g_E=0.0, ckpt_every=8, out=None,
                 prec="fp64", guess="canonical", method="hpcp"):
        """dL/dH of L = <G_D, D_K> + g_E Tr(H D_K), D_K after exactly
        `fixed_iters` steps from the guess (gcp_backward).  prec "fp64": the
        FP64 recursion and adjoint; "fp32": the split-FP16 tensor-core
        recursion (the iterates of prec="fp32" solves) and its adjoint.
        guess / method: those of the forward (solve's options)."""
        _check_matrix(H, "H")
        if G_D is not None:
            _check_matrix(G_D, "G_D")
            if G_D.dtype != H.dtype or G_D.stride(0) != H.stride(0):
                raise ValueError("G_D must match H's dtype and layout")
        if out is None:
            out = torch.empty_like(H)
        _check_matrix(out, "out")
        if out.dtype != H.dtype or out.stride(0) != H.stride(0):
            raise ValueError("out must match H's dtype and layout")
        o = make_options(prec=prec, fixed_iters=fixed_iters, ckpt_every=ckpt_every, guess=guess,
                         method=method)
        st = self.lib.gcp_backward(self.h, C.c_void_p(H.data_ptr()), H.shape[0], int(N),
                                   H.stride(0), _dtype_code(H),
                                   C.c_void_p(G_D.data_ptr() if G_D is not None else 0),
                                   float(g_E), C.c_void_p(out.data_ptr()), C.byref(o))
        self._check(st)
        return out

    def time_kernels(self, M, N, prec="fp16x3", reps=10, tol=1e-12):
        """Mean duration (ms) of the two products of one step, CUDA events on
        the current stream; needs a prior solve of size M on this handle.
        prec "fp16x3"/"bf16x3": GEMM1 and GEMM2 of a split step; "fp64": the
        FP64 products; "mixed_fp16"/"mixed_bf16": the digit-slice D^2, the
        (D^2 - D) D product and the stop-test product of an exact-slice
        refinement step and the number of digit-pair products of the slice
        product (four values); tol selects those pairs as a solve with that
        tolerance does."""
        ms = (C.c_double * 4)()
        p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        o = make_options(tol=tol)
        self._check(self.lib.gcp_time_kernels(self.h, int(M), int(N), p, int(reps), ms,
                                              C.byref(o)))
        if p in (PRECISIONS["mixed_fp16"], PRECISIONS["mixed_bf16"]):
            return ms[0], ms[1], ms[2], int(ms[3])
        return ms[0], ms[1]

    def set_batched_order(self, order=-1):
        """gcp_set_batched_order: -1 times the candidate work orders of the
        batched tensor-core products; 0, 1, 2 or 3 fixes one."""
        self._check(self.lib.gcp_set_batched_order(self.h, int(order)))

    def batched_order(self):
        """gcp_batched_order: (order used by the last split-precision batched
        solve, [GEMM1 ms of each candidate, -1 where not timed])."""
        c = C.c_int()
        ms = (C.c_double * 4)()
        self._check(self.lib.gcp_batched_order(self.h, C.byref(c), ms))
        return c.value, list(ms)

    def debug_timeout(self, M, wait_s=1e-3):
        """gcp_debug_timeout: run one split GEMM1 of size M whose waits are
        bounded by wait_s seconds while its drain warps wait on a barrier
        nobody arrives on; returns the status (GCP_ERR_TIMEOUT expected)."""
        o = make_options()
        return self.lib.gcp_debug_timeout(self.h, int(M), float(wait_s), C.byref(o))

    def history(self, cap=1000):
        buf = (C.c_double * (cap * HISTORY_FIELDS))()
        n = C.c_int()
        self._check(self.lib.gcp_get_history(self.h, buf, cap, C.byref(n)))
        keys = ("n", "T1", "T2", "T3", "R", "c", "E", "phase")
        return [dict(zip(keys, buf[i * HISTORY_FIELDS:(i + 1) * HISTORY_FIELDS]))
                for i in range(n.value)]


_default = None


def default_solver() -> Solver:
    global _default
    if _default is None:
        _default = Solver()
    return _default


def solve(H, N, **kw):
    """gcp.solve(H, N, **opts) -> (D, info) on the default handle."""
    return default_solver().solve(H, N, **kw)
