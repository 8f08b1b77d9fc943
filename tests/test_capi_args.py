"""Host-side fault handling of the C ABI (no GPU): malformed calls return
GCP_ERR_INVALID_ARG (or GCP_ERR_UNSUPPORTED) with a message, before any
device work.  The matrix pointers passed are never dereferenced because the
argument checks come first; the module skips itself on a machine with a GPU
so that a check that let a call through could not touch device memory."""
import ctypes as C
import math

import pytest

from paper_1512_07236_gb300 import gcp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.skipif(torch.cuda.is_available(),
                                reason="host-side argument checks run where no GPU is present")

FAKE = C.c_void_p(4096)  # a non-null address the checks reject before any use


@pytest.fixture(scope="module")
def lib():
    from paper_1512_07236_gb300 import _build
    _build.build()
    return gcp.load_library()


@pytest.fixture()
def handle(lib):
    h = C.c_void_p()
    assert lib.gcp_create(C.byref(h)) == gcp.OK
    yield h
    lib.gcp_destroy(h)


def _opts(**kw):
    o = gcp.make_options(stream=0)  # the default stream: no torch.cuda call
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _solve(lib, h, H=FAKE, M=64, N=16, ld=64, hd=gcp.F64, D=FAKE, ldd=64, dd=gcp.F64, **kw):
    res = gcp.Result()
    o = _opts(**kw)
    return lib.gcp_solve(h, H, M, N, ld, hd, D, ldd, dd, C.byref(res), C.byref(o))


@pytest.mark.parametrize("case", [
    dict(H=None), dict(D=None), dict(M=0), dict(N=-1), dict(N=65), dict(ld=63), dict(ldd=63),
    dict(hd=7), dict(dd=7), dict(prec=99), dict(prec=-1), dict(max_iter=-1),
    dict(history_cap=-1), dict(tol=math.nan), dict(tol=-1.0), dict(stop=2), dict(guess=3),
    dict(method=2), dict(prec=7), dict(refine_iters=-1), dict(check_symmetry=2),
    dict(sym_tol=-1e-3), dict(sym_tol=math.nan), dict(sym_tol=2.0),
])
def test_solve_rejects(lib, handle, case):
    assert _solve(lib, handle, **case) == gcp.ERR_INVALID_ARG
    assert b"bad arguments" in lib.gcp_last_error(handle)


def test_null_handle(lib):
    res = gcp.Result()
    o = gcp.make_options(stream=0)
    assert lib.gcp_solve(None, FAKE, 64, 16, 64, gcp.F64, FAKE, 64, gcp.F64, C.byref(res),
                         C.byref(o)) == gcp.ERR_INVALID_ARG
    assert lib.gcp_create(None) == gcp.ERR_INVALID_ARG
    assert lib.gcp_destroy(None) == gcp.ERR_INVALID_ARG


@pytest.mark.parametrize("M,N,guess", [(64, 0, 0), (64, 64, 0), (64, 16, 5)])
def test_init_guess_rejects(lib, handle, M, N, guess):
    info = (C.c_double * 8)()
    o = _opts(guess=guess)
    st = lib.gcp_init_guess(handle, FAKE, M, N, M, gcp.F64, FAKE, M, gcp.F64, info, C.byref(o))
    assert st == gcp.ERR_INVALID_ARG


@pytest.mark.parametrize("case", [dict(D=None), dict(M=0), dict(prec=42), dict(method=7)])
def test_step_rejects(lib, handle, case):
    out = (C.c_double * 8)()
    D = case.get("D", FAKE)
    M = case.get("M", 64)
    o = _opts(**{k: v for k, v in case.items() if k in ("prec", "method")})
    assert lib.gcp_step(handle, D, M, 16, 64, gcp.F64, out, C.byref(o)) == gcp.ERR_INVALID_ARG


def test_batched_rejects(lib, handle):
    n = 2
    Hs = (C.c_void_p * n)(FAKE.value, FAKE.value)
    Ds = (C.c_void_p * n)(FAKE.value, FAKE.value)
    Ms = (C.c_int * n)(64, 96)
    lds = (C.c_int * n)(64, 96)
    res = (gcp.Result * n)()
    o = gcp.make_options(stream=0)
    good_N = (C.c_int * n)(16, 24)
    assert lib.gcp_solve_batched(handle, 0, Hs, Ms, good_N, lds, gcp.F64, Ds, gcp.F64, res,
                                 C.byref(o)) == gcp.ERR_INVALID_ARG
    bad_N = (C.c_int * n)(16, 97)  # instance 1: N > M
    assert lib.gcp_solve_batched(handle, n, Hs, Ms, bad_N, lds, gcp.F64, Ds, gcp.F64, res,
                                 C.byref(o)) == gcp.ERR_INVALID_ARG
    assert b"bad instance 1" in lib.gcp_last_error(handle)


@pytest.mark.parametrize("kw,expect", [
    (dict(fixed_iters=0), gcp.ERR_INVALID_ARG),
    (dict(fixed_iters=5, prec=gcp.PRECISIONS["mixed_fp16"]), gcp.ERR_UNSUPPORTED),
    (dict(fixed_iters=5, prec=gcp.PRECISIONS["fp16x3"]), gcp.ERR_UNSUPPORTED),
    (dict(fixed_iters=5, guess=3), gcp.ERR_INVALID_ARG),
    (dict(fixed_iters=5, method=2), gcp.ERR_INVALID_ARG),
    (dict(fixed_iters=5, method=gcp.METHODS["pmcp"], prec=gcp.PRECISIONS["fp32"]),
     gcp.ERR_UNSUPPORTED),
])
def test_backward_rejects(lib, handle, kw, expect):
    o = _opts(**kw)
    assert lib.gcp_backward(handle, FAKE, 64, 16, 64, gcp.F64, None, 1.0, FAKE,
                            C.byref(o)) == expect


def test_defaults_of_the_added_options(lib):
    o = gcp.Options()
    lib.gcp_default_options(C.byref(o))
    assert o.refine_iters == 0 and o.check_symmetry == 0 and o.sym_tol == 0.0


def test_batched_rejects_added_options(lib, handle):
    n = 1
    Hs = (C.c_void_p * n)(FAKE.value)
    Ds = (C.c_void_p * n)(FAKE.value)
    Ms, Ns, lds = (C.c_int * n)(64), (C.c_int * n)(16), (C.c_int * n)(64)
    res = (gcp.Result * n)()
    for kw in (dict(prec=7), dict(refine_iters=-2), dict(check_symmetry=-1)):
        o = _opts(**kw)
        assert lib.gcp_solve_batched(handle, n, Hs, Ms, Ns, lds, gcp.F64, Ds, gcp.F64, res,
                                     C.byref(o)) == gcp.ERR_INVALID_ARG, kw


@pytest.mark.parametrize("M,wait_s", [(0, 1e-3), (-5, 1e-3), (256, 0.0), (256, -1.0),
                                      (256, 11.0), (256, math.nan)])
def test_debug_timeout_rejects(lib, handle, M, wait_s):
    o = gcp.make_options(stream=0)
    assert lib.gcp_debug_timeout(handle, M, wait_s, C.byref(o)) == gcp.ERR_INVALID_ARG
    assert lib.gcp_debug_timeout(None, 256, 1e-3, C.byref(o)) == gcp.ERR_INVALID_ARG


def test_batched_order_args(lib, handle):
    """gcp_set_batched_order takes -1, 0, 1, 2 or 3; gcp_batched_order reports the
    default (order 0, nothing timed) on a fresh handle; both are host-only."""
    for bad in (-2, 4, 100):
        assert lib.gcp_set_batched_order(handle, bad) == gcp.ERR_INVALID_ARG
    assert lib.gcp_set_batched_order(None, 0) == gcp.ERR_INVALID_ARG
    for good in (-1, 0, 1, 2, 3, -1):
        assert lib.gcp_set_batched_order(handle, good) == gcp.OK
    c = C.c_int(-7)
    ms = (C.c_double * 4)(1.0, 1.0, 1.0, 1.0)
    assert lib.gcp_batched_order(handle, C.byref(c), ms) == gcp.OK
    assert c.value == 0 and list(ms) == [-1.0, -1.0, -1.0, -1.0]
    assert lib.gcp_batched_order(handle, None, ms) == gcp.ERR_INVALID_ARG
    assert lib.gcp_batched_order(None, C.byref(c), ms) == gcp.ERR_INVALID_ARG
