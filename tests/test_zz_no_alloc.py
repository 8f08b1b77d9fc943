"""gcp_solve_noalloc: the allocation-free FP64 solve, for callers that must
not allocate device memory while solving (a memory pool that already holds
the GPU, a latency-bound loop that cannot take cudaMalloc's implicit
synchronisation, code without a library handle).

Calls the entry point directly through the C ABI and compares it with
gcp_solve (the handle-based path) on two calls in a row, within the FP64
parity tolerance of the other tests.  Kept in a file that sorts last so a
run that stops at the first failure has already run every other test; it
also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

from paper_1512_07236_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1512_07236_gb300 import gcp
    return gcp


def _noalloc(g, H, N, out, **opts):
    L = g.load_library()
    res = g.Result()
    o = g.make_options(**opts)
    err = C.create_string_buffer(256)
    st = L.gcp_solve_noalloc(C.c_void_p(H.data_ptr()), H.shape[0], int(N), H.stride(0),
                             g.F64 if H.dtype == torch.float64 else g.F32,
                             C.c_void_p(out.data_ptr()), out.stride(0),
                             g.F64 if out.dtype == torch.float64 else g.F32, C.byref(res),
                             C.byref(o), err, 256)
    torch.cuda.synchronize()
    return st, res, err.value.decode()


def test_noalloc_matches_solve_twice_in_a_row(lib):
    g = lib
    solver = g.Solver()
    cases = [(256, 64, (-1.0, -0.1), (0.1, 1.0), 1), (130, 33, (-1.0, -0.05), (0.05, 1.0), 2)]
    for M, N, occ, virt, seed in cases:
        H, eps, Q = inputs.rotated_spectrum(M, N, occ, virt, seed=seed)
        Ht = torch.from_numpy(H).cuda()
        Dref, iref = solver.solve(Ht, N, prec="fp64", tol=1e-12)
        Dn = torch.full((M, M), float("nan"), dtype=torch.float64, device="cuda")
        st, res, msg = _noalloc(g, Ht, N, Dn, prec="fp64", tol=1e-12)
        assert st == g.OK, msg
        assert res.status == g.OK and res.iters == iref["iters"]
        assert float((Dn - Dref).abs().max()) <= 1e-12
        assert abs(res.energy - iref["energy"]) <= 1e-12 * abs(iref["energy"])
        assert abs(res.trace - N) <= 1e-10


def test_noalloc_rejects_sizes_beyond_its_workspace(lib):
    g = lib
    H = torch.eye(520, dtype=torch.float64, device="cuda")
    D = torch.empty_like(H)
    st, res, msg = _noalloc(g, H, 100, D, prec="fp64")
    assert st == g.ERR_INVALID_ARG
    assert "exceeds" in msg and "512" in msg
