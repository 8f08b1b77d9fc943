"""The stop test after an exact-slice refinement step, through the C ABI.

After a step D -> D1 the residual ||D1^2 - D1||_F is formed from
W = D1^2 - D^2 (one split product over [D | Delta | Delta] x
[Delta | D | Delta], Delta = D1 - D) and the exact S = D^2 as S + W - D1.
Every check here recomputes the residual and the trace of the returned D
independently in FP64 on the host (numpy), so the reported figures are
pinned to the plain definition, not to the solver's own arithmetic."""
import math

import numpy as np
import pytest

from paper_1512_07236_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1512_07236_gb300 import gcp
    return gcp.Solver()


def _fp64_residual(D):
    return float(np.linalg.norm(D @ D - D))


@pytest.mark.parametrize("M,theta,gap,seed", [(300, 0.25, 0.05, 1), (640, 0.1, 0.02, 2),
                                              (1000, 0.6, 0.05, 3), (257, 0.5, 0.2, 4)])
@pytest.mark.parametrize("tol", [1e-6, 1e-8, 1e-10])
def test_reported_residual_and_trace(solver, M, theta, gap, seed, tol):
    N = int(round(theta * M))
    H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -gap / 2), (gap / 2, 1.0), seed=seed)
    D, info = solver.solve(torch.from_numpy(H).cuda(), N, prec="mixed_fp16", tol=tol,
                           history_cap=400)
    assert info["status"] == 0, info
    Dh = D.cpu().numpy()
    R = _fp64_residual(Dh)
    assert R <= tol * (1 + 1e-3)
    # the stop test's residual carries the FP32 rounding of W (~1e-7 of the
    # step, ~1e-7 sqrt(tol), a few 1e-3 of R here), the ~1e-14 per element
    # that the slice product S leaves with all digit pairs (Frobenius
    # ~1e-14 M), and what the digit pairs dropped for this tol add (at most
    # tol / 8 by the plan's estimate, which the solve subtracts from tol)
    assert abs(info["idem_fro"] - R) <= 5e-3 * R + 2e-14 * M + tol / 8, (info["idem_fro"], R)
    assert abs(info["trace"] - np.trace(Dh)) <= 1e-12 * N
    assert abs(np.trace(Dh) - N) <= 1e-9
    hist = solver.history(400)
    last = hist[-1]
    assert last["phase"] == 0 and last["R"] == pytest.approx(info["idem_fro"], rel=1e-15)
    if math.isnan(last["T3"]):
        # accepted by the stop-test product: its Tr D1^2 is the trace of the
        # exact square of the returned D
        assert abs(last["T2"] - np.trace(Dh @ Dh)) <= 1e-10 * N


def test_stop_test_product_ends_the_phase(solver):
    """The configuration of the dense workload at reduced size: one
    refinement step, accepted by the stop-test product (no second exact
    slice product)."""
    M, N = 2048, 512
    H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -0.005), (0.005, 1.0), seed=2)
    D, info = solver.solve(torch.from_numpy(H).cuda(), N, prec="mixed_fp16", tol=1e-6,
                           history_cap=400)
    assert info["status"] == 0
    assert info["iters_fp64"] == 1
    hist = solver.history(400)
    assert math.isnan(hist[-1]["T3"])
    assert sum(1 for h in hist if h["phase"] == 0) == 2  # one exact evaluation + the test
    Dh = D.cpu().numpy()
    assert (abs(info["idem_fro"] - _fp64_residual(Dh))
            <= 5e-3 * info["idem_fro"] + 2e-14 * M + 1e-6 / 8)
    E = float(eps[:N].sum())
    assert abs(info["energy"] - E) <= 1e-10 * abs(E)


def test_trace_stop_keeps_exact_evaluations(solver):
    """The stop-test product serves the idempotency criterion only; with the
    trace criterion every evaluation is an exact slice product."""
    M, N = 384, 96
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.05), (0.05, 1.0), seed=6)
    D, info = solver.solve(torch.from_numpy(H).cuda(), N, prec="mixed_fp16", tol=1e-9,
                           stop="trace", history_cap=400)
    assert info["status"] == 0
    hist = solver.history(400)
    assert not any(math.isnan(h["T3"]) for h in hist)
    Dh = D.cpu().numpy()
    assert abs(np.trace(Dh - Dh @ Dh)) <= 1e-9 * (1 + 1e-3)
