"""The iteration counts of Fig. 3 (p-bar) on the GPU: batched FP64 solves of
the paper's diagonal M = 100 test matrices (eigenvalues random in
[-2.5, eps_N] u [eps_N+1, 2.5], stop when Tr(D Dbar) <= 1e-6), HPCP and PMCP
steps, canonical and HPCP+ guesses, each instance's count against the
oracle's on the same matrix, and the relations the paper reports."""
import numpy as np
import pytest

from oracle import gcp_oracle as o
from paper_1512_07236_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

M, TOL, K = 100, 1e-6, 16


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1512_07236_gb300 import gcp
    return gcp.Solver()


def _counts(solver, theta, gap, method, guess):
    N = int(round(theta * M))
    Hs = [inputs.diagonal_spectrum(M, N, gap, seed=1000 + s)[0] for s in range(K)]
    Ds, infos = solver.solve_batched([torch.from_numpy(H).cuda() for H in Hs], [N] * K,
                                     prec="fp64", stop="trace", tol=TOL, method=method,
                                     guess=guess)
    gpu = [i["iters"] for i in infos]
    assert all(i["status"] == 0 for i in infos)
    ref = [o.solve(H, N, tol=TOL, stop="trace", method=method, guess=guess)["iters"]
           for H in Hs]
    return np.array(gpu), np.array(ref)


@pytest.mark.parametrize("theta,gap", [(0.05, 1.0), (0.5, 1.0), (0.5, 1e-2), (0.2, 1e-4)])
@pytest.mark.parametrize("method,guess", [("hpcp", "canonical"), ("pmcp", "canonical"),
                                          ("hpcp", "hpcp+")])
def test_counts_match_the_oracle(solver, theta, gap, method, guess):
    gpu, ref = _counts(solver, theta, gap, method, guess)
    assert np.abs(gpu - ref).max() <= 1


def test_paper_relations(solver):
    """At theta = 1/2 HPCP and PMCP take the same steps (about 10 at the
    wide-gap intercept); at theta = 0.05 HPCP needs about 23/37 of PMCP's;
    the count grows linearly in ln(1/gap)."""
    h5, _ = _counts(solver, 0.5, 1.0, "hpcp", "canonical")
    p5, _ = _counts(solver, 0.5, 1.0, "pmcp", "canonical")
    assert np.array_equal(h5, p5) and 6 <= h5.mean() <= 14
    h05, _ = _counts(solver, 0.05, 1.0, "hpcp", "canonical")
    p05, _ = _counts(solver, 0.05, 1.0, "pmcp", "canonical")
    assert abs(h05.mean() / p05.mean() - 23.0 / 37.0) < 0.12
    hs = [_counts(solver, 0.5, g, "hpcp", "canonical")[0].mean() for g in (1.0, 1e-2, 1e-4)]
    d1, d2 = hs[1] - hs[0], hs[2] - hs[1]
    assert d1 > 0 and d2 > 0 and abs(d1 - d2) <= 0.35 * max(d1, d2)
