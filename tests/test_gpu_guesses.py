"""HPCP+ and hole guesses, and the PMCP method, through the C ABI, against
the oracle (FP64 path to the FP64 bar; split and mixed modes to their
representation's bar)."""
import numpy as np
import pytest

from oracle import gcp_oracle as o
from paper_1512_07236_gb300 import inputs

from conftest import SUBSPACE_BF16, SUBSPACE_TARGET

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1512_07236_gb300 import gcp
    return gcp.Solver()


def _dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _rot(M, theta, gap, seed):
    N = int(round(theta * M))
    H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -gap / 2), (gap / 2, 1.0), seed=seed)
    return H, N, eps, Q


@pytest.mark.parametrize("theta", [0.05, 0.25, 0.5, 0.8, 0.97])
@pytest.mark.parametrize("guess", ["hpcp+", "hole"])
def test_init_guess_matches_oracle(solver, theta, guess):
    M = 160
    H, N, _, _ = _rot(M, theta, 0.1, 21)
    D0, info = solver.init_guess(_dev(H), N, guess=guess)
    ref, rinfo = o.hpcp_plus_guess(H, N, alpha=0.0 if guess == "hole" else None)
    assert np.abs(D0.cpu().numpy() - ref).max() <= 1e-13
    assert info["beta2"] == pytest.approx(rinfo["beta2"], rel=1e-12)


@pytest.mark.parametrize("method", ["hpcp", "pmcp"])
@pytest.mark.parametrize("guess", ["canonical", "hpcp+"])
@pytest.mark.parametrize("M,theta,gap,seed", [(96, 0.05, 0.2, 1), (130, 0.3, 0.1, 2),
                                              (200, 0.5, 0.1, 3), (257, 0.9, 0.05, 4)])
def test_fp64_solve_parity(solver, method, guess, M, theta, gap, seed):
    H, N, eps, Q = _rot(M, theta, gap, seed)
    ref = o.solve(H, N, tol=1e-12, guess=guess, method=method)
    D, info = solver.solve(_dev(H), N, prec="fp64", tol=1e-12, guess=guess, method=method)
    assert ref["status"] == "ok" and info["status"] == 0, info
    assert np.abs(D.cpu().numpy() - ref["D"]).max() <= 1e-10
    assert abs(info["energy"] - ref["E"]) <= 1e-12 * abs(ref["E"])
    assert abs(info["iters"] - ref["iters"]) <= 1
    if guess == "hpcp+":
        assert info["alpha"] == pytest.approx(ref["guess"]["alpha"], abs=1e-12)


@pytest.mark.parametrize("theta", [0.4, 0.5, 0.6])
def test_hole_purification_parity(solver, theta):
    """GCP_GUESS_HOLE purifies I - Dbar_0: the oracle's literal hole
    purification (Eq. hpcp3 on Dbar) gives the same D."""
    H, N, eps, Q = _rot(120, theta, 0.2, 31)
    ref = o.solve_holes(H, N, tol=1e-12)
    D, info = solver.solve(_dev(H), N, prec="fp64", tol=1e-12, guess="hole")
    assert info["status"] == 0 and ref["status"] == "ok"
    assert np.abs(D.cpu().numpy() - ref["D"]).max() <= 1e-10
    assert abs(info["iters"] - ref["iters"]) <= 1


def test_hole_guess_at_extreme_filling_is_ill_conditioned(solver):
    from paper_1512_07236_gb300 import gcp
    H, eps = inputs.diagonal_spectrum(100, 5, 1.0, seed=2)
    ref = o.solve(H, 5, tol=1e-6, stop="trace", guess="hole")
    D, info = solver.solve(_dev(H), 5, prec="fp64", tol=1e-6, stop="trace", guess="hole")
    assert ref["status"] == "ill_conditioned"
    assert info["status"] == gcp.ERR_ILL_CONDITIONED


@pytest.mark.parametrize("method,guess", [("pmcp", "canonical"), ("pmcp", "hpcp+"),
                                          ("hpcp", "hpcp+")])
@pytest.mark.parametrize("prec,lim", [("mixed_fp16", SUBSPACE_TARGET),
                                      ("mixed_bf16", SUBSPACE_BF16)])
def test_mixed_modes(solver, method, guess, prec, lim):
    H, N, eps, Q = _rot(512, 0.1, 0.05, 41)
    D, info = solver.solve(_dev(H), N, prec=prec, tol=1e-10, guess=guess, method=method)
    Dg = D.cpu().numpy()
    assert info["status"] == 0, info
    assert np.linalg.norm(Dg @ Dg - Dg) <= 2e-10
    assert abs(np.trace(Dg) - N) <= 1e-9
    Dref = Q[:, :N] @ Q[:, :N].T
    assert np.linalg.norm(Dg - Dref) / np.sqrt(N) <= lim
    assert np.abs(Dg - Dref).max() <= 3 * lim
    assert abs(info["energy"] - eps[:N].sum()) <= 1e-9 * abs(eps[:N].sum())


@pytest.mark.parametrize("prec,tol", [("fp16x3", 2e-6), ("bf16x3", 6e-5)])
def test_pmcp_split_step(solver, prec, tol):
    M = 300
    H, N, _, _ = _rot(M, 0.2, 0.1, 51)
    D, _ = o.canonical_guess(H, N)
    for _ in range(3):
        D = o.pm_step(D, o.coefficient_c(D))
    Dt = _dev(D, torch.float32)
    T1, T2, T3, R, c, applied = solver.step(Dt, N, prec=prec, method="pmcp")
    c_ref = o.coefficient_c(D)
    assert c == pytest.approx(c_ref, rel=1e-3)
    Dn = o.pm_step(D, c_ref)
    err = np.abs(Dt.cpu().numpy().astype(np.float64) - Dn).max()
    assert err <= tol * max(1.0, np.abs(Dn).max()), err


def test_unsupported_combinations(solver):
    """The FP64 adjoint differentiates PM steps; the FP32 one does not."""
    from paper_1512_07236_gb300 import gcp
    H, N, _, _ = _rot(64, 0.25, 0.2, 61)
    out = torch.empty(64, 64, dtype=torch.float64, device="cuda")
    o_ = gcp.make_options(prec="fp64", fixed_iters=5, method="pmcp")
    st = solver.lib.gcp_backward(solver.h, _dev(H).data_ptr(), 64, N, 64, gcp.F64, None, 1.0,
                                 out.data_ptr(), gcp.C.byref(o_))
    assert st == gcp.OK
    o_ = gcp.make_options(prec="fp32", fixed_iters=5, method="pmcp")
    st = solver.lib.gcp_backward(solver.h, _dev(H).data_ptr(), 64, N, 64, gcp.F64, None, 1.0,
                                 out.data_ptr(), gcp.C.byref(o_))
    assert st == gcp.ERR_UNSUPPORTED
