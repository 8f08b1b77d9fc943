"""Parity of the FP64 CUDA path (through the C ABI) with the FP64 oracle.

Bar (from the method's FP64 arithmetic): max|dD| <= 1e-10, |dE|/|E| <= 1e-12,
iteration count within +-1 (the stop decision can flip under rounding)."""
import numpy as np
import pytest

from oracle import gcp_oracle as o
from paper_1512_07236_gb300 import inputs

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


def test_config1_parity_with_oracle_and_jacobi(solver):
    """M=256, N=64, gap 0.2, ||D^2-D||_F <= 1e-12."""
    H, eps, Q = inputs.rotated_spectrum(256, 64, (-1.0, -0.1), (0.1, 1.0), seed=1)
    ref = o.solve(H, 64, tol=1e-12)
    D, info = solver.solve(_dev(H), 64, prec="fp64", tol=1e-12)
    Dg = D.cpu().numpy()
    assert info["status"] == 0
    assert np.abs(Dg - ref["D"]).max() <= 1e-10
    assert abs(info["energy"] - ref["E"]) <= 1e-12 * abs(ref["E"])
    assert abs(info["iters"] - ref["iters"]) <= 1
    Dj, Ej, _ = o.ground_state_projector(H, 64)
    assert np.abs(Dg - Dj).max() <= 1e-10
    assert abs(info["energy"] - Ej) <= 1e-11 * abs(Ej)
    assert abs(info["trace"] - 64) <= 1e-10


@pytest.mark.parametrize("M,N", [(33, 7), (100, 10), (257, 128), (130, 129), (64, 1)])
def test_ragged_sizes(solver, M, N):
    H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -0.15), (0.15, 1.0), seed=M + N)
    ref = o.solve(H, N, tol=1e-12)
    D, info = solver.solve(_dev(H), N, prec="fp64", tol=1e-12)
    # theta = 129/130 is a pathological filling: both sides hit max_iter
    expect = {o.STATUS_OK: 0, o.STATUS_NOT_CONVERGED: 2}[ref["status"]]
    assert info["status"] == expect
    assert np.abs(D.cpu().numpy() - ref["D"]).max() <= 1e-10
    assert abs(info["iters"] - ref["iters"]) <= 1
    assert abs(info["energy"] - ref["E"]) <= 1e-12 * max(1.0, abs(ref["E"]))


def test_guess_parity(solver):
    H, _, _ = inputs.rotated_spectrum(200, 50, seed=3)
    D0, info = solver.init_guess(_dev(H), 50)
    R0, rinfo = o.canonical_guess(H, 50)
    assert abs(info["mu"] - rinfo["mu"]) <= 1e-15
    assert abs(info["beta2"] - rinfo["beta2"]) <= 1e-14 * rinfo["beta2"]
    assert abs(info["hmin"] - rinfo["hmin"]) <= 1e-13
    assert abs(info["hmax"] - rinfo["hmax"]) <= 1e-13
    assert np.abs(D0.cpu().numpy() - R0).max() <= 1e-15


def test_single_step_parity(solver):
    H, _, _ = inputs.rotated_spectrum(150, 40, seed=4)
    D, _ = o.canonical_guess(H, 40)
    for _ in range(3):
        Dt = _dev(D)
        T1, T2, T3, R, c, applied = solver.step(Dt, 40, prec="fp64")
        S = D @ D
        assert T1 == pytest.approx(np.trace(D), rel=1e-13)
        assert T2 == pytest.approx(np.trace(S), rel=1e-13)
        assert T3 == pytest.approx(np.sum(S * D), rel=1e-13)
        assert R == pytest.approx(np.linalg.norm(S - D), rel=1e-10)
        c_ref = (np.trace(S) - np.sum(S * D)) / (np.trace(D) - np.trace(S))
        assert c == pytest.approx(c_ref, rel=1e-10)
        Dn = o.hpcp_step(D, c_ref)
        assert applied == 1.0
        assert np.abs(Dt.cpu().numpy() - Dn).max() <= 1e-13
        D = Dn


def test_history_invariants(solver):
    """Tr D_n = N every step, c_n in [0,1], E_n monotone, R quadratic at the end."""
    H, _, _ = inputs.rotated_spectrum(128, 32, (-1.0, -0.1), (0.1, 1.0), seed=5)
    D, info = solver.solve(_dev(H), 32, prec="fp64", tol=1e-12, history_cap=200)
    hist = solver.history(200)
    ref = o.solve(H, 32, tol=1e-12)
    assert len(hist) == info["iters"] + 1
    for hg, hr in zip(hist, ref["history"]):
        assert abs(hg["T1"] - 32) <= 1e-11
        assert hg["E"] == pytest.approx(hr["E"], rel=1e-12)
        if not np.isnan(hr["c"]) and hr["T1"] - hr["T2"] > 1e-3:
            # c is a ratio of two vanishing traces: compared while they are not rounding noise
            assert hg["c"] == pytest.approx(hr["c"], abs=1e-9)
            assert 0.0 <= hg["c"] <= 1.0
    E = [h["E"] for h in hist]
    assert all(E[i + 1] <= E[i] + 1e-12 for i in range(len(E) - 1))


def test_trace_stop_criterion(solver):
    H, _, _ = inputs.rotated_spectrum(90, 30, seed=6)
    ref = o.solve(H, 30, tol=1e-6, stop="trace")
    D, info = solver.solve(_dev(H), 30, prec="fp64", tol=1e-6, stop="trace")
    assert info["status"] == 0
    assert abs(info["iters"] - ref["iters"]) <= 1
    assert info["trace_ddbar"] <= 1e-6


def test_edge_fillings_and_no_gap(solver):
    H, _, _ = inputs.rotated_spectrum(40, 10, seed=8)
    D, info = solver.solve(_dev(H), 0, prec="fp64")
    assert info["status"] == 0 and float(D.abs().max()) == 0.0
    D, info = solver.solve(_dev(H), 40, prec="fp64")
    assert np.array_equal(D.cpu().numpy(), np.eye(40))
    assert info["energy"] == pytest.approx(np.trace(H), abs=1e-12)
    from paper_1512_07236_gb300 import gcp
    D, info = solver.solve(_dev(0.3 * np.eye(24)), 6, prec="fp64")
    assert info["status"] == gcp.ERR_NO_GAP
    assert np.abs(D.cpu().numpy() - 0.25 * np.eye(24)).max() <= 1e-15


def test_fp32_input_and_output(solver):
    H, _, _ = inputs.rotated_spectrum(120, 30, seed=9)
    H32 = H.astype(np.float32)
    ref = o.solve(H32.astype(np.float64), 30, tol=1e-12)
    D, info = solver.solve(_dev(H32, torch.float32), 30, prec="fp64", tol=1e-12,
                           out_dtype=torch.float32)
    assert D.dtype == torch.float32
    assert np.abs(D.cpu().numpy() - ref["D"]).max() <= 1e-6


def test_host_loop_matches_graph(solver):
    H, _, _ = inputs.rotated_spectrum(160, 40, seed=10)
    D1, i1 = solver.solve(_dev(H), 40, prec="fp64", use_graph=True)
    D2, i2 = solver.solve(_dev(H), 40, prec="fp64", use_graph=False)
    assert i1["iters"] == i2["iters"]
    assert torch.equal(D1, D2)


def test_fixed_iterations_and_max_iter(solver):
    from paper_1512_07236_gb300 import gcp
    H, _, _ = inputs.rotated_spectrum(64, 16, seed=11)
    ref = o.solve(H, 16, fixed_iters=5)
    D, info = solver.solve(_dev(H), 16, prec="fp64", fixed_iters=5)
    assert info["iters"] == 5
    assert np.abs(D.cpu().numpy() - ref["D"]).max() <= 1e-13
    D, info = solver.solve(_dev(H), 16, prec="fp64", max_iter=2)
    assert info["status"] == gcp.ERR_NOT_CONVERGED and info["iters"] == 2


def test_bad_arguments_rejected(solver):
    from paper_1512_07236_gb300 import gcp
    H = _dev(np.eye(8))
    with pytest.raises(gcp.GCPError):
        solver.solve(H, 9, prec="fp64")
    with pytest.raises(gcp.GCPError):
        solver.solve(H, 2, prec=17)


@pytest.mark.parametrize("prec", ["fp64", "mixed_fp16"])
def test_nonfinite_hamiltonian_is_a_status(solver, prec):
    """A NaN in H makes the first evaluation's traces non-finite: the control
    kernel stops with GCP_ERR_NONFINITE and the handle stays usable."""
    from paper_1512_07236_gb300 import gcp
    H, _, _ = inputs.rotated_spectrum(64, 16, seed=12)
    Hn = H.copy()
    Hn[3, 5] = Hn[5, 3] = np.nan
    with pytest.raises(gcp.GCPError) as err:
        solver.solve(_dev(Hn), 16, prec=prec)
    assert err.value.status == gcp.ERR_NONFINITE
    D, info = solver.solve(_dev(H), 16, prec="fp64")
    assert info["status"] == 0
