"""Split-precision tcgen05 path (through the C ABI) against the FP64 oracle.

Tolerances follow from the arithmetic: the split-FP16 state carries about
22 significant bits of the shifted iterate X = D - theta I and the products
accumulate in FP32 (u = 2^-24), so one step agrees with FP64 to ~1e-6
relative; split-BF16 carries ~16 bits (~1e-5).  The mixed modes finish in
FP64, so idempotency, trace and energy reach FP64-refinement accuracy while
the eigenvector subspace keeps the rounding rotation of the split phase
(bounded here by max|dD| <= 3e-6 at gap >= 0.05)."""
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


@pytest.mark.parametrize("prec,tol", [("fp16x3", 2e-6), ("bf16x3", 6e-5)])
@pytest.mark.parametrize("M", [256, 300, 640])
def test_single_split_step(solver, prec, tol, M):
    """One tensor-core step from a mid-purification D (several 128x256 tiles;
    M = 300 pads to 384, so the last 256-wide column block reaches past the
    matrix; 640 pads to itself with an odd number of 128-row blocks)."""
    N = M // 4
    H, _, _ = inputs.rotated_spectrum(M, N, seed=M)
    D, _ = o.canonical_guess(H, N)
    for _ in range(4):
        D = o.hpcp_step(D, o.coefficient_c(D))
    Dt = _dev(D, torch.float32)
    T1, T2, T3, R, c, applied = solver.step(Dt, N, prec=prec)
    S = D @ D
    c_ref = (np.trace(S) - np.sum(S * D)) / (np.trace(D) - np.trace(S))
    assert applied == 1.0
    assert T1 == pytest.approx(np.trace(D), rel=1e-6)
    assert T2 == pytest.approx(np.trace(S), rel=1e-5)
    assert R == pytest.approx(np.linalg.norm(S - D), rel=1e-3)
    assert c == pytest.approx(c_ref, rel=1e-3)
    Dn = o.hpcp_step(D, c_ref)
    err = np.abs(Dt.cpu().numpy().astype(np.float64) - Dn).max()
    assert err <= tol * max(1.0, np.abs(Dn).max()), err


@pytest.mark.parametrize("refine", ["slices", "fp64"])
@pytest.mark.parametrize("prec", ["mixed_fp16", "mixed_bf16"])
@pytest.mark.parametrize("M,N,gap,seed", [(256, 64, 0.2, 1), (512, 128, 0.1, 2), (700, 175, 0.05, 3)])
def test_mixed_solve_parity(solver, prec, refine, M, N, gap, seed):
    H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -gap / 2), (gap / 2, 1.0), seed=seed)
    ref = o.solve(H, N, tol=1e-12)
    D, info = solver.solve(_dev(H), N, prec=prec, tol=1e-10, refine=refine)
    Dg = D.cpu().numpy()
    assert info["status"] == 0, info
    assert info["idem_fro"] <= 1e-10
    # the device residual is the refinement's own; recheck it in plain FP64
    assert np.linalg.norm(Dg @ Dg - Dg) <= 2e-10
    assert abs(np.trace(Dg) - N) <= 1e-9
    dmax = np.abs(Dg - ref["D"]).max()
    dfro = np.linalg.norm(Dg - ref["D"]) / np.sqrt(N)
    # the subspace keeps the rotation left by the split phase; its size is
    # set by the representation (2^-22 fp16, 2^-17 bf16) and by the
    # truncating FP32 accumulation of the tensor cores
    if prec == "mixed_fp16":
        assert dfro <= SUBSPACE_TARGET and dmax <= 3 * SUBSPACE_TARGET, (dmax, dfro)
    else:  # mixed_bf16 misses the target (see conftest)
        assert dfro <= SUBSPACE_BF16 and dmax <= SUBSPACE_BF16, (dmax, dfro)
    assert abs(info["energy"] - ref["E"]) <= 1e-9 * abs(ref["E"])
    assert info["iters_lowp"] >= 1 and info["iters_fp64"] >= 1


def test_split_only_reaches_its_floor(solver):
    """FP16X3 alone stops when the products can do no better; the result is
    near-idempotent at the FP32 level and its trace stays at N."""
    M, N = 512, 128
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.05), (0.05, 1.0), seed=12)
    ref = o.solve(H, N, tol=1e-12)
    D, info = solver.solve(_dev(H), N, prec="fp16x3", tol=1e-12, out_dtype=torch.float32)
    assert info["iters_fp64"] == 0
    assert info["idem_fro"] <= 1e-4
    Dg = D.cpu().numpy().astype(np.float64)
    assert abs(np.trace(Dg) - N) <= 1e-3
    assert np.abs(Dg - ref["D"]).max() <= 1e-5


def test_mixed_history_phases(solver):
    M, N = 384, 96
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.05), (0.05, 1.0), seed=13)
    D, info = solver.solve(_dev(H), N, prec="mixed_fp16", tol=1e-11, history_cap=300,
                           refine="fp64")
    hist = solver.history(300)
    phases = [int(h["phase"]) for h in hist]
    assert phases[0] == 1 and phases[-1] == 0
    assert sum(1 for p in phases if p == 1) >= info["iters_lowp"]
    for h in hist:
        assert abs(h["T1"] - N) <= 1e-3
    E = [h["E"] for h in hist if h["phase"] == 1]
    assert all(E[i + 1] <= E[i] + 1e-6 for i in range(len(E) - 1))


def test_mixed_with_float32_hamiltonian(solver):
    """Tight-binding style FP32 input (small lattice)."""
    H = inputs.tight_binding_cubic(L=8, seed=3)  # M = 512, N = 256
    M = H.shape[0]
    ref = o.solve(H.astype(np.float64), M // 2, tol=1e-12)
    D, info = solver.solve(_dev(H, torch.float32), M // 2, prec="mixed_fp16", tol=1e-10)
    assert info["status"] == 0
    assert abs(info["energy"] - ref["E"]) / M <= 1e-10
    Dg = D.cpu().numpy()
    assert np.linalg.norm(Dg - ref["D"]) / np.sqrt(M // 2) <= SUBSPACE_TARGET
    assert np.abs(Dg - ref["D"]).max() <= 3 * SUBSPACE_TARGET


def test_slice_refinement_agrees_with_fp64_refinement(solver):
    """Both refinements purify the same split-phase result: the exact-slice
    McWeeny steps and the FP64 HPCP steps land on the same projector."""
    M, N = 1000, 250
    H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -0.02), (0.02, 1.0), seed=21)
    Ds, i_s = solver.solve(_dev(H), N, prec="mixed_fp16", tol=1e-10, refine="slices")
    Df, i_f = solver.solve(_dev(H), N, prec="mixed_fp16", tol=1e-10, refine="fp64")
    assert i_s["status"] == 0 and i_f["status"] == 0
    assert i_s["iters_lowp"] == i_f["iters_lowp"]
    a, b = Ds.cpu().numpy(), Df.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-9
    assert abs(np.trace(a) - N) <= 1e-9
    assert abs(i_s["energy"] - i_f["energy"]) <= 1e-12 * abs(i_f["energy"])
