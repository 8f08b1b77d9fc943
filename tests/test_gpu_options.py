"""The option surface of the C ABI on the GPU: GCP_MIXED_AUTO, refine_iters,
the H-symmetry check, and the bounded-wait path of the tensor-core kernel
(gcp_debug_timeout), each through the library's own entry points."""
import numpy as np
import pytest

from oracle import gcp_oracle as o
from paper_1512_07236_gb300 import inputs

from conftest import SUBSPACE_TARGET

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1512_07236_gb300 import gcp
    return gcp


@pytest.fixture(scope="module")
def solver(g):
    return g.Solver()


def _rot(M, N, gap, seed):
    return inputs.rotated_spectrum(M, N, (-1.0, -gap / 2), (gap / 2, 1.0), seed=seed)


def test_mixed_auto_small_m_runs_fp64(solver):
    """Below M = 512 the automatic choice is the FP64 path: the same result,
    bit for bit, as prec='fp64', and no split-precision steps."""
    H, eps, Q = _rot(256, 64, 0.2, 1)
    Ht = torch.from_numpy(H).cuda()
    Da, ia = solver.solve(Ht, 64, prec="mixed_auto", tol=1e-12)
    Df, i_f = solver.solve(Ht, 64, prec="fp64", tol=1e-12)
    assert ia["status"] == 0 and ia["iters_lowp"] == 0
    assert torch.equal(Da, Df) and ia["iters"] == i_f["iters"]


def test_mixed_auto_large_m_runs_mixed(solver):
    """From M = 512 (and tol >= 1e-10) it is the split-FP16 path with
    refinement, held to the stated subspace tolerance."""
    M, N = 640, 160
    H, eps, Q = _rot(M, N, 0.05, 2)
    Ht = torch.from_numpy(H).cuda()
    D, info = solver.solve(Ht, N, prec="mixed_auto", tol=1e-10)
    assert info["status"] == 0 and info["iters_lowp"] > 0 and info["iters_fp64"] >= 1
    Dg = D.cpu().numpy()
    Dref = Q[:, :N] @ Q[:, :N].T
    assert np.linalg.norm(Dg - Dref) / np.sqrt(N) <= SUBSPACE_TARGET
    # a tolerance below the refinement's floor selects FP64 instead
    D2, i2 = solver.solve(Ht, N, prec="mixed_auto", tol=1e-12)
    assert i2["status"] == 0 and i2["iters_lowp"] == 0


def test_refine_iters_caps_the_refinement(solver, g):
    M, N = 512, 128
    H, eps, Q = _rot(M, N, 0.1, 3)
    Ht = torch.from_numpy(H).cuda()
    D, info = solver.solve(Ht, N, prec="mixed_fp16", tol=1e-10)
    assert info["status"] == 0 and info["iters_fp64"] >= 1
    need = info["iters_fp64"]
    # a cap the solve needs no more than: same result
    D1, i1 = solver.solve(Ht, N, prec="mixed_fp16", tol=1e-10, refine_iters=need)
    assert i1["status"] == 0 and torch.equal(D, D1)
    # an unreachable tolerance with one refinement step: NOT_CONVERGED after
    # exactly one step, the iterate still returned
    D2, i2 = solver.solve(Ht, N, prec="mixed_fp16", tol=1e-15, refine_iters=1)
    assert i2["status"] == g.ERR_NOT_CONVERGED and i2["iters_fp64"] == 1
    assert abs(float(torch.trace(D2)) - N) <= 1e-8


def test_symmetry_check(solver, g):
    M, N = 300, 75
    H, eps, Q = _rot(M, N, 0.1, 4)
    Ht = torch.from_numpy(H).cuda()
    D, info = solver.solve(Ht, N, prec="fp64", tol=1e-12, check_symmetry=True)
    assert info["status"] == 0
    Ha = Ht.clone()
    Ha[3, 200] += 1e-3  # one asymmetric pair
    with pytest.raises(g.GCPError) as e:
        solver.solve(Ha, N, prec="fp64", tol=1e-12, check_symmetry=True)
    assert e.value.status == g.ERR_INVALID_ARG and "not symmetric" in str(e.value)
    # a relative bound above the defect lets it through
    amax = float(Ha.abs().max())
    D2, i2 = solver.solve(Ha, N, prec="fp64", tol=1e-12, check_symmetry=True,
                          sym_tol=2e-3 / amax)
    # (the FP64 path reads all of this non-symmetric H and may stagnate short
    # of tol: the check only has to let the call through)
    assert i2["status"] in (g.OK, g.ERR_NOT_CONVERGED)
    # FP32 storage, batched form
    Hf = Ht.float().contiguous()
    Haf = Ha.float().contiguous()
    with pytest.raises(g.GCPError) as e:
        solver.solve_batched([Hf, Haf], [N, N], prec="fp64", tol=1e-10, check_symmetry=True)
    assert "instance 1" in str(e.value)


def test_timeout_path_then_a_correct_solve(solver, g):
    """A bounded device-side wait that no thread will satisfy: the kernel
    gives up after ~1 ms, reports GCP_ERR_TIMEOUT, frees its TMEM and returns;
    the same handle then solves correctly."""
    M, N = 512, 128
    H, eps, Q = _rot(M, N, 0.1, 5)
    Ht = torch.from_numpy(H).cuda()
    st = solver.debug_timeout(M, 1e-3)
    torch.cuda.synchronize()
    assert st == g.ERR_TIMEOUT
    assert b"gave up" in solver.lib.gcp_last_error(solver.h)
    D, info = solver.solve(Ht, N, prec="mixed_fp16", tol=1e-10)
    assert info["status"] == 0
    ref = o.solve(H, N, tol=1e-12)
    Dg = D.cpu().numpy()
    assert np.linalg.norm(Dg - ref["D"]) / np.sqrt(N) <= SUBSPACE_TARGET
    assert abs(info["energy"] - ref["E"]) <= 1e-9 * abs(ref["E"])
    # and again, with a different size, on the same handle
    assert solver.debug_timeout(1024, 2e-3) == g.ERR_TIMEOUT
    D, info = solver.solve(Ht, N, prec="fp64", tol=1e-12)
    assert info["status"] == 0
    assert np.abs(D.cpu().numpy() - ref["D"]).max() <= 1e-10
