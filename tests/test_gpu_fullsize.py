"""Full-size workloads through the C ABI, in the configuration bench.py times.

At these sizes the oracle is too slow for element-by-element parity, so the
checks are the properties the result must have at any size, plus sampled
entries of the exact projector that can be formed one by one:
  * the dense Q diag(eps) Q^T Hamiltonian (M = 8192, N = 2048, gap 0.01):
    D_ij = sum_{k < N} Q_ik Q_jk and E = sum_{k < N} eps_k are known exactly;
  * the tight-binding insulator (20^3 sites, FP32 storage, half filling):
    E against the sum of the lowest N eigenvalues from a library eigensolver.
Each check is an independent FP64 recomputation (a plain FP64 product for
||D^2 - D||_F, a trace of the returned D), not the solver's own figures."""
import numpy as np
import pytest

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


@pytest.fixture(scope="module")
def dense8192():
    M, N, gap = 8192, 2048, 0.01
    H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -gap / 2), (gap / 2, 1.0), seed=2,
                                        qr_backend="torch")
    return M, N, H, eps, Q


def _checks(D, N, Ht):
    D2 = D @ D
    R = float(torch.linalg.norm(D2 - D))
    tr = float(torch.trace(D))
    comm = float(torch.linalg.norm(Ht @ D - D @ Ht))
    return R, tr, comm


# mixed_fp16 is held to the stated target; mixed_bf16 misses it (see conftest)
@pytest.mark.parametrize("prec,fro_lim", [("mixed_fp16", SUBSPACE_TARGET),
                                          ("mixed_bf16", SUBSPACE_BF16)])
def test_dense_8192_mixed(solver, dense8192, prec, fro_lim):
    M, N, H, eps, Q = dense8192
    Ht = torch.from_numpy(H).cuda()
    D, info = solver.solve(Ht, N, prec=prec, tol=1e-6)
    assert info["status"] == 0, info
    R, tr, comm = _checks(D, N, Ht)
    assert R <= 1e-6, R
    assert abs(tr - N) <= 1e-9, tr - N
    E_ref = float(eps[:N].sum())
    assert abs(info["energy"] - E_ref) <= 1e-8 * abs(E_ref)
    # subspace error against the exact projector; the split phase's rounding
    # rotation is what remains once the refinement has made D idempotent
    Qo = torch.from_numpy(Q[:, :N]).cuda()
    fro = float(torch.linalg.norm(D - Qo @ Qo.T)) / np.sqrt(N)
    assert fro <= fro_lim, fro
    assert comm <= 10 * fro * np.sqrt(N)
    # sampled entries, each formed on the host from the construction
    rng = np.random.default_rng(5)
    idx = rng.integers(0, M, size=(64, 2))
    Dh = D.cpu().numpy()
    for i, j in idx:
        exact = float(np.dot(Q[i, :N], Q[j, :N]))
        assert abs(Dh[i, j] - exact) <= 50 * fro_lim, (i, j)


def test_dense_8192_fp64_refinements_agree(solver, dense8192):
    """Exact-slice and FP64 refinement of the same split phase agree."""
    M, N, H, eps, Q = dense8192
    Ht = torch.from_numpy(H).cuda()
    Ds, i_s = solver.solve(Ht, N, prec="mixed_fp16", tol=1e-8, refine="slices")
    Df, i_f = solver.solve(Ht, N, prec="mixed_fp16", tol=1e-8, refine="fp64")
    assert i_s["status"] == 0 and i_f["status"] == 0
    assert float((Ds - Df).abs().max()) <= 1e-8
    assert abs(i_s["energy"] - i_f["energy"]) <= 1e-11 * abs(i_f["energy"])


def test_tight_binding_8000(solver):
    Hf = inputs.tight_binding_cubic(L=20, seed=3)
    M = Hf.shape[0]
    N = M // 2
    Ht = torch.from_numpy(Hf).cuda()
    assert Ht.dtype == torch.float32
    D, info = solver.solve(Ht, N, prec="mixed_fp16", tol=1e-6)
    assert info["status"] == 0, info
    H64 = Ht.double()
    R, tr, comm = _checks(D, N, H64)
    assert R <= 1e-6 and abs(tr - N) <= 1e-9, (R, tr - N)
    lam = torch.linalg.eigvalsh(H64)
    E_ref = float(lam[:N].sum())
    assert float(lam[N] - lam[N - 1]) > 0.5  # the staggered potential opens a gap
    assert abs(info["energy"] - E_ref) / M <= 1e-9
    assert abs(float((D * H64).sum()) - info["energy"]) <= 1e-9 * abs(E_ref)
