"""gcp_solve_batched (through the C ABI): many Hamiltonians of uneven size
in one call, per-instance c_n and stop test.

Each instance runs the same recursion as gcp_solve on the same tiles, so a
batched solve must equal a loop of single solves exactly, and the FP64
batch must meet the FP64 parity bar against the oracle."""
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


def _instances(seed=0):
    """Uneven sizes (ragged tails, one instance per Mp class up to 512),
    N = round(M/4), gaps drawn in [0.05, 0.2]."""
    rng = np.random.default_rng(seed)
    Ms = [64, 96, 130, 200, 256, 300, 384, 512]
    out = []
    for k, M in enumerate(Ms):
        g = float(rng.uniform(0.05, 0.2))
        N = int(round(M / 4))
        H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -g / 2), (g / 2, 1.0), seed=100 + k)
        out.append((H, N, eps, Q))
    return out


@pytest.fixture(scope="module")
def batch():
    return _instances()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_batched_fp64_matches_oracle(solver, batch):
    Hs = [_dev(H) for H, _, _, _ in batch]
    Ds, infos = solver.solve_batched(Hs, [N for _, N, _, _ in batch], prec="fp64", tol=1e-12)
    for (H, N, eps, Q), D, info in zip(batch, Ds, infos):
        ref = o.solve(H, N, tol=1e-12)
        assert info["status"] == 0
        assert np.abs(D.cpu().numpy() - ref["D"]).max() <= 1e-10
        assert abs(info["iters"] - ref["iters"]) <= 1
        assert abs(info["energy"] - ref["E"]) <= 1e-12 * abs(ref["E"])


@pytest.mark.parametrize("prec,refine", [("fp64", "fp64"), ("mixed_fp16", "fp64"),
                                         ("mixed_fp16", "slices"), ("mixed_bf16", "slices"),
                                         ("fp16x3", "fp64")])
def test_batched_equals_loop_of_single_solves(solver, batch, prec, refine):
    Hs = [_dev(H) for H, _, _, _ in batch]
    Ns = [N for _, N, _, _ in batch]
    kw = dict(prec=prec, tol=1e-10 if prec != "fp16x3" else 1e-12, refine=refine)
    Ds, infos = solver.solve_batched(Hs, Ns, **kw)
    for H, N, D, info in zip(Hs, Ns, Ds, infos):
        D1, i1 = solver.solve(H, N, out_dtype=D.dtype, **kw)
        assert info["iters"] == i1["iters"] and info["status"] == i1["status"]
        assert torch.equal(D, D1)


def test_batched_mixed_accuracy(solver, batch):
    Hs = [_dev(H) for H, _, _, _ in batch]
    Ds, infos = solver.solve_batched(Hs, [N for _, N, _, _ in batch], prec="mixed_fp16",
                                     tol=1e-10)
    for (H, N, eps, Q), D, info in zip(batch, Ds, infos):
        Dref = Q[:, :N] @ Q[:, :N].T
        Dg = D.cpu().numpy()
        assert info["status"] == 0
        assert info["idem_fro"] <= 1e-10
        assert abs(np.trace(Dg) - N) <= 1e-9
        assert np.linalg.norm(Dg - Dref) / np.sqrt(N) <= SUBSPACE_TARGET
        assert abs(info["energy"] - eps[:N].sum()) <= 1e-9 * abs(eps[:N].sum())


def test_batched_pmcp_equals_loop(solver, batch):
    Hs = [_dev(H) for H, _, _, _ in batch[:4]]
    Ns = [N for _, N, _, _ in batch[:4]]
    for prec in ("fp64", "mixed_fp16"):
        Ds, infos = solver.solve_batched(Hs, Ns, prec=prec, tol=1e-10, method="pmcp")
        for H, N, D, info in zip(Hs, Ns, Ds, infos):
            D1, i1 = solver.solve(H, N, out_dtype=D.dtype, prec=prec, tol=1e-10, method="pmcp")
            assert info["iters"] == i1["iters"] and info["status"] == i1["status"] == 0
            assert torch.equal(D, D1)


@pytest.mark.parametrize("guess", ["hpcp+", "hole"])
def test_batched_guesses_equal_loop(solver, batch, guess):
    """HPCP+ (Eq. hpcpguess) and hole guesses in a batch: the same
    coefficients, steps and results as single solves (the hole guess may be
    ill-conditioned at theta = 1/4; the status must then agree too)."""
    Hs = [_dev(H) for H, _, _, _ in batch[:5]]
    Ns = [N for _, N, _, _ in batch[:5]]
    for prec in ("fp64", "mixed_fp16"):
        Ds, infos = solver.solve_batched(Hs, Ns, prec=prec, tol=1e-10, guess=guess)
        for H, N, D, info in zip(Hs, Ns, Ds, infos):
            D1, i1 = solver.solve(H, N, out_dtype=D.dtype, prec=prec, tol=1e-10, guess=guess)
            assert info["status"] == i1["status"]
            assert info["alpha"] == i1["alpha"] and info["beta2"] == i1["beta2"]
            if i1["status"] == 0:
                assert info["iters"] == i1["iters"]
                assert torch.equal(D, D1)


def test_batched_edge_instances_do_not_disturb_others(solver, batch):
    """N = 0, N = M and H = mu I inside a batch: each gets its own status;
    the others are unaffected."""
    from paper_1512_07236_gb300 import gcp
    H0, N0, _, _ = batch[2]
    H1, N1, _, _ = batch[4]
    Hs = [_dev(H0), _dev(np.eye(40) * 0.5), _dev(H1), _dev(H0), _dev(H0)]
    Ns = [N0, 10, N1, 0, H0.shape[0]]
    Ds, infos = solver.solve_batched(Hs, Ns, prec="fp64", tol=1e-12)
    assert infos[1]["status"] == gcp.ERR_NO_GAP
    assert np.abs(Ds[1].cpu().numpy() - 0.25 * np.eye(40)).max() <= 1e-15
    assert float(Ds[3].abs().max()) == 0.0
    assert np.array_equal(Ds[4].cpu().numpy(), np.eye(H0.shape[0]))
    for k, (H, N) in ((0, (H0, N0)), (2, (H1, N1))):
        D1, i1 = solver.solve(_dev(H), N, prec="fp64", tol=1e-12)
        assert infos[k]["status"] == 0 and torch.equal(Ds[k], D1)


def test_batched_host_loop_matches_graph(solver, batch):
    Hs = [_dev(H) for H, _, _, _ in batch[:4]]
    Ns = [N for _, N, _, _ in batch[:4]]
    D1, i1 = solver.solve_batched(Hs, Ns, prec="mixed_fp16", tol=1e-10, use_graph=True)
    D2, i2 = solver.solve_batched(Hs, Ns, prec="mixed_fp16", tol=1e-10, use_graph=False)
    for a, b, x, y in zip(D1, D2, i1, i2):
        assert x["iters"] == y["iters"]
        assert torch.equal(a, b)


def _tc_tiles(M):
    """Tensor-core tiles of one instance: 128 x 256 tiles of the padded
    matrix that reach the upper block triangle."""
    Mp = -(-M // 256) * 256
    NI, NJ = Mp // 128, Mp // 256
    return sum(min(2 * j + 2, NI) for j in range(NJ))


def test_batched_work_orders_agree(solver):
    """The batched tensor-core products take their tiles in one of four
    orders (scheduling only): every order gives the same D bit for bit, a
    fixed order is reported back untimed, and the timed choice on a batch of
    at least two tiles per SM measures every candidate and keeps the
    fastest."""
    items = inputs.batched_rotated(96, sizes=tuple(range(64, 1025, 96)), seed=11,
                                   qr_backend="torch")
    Hs = [_dev(H) for H, _, _, _ in items]
    Ns = [N for _, N, _, _ in items]
    kw = dict(prec="mixed_fp16", tol=1e-8)
    try:
        ref = None
        for order in (0, 1, 2, 3):
            solver.set_batched_order(order)
            Ds, infos = solver.solve_batched(Hs, Ns, **kw)
            c, ms = solver.batched_order()
            assert c == order and ms == [-1.0, -1.0, -1.0, -1.0]
            assert all(i["status"] == 0 for i in infos)
            if ref is None:
                ref = Ds
            else:
                assert all(torch.equal(a, b) for a, b in zip(Ds, ref))
        solver.set_batched_order(-1)
        Ds, infos = solver.solve_batched(Hs, Ns, **kw)
        c, ms = solver.batched_order()
        assert all(torch.equal(a, b) for a, b in zip(Ds, ref))
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        assert sum(_tc_tiles(H.shape[0]) for H in Hs) >= 2 * nsm
        assert all(m > 0 for m in ms) and ms[c] == min(ms)
    finally:
        solver.set_batched_order(-1)
