"""gcp_backward (through the C ABI): the hand-written adjoint of the
fixed-iteration recursion, against the oracle's reverse mode, central
differences of the GPU forward, Hellmann-Feynman and Daleckii-Krein."""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("M,N,K,ck", [(40, 10, 10, 4), (77, 20, 12, 8), (64, 16, 30, 8)])
def test_adjoint_matches_oracle_reverse_mode(solver, M, N, K, ck):
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.2), (0.2, 1.0), seed=M)
    G = inputs.symmetric_gaussian(M, 0.3, seed=M + 1)
    ref, _ = o.reverse_mode_grad(H, N, K, G_D=G, g_E=1.0)
    gH = solver.backward(_dev(H), N, K, G_D=_dev(G), g_E=1.0, ckpt_every=ck).cpu().numpy()
    assert np.abs(gH - gH.T).max() == 0.0
    assert np.abs(gH - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())


def test_adjoint_checkpoint_interval_does_not_matter(solver):
    M, N, K = 50, 12, 17
    H, _, _ = inputs.rotated_spectrum(M, N, seed=3)
    G = inputs.symmetric_gaussian(M, 0.2, seed=4)
    a = solver.backward(_dev(H), N, K, G_D=_dev(G), g_E=0.5, ckpt_every=1)
    b = solver.backward(_dev(H), N, K, G_D=_dev(G), g_E=0.5, ckpt_every=5)
    c = solver.backward(_dev(H), N, K, G_D=_dev(G), g_E=0.5, ckpt_every=64)
    assert torch.equal(a, b) and torch.equal(a, c)


def test_adjoint_matches_central_differences_of_gpu_forward(solver):
    """FD of the GPU FP64 forward itself (no oracle), 6 symmetric directions."""
    M, N, K = 48, 12, 15
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.25), (0.25, 1.0), seed=11)
    G = inputs.symmetric_gaussian(M, 0.3, seed=12)
    Gt = _dev(G)
    gH = solver.backward(_dev(H), N, K, G_D=Gt, g_E=1.0).cpu().numpy()

    def loss(Hx):
        D, info = solver.solve(_dev(Hx), N, prec="fp64", fixed_iters=K)
        return float((D * Gt).sum()) + info["energy"]

    rng = np.random.default_rng(13)
    h = 1e-5
    for _ in range(6):
        E = rng.standard_normal((M, M))
        E = E + E.T
        E /= np.linalg.norm(E)
        fd = (loss(H + h * E) - loss(H - h * E)) / (2 * h)
        assert float(np.sum(gH * E)) == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_hellmann_feynman(solver):
    """dE/dH = D once D_K is converged (the implicit part vanishes)."""
    M, N = 40, 10
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.3), (0.3, 1.0), seed=21)
    gH = solver.backward(_dev(H), N, 40, G_D=None, g_E=1.0).cpu().numpy()
    D, _ = solver.solve(_dev(H), N, prec="fp64", fixed_iters=40)
    assert np.abs(gH - D.cpu().numpy()).max() <= 1e-9


def test_daleckii_krein_at_convergence(solver):
    M, N = 96, 24
    H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -0.2), (0.2, 1.0), seed=31)
    V = inputs.symmetric_gaussian(M, 0.1, seed=32)
    gH = solver.backward(_dev(H), N, 40, G_D=_dev(V), g_E=1.0).cpu().numpy()
    ref = o.daleckii_krein_grad(Q, eps, N, V)
    assert np.abs(gH - ref).max() <= 1e-8


def test_autograd_function(solver):
    from paper_1512_07236_gb300.autograd import gcp_density
    M, N, K = 24, 6, 8
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.3), (0.3, 1.0), seed=41)
    V = inputs.symmetric_gaussian(M, 0.2, seed=42)
    Ht = _dev(H).requires_grad_(True)
    Vt = _dev(V)
    D, E = gcp_density(Ht, N, K)
    L = (D * Vt).sum() + E
    L.backward()
    ref, _ = o.reverse_mode_grad(H, N, K, G_D=V, g_E=1.0)
    assert np.abs(Ht.grad.cpu().numpy() - ref).max() <= 1e-9


def test_config5_sized_adjoint(solver):
    """M=2048, N=512, gap 0.05, L = Tr(D H) + Tr(D V), 40 FP64 steps with a
    checkpoint every 8: Daleckii-Krein on sampled entries and central
    differences along two symmetric directions."""
    M, N, K = 2048, 512, 40
    H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -0.025), (0.025, 1.0), seed=5,
                                        qr_backend="torch")
    V = inputs.symmetric_gaussian(M, 0.1, seed=6)
    Ht, Vt = _dev(H), _dev(V)
    gH = solver.backward(Ht, N, K, G_D=Vt, g_E=1.0, ckpt_every=8).cpu().numpy()
    # Daleckii-Krein at convergence, on a sample of rows
    rows = np.random.default_rng(7).choice(M, 16, replace=False)
    Vq = Q.T @ V @ Q
    f = np.zeros(M)
    f[:N] = 1.0
    de = eps[:, None] - eps[None, :]
    df = f[:, None] - f[None, :]
    F = np.where(df != 0, df / np.where(de == 0, 1.0, de), 0.0)
    FV = F * Vq
    for r in rows:
        ref_row = Q[r, :N] @ Q[:, :N].T + (Q[r, :] @ FV) @ Q.T
        assert np.abs(gH[r] - ref_row).max() <= 1e-6
    rng = np.random.default_rng(8)
    h = 1e-4

    def loss(Hx):
        D, info = solver.solve(_dev(Hx), N, prec="fp64", fixed_iters=K)
        return float((D * Vt).sum()) + info["energy"]

    for _ in range(2):
        E = rng.standard_normal((M, M))
        E = E + E.T
        E /= np.linalg.norm(E)
        fd = (loss(H + h * E) - loss(H - h * E)) / (2 * h)
        assert float(np.sum(gH * E)) == pytest.approx(fd, rel=1e-6)
