"""gcp_backward (through the C ABI): the hand-written adjoints of the
fixed-iteration recursion, FP64 (against the oracle's reverse mode, central
differences of the GPU forward, Hellmann-Feynman and Daleckii-Krein) and FP32
on the tensor cores (against the FP64 adjoint, Daleckii-Krein and the same
central differences), plus the conserved-trace invariant for both."""
import time

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


# The FP32 adjoint against FP64 references: the FP32 state (unit roundoff
# 6e-8) and the split-FP16 products leave ~1e-6 relative in D_K itself, which
# enters dL/dH directly through g_E D_K; measured 1-3e-6 relative (max entry
# and Frobenius) on every case below.  The bar keeps a factor of ~4 above.
FP32_BAR = 1e-5


@pytest.mark.parametrize("M,N,K,ck", [(40, 10, 10, 4), (77, 20, 12, 8), (64, 16, 30, 8)])
def test_adjoint_matches_oracle_reverse_mode(solver, M, N, K, ck):
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.2), (0.2, 1.0), seed=M)
    G = inputs.symmetric_gaussian(M, 0.3, seed=M + 1)
    ref, _ = o.reverse_mode_grad(H, N, K, G_D=G, g_E=1.0)
    gH = solver.backward(_dev(H), N, K, G_D=_dev(G), g_E=1.0, ckpt_every=ck).cpu().numpy()
    assert np.abs(gH - gH.T).max() == 0.0
    assert np.abs(gH - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("M,N,guess,method", [
    (40, 10, "canonical", "pmcp"),  # c <= 1/2 branch of Eq. pm1
    (40, 30, "canonical", "pmcp"),  # c > 1/2 branch
    (45, 11, "hpcp+", "hpcp"),      # alpha an interior root of Eq. hpcpguessalpha
    (45, 22, "hpcp+", "hpcp"),      # middle filling, alpha = 1/2
    (45, 34, "hpcp+", "pmcp"),
    (48, 24, "hole", "hpcp"),
    (48, 24, "hole", "pmcp"),
])
def test_adjoint_guesses_and_pmcp_match_oracle(solver, M, N, guess, method):
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.2), (0.2, 1.0), seed=M + N)
    G = inputs.symmetric_gaussian(M, 0.3, seed=M + N + 1)
    K = 12
    ref, _ = o.reverse_mode_grad(H, N, K, G_D=G, g_E=1.0, guess=guess, method=method)
    gH = solver.backward(_dev(H), N, K, G_D=_dev(G), g_E=1.0, ckpt_every=5, guess=guess,
                         method=method).cpu().numpy()
    assert np.abs(gH - gH.T).max() <= 1e-14 * max(1.0, np.abs(ref).max())
    assert np.abs(gH - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max())
    # the conserved trace
    I = torch.eye(M, dtype=torch.float64, device="cuda")
    gT = solver.backward(_dev(H), N, K, G_D=I, g_E=0.0, guess=guess, method=method)
    assert float(gT.abs().max()) <= 1e-12


def test_fp32_adjoint_hpcp_plus_guess(solver):
    """The FP32 adjoint from the HPCP+ guess against the FP64 one."""
    M, N, K = 300, 75, 25
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.1), (0.1, 1.0), seed=91)
    G = inputs.symmetric_gaussian(M, 0.3, seed=92)
    H32, G32 = _dev(H).float(), _dev(G).float()
    ref = solver.backward(H32.double(), N, K, G_D=G32.double(), g_E=1.0,
                          guess="hpcp+").cpu().numpy()
    g = solver.backward(H32, N, K, G_D=G32, g_E=1.0, prec="fp32",
                        guess="hpcp+").double().cpu().numpy()
    assert np.abs(g - ref).max() <= FP32_BAR * np.abs(ref).max()


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


@pytest.mark.parametrize("M,N,K,ck,gap", [(200, 50, 20, 8, 0.2), (300, 75, 25, 4, 0.1),
                                          (513, 128, 30, 8, 0.1), (256, 64, 12, 5, 0.2),
                                          (1000, 250, 40, 16, 0.05)])
def test_fp32_adjoint_matches_fp64_adjoint(solver, M, N, K, ck, gap):
    """The FP32 adjoint (products on the tensor cores, padded to a multiple
    of 128: M = 300 and 513 pad to 384 and 640, where the last 256-wide
    column block reaches past the matrix; 1000 leaves ragged tiles) against
    the FP64 one on
    the same FP32-rounded inputs.  K either stops before the McWeeny endgame
    of the FP32 recursion or runs well past convergence, where both
    recursions have the same limit."""
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -gap / 2), (gap / 2, 1.0), seed=M)
    G = inputs.symmetric_gaussian(M, 0.3, seed=M + 1)
    H32, G32 = _dev(H).float(), _dev(G).float()
    ref = solver.backward(H32.double(), N, K, G_D=G32.double(), g_E=1.0,
                          ckpt_every=ck).cpu().numpy()
    g = solver.backward(H32, N, K, G_D=G32, g_E=1.0, ckpt_every=ck, prec="fp32")
    assert g.dtype == torch.float32
    gn = g.double().cpu().numpy()
    assert np.abs(gn - gn.T).max() == 0.0
    assert np.abs(gn - ref).max() <= FP32_BAR * np.abs(ref).max()


def test_fp32_adjoint_checkpoint_interval_does_not_matter(solver):
    """The recomputed iterates are the forward's bit for bit."""
    M, N, K = 300, 75, 30
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.05), (0.05, 1.0), seed=61)
    G = inputs.symmetric_gaussian(M, 0.2, seed=62)
    Ht, Gt = _dev(H).float(), _dev(G).float()
    a = solver.backward(Ht, N, K, G_D=Gt, g_E=0.5, ckpt_every=1, prec="fp32")
    b = solver.backward(Ht, N, K, G_D=Gt, g_E=0.5, ckpt_every=7, prec="fp32")
    c = solver.backward(Ht, N, K, G_D=Gt, g_E=0.5, ckpt_every=64, prec="fp32")
    assert torch.equal(a, b) and torch.equal(a, c)


@pytest.mark.parametrize("K", [10, 40])
def test_gradient_of_the_conserved_trace_vanishes(solver, K):
    """L = Tr D_K = N for every H, so dL/dH = 0: G_D = I, g_E = 0.  FP64
    to rounding; FP32 to the rounding of its products (the McWeeny steps of
    the FP32 endgame change Tr D only at second order in ||D^2 - D||)."""
    M, N = 384, 96
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.1), (0.1, 1.0), seed=71)
    I = torch.eye(M, dtype=torch.float64, device="cuda")
    g64 = solver.backward(_dev(H), N, K, G_D=I, g_E=0.0)
    assert float(g64.abs().max()) <= 1e-12
    g32 = solver.backward(_dev(H).float(), N, K, G_D=I.float(), g_E=0.0, prec="fp32")
    assert float(g32.abs().max()) <= 1e-6


def test_autograd_function_float32(solver):
    """A float32 H runs the FP32 recursion forward and the FP32 adjoint
    backward: the same D as gcp_solve and the same gradient as gcp_backward."""
    from paper_1512_07236_gb300.autograd import gcp_density
    M, N, K = 320, 80, 30
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.1), (0.1, 1.0), seed=81)
    V = inputs.symmetric_gaussian(M, 0.2, seed=82)
    Ht = _dev(H).float().requires_grad_(True)
    Vt = _dev(V).float()
    D, E = gcp_density(Ht, N, K)
    assert D.dtype == torch.float32
    (D * Vt).sum().add(E).backward()
    ref = solver.backward(Ht.detach(), N, K, G_D=Vt, g_E=1.0, prec="fp32")
    assert torch.equal(Ht.grad, ref)
    D2, _ = solver.solve(Ht.detach(), N, prec="fp32", fixed_iters=K)
    assert torch.equal(D, D2)


@pytest.fixture(scope="module")
def cfg5(solver):
    """M=2048, N=512, gap 0.05, L = Tr(D H) + Tr(D V), 40 steps with a
    checkpoint every 8, in FP64 and in FP32 (the tensor-core adjoint, on H
    and V rounded to FP32); the oracle's Daleckii-Krein gradient at
    convergence; central differences of the GPU FP64 forward along 32 random
    symmetric unit directions, h = 1e-4, each with both adjoints' directional
    derivatives."""
    M, N, K = 2048, 512, 40
    H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -0.025), (0.025, 1.0), seed=5,
                                        qr_backend="torch")
    V = inputs.symmetric_gaussian(M, 0.1, seed=6)
    Ht, Vt = _dev(H), _dev(V)
    gH = solver.backward(Ht, N, K, G_D=Vt, g_E=1.0, ckpt_every=8).cpu().numpy()
    H32, V32 = Ht.float(), Vt.float()
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g32 = solver.backward(H32, N, K, G_D=V32, g_E=1.0, ckpt_every=8, prec="fp32")
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    g32 = g32.double().cpu().numpy()
    dk = o.daleckii_krein_grad(Q, eps, N, V)

    def loss(Hx):
        D, info = solver.solve(_dev(Hx), N, prec="fp64", fixed_iters=K)
        return float((D * Vt).sum()) + info["energy"]

    rng = np.random.default_rng(8)
    h = 1e-4
    fd, ad64, ad32 = [], [], []
    for _ in range(32):
        E = rng.standard_normal((M, M))
        E = E + E.T
        E /= np.linalg.norm(E)
        fd.append((loss(H + h * E) - loss(H - h * E)) / (2 * h))
        ad64.append(float(np.sum(gH * E)))
        ad32.append(float(np.sum(g32 * E)))
    return dict(gH=gH, g32=g32, dk=dk, fd=np.array(fd), ad64=np.array(ad64),
                ad32=np.array(ad32), t32=min(times))


def test_config5_fp64_daleckii_krein(cfg5):
    """After 40 steps D_K is converged to FP64 rounding: the adjoint equals
    first-order perturbation theory of the exact projector, every entry."""
    assert np.abs(cfg5["gH"] - cfg5["dk"]).max() <= 1e-6


def test_config5_fp64_central_differences(cfg5):
    rel = np.abs(cfg5["ad64"] - cfg5["fd"]) / np.abs(cfg5["fd"])
    assert rel.max() <= 1e-6


def test_config5_fp32_daleckii_krein_and_central_differences(cfg5):
    """The FP32 tensor-core adjoint of the FP32 recursion: every entry within
    FP32_BAR of Daleckii-Krein and of the FP64 adjoint; the 32 directional
    derivatives within FP32_BAR of the central differences, relative to their
    root mean square (a random direction's derivative <dL/dH, E> can come
    close to zero, and the error <err, E> does not shrink with it: measured
    per-direction ratios 4e-7 .. 2.6e-5, median ~2e-6)."""
    scale = np.abs(cfg5["dk"]).max()
    assert np.abs(cfg5["g32"] - cfg5["dk"]).max() <= FP32_BAR * scale
    assert np.abs(cfg5["g32"] - cfg5["gH"]).max() <= FP32_BAR * scale
    fd = cfg5["fd"]
    err = np.abs(cfg5["ad32"] - fd)
    assert err.max() <= FP32_BAR * np.sqrt(np.mean(fd ** 2))
    assert np.median(err / np.abs(fd)) <= FP32_BAR


def test_config5_fp32_time(cfg5):
    """Forward with checkpoints plus adjoint, M = 2048, 40 steps."""
    assert cfg5["t32"] <= 0.3
