"""Pins for the FP64 oracle: each check ties it to something other than
itself -- a hand-worked example, an independent formula from another part
of the paper, a library eigensolver, brute force, or a closed form."""
import json
import math
import os

import numpy as np
import pytest

from oracle import gcp_oracle as o
from paper_1512_07236_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _rand_sym_spectrum(M, seed, lo=0.05, hi=0.95):
    """A symmetric D with eigenvalues in (lo, hi) (a mid-purification state)."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((M, M)))
    lam = rng.uniform(lo, hi, M)
    return (Q * lam) @ Q.T


# ----------------------------------------------------------------- guess ----
def test_guess_2x2_hand_worked():
    g = _gold("guess_2x2.json")
    H = np.array(g["H"])
    D0, info = o.canonical_guess(H, g["N"])
    assert info["mu"] == pytest.approx(g["mu"], abs=1e-15)
    assert info["hmin"] == pytest.approx(g["hmin"], abs=1e-15)
    assert info["hmax"] == pytest.approx(g["hmax"], abs=1e-15)
    assert info["beta2"] == pytest.approx(g["beta2"], abs=1e-15)
    np.testing.assert_allclose(D0, np.array(g["D0"]), atol=1e-15)


def test_limit_2x2_hand_worked():
    g = _gold("guess_2x2.json")
    H = np.array(g["H"])
    r = o.solve(H, g["N"], tol=1e-13)
    assert r["status"] == o.STATUS_OK
    np.testing.assert_allclose(r["D"], np.array(g["D_star"]), atol=1e-12)
    assert r["E"] == pytest.approx(g["E_star"], abs=1e-12)


def test_gershgorin_bounds_contain_spectrum_and_are_exact_for_diagonal():
    H, eps, _ = inputs.rotated_spectrum(48, 12, seed=11)
    hmin, hmax = o.gershgorin_bounds(H)
    w = np.linalg.eigvalsh(H)
    assert hmin <= w[0] and w[-1] <= hmax
    Hd, epsd = inputs.diagonal_spectrum(30, 7, 0.3, seed=5)
    hmin, hmax = o.gershgorin_bounds(Hd)
    assert hmin == epsd[0] and hmax == epsd[-1]
    # a hand-sized 3x3 disc bound
    H3 = np.array([[2.0, -1.0, 0.5], [-1.0, 0.0, 0.25], [0.5, 0.25, -3.0]])
    assert o.gershgorin_bounds(H3) == (-3.75, 3.5)


@pytest.mark.parametrize("M,N,seed", [(40, 10, 1), (64, 5, 2), (64, 59, 3), (33, 16, 4)])
def test_guess_constraints(M, N, seed):
    """Tr D0 = N (Eq. pmcpcons1), spec(D0) in [0,1], Tr D0 > Tr D0^2 > Tr D0^3
    (Eq. pmcpcons2), Tr D0^3 > 2 Tr D0^2 - Tr D0 (Eq. pmcpcons3), c_0 in [0,1]."""
    H, _, _ = inputs.rotated_spectrum(M, N, seed=seed)
    D0, info = o.canonical_guess(H, N)
    assert abs(np.trace(D0) - N) <= 1e-12 * N
    w = np.linalg.eigvalsh(D0)
    assert w[0] >= -1e-14 and w[-1] <= 1 + 1e-14
    t1, t2, t3 = np.trace(D0), np.trace(D0 @ D0), np.trace(D0 @ D0 @ D0)
    assert t1 > t2 > t3
    assert t3 > 2 * t2 - t1
    c0 = o.coefficient_c(D0)
    assert 0.0 <= c0 <= 1.0


def test_no_gap_returns_theta_identity_fixed_point():
    M, N = 12, 3
    H = 0.7 * np.eye(M)
    r = o.solve(H, N)
    assert r["status"] == o.STATUS_NO_GAP
    np.testing.assert_allclose(r["D"], (N / M) * np.eye(M), atol=1e-15)
    # theta*I is an exact fixed point of the step whatever c the formula gives
    D = (N / M) * np.eye(M)
    np.testing.assert_allclose(o.hpcp_step(D, N / M), D, atol=1e-15)


def test_trivial_fillings():
    H, _, _ = inputs.rotated_spectrum(10, 3, seed=2)
    r0 = o.solve(H, 0)
    rM = o.solve(H, 10)
    assert np.all(r0["D"] == 0) and r0["E"] == 0
    np.testing.assert_array_equal(rM["D"], np.eye(10))
    assert rM["E"] == pytest.approx(np.trace(H))


# ------------------------------------------------------------------ step ----
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_closed_form_equals_lagrangian_descent(seed):
    """Eq. hpcp3 (written with Dbar) equals Eq. hpcp1a (half a gradient
    step on the Lagrangian of Eq. mcw4b with gamma from Eq. mcwgama)."""
    D = _rand_sym_spectrum(24, seed)
    c = o.coefficient_c(D)
    a = o.hpcp_step(D, c)
    b = o.lagrangian_step(D, o.gamma_from_c(c))
    np.testing.assert_allclose(a, b, atol=1e-13)


@pytest.mark.parametrize("seed", [3, 4])
def test_gradient_is_traceless(seed):
    """d = Tr(grad L)/Tr(D - D^2) vanishes for every D once gamma follows
    Eq. mcwgama (text after Eq. mcwgamc)."""
    D = _rand_sym_spectrum(20, seed)
    g = o.lagrangian_gradient(D, o.gamma_from_c(o.coefficient_c(D)))
    assert abs(np.trace(g)) < 1e-12
    # and with another gamma the trace is not conserved
    g2 = o.lagrangian_gradient(D, 0.1)
    assert abs(np.trace(g2)) > 1e-3


@pytest.mark.parametrize("lo,hi", [(0.05, 0.45), (0.5, 0.95), (0.05, 0.95)])
def test_pm_combination_identity(lo, hi):
    """Appendix A: (1-c) pm1a + c pm3a = HPCP for c <= 1/2 and
    c pm1b + (1-c) pm3b = HPCP for c > 1/2."""
    D = _rand_sym_spectrum(18, 7, lo, hi)
    c = o.coefficient_c(D)
    pm = o.pm_step(D, c)
    dual = o.pm_dual_constrained_step(D, c)
    comb = (1 - c) * pm + c * dual if c <= 0.5 else c * pm + (1 - c) * dual
    np.testing.assert_allclose(comb, o.hpcp_step(D, c), atol=1e-11)


def test_c_half_is_mcweeny():
    """At c = 1/2 (gamma = 0) the step is McWeeny purification, Eq. mcweeny3."""
    D = _rand_sym_spectrum(16, 9)
    np.testing.assert_allclose(o.hpcp_step(D, 0.5), o.mcweeny_step(D), atol=1e-13)


def test_diagonal_matrix_step_is_scalar_step():
    """For diagonal D the matrix step acts entrywise on the diagonal (brute force)."""
    rng = np.random.default_rng(3)
    x = rng.uniform(0.02, 0.98, 25)
    D = np.diag(x)
    xs, cs = o.scalar_recursion(x, 1)
    c = o.coefficient_c(D)
    assert c == pytest.approx(cs[0], rel=1e-13)
    np.testing.assert_allclose(np.diag(o.hpcp_step(D, c)), xs, atol=1e-14)


# ------------------------------------------------------------- recursion ----
@pytest.fixture(scope="module")
def run64():
    H, eps, Q = inputs.rotated_spectrum(64, 16, (-1.0, -0.1), (0.1, 1.0), seed=1)
    return H, eps, Q, o.solve(H, 16, tol=1e-12)


def test_trace_conserved_every_step(run64):
    """Tr D_n = N for all n (text after Eq. hpcp1a)."""
    _, _, _, r = run64
    for h in r["history"]:
        assert abs(h["T1"] - 16) <= 1e-12 * 16


def test_c_in_unit_interval_and_tends_to_half(run64):
    """c is PM's unstable fixed point, in [0,1] (text after Fig. 1); in the
    McWeeny regime at the end gamma -> 0, i.e. c -> 1/2."""
    _, _, _, r = run64
    cs = [h["c"] for h in r["history"] if not math.isnan(h["c"])]
    assert all(0.0 <= c <= 1.0 for c in cs)
    assert abs(cs[-1] - 0.5) < 1e-3


def test_energy_monotone(run64):
    """E_n = Tr(H D_n) decreases monotonically (variational, Fig. 3b)."""
    _, _, _, r = run64
    E = [h["E"] for h in r["history"]]
    assert all(E[i + 1] <= E[i] + 1e-13 for i in range(len(E) - 1))


def test_quadratic_final_phase(run64):
    """Quadratic convergence (text after Eq. hpcp3): R_{n+1} <= C R_n^2 once
    R is small."""
    _, _, _, r = run64
    R = [h["R"] for h in r["history"]]
    pairs = [(R[i], R[i + 1]) for i in range(len(R) - 1) if 1e-9 < R[i] < 1e-2]
    assert pairs, R
    for a, b in pairs:
        assert b <= 10.0 * a * a + 1e-14


def test_limit_is_ground_state(run64):
    """D_inf equals the projector on the N lowest eigenvectors, D^2 = D,
    [H, D] = 0, E = sum of the N lowest eigenvalues, and the tests of
    Eq. testa / testb."""
    H, eps, Q, r = run64
    D = r["D"]
    assert r["status"] == o.STATUS_OK
    Dref = Q[:, :16] @ Q[:, :16].T
    assert np.abs(D - Dref).max() < 1e-12
    assert np.linalg.norm(D @ D - D) < 1e-12
    assert np.linalg.norm(H @ D - D @ H) < 1e-12
    assert r["E"] == pytest.approx(eps[:16].sum(), abs=1e-12)
    fro = np.linalg.norm(D)
    assert abs(fro - math.sqrt(np.trace(D))) < 1e-6        # Eq. testa
    assert abs(fro ** 2 - 16) < 1e-6                       # Eq. testb (read as ||D||^2 - N)


def test_limit_matches_jacobi_at_256():
    """Config-1 sized case (M=256, N=64, gap 0.2): the oracle's recursion and
    its own Jacobi eigensolver agree."""
    H, eps, Q = inputs.rotated_spectrum(256, 64, (-1.0, -0.1), (0.1, 1.0), seed=1)
    r = o.solve(H, 64, tol=1e-12)
    Dj, Ej, _ = o.ground_state_projector(H, 64)
    assert r["status"] == o.STATUS_OK
    assert np.abs(r["D"] - Dj).max() < 1e-11
    assert abs(r["E"] - Ej) < 1e-11 * abs(Ej)


def test_testc_on_diagonal_hamiltonian():
    """Eq. testc: for a diagonal H the converged diagonal is the occupation
    pattern of the N lowest levels."""
    H, eps = inputs.diagonal_spectrum(100, 30, 0.5, seed=9)
    r = o.solve(H, 30, tol=1e-10)
    occ = (np.diag(H) <= eps[29]).astype(float)
    assert np.linalg.norm(np.diag(r["D"]) - occ) < 1e-6


def test_scalar_recursion_predicts_matrix_run(run64):
    """Every D_n = Q diag(x_n) Q^T: the eigenvalue recursion reproduces c_n
    while Tr(D Dbar) is far above rounding, and the count of steps."""
    H, eps, Q, r = run64
    _, info = o.canonical_guess(H, 16)
    x0 = o.guess_eigenvalues(eps, 16, info)
    xs, cs = o.scalar_recursion(x0, r["iters"])
    for h, c in zip(r["history"], cs):
        if h["T1"] - h["T2"] > 1e-6:
            assert h["c"] == pytest.approx(c, abs=1e-8)
    # the eigenvalue run meets the same stop test within one step
    x = np.array(x0)
    n = 0
    while np.sqrt(np.sum((x * x - x) ** 2)) > 1e-12 and n < 100:
        x, _ = o.scalar_recursion(x, 1)
        n += 1
    assert abs(n - r["iters"]) <= 1


def test_lambda_d0_within_unit_interval_from_eigs(run64):
    H, eps, Q, _ = run64
    _, info = o.canonical_guess(H, 16)
    x0 = o.guess_eigenvalues(eps, 16, info)
    assert x0.min() >= 0 and x0.max() <= 1
    assert np.sum(x0) == pytest.approx(16, abs=1e-12)


def test_paper_iteration_counts_context():
    """Paper's p-bar on diagonal M=100 matrices (stop Tr(D Dbar) <= 1e-6):
    at theta=0.5 the HPCP and PM counts coincide (both about 10); at
    theta=0.05 HPCP needs about 23/37 of PMCP's steps; p-bar grows with
    ln(1/gap).  Ratios are pinned, absolute counts only to a band."""
    g = _gold("paper_iteration_counts.json")

    def pm_count(H, N, tol):
        D, _ = o.canonical_guess(H, N)
        for n in range(300):
            S = D @ D
            den = np.trace(D) - np.trace(S)
            if den <= tol:
                return n
            D = o.pm_step(D, (np.trace(S) - np.sum(S * D)) / den)
        return 300

    def mean_counts(theta, gap, k=16):
        a, b = [], []
        for s in range(k):
            N = int(round(theta * g["M"]))
            H, _ = inputs.diagonal_spectrum(g["M"], N, gap, seed=1000 + s)
            a.append(o.solve(H, N, tol=g["tol_trace"], stop="trace")["iters"])
            b.append(pm_count(H, N, g["tol_trace"]))
        return np.mean(a), np.mean(b)

    h5, p5 = mean_counts(0.5, 1.0)
    assert h5 == p5 and 6 <= h5 <= 14
    h05, p05 = mean_counts(0.05, 1.0)
    ratio_paper = g["points"][1]["pbar_hpcp"] / 37.0
    assert abs(h05 / p05 - ratio_paper) < 0.12
    assert 10 <= h05 <= 50
    hs = [mean_counts(0.5, gap, 8)[0] for gap in (1.0, 1e-2, 1e-4)]
    assert hs[0] < hs[1] < hs[2]
    d1, d2 = hs[1] - hs[0], hs[2] - hs[1]
    assert abs(d1 - d2) <= 0.35 * max(d1, d2)   # linear in ln(1/gap)


# ----------------------------------------------------------------- Jacobi ---
@pytest.mark.parametrize("M", [1, 2, 7, 30])
def test_jacobi_against_library(M):
    rng = np.random.default_rng(M)
    A = rng.standard_normal((M, M))
    A = A + A.T
    w, V = o.jacobi_eigh(A)
    np.testing.assert_allclose(w, np.linalg.eigvalsh(A), atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(M), atol=1e-12)
    np.testing.assert_allclose(V @ np.diag(w) @ V.T, A, atol=1e-12)


# ------------------------------------------------------------ derivatives --
def _loss(H, N, n_iter, G):
    r = o.solve(H, N, fixed_iters=n_iter, record=False)
    return float(np.sum(G * r["D"])) + r["E"]


def _loss_gm(H, N, n_iter, G, guess, method):
    r = o.solve(H, N, fixed_iters=n_iter, record=False, guess=guess, method=method)
    return float(np.sum(G * r["D"])) + r["E"]


@pytest.mark.parametrize("M,N,guess,method", [
    (14, 4, "canonical", "pmcp"),   # c <= 1/2 branch of Eq. pm1
    (14, 10, "canonical", "pmcp"),  # c > 1/2 branch
    (15, 4, "hpcp+", "hpcp"),       # alpha an interior root of Eq. hpcpguessalpha
    (15, 7, "hpcp+", "hpcp"),       # middle filling: alpha = 1/2
    (15, 11, "hpcp+", "pmcp"),      # the other target, PM steps
    (16, 8, "hole", "hpcp"),
    (16, 8, "hole", "pmcp"),
])
def test_reverse_mode_guesses_and_pmcp_match_central_differences(M, N, guess, method):
    """The adjoint of the PM step (both branches of Eq. pm1, through c_n) and
    of the HPCP+ and hole guesses (through alpha and the Gershgorin branch
    they use) against central differences of the oracle's own forward."""
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.2), (0.2, 1.0), seed=21)
    G = inputs.symmetric_gaussian(M, 0.3, seed=22)
    K = 6
    gH, fwd = o.reverse_mode_grad(H, N, K, G_D=G, g_E=1.0, guess=guess, method=method)
    ref = o.solve(H, N, fixed_iters=K, guess=guess, method=method)["D"]
    assert np.abs(fwd["D"] - ref).max() <= 1e-14
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(6):
        E = rng.standard_normal((M, M))
        E = E + E.T
        E /= np.linalg.norm(E)
        fd = (_loss_gm(H + h * E, N, K, G, guess, method)
              - _loss_gm(H - h * E, N, K, G, guess, method)) / (2 * h)
        assert float(np.sum(gH * E)) == pytest.approx(fd, rel=1e-6, abs=1e-8)
    # every guess has Tr D_0 = N and both steps keep the trace: Tr D_K is
    # constant, its gradient zero
    gT, _ = o.reverse_mode_grad(H, N, K, G_D=np.eye(M), g_E=0.0, guess=guess, method=method)
    assert np.abs(gT).max() <= 1e-11


def test_reverse_mode_matches_central_differences():
    M, N, K = 14, 4, 6
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.2), (0.2, 1.0), seed=21)
    G = inputs.symmetric_gaussian(M, 0.3, seed=22)
    gH, fwd = o.reverse_mode_grad(H, N, K, G_D=G, g_E=1.0)
    assert fwd["D"] == pytest.approx(o.solve(H, N, fixed_iters=K)["D"], abs=1e-15)
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(6):
        E = rng.standard_normal((M, M))
        E = E + E.T
        E /= np.linalg.norm(E)
        fd = (_loss(H + h * E, N, K, G) - _loss(H - h * E, N, K, G)) / (2 * h)
        an = float(np.sum(gH * E))
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_hellmann_feynman_at_convergence():
    """dE/dH = D at convergence: the implicit part of the derivative of
    E = Tr(D H) vanishes because D is a stationary projector."""
    M, N = 20, 6
    H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -0.3), (0.3, 1.0), seed=31)
    gH, fwd = o.reverse_mode_grad(H, N, 40, G_D=None, g_E=1.0)
    np.testing.assert_allclose(gH, fwd["D"], atol=1e-9)


def test_daleckii_krein_matches_fd_of_exact_projector_and_reverse_mode():
    M, N = 16, 5
    H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -0.25), (0.25, 1.0), seed=41)
    V = inputs.symmetric_gaussian(M, 0.1, seed=42)
    g_dk = o.daleckii_krein_grad(Q, eps, N, V)

    def exact_loss(Hx):
        w, U = np.linalg.eigh(Hx)
        D = U[:, :N] @ U[:, :N].T
        return float(np.sum(D * (Hx + V)))

    rng = np.random.default_rng(6)
    h = 1e-5
    for _ in range(5):
        E = rng.standard_normal((M, M))
        E = E + E.T
        E /= np.linalg.norm(E)
        fd = (exact_loss(H + h * E) - exact_loss(H - h * E)) / (2 * h)
        assert float(np.sum(g_dk * E)) == pytest.approx(fd, rel=1e-6, abs=1e-9)
    g_rm, _ = o.reverse_mode_grad(H, N, 40, G_D=V, g_E=1.0)
    np.testing.assert_allclose(g_rm, g_dk, atol=1e-8)


@pytest.mark.parametrize("K", [3, 12, 40])
def test_gradient_of_the_conserved_trace_vanishes(K):
    """Every step of Eq. hpcp3 with c_n from Eq. mcwgamb keeps Tr D = N, and
    the guess has Tr D_0 = N for every H: L = Tr D_K is constant, so dL/dH = 0.
    A dropped or mis-signed dc_n/dD term, or a guess adjoint that loses the
    trace constraint, leaves an O(1) gradient here."""
    M, N = 18, 5
    H, _, _ = inputs.rotated_spectrum(M, N, (-1.0, -0.2), (0.2, 1.0), seed=51)
    gH, _ = o.reverse_mode_grad(H, N, K, G_D=np.eye(M), g_E=0.0)
    assert np.abs(gH).max() <= 1e-11
