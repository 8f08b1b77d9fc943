"""FP64 CPU oracle for generalized canonical purification (GCP / HPCP).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this module.  It shares no code with the CUDA path and imports nothing from
the ``paper_1512_07236_gb300`` package.

Plain, slow, obviously correct numpy in float64.  A matrix product
(``@``) is used as a library step; there is no blocking, fusion or
reordering beyond the paper's formulas.  Notation follows the paper:
M basis states (matrix dimension), N occupied states, theta = N/M,
D the density matrix, Dbar = I - D the hole density matrix (Eq. closure).

Functions and the passages they follow:

* ``gershgorin_bounds``      Gershgorin disc bounds used in Eq. pmcpguess.
* ``canonical_guess``        Eq. dmguess with the coefficients of Eq. pmcpguess.
* ``hole_guess``             the hole guess (beta_1 = thetabar,
                             beta_2 = -max{...}) before Eq. hpcpguess.
* ``hpcp_plus_guess``        Eq. hpcpguess with the alpha search of
                             Eq. hpcpguessalpha.
* ``solve_holes``            hole purification (Eq. hpcp3 on Dbar).
* ``coefficient_c``          Eq. mcwgamb (c_n, the PM unstable fixed point).
* ``gamma_from_c``           Eq. mcwgama with d = 0.
* ``hpcp_step``              Eq. hpcp3 (closed-form hole-particle step).
* ``lagrangian_step``        Eq. hpcp1a with the gradient of Eq. mcwgrada.
* ``mcweeny_step``           Eq. mcweeny3.
* ``pm_step`` / ``pm_dual_constrained_step``  Appendix A, Eqs. pm1 and pm3.
* ``solve``                  the recursion of Eq. hpcp3 from the guess,
                             terminated as in the text after Eq. hpcp3.
* ``jacobi_eigh``            cyclic Jacobi eigensolver (the exact limit).
* ``ground_state_projector`` the N-representable ground state D* and E*.
* ``scalar_recursion``       the same recursion on eigenvalues (every iterate
                             is a polynomial in H, so it acts eigenvalue-wise).
* ``reverse_mode_grad``      reverse-mode derivative through a fixed number of
                             steps and the guess.
* ``daleckii_krein_grad``    first-order perturbation theory of the converged
                             projector (divided differences).

Readings where the paper is silent (shared with the CUDA path by
specification, not by code):

1. c_n uses the computed Tr D_n, not N; the step then conserves the
   trace for any value of c (Eqs. mcwgamb, hpcp1a).
2. Two stop tests are offered: ||D^2 - D||_F <= tol (computed elementwise)
   and |Tr(D Dbar)| <= tol (the paper's test; Tr(D Dbar) >= 0 while the
   spectrum of D lies in [0, 1], but the hole and mixed guesses of
   Eq. hpcpguess can start outside it, where a negative Tr(D Dbar) is not
   convergence).
3. 0/0 guard: when |den| = |Tr(D - D^2)| <= den_min with
   den_min = 16 * M * u * max(1, Tr D) (u = 2^-53) and the stop test still
   fails, the step uses c = 1/2 (the McWeeny step of Eq. mcweeny3, which the
   recursion reaches as gamma -> 0): c itself would be rounding noise over
   rounding noise.  An initial c outside [0, 1] is reported as
   ill-conditioned (Eqs. pmcpcons1-3 violated).
4. Stagnation: once R < 1e-8, two consecutive non-decreasing R stop the
   loop (converged if R <= tol).
5. H = mu*I (Gershgorin interval of width <= 8 M u max(1, max|H_ii|)):
   D = theta*I is returned with status "no_gap"; theta*I is an exact fixed
   point.
6. Test Eq. testb is read as ||D||_F^2 - N (= Tr D^2 - N).
7. E = Tr(H D) without a spin factor.
8. Eq. hpcpguessalpha (garbled case conditions): delta = 2/3; the target
   Tr(D+_0^2) = N - delta N applies for theta <= 1 - delta, the target
   N - delta Nbar for theta >= delta (each has a real solution only there),
   and alpha = 1/2 (the paper's naive value, good for 0.3 < theta < 0.7) in
   between.
"""
from __future__ import annotations

import math

import numpy as np

U_FP64 = 2.0 ** -53

STATUS_OK = "ok"
STATUS_NOT_CONVERGED = "not_converged"
STATUS_ILL_CONDITIONED = "ill_conditioned"
STATUS_NO_GAP = "no_gap"


# ----------------------------------------------------------------------------
# Initial guess (Eq. dmguess, Eq. pmcpguess)
# ----------------------------------------------------------------------------
def gershgorin_bounds(H):
    """Lower/upper bounds of spec(H) from Gershgorin's disc theorem:
    every eigenvalue lies in some disc |z - H_ii| <= r_i with
    r_i = sum_{j != i} |H_ij|.  Returns (H_min, H_max)."""
    H = np.asarray(H, dtype=np.float64)
    diag = np.diag(H)
    r = np.abs(H).sum(axis=1) - np.abs(diag)
    return float(np.min(diag - r)), float(np.max(diag + r))


def canonical_guess(H, N):
    """D_0 = beta_1 I + beta_2 (mu I - H)   (Eq. dmguess)

    with beta_1 = theta, beta_2 = min(theta/(H_max - mu),
    thetabar/(mu - H_min)) and mu = Tr H / M   (Eq. pmcpguess).
    Returns (D0, info) with info = dict(mu, theta, beta1, beta2, hmin, hmax,
    no_gap).
    """
    H = np.asarray(H, dtype=np.float64)
    M = H.shape[0]
    theta = N / M
    thetabar = 1.0 - theta
    mu = float(np.trace(H)) / M
    hmin, hmax = gershgorin_bounds(H)
    den_up = hmax - mu
    den_lo = mu - hmin
    # a spectrum bound of zero width (H = mu I up to rounding) leaves beta2
    # undefined: reported as "no gap" with beta2 = 0, i.e. D0 = theta I
    scale = max(1.0, float(np.max(np.abs(np.diag(H)))))
    no_gap = (hmax - hmin) <= 8.0 * M * U_FP64 * scale
    cands = []
    if not no_gap:
        if den_up > 0:
            cands.append(theta / den_up)
        if den_lo > 0:
            cands.append(thetabar / den_lo)
    beta2 = 0.0 if no_gap else min(cands)
    D0 = theta * np.eye(M) + beta2 * (mu * np.eye(M) - H)
    return D0, dict(mu=mu, theta=theta, beta1=theta, beta2=beta2, hmin=hmin, hmax=hmax,
                    no_gap=no_gap)


def hole_guess(H, N):
    """Initial hole density matrix Dbar_0 = beta_1 I + beta_2 (mu I - H) with
    beta_1 = thetabar and beta_2 = -max(theta/(H_max - mu),
    thetabar/(mu - H_min))   (Eqs. dmguess and pmcpguess for the hole
    matrix, in the text before Eq. hpcpguess).  Returns (Dbar0, info)."""
    H = np.asarray(H, dtype=np.float64)
    M = H.shape[0]
    _, info = canonical_guess(H, N)
    theta = info["theta"]
    mu = info["mu"]
    bt = theta / (info["hmax"] - mu)
    bb = (1.0 - theta) / (mu - info["hmin"])
    bmax = max(bt, bb)
    Dbar0 = (1.0 - theta) * np.eye(M) - bmax * (mu * np.eye(M) - H)
    return Dbar0, dict(info, beta1_hole=1.0 - theta, beta2_hole=-bmax, beta_max=bmax,
                       beta_min=min(bt, bb))


def hpcp_plus_guess(H, N, delta=2.0 / 3.0, alpha=None):
    """Mixed guess D+_0 = alpha D_0 + (1 - alpha)(I - Dbar_0)   (Eq. hpcpguess).

    Without ``alpha``, alpha is searched in [0, 1] so that Tr(D+_0^2) equals
    N - delta N when theta <= 1 - delta, or N - delta Nbar when theta >= delta
    (Eq. hpcpguessalpha; Nbar = M - N), and alpha = 1/2 in between.  As the
    paper does it: Tr((alpha A + (1 - alpha) B)^2) with A = D_0,
    B = I - Dbar_0 is the quadratic
      alpha^2 Tr(A^2) + 2 alpha (1 - alpha) Tr(AB) + (1 - alpha)^2 Tr(B^2)
    in alpha (one extra product, A B), solved with numpy.roots; its root in
    [0, 1] is taken (the trace is monotone in alpha there), else the end of
    [0, 1] nearer to the target.  Returns (D0, info) with alpha."""
    H = np.asarray(H, dtype=np.float64)
    M = H.shape[0]
    A, info = canonical_guess(H, N)
    if info["no_gap"]:
        return A, dict(info, alpha=1.0)
    Dbar0, hinfo = hole_guess(H, N)
    B = np.eye(M) - Dbar0
    theta = info["theta"]
    if alpha is None:
        if theta <= 1.0 - delta:
            target = N - delta * N
        elif theta >= delta:
            target = N - delta * (M - N)
        else:
            target = None
        if target is None:
            alpha = 0.5
        else:
            tAA = float(np.trace(A @ A))
            tBB = float(np.trace(B @ B))
            tAB = float(np.trace(A @ B))
            coef = [tAA - 2.0 * tAB + tBB, 2.0 * tAB - 2.0 * tBB, tBB - target]
            roots = [r.real for r in np.roots(coef) if abs(r.imag) < 1e-12]
            inside = [r for r in roots if -1e-12 <= r <= 1.0 + 1e-12]
            if inside:
                alpha = min(max(inside[0], 0.0), 1.0)
            else:
                # Tr at alpha = 0 (largest spread) vs the target
                alpha = 0.0 if target >= tBB else 1.0
    D0 = alpha * A + (1.0 - alpha) * B
    return D0, dict(info, alpha=float(alpha), beta2=alpha * info["beta2"]
                    + (1.0 - alpha) * hinfo["beta_max"], beta_max=hinfo["beta_max"])


# ----------------------------------------------------------------------------
# One step of the recursion
# ----------------------------------------------------------------------------
def coefficient_c(D):
    """c = Tr(D^2 - D^3) / Tr(D - D^2)   (Eq. mcwgamb)."""
    D2 = D @ D
    D3 = D2 @ D
    return float(np.trace(D2 - D3) / np.trace(D - D2))


def gamma_from_c(c, d=0.0):
    """gamma = 1/3 - 2c/3 - d/6   (Eq. mcwgama); d = 0 for every D."""
    return 1.0 / 3.0 - 2.0 * c / 3.0 - d / 6.0


def hpcp_step(D, c):
    """D_{n+1} = D + 2 (D^2 Dbar - c D Dbar), Dbar = I - D   (Eq. hpcp3)."""
    M = D.shape[0]
    Dbar = np.eye(M) - D
    return D + 2.0 * (D @ D @ Dbar - c * (D @ Dbar))


def lagrangian_gradient(D, gamma):
    """grad L = grad Omega - 6 gamma (D - D^2), grad Omega = 2(2D^3 - 3D^2 + D)
    (Eqs. mcw2b, mcwgrada)."""
    D2 = D @ D
    D3 = D2 @ D
    return 2.0 * (2.0 * D3 - 3.0 * D2 + D) - 6.0 * gamma * (D - D2)


def lagrangian_step(D, gamma):
    """D_{n+1} = D - (1/2) grad L(D; gamma)   (Eq. hpcp1a)."""
    return D - 0.5 * lagrangian_gradient(D, gamma)


def mcweeny_step(D):
    """D_{n+1} = 3 D^2 - 2 D^3   (Eq. mcweeny3)."""
    D2 = D @ D
    return 3.0 * D2 - 2.0 * (D2 @ D)


def pm_step(D, c):
    """Palser-Manolopoulos canonical purification, Appendix A Eq. pm1:
    c <= 1/2: D+ = [-D^3 + (1+c) D^2 + (1-2c) D] / (1-c)
    c >  1/2: D+ = [-D^3 + (1+c) D^2] / c"""
    D2 = D @ D
    D3 = D2 @ D
    if c <= 0.5:
        return (-D3 + (1.0 + c) * D2 + (1.0 - 2.0 * c) * D) / (1.0 - c)
    return (-D3 + (1.0 + c) * D2) / c


def pm_dual_constrained_step(D, c):
    """PM on the hole matrix constrained to D = I - Dbar, Appendix A Eq. pm3:
    c <= 1/2: D+ = I - [-(I-D)^3/c + (2-c)/c (I-D)^2 - (1-2c)/c (I-D)]
    c >  1/2: D+ = I - [-(I-D)^3/(1-c) + (2-c)/(1-c) (I-D)^2]"""
    M = D.shape[0]
    I = np.eye(M)
    B = I - D
    B2 = B @ B
    B3 = B2 @ B
    if c <= 0.5:
        return I - (-B3 / c + (2.0 - c) / c * B2 - (1.0 - 2.0 * c) / c * B)
    return I - (-B3 / (1.0 - c) + (2.0 - c) / (1.0 - c) * B2)


# ----------------------------------------------------------------------------
# The recursion with termination
# ----------------------------------------------------------------------------
def solve(H, N, tol=1e-12, stop="idem_fro", max_iter=100, fixed_iters=0, D0=None,
          record=True, guess="canonical", method="hpcp"):
    """Purify the canonical guess of H with the recursion of Eq. hpcp3.

    ``guess``: "canonical" (Eq. dmguess / Eq. pmcpguess), "hpcp+"
    (Eq. hpcpguess with the search of Eq. hpcpguessalpha) or "hole"
    (I - Dbar_0: the particle iterate of hole purification, see
    ``solve_holes``).  ``method``: "hpcp" (Eq. hpcp3) or "pmcp" (the
    Palser-Manolopoulos step of Eq. pm1 with the same c_n).

    Per iteration n (all in float64):
      S  = D D
      T1 = Tr D,  T2 = Tr S,  T3 = sum_ij S_ij D_ij (= Tr D^3, D symmetric)
      R  = ||S - D||_F (elementwise; Omega = R^2 is Eq. mcw1b)
      stop test (R <= tol, or Tr(D Dbar) = T1 - T2 <= tol)
      c  = (T2 - T3) / (T1 - T2)                 (Eq. mcwgamb)
      D  = (1 - 2c) D + (2 + 2c) S - 2 S D        (Eq. hpcp3 expanded)

    ``fixed_iters > 0`` runs exactly that many steps with no stop test
    (steps after the 0/0 guard trips become identity steps).
    Returns a dict: D, E, iters, status, history (list of per-step dicts
    with n, T1, T2, T3, R, c, E), guess info.
    """
    H = np.asarray(H, dtype=np.float64)
    M = H.shape[0]
    if not (0 <= N <= M):
        raise ValueError("need 0 <= N <= M")
    if N == 0 or N == M:
        D = np.zeros((M, M)) if N == 0 else np.eye(M)
        return dict(D=D, E=float(np.sum(D * H)), iters=0, status=STATUS_OK, history=[],
                    guess=None)
    if D0 is None:
        if guess == "canonical":
            D, info = canonical_guess(H, N)
        elif guess == "hpcp+":
            D, info = hpcp_plus_guess(H, N)
        elif guess == "hole":
            D, info = hpcp_plus_guess(H, N, alpha=0.0)
        else:
            raise ValueError("unknown guess")
    else:
        D, info = np.array(D0, dtype=np.float64), None
    if info is not None and info["no_gap"]:
        return dict(D=D, E=float(np.sum(D * H)), iters=0, status=STATUS_NO_GAP, history=[],
                    guess=info)
    hist = []
    status = STATUS_NOT_CONVERGED
    n = 0
    R_prev = [math.inf, math.inf]
    while True:
        S = D @ D
        T1 = float(np.trace(D))
        T2 = float(np.trace(S))
        T3 = float(np.sum(S * D))
        R = float(np.sqrt(np.sum((S - D) ** 2)))
        den = T1 - T2
        rec = dict(n=n, T1=T1, T2=T2, T3=T3, R=R, c=float("nan"),
                   E=float(np.sum(D * H)) if record else float("nan"))
        if fixed_iters > 0:
            if n >= fixed_iters:
                hist.append(rec)
                status = STATUS_OK
                break
        else:
            crit = R if stop == "idem_fro" else abs(den)
            if crit <= tol:
                hist.append(rec)
                status = STATUS_OK
                break
            if R < 1e-8 and R >= R_prev[0] and R_prev[0] >= R_prev[1]:
                hist.append(rec)
                status = STATUS_OK if R <= tol else STATUS_NOT_CONVERGED
                break
            if n >= max_iter:
                hist.append(rec)
                status = STATUS_NOT_CONVERGED
                break
        den_min = 16.0 * M * U_FP64 * max(1.0, T1)
        if abs(den) <= den_min:
            if fixed_iters > 0:
                hist.append(rec)
                n += 1
                continue  # identity step
            # Tr(D Dbar) is at rounding level but R > tol: c would be noise
            # over noise, so take the McWeeny step (c = 1/2, gamma = 0), the
            # regime the recursion itself ends in (Eq. mcweeny3)
            c = 0.5
        else:
            c = (T2 - T3) / den
        rec["c"] = c
        hist.append(rec)
        if n == 0 and not (0.0 <= c <= 1.0) and fixed_iters == 0:
            status = STATUS_ILL_CONDITIONED
            break
        P = S @ D
        if method == "pmcp":
            if c <= 0.5:
                D = ((1.0 - 2.0 * c) * D + (1.0 + c) * S - P) / (1.0 - c)
            else:
                D = ((1.0 + c) * S - P) / c
        else:
            D = (1.0 - 2.0 * c) * D + (2.0 + 2.0 * c) * S - 2.0 * P
        R_prev = [R, R_prev[0]]
        n += 1
    return dict(D=D, E=float(np.sum(D * H)), iters=n, status=status, history=hist, guess=info)


def solve_holes(H, N, **kw):
    """Hole purification: Eq. hpcp3 applied to Dbar from the hole guess
    (text before Eq. hpcpguess), N_bar = M - N holes; returns the particle
    result D = I - Dbar_inf (Eq. closure) in the same dict layout as solve."""
    H = np.asarray(H, dtype=np.float64)
    M = H.shape[0]
    if N == 0 or N == M:
        return solve(H, N, **kw)
    Dbar0, info = hole_guess(H, N)
    r = solve(H, M - N, D0=Dbar0, **kw)
    D = np.eye(M) - r["D"]
    return dict(r, D=D, E=float(np.sum(D * H)), guess=info)


def energy(D, H):
    """E = Tr(H D) = sum_ij D_ij H_ij for symmetric matrices."""
    return float(np.sum(np.asarray(D, np.float64) * np.asarray(H, np.float64)))


# ----------------------------------------------------------------------------
# The exact limit: cyclic Jacobi eigensolver
# ----------------------------------------------------------------------------
def _round_robin_pairs(M):
    """Brent-Luk tournament ordering: M-1 rounds (M even) of M/2 disjoint
    index pairs, together covering every pair once per sweep."""
    Me = M + (M % 2)
    players = list(range(Me))
    rounds = []
    for _ in range(Me - 1):
        pairs = []
        for k in range(Me // 2):
            p, q = players[k], players[Me - 1 - k]
            if p < M and q < M:
                pairs.append((min(p, q), max(p, q)))
        rounds.append(np.array(pairs, dtype=np.int64).reshape(-1, 2))
        players = [players[0]] + [players[-1]] + players[1:-1]
    return rounds


def jacobi_eigh(A, tol=1e-14, max_sweeps=60):
    """Cyclic Jacobi eigensolver for a real symmetric matrix.

    Classic two-sided rotations: for a pair (p, q) the angle zeroes A_pq
    (t = sgn(tau)/(|tau| + sqrt(1 + tau^2)), tau = (A_qq - A_pp)/(2 A_pq)).
    The pairs of one sweep are visited in tournament order, M/2 disjoint
    rotations at a time.  Sweeps run until off(A) < tol * ||A||_F.
    Returns (eigenvalues ascending, eigenvectors as columns).
    """
    A = np.array(A, dtype=np.float64)
    M = A.shape[0]
    V = np.eye(M)
    if M == 1:
        return np.diag(A).copy(), V
    normA = np.linalg.norm(A)
    rounds = _round_robin_pairs(M)
    for _ in range(max_sweeps):
        off = math.sqrt(max(0.0, np.sum(A * A) - np.sum(np.diag(A) ** 2)))
        if off <= tol * max(normA, 1e-300):
            break
        for pr in rounds:
            if pr.size == 0:
                continue
            p, q = pr[:, 0], pr[:, 1]
            apq = A[p, q]
            app = A[p, p]
            aqq = A[q, q]
            nz = np.abs(apq) > 1e-300
            tau = np.where(nz, (aqq - app) / (2.0 * np.where(nz, apq, 1.0)), 0.0)
            t = np.where(nz, np.where(tau >= 0, 1.0, -1.0) / (np.abs(tau) + np.hypot(1.0, tau)),
                         0.0)
            cs = 1.0 / np.sqrt(1.0 + t * t)
            sn = t * cs
            # rows: A <- J^T A
            Ap = A[p, :].copy()
            Aq = A[q, :].copy()
            A[p, :] = cs[:, None] * Ap - sn[:, None] * Aq
            A[q, :] = sn[:, None] * Ap + cs[:, None] * Aq
            # columns: A <- A J
            Ap = A[:, p].copy()
            Aq = A[:, q].copy()
            A[:, p] = cs[None, :] * Ap - sn[None, :] * Aq
            A[:, q] = sn[None, :] * Ap + cs[None, :] * Aq
            A[p, q] = 0.0
            A[q, p] = 0.0
            Vp = V[:, p].copy()
            Vq = V[:, q].copy()
            V[:, p] = cs[None, :] * Vp - sn[None, :] * Vq
            V[:, q] = sn[None, :] * Vp + cs[None, :] * Vq
    w = np.diag(A).copy()
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]


def ground_state_projector(H, N, eig=None):
    """D* = sum_{k <= N} v_k v_k^T over the N lowest eigenvectors and
    E* = sum_{k <= N} eps_k: the N-representable idempotent ground state the
    recursion converges to (Eq. mcw4a at its minimum, Eq. testa-c)."""
    w, V = jacobi_eigh(H) if eig is None else eig
    Vo = V[:, :N]
    return Vo @ Vo.T, float(np.sum(w[:N])), (w, V)


# ----------------------------------------------------------------------------
# Scalar recursion on the eigenvalues
# ----------------------------------------------------------------------------
def scalar_recursion(x0, n_steps):
    """Apply the recursion to eigenvalues: c = sum x^2(1-x) / sum x(1-x),
    x <- (1-2c) x + (2+2c) x^2 - 2 x^3.  D_0 is a polynomial in H, hence so is
    every D_n, and the matrix recursion acts on H's eigenvalues one by one.
    Returns (x_n, list of c_n)."""
    x = np.array(x0, dtype=np.float64)
    cs = []
    for _ in range(n_steps):
        c = float(np.sum(x * x * (1 - x)) / np.sum(x * (1 - x)))
        cs.append(c)
        x = (1 - 2 * c) * x + (2 + 2 * c) * x * x - 2 * x ** 3
    return x, cs


def guess_eigenvalues(eps, N, info):
    """Eigenvalues of D_0 = theta I + beta2 (mu I - H) given those of H."""
    return info["theta"] + info["beta2"] * (info["mu"] - np.asarray(eps, np.float64))


# ----------------------------------------------------------------------------
# Derivatives
# ----------------------------------------------------------------------------
def _sym(A):
    return 0.5 * (A + A.T)


def _step_coefficients(c, method):
    """(a, b, g3) of D+ = a D + b D^2 + g3 D^3 for c and the method, and
    their derivatives with respect to c.
      HPCP (Eq. hpcp3): a = 1 - 2c, b = 2 + 2c, g3 = -2.
      PMCP (Eq. pm1):   c <= 1/2: a = (1-2c)/(1-c), b = (1+c)/(1-c),
                                  g3 = -1/(1-c);
                        c >  1/2: a = 0, b = (1+c)/c, g3 = -1/c."""
    if method == "pmcp":
        if c <= 0.5:
            k = 1.0 - c
            return ((1.0 - 2.0 * c) / k, (1.0 + c) / k, -1.0 / k,
                    -1.0 / k ** 2, 2.0 / k ** 2, -1.0 / k ** 2)
        return 0.0, (1.0 + c) / c, -1.0 / c, 0.0, -1.0 / c ** 2, 1.0 / c ** 2
    return 1.0 - 2.0 * c, 2.0 + 2.0 * c, -2.0, -2.0, 2.0, 0.0


def step_adjoint(D, G, T1, T2, c, method="hpcp"):
    """Pull G = dL/dD_{n+1} back through D_{n+1} = aD + bD^2 + g3 D^3 with
    the coefficients of the method (``_step_coefficients``) and
    c = (T2-T3)/(T1-T2) a function of D (Eq. mcwgamb):
      polynomial part: aG + b(GD + DG) + g3(GD^2 + DGD + D^2G)
      c part: s * dc/dD, s = dL/dc = sum G o (a'D + b'D^2 + g3'D^3),
              dc/dD = [(2D - 3D^2) - c(I - 2D)] / (T1 - T2).
    Returns the symmetric dL/dD_n."""
    M = D.shape[0]
    I = np.eye(M)
    a, b, g3, da, db, dg3 = _step_coefficients(c, method)
    D2 = D @ D
    D3 = D2 @ D
    poly = a * G + b * (G @ D + D @ G) + g3 * (G @ D2 + D @ G @ D + D2 @ G)
    s = float(np.sum(G * (da * D + db * D2 + dg3 * D3)))
    dc = ((2.0 * D - 3.0 * D2) - c * (I - 2.0 * D)) / (T1 - T2)
    return _sym(poly + s * dc)


def _branch_guess_adjoint(H, N, G0, which):
    """Pull G0 = dL/dD_0 back through D_0 = theta I + b (mu I - H) with
    b = beta_min ("min": the canonical guess, Eqs. dmguess and pmcpguess) or
    b = beta_max ("max": I - Dbar_0 of the hole guess), mu = Tr H / M,
    beta_min / beta_max the smaller / larger of theta/(H_max - mu) and
    thetabar/(mu - H_min), H_max/H_min from the Gershgorin row of the
    extreme disc (a subgradient at |H_ij| = 0).  Returns the symmetric
    dL/dH."""
    H = np.asarray(H, dtype=np.float64)
    M = H.shape[0]
    _, info = canonical_guess(H, N)
    theta, mu = info["theta"], info["mu"]
    hmin, hmax = info["hmin"], info["hmax"]
    b_up = theta / (hmax - mu) if hmax - mu > 0 else math.inf
    b_lo = (1 - theta) / (mu - hmin) if mu - hmin > 0 else math.inf
    use_up = b_up <= b_lo
    if which == "max" and math.isfinite(max(b_up, b_lo)):
        use_up = not use_up
    b = b_up if use_up else b_lo
    I = np.eye(M)
    gH = -b * G0
    g_mu = b * float(np.trace(G0))
    g_b = float(np.sum(G0 * (mu * I - H)))
    diag = np.diag(H)
    r = np.abs(H).sum(axis=1) - np.abs(diag)
    if use_up:
        # b = theta / (hmax - mu)
        g_mu += g_b * theta / (hmax - mu) ** 2
        g_hmax = -g_b * theta / (hmax - mu) ** 2
        i = int(np.argmax(diag + r))
        row = np.sign(H[i, :])
        row[i] = 1.0
        gH[i, :] += g_hmax * row
    else:
        # b = thetabar / (mu - hmin)
        g_mu += -g_b * (1 - theta) / (mu - hmin) ** 2
        g_hmin = g_b * (1 - theta) / (mu - hmin) ** 2
        i = int(np.argmin(diag - r))
        row = -np.sign(H[i, :])
        row[i] = 1.0
        gH[i, :] += g_hmin * row
    gH += g_mu * I / M
    return _sym(gH)


def guess_adjoint(H, N, G0, guess="canonical"):
    """Pull G0 = dL/dD_0 back through the guess.  "canonical" and "hole"
    are the two branches of ``_branch_guess_adjoint``.  "hpcp+" (Eq. hpcpguess)
    is D_0 = alpha A + (1 - alpha) B with A the canonical guess and
    B = I - Dbar_0: at fixed alpha the weighted branch adjoints, and where
    alpha is the root of q(alpha, H) = Tr(D_0^2) - target = 0 of
    Eq. hpcpguessalpha (not clamped, not the fixed 1/2 of the middle
    fillings) the implicit derivative dalpha/dH = -(dq/dH) / (dq/dalpha),
    dq/dalpha = 2 Tr(D_0 (A - B)), dq/dH = 2 (alpha adj_A(D_0) +
    (1 - alpha) adj_B(D_0)).  Returns the symmetric dL/dH."""
    if guess == "canonical":
        return _branch_guess_adjoint(H, N, G0, "min")
    if guess == "hole":
        return _branch_guess_adjoint(H, N, G0, "max")
    if guess != "hpcp+":
        raise ValueError("unknown guess")
    H = np.asarray(H, dtype=np.float64)
    M = H.shape[0]
    D0, info = hpcp_plus_guess(H, N)
    alpha = info["alpha"]
    A, _ = canonical_guess(H, N)
    B = np.eye(M) - hole_guess(H, N)[0]
    g = alpha * _branch_guess_adjoint(H, N, G0, "min") + \
        (1.0 - alpha) * _branch_guess_adjoint(H, N, G0, "max")
    theta, delta = N / M, 2.0 / 3.0
    has_target = theta <= 1.0 - delta or theta >= delta
    if has_target and 0.0 < alpha < 1.0:
        dq_dalpha = 2.0 * float(np.sum(D0 * (A - B)))
        dq_dH = 2.0 * (alpha * _branch_guess_adjoint(H, N, D0, "min")
                       + (1.0 - alpha) * _branch_guess_adjoint(H, N, D0, "max"))
        dL_dalpha = float(np.sum(G0 * (A - B)))
        g = g - dL_dalpha * dq_dH / dq_dalpha
    return _sym(g)


def reverse_mode_grad(H, N, n_iter, G_D=None, g_E=0.0, guess="canonical", method="hpcp"):
    """dL/dH for L = <G_D, D_K> + g_E * Tr(D_K H), D_K after exactly
    ``n_iter`` steps of the method (Eq. hpcp3, or Eq. pm1 for "pmcp") from the
    guess.  Plain reverse mode: the forward pass stores every iterate, the
    backward pass applies ``step_adjoint`` in reverse and ``guess_adjoint``
    last.  Returns (dL/dH symmetric, forward result dict)."""
    H = np.asarray(H, dtype=np.float64)
    M = H.shape[0]
    if guess == "canonical":
        D, _ = canonical_guess(H, N)
    elif guess == "hpcp+":
        D, _ = hpcp_plus_guess(H, N)
    elif guess == "hole":
        D, _ = hpcp_plus_guess(H, N, alpha=0.0)
    else:
        raise ValueError("unknown guess")
    Ds, aux = [], []
    for _ in range(n_iter):
        S = D @ D
        T1 = float(np.trace(D))
        T2 = float(np.trace(S))
        T3 = float(np.sum(S * D))
        den = T1 - T2
        Ds.append(D)
        if abs(den) <= 16.0 * M * U_FP64 * max(1.0, T1):
            aux.append(None)  # identity step past the 0/0 guard (|den|, as in solve)
            continue
        c = (T2 - T3) / den
        aux.append((T1, T2, c))
        a, b, g3 = _step_coefficients(c, method)[:3]
        D = a * D + b * S + g3 * (S @ D)
    DK = D
    G = np.zeros((M, M)) if G_D is None else np.array(G_D, dtype=np.float64)
    G = G + g_E * H
    for D_n, ax in zip(reversed(Ds), reversed(aux)):
        if ax is None:
            continue
        G = step_adjoint(D_n, G, *ax, method=method)
    gH = guess_adjoint(H, N, G, guess=guess) + g_E * _sym(DK)
    return gH, dict(D=DK, E=float(np.sum(DK * H)))


def daleckii_krein_grad(Q, eps, N, V):
    """dL/dH at convergence for L = Tr(D H) + Tr(D V), D the projector on the
    N lowest eigenvectors of H = Q diag(eps) Q^T.  First-order perturbation
    theory: dD[dH] = Q (F o (Q^T dH Q)) Q^T with the divided differences
    F_ij = (f_i - f_j)/(eps_i - eps_j), f = 1 on occupied and 0 on virtual
    levels (F = 0 within a block).  Hence dL/dH = D + Q (F o (Q^T (H+V) Q)) Q^T;
    the H part drops because Q^T H Q is diagonal and F_ii = 0."""
    Q = np.asarray(Q, np.float64)
    eps = np.asarray(eps, np.float64)
    M = Q.shape[0]
    f = np.zeros(M)
    f[:N] = 1.0
    de = eps[:, None] - eps[None, :]
    df = f[:, None] - f[None, :]
    F = np.zeros((M, M))
    mask = df != 0
    F[mask] = df[mask] / de[mask]
    Vt = Q.T @ np.asarray(V, np.float64) @ Q
    D = Q[:, :N] @ Q[:, :N].T
    return _sym(D + Q @ (F * Vt) @ Q.T)
