"""Pins for the oracle's hole guess, HPCP+ guess (Eq. hpcpguess with the
search of Eq. hpcpguessalpha), hole purification and the PMCP method.

Each check is fixed by the paper or by the mathematics, not by re-running
the oracle's own formula: traces by brute-force products, spectra by a
library eigensolver against the closed forms written out here, limits
against the Jacobi projector, the particle-hole duality (c + cbar = 1) by
comparing two different loops, and the iteration-count ordering of Fig. 3."""
import numpy as np
import pytest

from oracle import gcp_oracle as o
from paper_1512_07236_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rot(M, N, gap, seed):
    H, eps, Q = inputs.rotated_spectrum(M, N, (-1.0, -gap / 2), (gap / 2, 1.0), seed=seed)
    return H, eps, Q


def _betas(eps, N):
    """beta_min, beta_max from the Gershgorin bounds of a diagonal H, written
    out from Eq. pmcpguess (for a diagonal matrix the discs are exact)."""
    M = len(eps)
    th = N / M
    mu = float(np.mean(eps))
    bt = th / (eps.max() - mu)
    bb = (1 - th) / (mu - eps.min())
    return min(bt, bb), max(bt, bb), mu, th


@pytest.mark.parametrize("theta", [0.1, 0.25, 0.6, 0.9])
def test_hole_guess_closed_form_and_trace(theta):
    M = 60
    N = int(round(theta * M))
    H, eps = inputs.diagonal_spectrum(M, N, 0.3, seed=3)
    Db, info = o.hole_guess(H, N)
    bmin, bmax, mu, th = _betas(eps, N)
    # eigenvalues thetabar - beta_max (mu - eps): diagonal H keeps its order
    assert np.allclose(np.sort(np.linalg.eigvalsh(Db)),
                       np.sort((1 - th) - bmax * (mu - eps)), atol=1e-13)
    assert abs(np.trace(Db) - (M - N)) <= 1e-12 * M
    assert info["beta2_hole"] == pytest.approx(-bmax)


@pytest.mark.parametrize("theta,seed", [(0.05, 1), (0.2, 2), (0.3, 3), (0.5, 4), (0.7, 5),
                                        (0.85, 6), (0.97, 7)])
def test_hpcp_plus_guess_targets(theta, seed):
    M = 100
    N = int(round(theta * M))
    H, eps = inputs.diagonal_spectrum(M, N, 1.0, seed=seed)
    D0, info = o.hpcp_plus_guess(H, N)
    a = info["alpha"]
    assert 0.0 <= a <= 1.0
    bmin, bmax, mu, th = _betas(eps, N)
    # the mixture is theta I + b (mu I - H), b = alpha beta_min + (1-alpha) beta_max
    b = a * bmin + (1 - a) * bmax
    assert np.allclose(np.sort(np.linalg.eigvalsh(D0)), np.sort(th + b * (mu - eps)),
                       atol=1e-13)
    assert abs(np.trace(D0) - N) <= 1e-12 * M
    t2 = float(np.trace(D0 @ D0))
    delta = 2.0 / 3.0
    if th <= 1 - delta and 0.0 < a < 1.0:
        assert t2 == pytest.approx(N - delta * N, rel=1e-12)
    elif th >= delta and 0.0 < a < 1.0:
        assert t2 == pytest.approx(N - delta * (M - N), rel=1e-12)
    elif 1 - delta < th < delta:
        assert a == 0.5
    # footnote to Eq. hpcpguess: the spectrum lies in [-1/2, 3/2]
    lam = np.linalg.eigvalsh(D0)
    assert lam.min() >= -0.5 - 1e-12 and lam.max() <= 1.5 + 1e-12
    # and the first inequality of Eq. pmcpcons2 holds: Tr D0 > Tr D0^2
    assert np.trace(D0) > t2


def test_hpcp_plus_alpha_one_is_canonical_and_spectrum_bound_for_any_alpha():
    H, eps, Q = _rot(80, 20, 0.1, 9)
    D1, _ = o.hpcp_plus_guess(H, 20, alpha=1.0)
    Dc, _ = o.canonical_guess(H, 20)
    assert np.abs(D1 - Dc).max() == 0.0
    for a in np.linspace(0, 1, 7):
        D, _ = o.hpcp_plus_guess(H, 20, alpha=a)
        lam = np.linalg.eigvalsh(D)
        assert lam.min() >= -0.5 - 1e-12 and lam.max() <= 1.5 + 1e-12


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7])
def test_hole_purification_is_the_dual_of_particle_purification(theta):
    """Purifying Dbar with Eq. hpcp3 and purifying D from I - Dbar_0 are the
    same recursion (cbar = 1 - c); both reach the ground-state projector."""
    M = 64
    N = int(round(theta * M))
    H, eps, Q = _rot(M, N, 0.2, 11)
    rh = o.solve_holes(H, N, tol=1e-12)
    rp = o.solve(H, N, tol=1e-12, guess="hole")
    assert rh["status"] == "ok" and rp["status"] == "ok"
    assert abs(rh["iters"] - rp["iters"]) <= 1
    assert np.abs(rh["D"] - rp["D"]).max() <= 1e-10
    Dstar = Q[:, :N] @ Q[:, :N].T
    assert np.abs(rh["D"] - Dstar).max() <= 1e-10
    # cbar_n + c_n = 1 along the two runs while c is well defined
    for a, b in zip(rh["history"][:4], rp["history"][:4]):
        assert a["c"] + b["c"] == pytest.approx(1.0, abs=1e-9)


def test_hole_guess_far_from_half_filling_is_reported_not_stopped():
    """With beta_2 = -max{...} the hole guess leaves [0, 1] at extreme
    filling; Tr(D Dbar) < 0 there must not read as convergence."""
    H, eps = inputs.diagonal_spectrum(100, 5, 1.0, seed=2)
    r = o.solve(H, 5, tol=1e-6, stop="trace", guess="hole")
    assert r["status"] == "ill_conditioned"


@pytest.mark.parametrize("guess", ["canonical", "hpcp+"])
@pytest.mark.parametrize("theta", [0.05, 0.5, 0.9])
def test_pmcp_and_hpcp_plus_reach_the_ground_state(theta, guess):
    M = 64
    N = int(round(theta * M))
    H, eps, Q = _rot(M, N, 0.2, 13)
    Dstar = Q[:, :N] @ Q[:, :N].T
    for method in ("hpcp", "pmcp"):
        r = o.solve(H, N, tol=1e-12, guess=guess, method=method)
        assert r["status"] == "ok"
        assert np.abs(r["D"] - Dstar).max() <= 1e-10
        # both recursions conserve the trace step by step
        for h in r["history"]:
            assert abs(h["T1"] - N) <= 1e-10


def test_iteration_counts_follow_fig3():
    """Fig. 3 (M = 100 diagonal, gap ~ 1, tol 1e-6 on Tr(D Dbar)): PMCP needs
    more steps than HPCP away from half filling, the same at theta = 1/2;
    the HPCP+ guess cuts the count at extreme filling (theta <= 0.3 or
    >= 0.7) and leaves it at theta = 1/2."""
    def mean_iters(theta, **kw):
        M = 100
        N = int(round(theta * M))
        its = []
        for seed in range(6):
            H, _ = inputs.diagonal_spectrum(M, N, 1.0, seed=seed)
            r = o.solve(H, N, tol=1e-6, stop="trace", **kw)
            assert r["status"] == "ok"
            its.append(r["iters"])
        return float(np.mean(its))

    for th in (0.05, 0.95):
        h, p = mean_iters(th), mean_iters(th, method="pmcp")
        hp, pp = mean_iters(th, guess="hpcp+"), mean_iters(th, method="pmcp", guess="hpcp+")
        assert p > 1.3 * h
        assert hp < 0.8 * h and pp < 0.8 * p
    assert mean_iters(0.5) == mean_iters(0.5, method="pmcp") == mean_iters(0.5, guess="hpcp+")
    assert mean_iters(0.01, guess="hpcp+") < 0.6 * mean_iters(0.01)
