"""The mathematics of the stop test after an exact-slice refinement step
(no GPU): numpy FP64 on near-idempotent iterates built from a seeded
rotation, for the step the refinement takes (Eq. hpcp3 with 1 - 2c = a,
|a| <= 0.1 around the McWeeny step of Eq. mcweeny3):

    X = S - D, S = D^2,  D1 = S - 2 X D - a X,  Delta = D1 - D.

Pinned here: |Delta| <= 1.2 ||X||_F (so the operand scale 2^13 / 2^e with
2^e > 2R keeps every scaled entry below 2^13); the K-concatenation
[D | Delta | Delta] [Delta | D | Delta]^T equals D1^2 - D^2; and
||S + W - D1||_F is the residual ||D1^2 - D1||_F of the new iterate."""
import math

import numpy as np
import pytest

from paper_1512_07236_gb300 import inputs


def _near_projector(M, N, eps, seed):
    rng = np.random.default_rng(seed)
    _, _, Q = inputs.rotated_spectrum(M, N, (-1.0, -0.1), (0.1, 1.0), seed=seed)
    lam = np.zeros(M)
    lam[:N] = 1.0
    lam += eps * rng.standard_normal(M)  # eigenvalues within ~eps of 0 or 1
    return (Q * lam) @ Q.T


def _step(D, a):
    S = D @ D
    X = S - D
    D1 = S - 2.0 * X @ D - a * X
    return S, X, 0.5 * (D1 + D1.T)


@pytest.mark.parametrize("a", [-0.1, 0.0, 0.1])
@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-6])
def test_delta_bound_and_scale(a, eps):
    D = _near_projector(160, 40, eps, seed=3)
    S, X, D1 = _step(D, a)
    R = np.linalg.norm(X)
    Delta = D1 - D
    assert np.abs(Delta).max() <= 1.2 * R
    e = math.frexp(2.0 * R)[1]  # 2R < 2^e
    s = 2.0 ** (13 - e)
    assert np.abs(Delta * s).max() < 2.0 ** 13


@pytest.mark.parametrize("a", [-0.05, 0.0, 0.08])
def test_concatenated_product_is_the_difference_of_squares(a):
    D = _near_projector(96, 30, 1e-3, seed=5)
    S, X, D1 = _step(D, a)
    Delta = D1 - D
    A = np.hstack([D, Delta, Delta])   # rows i: [D_i | Delta_i | Delta_i]
    B = np.hstack([Delta, D, Delta])   # rows j: [Delta_j | D_j | Delta_j]
    W = A @ B.T
    ref = D1 @ D1 - D @ D
    assert np.abs(W - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max()) * 96
    assert np.allclose(W, W.T, rtol=0, atol=1e-15 * 96)
    # the stop test's residual is the residual of the new iterate
    R1 = np.linalg.norm(S + W - D1)
    assert R1 == pytest.approx(np.linalg.norm(D1 @ D1 - D1), rel=1e-6, abs=1e-14)


def test_mcweeny_image_of_the_residual():
    """At a = 0 the residual maps as X1 = X^2 (4X - 3I) (D and X commute),
    so one step from R reaches ~3 R^2: the hand-over rule R <= sqrt(tol/3)/2
    leaves the first refinement step at ~tol/4."""
    D = _near_projector(128, 32, 1e-3, seed=7)
    S, X, D1 = _step(D, 0.0)
    X1 = D1 @ D1 - D1
    pred = X @ X @ (4.0 * X - 3.0 * np.eye(128))
    assert np.abs(X1 - pred).max() <= 1e-12
    R = np.linalg.norm(X)
    assert np.linalg.norm(X1) <= 3.0 * R * R * (1.0 + 4.0 * R / 3.0)
