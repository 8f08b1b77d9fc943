"""Seeded synthetic Hamiltonians for the GCP solver and its tests.

This module only draws inputs.  It holds none of the purification
arithmetic, and both the CUDA path and the FP64 oracle consume what it
returns.  Every generator is a pure function of its seed (numpy PCG64).

Workload families (all real symmetric H in an orthonormal basis, the
setting of the paper's problem statement, footnote to Eq. mcw1b):

* ``rotated_spectrum``: H = Q diag(eps) Q^T with Q from the Householder
  QR of a seeded N(0,1) matrix, occupied eigenvalues uniform in one
  interval and virtual ones in another, separated by a gap.  This is the
  dense analogue of the paper's test Hamiltonians (Sec. "To assess the
  efficiency ...": eigenvalues drawn at random in [-2.5, eps_N] and
  [eps_N+1, 2.5]), rotated so that the matrix is dense.
* ``diagonal_spectrum``: the paper's own test matrices, M x M with
  vanishing off-diagonal elements and eigenvalues drawn in
  [-2.5, eps_N] u [eps_N+1, 2.5] (the Fig. 3 protocol).
* ``tight_binding_cubic``: a simple-cubic lattice insulator with
  nearest-neighbour hopping, staggered onsite energies and disorder.
* ``batched_rotated``: many independent rotated spectra of uneven size.

Reading of the paper (where it does not fix the placement of the
frontier levels): the extreme draws are pinned so that eps_N and eps_N+1
are exactly the interval ends, which makes the gap exact.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "haar_like_q",
    "rotated_spectrum",
    "diagonal_spectrum",
    "tight_binding_cubic",
    "batched_rotated",
    "symmetric_gaussian",
]


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def haar_like_q(M: int, seed: int, qr_backend: str = "numpy") -> np.ndarray:
    """Orthogonal Q from the Householder QR of a seeded N(0,1) M x M matrix.

    ``qr_backend='torch'`` runs the same factorisation with torch (on CUDA
    when available) to keep large inputs quick to build; the Gaussian draw
    is identical, only the rounding of the factorisation differs.  The
    column signs of Q are irrelevant because H = Q diag(eps) Q^T does not
    depend on them.
    """
    A = _rng(seed).standard_normal((M, M))
    if qr_backend == "numpy":
        Q, _ = np.linalg.qr(A)
        return Q
    import torch

    At = torch.from_numpy(A)
    if torch.cuda.is_available():
        try:
            return torch.linalg.qr(At.cuda())[0].cpu().numpy()
        except RuntimeError:
            pass  # the CUDA linear-algebra library may be unloadable (e.g. under a profiler)
    return torch.linalg.qr(At)[0].numpy()


def _two_band_eigs(rng, M, N, occ, virt):
    """N occupied levels uniform in ``occ`` and M-N virtual ones uniform in
    ``virt``; the highest occupied is pinned to occ[1] and the lowest
    virtual to virt[0]; returned sorted ascending."""
    lo_o, hi_o = occ
    lo_v, hi_v = virt
    eo = rng.uniform(lo_o, hi_o, size=N)
    ev = rng.uniform(lo_v, hi_v, size=M - N)
    if N > 0:
        eo[np.argmax(eo)] = hi_o
    if M - N > 0:
        ev[np.argmin(ev)] = lo_v
    return np.sort(np.concatenate([eo, ev]))


def rotated_spectrum(M: int, N: int, occ=(-1.0, -0.1), virt=(0.1, 1.0), seed: int = 1,
                     qr_backend: str = "numpy"):
    """Dense H = Q diag(eps) Q^T with a two-band spectrum.

    Returns ``(H, eps, Q)``: H float64 (exactly symmetric), eps ascending,
    Q orthogonal with H's eigenvector k in column k.
    """
    rng = _rng(seed)
    eps = _two_band_eigs(rng, M, N, occ, virt)
    Q = haar_like_q(M, seed + 7919, qr_backend)
    H = (Q * eps) @ Q.T
    H = 0.5 * (H + H.T)
    return H, eps, Q


def diagonal_spectrum(M: int, N: int, gap: float, seed: int, half_width: float = 2.5):
    """The paper's Fig. 3 test matrices: diagonal H, eigenvalues random in
    [-2.5, eps_N] u [eps_N+1, 2.5] with eps_N+1 - eps_N = gap, centred on 0.

    The diagonal order is shuffled (a diagonal H has no preferred order);
    returns ``(H, eps_sorted)``.
    """
    rng = _rng(seed)
    eps = _two_band_eigs(rng, M, N, (-half_width, -gap / 2), (gap / 2, half_width))
    d = rng.permutation(eps)
    return np.diag(d), eps


def tight_binding_cubic(L: int = 20, t: float = -1.0, delta: float = 0.5, disorder: float = 0.1,
                        seed: int = 3, dtype=np.float32):
    """Simple-cubic L^3 lattice, periodic boundaries, hopping t to the six
    nearest neighbours, onsite +delta on even and -delta on odd sites of the
    bipartite lattice plus uniform disorder in [-disorder, disorder].
    Site index i = x + L*y + L*L*z.  Stored dense."""
    M = L ** 3
    rng = _rng(seed)
    H = np.zeros((M, M), dtype=np.float64)
    idx = np.arange(M)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    onsite = np.where((x + y + z) % 2 == 0, delta, -delta) + rng.uniform(-disorder, disorder, M)
    H[idx, idx] = onsite
    for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        j = ((x + dx) % L) + L * ((y + dy) % L) + L * L * ((z + dz) % L)
        H[idx, j] = t
        H[j, idx] = t
    return H.astype(dtype)


def batched_rotated(batch: int = 512, sizes=tuple(range(64, 1025, 32)), theta: float = 0.25,
                    gap_range=(0.02, 0.2), seed: int = 4, qr_backend: str = "numpy"):
    """Independent rotated spectra of uneven size: M drawn uniformly from
    ``sizes``, N = round(theta*M), gap uniform in ``gap_range`` centred at 0,
    spectrum in [-1, 1].  Returns a list of ``(H, N, eps, Q)``."""
    rng = _rng(seed)
    Ms = rng.choice(np.asarray(sizes), size=batch)
    gaps = rng.uniform(*gap_range, size=batch)
    out = []
    for b in range(batch):
        M = int(Ms[b])
        N = int(round(theta * M))
        g = float(gaps[b])
        H, eps, Q = rotated_spectrum(M, N, (-1.0, -g / 2), (g / 2, 1.0), seed=seed * 100003 + b,
                                     qr_backend=qr_backend)
        out.append((H, N, eps, Q))
    return out


def symmetric_gaussian(M: int, sigma: float, seed: int) -> np.ndarray:
    """Symmetric matrix with V_ij = V_ji ~ N(0, sigma^2) drawn for i <= j."""
    rng = _rng(seed)
    A = rng.normal(0.0, sigma, size=(M, M))
    U = np.triu(A)
    return U + np.triu(U, 1).T
