"""O3: the U = 0 limit of Eq. (FHM) in closed form (test infrastructure).

At U = 0 the two spin species hop independently with the one-body matrix
h = -J * (adjacency of the open chain).  For a Slater-determinant start such as
the Neel state of Eq. (neel) the one-body correlation matrix
G_sigma(t)_{ij} = <c^dag_{i sigma} c_{j sigma}>(t) obeys
G(t) = exp(i h t) G(0) exp(-i h t), with G_up(0) = diag(1 on sublattice A)
and G_dn(0) = diag(1 on sublattice B).  Then

* n_{i sigma}(t) = G_sigma(t)_{ii},
* docc_i = n_{i up} n_{i dn} (the two species are uncorrelated),
* the entanglement entropy of a cut is the sum over species of
  -sum_nu [nu ln nu + (1-nu) ln(1-nu)] over the eigenvalues nu of the block
  of G_sigma restricted to the left sites (Peschel's formula for Gaussian
  states),
* E = sum_sigma Tr(h G_sigma).
"""
from __future__ import annotations

import numpy as np


def hopping_matrix(L: int, J: float) -> np.ndarray:
    h = np.zeros((L, L))
    for i in range(L - 1):
        h[i, i + 1] = h[i + 1, i] = -J
    return h


def correlation_matrices(L: int, J: float, t: float):
    h = hopping_matrix(L, J)
    w, V = np.linalg.eigh(h)
    Ut = V @ np.diag(np.exp(1j * w * t)) @ V.T  # exp(i h t)
    G_up0 = np.diag([1.0 if i % 2 == 0 else 0.0 for i in range(L)])
    G_dn0 = np.diag([0.0 if i % 2 == 0 else 1.0 for i in range(L)])
    return Ut @ G_up0 @ Ut.conj().T, Ut @ G_dn0 @ Ut.conj().T


def _species_entropy(G: np.ndarray, k: int) -> float:
    nu = np.linalg.eigvalsh(G[:k, :k])
    s = 0.0
    for x in nu:
        for y in (x, 1.0 - x):
            if y > 1e-300:
                s -= y * np.log(y)
    return s


def observables(L: int, J: float, t: float) -> dict:
    Gu, Gd = correlation_matrices(L, J, t)
    n_up = np.real(np.diag(Gu))
    n_dn = np.real(np.diag(Gd))
    h = hopping_matrix(L, J)
    return {
        "n_up": n_up,
        "n_dn": n_dn,
        "docc": n_up * n_dn,
        "sz": 0.5 * (n_up - n_dn),
        "n": n_up + n_dn,
        "s_ent": np.array([_species_entropy(Gu, k) + _species_entropy(Gd, k) for k in range(1, L)]),
        "energy": float(np.real(np.trace(h @ Gu) + np.trace(h @ Gd))),
    }
