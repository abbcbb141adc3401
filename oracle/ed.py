"""O1: exact diagonalisation of the open Fermi-Hubbard chain (test infrastructure).

Restates, as plainly as possible:

* Eq. (FHM), Sec. 2: H = -J sum_{<ij>,sigma} (c^dag_{i sigma} c_{j sigma} + h.c.)
  + U sum_i n_{i up} n_{i dn}, open chain, nearest neighbours.
* Eq. (neel), Sec. 2.1: the Neel state prod_{i in A} c^dag_{i up}
  prod_{j in B} c^dag_{j dn} |0>, sublattice A = even sites (0-indexed).
* Sec. S2.1: N and S^z are conserved; the pseudospin operators
  T^+ = sum_i (-1)^i c^dag_{i up} c^dag_{i dn}, T^- = (T^+)^dag, T^z = (N-L)/2.

Fermion modes are ordered p = 2*i + sigma (sigma = 0 up, 1 down), the
Jordan-Wigner order.  A Fock state is an integer whose bit p is n_p, and its
amplitude is taken with respect to the ordered product of creation operators
(lowest mode leftmost) acting on the vacuum.  Time evolution is the plain
definition psi(t) = V exp(-i E t) V^dag psi(0) from a full eigendecomposition.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def mode(i: int, sigma: int) -> int:
    """Jordan-Wigner index of the mode (site i, spin sigma), sigma 0=up 1=down."""
    return 2 * i + sigma


def _parity_below(state: int, p: int) -> int:
    """(-1)^(number of occupied modes with index < p)."""
    return -1 if bin(state & ((1 << p) - 1)).count("1") % 2 else 1


def apply_cdag(p: int, state: int):
    """c^dag_p |state> = sign |state'>; returns (0, None) if mode p is occupied."""
    if state >> p & 1:
        return 0, None
    return _parity_below(state, p), state | (1 << p)


def apply_c(p: int, state: int):
    """c_p |state> = sign |state'>; returns (0, None) if mode p is empty."""
    if not state >> p & 1:
        return 0, None
    return _parity_below(state, p), state & ~(1 << p)


def sector_basis(L: int, n_up: int, n_dn: int) -> list[int]:
    """All Fock states with n_up up-spins and n_dn down-spins, sorted."""
    out = []
    for ups in itertools.combinations(range(L), n_up):
        for dns in itertools.combinations(range(L), n_dn):
            s = 0
            for i in ups:
                s |= 1 << mode(i, 0)
            for i in dns:
                s |= 1 << mode(i, 1)
            out.append(s)
    return sorted(out)


def hamiltonian(L: int, J: float, U: float, basis: list[int]) -> np.ndarray:
    """Dense matrix of Eq. (FHM) on the given (closed) list of Fock states."""
    index = {s: k for k, s in enumerate(basis)}
    H = np.zeros((len(basis), len(basis)))
    for k, s in enumerate(basis):
        # interaction: diagonal
        H[k, k] += U * sum((s >> mode(i, 0) & 1) * (s >> mode(i, 1) & 1) for i in range(L))
        # hopping on each bond, both directions, both spins
        for i in range(L - 1):
            for sigma in (0, 1):
                for p, q in ((mode(i, sigma), mode(i + 1, sigma)), (mode(i + 1, sigma), mode(i, sigma))):
                    s1, t = apply_c(q, s)
                    if s1 == 0:
                        continue
                    s2, u = apply_cdag(p, t)
                    if s2 == 0:
                        continue
                    H[index[u], k] += -J * s1 * s2
    return H


def neel_state(L: int, basis: list[int]) -> np.ndarray:
    """Eq. (neel): prod_{i in A} c^dag_{i up} prod_{j in B} c^dag_{j dn} |0>.

    Operators are applied right to left (the B product acts first), each
    product in increasing site order, A = even sites.
    """
    ops = [mode(i, 0) for i in range(0, L, 2)] + [mode(j, 1) for j in range(1, L, 2)]
    sign, s = 1, 0
    for p in reversed(ops):
        sg, s = apply_cdag(p, s)
        sign *= sg
    psi = np.zeros(len(basis), dtype=complex)
    psi[basis.index(s)] = sign
    return psi


def product_state(L: int, occ, basis: list[int]) -> np.ndarray:
    """A Fock product state: occ[i] in {0: empty, 1: up, 2: down, 3: up and down}.
    The creators are applied right to left in increasing mode order (a global sign
    only)."""
    ops = [mode(i, sg) for i in range(L) for sg in (0, 1) if (occ[i] >> sg) & 1]
    sign, s = 1, 0
    for p in reversed(ops):
        sg, s = apply_cdag(p, s)
        sign *= sg
    psi = np.zeros(len(basis), dtype=complex)
    psi[basis.index(s)] = sign
    return psi


def vacancy_occupations(L: int) -> list[int]:
    """The second initial state of the benchmark (Sec. S1): the Neel pattern (up on even
    sites, down on odd sites) with the centre site L // 2 empty (L odd)."""
    occ = [1 if i % 2 == 0 else 2 for i in range(L)]
    occ[L // 2] = 0
    return occ


def evolve(H: np.ndarray, psi0: np.ndarray, times) -> list[np.ndarray]:
    """psi(t) = V exp(-i E t) V^dag psi0 from the full spectrum of H."""
    E, V = np.linalg.eigh(H)
    c0 = V.conj().T @ psi0
    return [V @ (np.exp(-1j * E * t) * c0) for t in times]


def observables(psi: np.ndarray, basis: list[int], L: int, H: np.ndarray | None = None) -> dict:
    """n_{i up}, n_{i dn}, docc_i = <n_up n_dn>, S^z_i, n_i, entanglement entropy
    of every cut k = 1..L-1 (sites < k on the left), and <H> if H is given."""
    prob = np.abs(psi) ** 2
    bits = np.array(basis, dtype=np.int64)
    n_up = np.array([np.sum(prob * (bits >> mode(i, 0) & 1)) for i in range(L)])
    n_dn = np.array([np.sum(prob * (bits >> mode(i, 1) & 1)) for i in range(L)])
    docc = np.array([np.sum(prob * ((bits >> mode(i, 0) & 1) & (bits >> mode(i, 1) & 1))) for i in range(L)])
    ent = []
    for k in range(1, L):
        ent.append(entanglement_entropy(psi, basis, k))
    out = {
        "n_up": n_up,
        "n_dn": n_dn,
        "docc": docc,
        "sz": 0.5 * (n_up - n_dn),
        "n": n_up + n_dn,
        "s_ent": np.array(ent),
        "norm": float(np.sum(prob)),
    }
    if H is not None:
        out["energy"] = float(np.real(np.vdot(psi, H @ psi)))
    return out


def entanglement_entropy(psi: np.ndarray, basis: list[int], k: int) -> float:
    """von Neumann entropy (natural log) of the cut after site k-1.

    The left part holds modes 0..2k-1; with the Jordan-Wigner ordering the
    ordered-creation Fock basis is a tensor product of left and right
    occupation patterns, so the Schmidt values are the singular values of the
    amplitude matrix M[left pattern, right pattern].
    """
    mask = (1 << (2 * k)) - 1
    lefts = sorted({s & mask for s in basis})
    rights = sorted({s >> (2 * k) for s in basis})
    li = {v: n for n, v in enumerate(lefts)}
    ri = {v: n for n, v in enumerate(rights)}
    M = np.zeros((len(lefts), len(rights)), dtype=complex)
    for amp, s in zip(psi, basis):
        M[li[s & mask], ri[s >> (2 * k)]] = amp
    sv = np.linalg.svd(M, compute_uv=False)
    p = sv ** 2
    p = p[p > 1e-300]
    return float(-np.sum(p * np.log(p)))


# ---------------------------------------------------------------------------
# Full Fock space operators (small L): used to check the symmetry algebra of
# Sec. S2.1 on the Hamiltonian itself.
# ---------------------------------------------------------------------------

def fock_operator_c(L: int, p: int) -> np.ndarray:
    """Dense matrix of c_p on the full 4^L Fock space (ordered-creation basis)."""
    dim = 1 << (2 * L)
    C = np.zeros((dim, dim))
    for s in range(dim):
        sg, t = apply_c(p, s)
        if sg:
            C[t, s] = sg
    return C


def fock_hamiltonian(L: int, J: float, U: float) -> np.ndarray:
    """Eq. (FHM) assembled from operator products on the full Fock space."""
    c = [fock_operator_c(L, p) for p in range(2 * L)]
    cd = [m.T for m in c]
    dim = 1 << (2 * L)
    H = np.zeros((dim, dim))
    for i in range(L - 1):
        for sigma in (0, 1):
            a, b = mode(i, sigma), mode(i + 1, sigma)
            H += -J * (cd[a] @ c[b] + cd[b] @ c[a])
    for i in range(L):
        H += U * (cd[mode(i, 0)] @ c[mode(i, 0)]) @ (cd[mode(i, 1)] @ c[mode(i, 1)])
    return H


def fock_pseudospin(L: int):
    """(T^+, T^-, T^z) of Sec. S2.1 with the (-1)^i phase, 0-indexed sites."""
    c = [fock_operator_c(L, p) for p in range(2 * L)]
    cd = [m.T for m in c]
    dim = 1 << (2 * L)
    Tp = np.zeros((dim, dim))
    for i in range(L):
        Tp += (-1) ** i * cd[mode(i, 0)] @ cd[mode(i, 1)]
    N = sum(cd[p] @ c[p] for p in range(2 * L))
    Tz = 0.5 * (N - L * np.eye(dim))
    return Tp, Tp.T.copy(), Tz


def fock_spin(L: int):
    """(S^+, S^-, S^z) total spin operators on the full Fock space."""
    c = [fock_operator_c(L, p) for p in range(2 * L)]
    cd = [m.T for m in c]
    dim = 1 << (2 * L)
    Sp = np.zeros((dim, dim))
    Sz = np.zeros((dim, dim))
    for i in range(L):
        Sp += cd[mode(i, 0)] @ c[mode(i, 1)]
        Sz += 0.5 * (cd[mode(i, 0)] @ c[mode(i, 0)] - cd[mode(i, 1)] @ c[mode(i, 1)])
    return Sp, Sp.T.copy(), Sz


def sector_dimension(L: int, n_up: int, n_dn: int) -> int:
    return math.comb(L, n_up) * math.comb(L, n_dn)
