"""O2: dense (unblocked) MPS two-site TDVP for Eq. (FHM) (test infrastructure).

Restates Sec. S2.2 (Adaptive TDVP algorithm) with no symmetry blocking:

* the MPS of Eq. (MPS) with local dimension d = 4, site basis index
  s = n_up + 2 n_dn, i.e. |0>, |up>, |dn>, |up dn> = c^dag_up c^dag_dn |0>;
* an MPO of Eq. (FHM) with Jordan-Wigner parity strings, W = 6 channels
  [B, c^dag_up, c^dag_dn, c_up, c_dn, E] (B: nothing placed yet, E: term
  complete);
* second-order two-site TDVP: a left-to-right half sweep and a right-to-left
  half sweep, each with tau = dt/2.  At every bond the two-site tensor is
  evolved forward by exp(-i tau H_eff), split by SVD with truncation, and the
  new centre tensor is evolved backward by exp(+i tau H_eff^(1)) with the
  one-site effective Hamiltonian, except at the last bond of each half sweep;
* the Krylov exponential is Lanczos with full re-orthogonalisation (twice),
  adaptively stopped when beta_k |[exp(-i tau T_k)]_{k,1}| < tol (Sec. S2.2
  says the Krylov dimension is chosen adaptively); exp(-i tau T_k) e_1 is taken
  from the eigendecomposition of the tridiagonal T_k;
* truncation on the truncated weight (Sec. S2.4): singular values sorted in
  descending order, the smallest tail with sum s^2 <= eps * sum s^2 is
  dropped, at most chi_max are kept and at least one; the kept values are
  rescaled to unit norm.

Observables are taken from the full state vector (small L only).
"""
from __future__ import annotations

import numpy as np

from . import truncation

D = 4  # local dimension


# ---------------------------------------------------------------------------
# local operators on one site, index s = n_up + 2 n_dn
# ---------------------------------------------------------------------------

def local_ops():
    """Annihilators a_up, a_dn (with the in-site Jordan-Wigner sign), parity F."""
    a_up = np.zeros((D, D))
    a_dn = np.zeros((D, D))
    F = np.zeros((D, D))
    for s in range(D):
        nu, nd = s & 1, s >> 1 & 1
        F[s, s] = (-1) ** (nu + nd)
        if nu:  # up is the lower mode: no sign inside the site
            a_up[s - 1, s] = 1.0
        if nd:  # down sits above up: sign (-1)^{n_up}
            a_dn[s - 2, s] = (-1) ** nu
    return a_up, a_dn, F


def mpo_tensor(J: float, U: float) -> np.ndarray:
    """Bulk MPO W[w, w', s', s] = <s'| W_{w w'} |s>, channels [B, cd_up, cd_dn, c_up, c_dn, E].

    Term c^dag_{i s} c_{i+1 s} = (a^dag_s F)_i (a_s)_{i+1} and its conjugate
    c^dag_{i+1 s} c_{i s} = (F a_s)_i (a^dag_s)_{i+1}.
    """
    a_up, a_dn, F = local_ops()
    I = np.eye(D)
    W = np.zeros((6, 6, D, D))
    W[0, 0] = I
    W[5, 5] = I
    n_up = a_up.T @ a_up
    n_dn = a_dn.T @ a_dn
    W[0, 5] = U * n_up @ n_dn
    for k, a in enumerate((a_up, a_dn)):
        W[0, 1 + k] = -J * a.T @ F
        W[1 + k, 5] = a
        W[0, 3 + k] = -J * F @ a
        W[3 + k, 5] = a.T
    return W


def mpo_dense(L: int, J: float, U: float) -> np.ndarray:
    """Full 4^L x 4^L matrix of the MPO (small L), rows/cols in C order of (s_0..s_{L-1})."""
    W = mpo_tensor(J, U)
    # contract left to right: T[w, rows, cols]
    T = W[0][:, :, :]  # [w', s', s]
    for _ in range(1, L):
        T = np.einsum("wxy,wvab->vxayb", T, W).reshape(6, T.shape[1] * D, T.shape[2] * D)
    return T[5]


# ---------------------------------------------------------------------------
# MPS helpers
# ---------------------------------------------------------------------------

def neel_mps(L: int) -> list[np.ndarray]:
    """Eq. (neel) as a bond-dimension-1 MPS: even sites |up> (s=1), odd |dn> (s=2)."""
    out = []
    for i in range(L):
        A = np.zeros((1, D, 1), dtype=complex)
        A[0, 1 if i % 2 == 0 else 2, 0] = 1.0
        out.append(A)
    return out


def product_mps(occ) -> list[np.ndarray]:
    """A Fock product state as a bond-dimension-1 MPS; occ[i] in {0, 1 (up), 2 (down),
    3 (both)} is the local basis index s = n_up + 2 n_dn."""
    out = []
    for o in occ:
        A = np.zeros((1, D, 1), dtype=complex)
        A[0, o, 0] = 1.0
        out.append(A)
    return out


def full_state(mps: list[np.ndarray]) -> np.ndarray:
    """Contract the MPS to the full vector indexed by the Fock integer sum_i s_i 4^i."""
    psi = mps[0][0]  # [s0, b]
    for A in mps[1:]:
        psi = np.einsum("xb,bsc->xsc", psi, A).reshape(-1, A.shape[2])
    psi = psi[:, 0]
    L = len(mps)
    # C-order index is sum_i s_i 4^(L-1-i); reorder to sum_i s_i 4^i
    return psi.reshape((D,) * L).transpose(tuple(range(L - 1, -1, -1))).reshape(-1)


def observables_full(psi: np.ndarray, L: int, W: np.ndarray | None = None, mps=None) -> dict:
    """Observables of a full Fock vector indexed by sum_i s_i 4^i."""
    prob = np.abs(psi) ** 2
    idx = np.arange(psi.size)
    s = [(idx >> (2 * i)) & 3 for i in range(L)]
    n_up = np.array([np.sum(prob * (s[i] & 1)) for i in range(L)])
    n_dn = np.array([np.sum(prob * (s[i] >> 1 & 1)) for i in range(L)])
    docc = np.array([np.sum(prob * (s[i] == 3)) for i in range(L)])
    ent = []
    for k in range(1, L):
        M = psi.reshape(D ** (L - k), D ** k)  # rows: right part, cols: left part
        sv = np.linalg.svd(M, compute_uv=False)
        p = sv ** 2
        p = p[p > 1e-300]
        ent.append(float(-np.sum(p * np.log(p))))
    out = {"n_up": n_up, "n_dn": n_dn, "docc": docc, "sz": 0.5 * (n_up - n_dn),
           "n": n_up + n_dn, "s_ent": np.array(ent), "norm": float(np.sum(prob))}
    if W is not None and mps is not None:
        out["energy"] = energy(mps, W)
    return out


# ---------------------------------------------------------------------------
# environments and effective Hamiltonians (Sec. S2.3)
# ---------------------------------------------------------------------------

def left_edge(W):
    E = np.zeros((1, W.shape[0], 1), dtype=complex)
    E[0, 0, 0] = 1.0
    return E


def right_edge(W):
    E = np.zeros((1, W.shape[0], 1), dtype=complex)
    E[0, W.shape[0] - 1, 0] = 1.0
    return E


def update_left(Lenv, A, W):
    """L'[b', w', b] = sum conj(A[a', s', b']) L[a', w, a] W[w, w', s', s] A[a, s, b]."""
    X = np.tensordot(Lenv, A, axes=([2], [0]))            # [a', w, s, b]
    Y = np.tensordot(X, W, axes=([1, 2], [0, 3]))          # [a', b, w', s']
    return np.tensordot(A.conj(), Y, axes=([0, 1], [0, 3])).transpose(0, 2, 1)  # [b', w', b]


def update_right(Renv, B, W):
    """R'[a, w, a'] = sum B[a, s, b] W[w, w', s', s] R[b, w', b'] conj(B[a', s', b'])."""
    X = np.tensordot(B, Renv, axes=([2], [0]))             # [a, s, w', b']
    Y = np.tensordot(X, W, axes=([1, 2], [3, 1]))          # [a, b', w, s']
    return np.tensordot(Y, B.conj(), axes=([1, 3], [2, 1]))  # [a, w, a']


def heff2(Lenv, W1, W2, Renv, theta):
    """theta'[a',s1',s2',b'] = sum L[a',w,a] W1[w,w1,s1',s1] W2[w1,w2,s2',s2] R[b,w2,b'] theta[a,s1,s2,b]."""
    X = np.tensordot(Lenv, theta, axes=([2], [0]))         # [a', w, s1, s2, b]
    X = np.tensordot(X, W1, axes=([1, 2], [0, 3]))         # [a', s2, b, w1, s1']
    X = np.tensordot(X, W2, axes=([3, 1], [0, 3]))         # [a', b, s1', w2, s2']
    X = np.tensordot(X, Renv, axes=([1, 3], [0, 1]))       # [a', s1', s2', b']
    return X


def heff1(Lenv, W, Renv, M):
    """M'[a',s',b'] = sum L[a',w,a] W[w,w',s',s] R[b,w',b'] M[a,s,b]."""
    X = np.tensordot(Lenv, M, axes=([2], [0]))             # [a', w, s, b]
    X = np.tensordot(X, W, axes=([1, 2], [0, 3]))          # [a', b, w', s']
    X = np.tensordot(X, Renv, axes=([1, 2], [0, 1]))       # [a', s', b']
    return X


def heff0(Lenv, Renv, C):
    """Zero-site effective Hamiltonian on the bond matrix between two sites:
    C'[a',b'] = sum L[a',w,a] C[a,b] R[b,w,b'] (the projector term of the bond in
    the one-site projector-splitting integrator, Sec. S2.2)."""
    X = np.tensordot(Lenv, C, axes=([2], [0]))             # [a', w, b]
    return np.tensordot(X, Renv, axes=([1, 2], [1, 0]))    # [a', b']


def energy(mps, W) -> float:
    E = left_edge(W)
    for A in mps:
        E = update_left(E, A, W)
    return float(np.real(E[0, W.shape[0] - 1, 0]))


# ---------------------------------------------------------------------------
# Krylov exponential (Lanczos, full re-orthogonalisation)
# ---------------------------------------------------------------------------

def expm_tridiag_e1(alpha, beta, tau):
    """exp(-i tau T) e_1 for the symmetric tridiagonal T(alpha, beta) via eigh."""
    k = len(alpha)
    T = np.diag(alpha) + np.diag(beta[: k - 1], 1) + np.diag(beta[: k - 1], -1)
    lam, Q = np.linalg.eigh(T)
    return Q @ (np.exp(-1j * tau * lam) * Q[0, :])


def krylov_expm(apply_h, v, tau, kmax=20, tol=1e-12, info=None):
    """exp(-i tau H) v with Lanczos; stops at the first k whose error estimate
    beta_k |c_k| is below tol, on an invariant subspace (beta_k < 1e-14), or at kmax."""
    shape = v.shape
    beta0 = np.linalg.norm(v)
    if beta0 == 0.0:
        return v.copy()
    V = [v.reshape(-1) / beta0]
    alpha, beta = [], []
    c = None
    for k in range(1, kmax + 1):
        w = apply_h(V[-1].reshape(shape)).reshape(-1)
        a = float(np.real(np.vdot(V[-1], w)))
        alpha.append(a)
        w = w - a * V[-1]
        if k > 1:
            w = w - beta[-1] * V[-2]
        Vm = np.array(V)
        for _ in range(2):
            w = w - Vm.T @ (Vm.conj() @ w)
        b = float(np.linalg.norm(w))
        beta.append(b)
        c = expm_tridiag_e1(np.array(alpha), np.array(beta), tau)
        err = b * abs(c[-1])
        if err < tol or b < 1e-14 or k == kmax:
            break
        V.append(w / b)
    if info is not None:
        info["krylov_dim"] = len(alpha)
    out = beta0 * (np.array(V).T @ c)
    return out.reshape(shape)


# ---------------------------------------------------------------------------
# truncation (Sec. S2.4)
# ---------------------------------------------------------------------------

def truncation_count(s: np.ndarray, chi_max: int, eps: float) -> int:
    """Number of leading singular values kept (s sorted descending)."""
    w = s ** 2
    total = np.sum(w)
    n = len(s)
    # drop the longest tail whose weight stays within eps * total
    tail = 0.0
    keep = n
    for k in range(n - 1, 0, -1):
        if tail + w[k] <= eps * total:
            tail += w[k]
            keep = k
        else:
            break
    return max(1, min(keep, chi_max))


def split_svd(theta, chi_max, eps, absorb, degeneracy=0.0):
    """theta[a,s1,s2,b] -> (X[a,s1,c], Y[c,s2,b]); absorb = 'right' puts S into Y, 'left' into X.

    degeneracy > 0: the cut never separates singular values whose squares agree to
    that relative tolerance (degenerate symmetry multiplets are kept or dropped
    together, ``truncation.select_multiplets``)."""
    a, d1, d2, b = theta.shape
    U, s, Vh = np.linalg.svd(theta.reshape(a * d1, d2 * b), full_matrices=False)
    if degeneracy > 0.0:
        n = truncation.dense_keep_count(s, chi_max, eps, degeneracy)
    else:
        n = truncation_count(s, chi_max, eps)
    discarded = float(np.sum(s[n:] ** 2))
    U, s, Vh = U[:, :n], s[:n], Vh[:n]
    s = s / np.linalg.norm(s)
    if absorb == "right":
        X, Y = U, np.diag(s) @ Vh
    else:
        X, Y = U @ np.diag(s), Vh
    return X.reshape(a, d1, n), Y.reshape(n, d2, b), discarded, s


# ---------------------------------------------------------------------------
# the sweep
# ---------------------------------------------------------------------------

class DenseTDVP:
    """Two-site TDVP on a dense MPS; the orthogonality centre rests on site 0."""

    def __init__(self, L, J, U, kmax=20, krylov_tol=1e-12, occ=None, degeneracy=0.0):
        self.L, self.J, self.U = L, J, U
        self.degeneracy = degeneracy  # > 0: degenerate singular values are cut together
        self.W = mpo_tensor(J, U)
        self.kmax, self.tol = kmax, krylov_tol
        # product state (Neel by default): every tensor is both left- and right-canonical
        self.mps = neel_mps(L) if occ is None else product_mps(occ)
        self.max_discarded = 0.0
        self.krylov_dims = []
        self._build_right_envs()

    def _build_right_envs(self):
        L, W = self.L, self.W
        self.R = [None] * (L + 1)
        self.R[L] = right_edge(W)
        for i in range(L - 1, 0, -1):
            self.R[i] = update_right(self.R[i + 1], self.mps[i], W)
        self.Lenv = [None] * (L + 1)
        self.Lenv[0] = left_edge(W)

    def _expm(self, apply_h, v, tau):
        info = {}
        out = krylov_expm(apply_h, v, tau, self.kmax, self.tol, info)
        self.krylov_dims.append(info["krylov_dim"])
        return out

    def bond_lr(self, i, tau, chi_max, eps, backward):
        """Left-to-right two-site update at bond (i, i+1); centre moves from i to i+1."""
        mps, W = self.mps, self.W
        theta = np.einsum("asc,ctb->astb", mps[i], mps[i + 1])
        Le, Re = self.Lenv[i], self.R[i + 2]
        theta = self._expm(lambda x: heff2(Le, W, W, Re, x), theta, tau)
        A, M, disc, s = split_svd(theta, chi_max, eps, "right", self.degeneracy)
        self.max_discarded = max(self.max_discarded, disc)
        self.last_s = s
        mps[i], mps[i + 1] = A, M
        self.Lenv[i + 1] = update_left(self.Lenv[i], A, W)
        if backward:
            Le1 = self.Lenv[i + 1]
            mps[i + 1] = self._expm(lambda x: heff1(Le1, W, Re, x), mps[i + 1], -tau)

    def bond_rl(self, i, tau, chi_max, eps, backward):
        """Right-to-left two-site update at bond (i, i+1); centre moves from i+1 to i."""
        mps, W = self.mps, self.W
        theta = np.einsum("asc,ctb->astb", mps[i], mps[i + 1])
        Le, Re = self.Lenv[i], self.R[i + 2]
        theta = self._expm(lambda x: heff2(Le, W, W, Re, x), theta, tau)
        M, B, disc, s = split_svd(theta, chi_max, eps, "left", self.degeneracy)
        self.max_discarded = max(self.max_discarded, disc)
        self.last_s = s
        mps[i], mps[i + 1] = M, B
        self.R[i + 1] = update_right(self.R[i + 2], B, W)
        if backward:
            Re1 = self.R[i + 1]
            mps[i] = self._expm(lambda x: heff1(Le, W, Re1, x), mps[i], -tau)

    def step(self, dt, chi_max, eps):
        L = self.L
        tau = dt / 2
        for i in range(L - 1):
            self.bond_lr(i, tau, chi_max, eps, i < L - 2)
        for i in range(L - 2, -1, -1):
            self.bond_rl(i, tau, chi_max, eps, i > 0)

    # ----- one-site TDVP (Sec. S2.2: after the bond dimension saturates) -----
    # Left to right with tau: the centre site is evolved forward, QR-split into a
    # left-orthonormal A and a bond matrix C, C is evolved backward with the
    # zero-site H_eff and absorbed into the next site; the last site of the half
    # sweep is evolved forward only.  Right to left mirrors it with an LQ split.
    # The bond dimensions never change (QR keeps min(rows, cols) columns).

    def site_lr(self, i, tau, shift):
        mps, W = self.mps, self.W
        Le, Re = self.Lenv[i], self.R[i + 1]
        mps[i] = self._expm(lambda x: heff1(Le, W, Re, x), mps[i], tau)
        if not shift:
            return
        a, d, b = mps[i].shape
        Q, C = np.linalg.qr(mps[i].reshape(a * d, b))
        mps[i] = Q.reshape(a, d, Q.shape[1])
        self.Lenv[i + 1] = update_left(Le, mps[i], W)
        L1 = self.Lenv[i + 1]
        C = self._expm(lambda x: heff0(L1, Re, x), C, -tau)
        mps[i + 1] = np.tensordot(C, mps[i + 1], axes=([1], [0]))

    def site_rl(self, i, tau, shift):
        mps, W = self.mps, self.W
        Le, Re = self.Lenv[i], self.R[i + 1]
        mps[i] = self._expm(lambda x: heff1(Le, W, Re, x), mps[i], tau)
        if not shift:
            return
        a, d, b = mps[i].shape
        Q, C = np.linalg.qr(mps[i].reshape(a, d * b).conj().T)  # M = C^H Q^H
        B = Q.conj().T
        mps[i] = B.reshape(B.shape[0], d, b)
        self.R[i] = update_right(Re, mps[i], W)
        R1 = self.R[i]
        Cl = self._expm(lambda x: heff0(Le, R1, x), C.conj().T, -tau)
        mps[i - 1] = np.tensordot(mps[i - 1], Cl, axes=([2], [0]))

    def step1(self, dt):
        """One second-order one-site TDVP time step (centre on site 0 before and after)."""
        L = self.L
        tau = dt / 2
        for i in range(L):
            self.site_lr(i, tau, i < L - 1)
        for i in range(L - 1, -1, -1):
            self.site_rl(i, tau, i > 0)

    def bond_dims(self):
        return [A.shape[2] for A in self.mps[:-1]]

    def observables(self):
        return observables_full(full_state(self.mps), self.L, self.W, self.mps)
