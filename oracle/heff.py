"""O4: brute-force effective-Hamiltonian application (test infrastructure).

Sec. S2.3 names the environment updates and the Krylov application of the
effective Hamiltonian as the dominant contractions.  Their plain definition,
written as dense einsums over m-resolved indices, is

  theta'[a',s1',s2',b'] = sum L[a',w,a] W[w,w1,s1',s1] W[w1,w2,s2',s2] R[b,w2,b'] theta[a,s1,s2,b]

(two-site) and M'[a',s',b'] = sum L[a',w,a] W[w,w',s',s] R[b,w',b'] M[a,s,b]
(one-site).

The engine stores U(1)xSU(2) tensors in the reduced form of Eq. (symdecomp)
(Sec. S2.1): one block per multiplet label, no m index.  To compare, this
module expands reduced blocks into m-resolved dense arrays with the
Clebsch-Gordan coefficients of ``oracle.cg``, using the tree conventions that
define the reduced format:

  A/M[(a,alpha),s,(b,beta)]    = A~[a,s,b]   <j_a alpha; j_s sigma | j_b beta>
  theta[(a,alpha),s1,s2,(b,beta)] = sum_c theta~[a,s1,c,s2,b]
                     sum_gamma <j_a alpha; j_s1 sigma1 | j_c gamma><j_c gamma; j_s2 sigma2 | j_b beta>
  L[(a',alpha'),(w,mu),(a,alpha)] = L~[a',w,a] <j_a alpha; j_w mu | j_a' alpha'>
  R[(b,beta),(w,mu),(b',beta')]   = R~[b,w,b'] <j_b beta; j_w mu | j_b' beta'>

and the Hamiltonian in the particle-hole (Shiba) frame c_{i dn} ->
(-1)^i c^dag_{i dn}, in which the charge SU(2) of Sec. S2.1 becomes the
ordinary spin SU(2):

  H' = -J sum_{i,s} (c^dag_{i s} c_{i+1 s} + h.c.) - U sum_i n_{i up} n_{i dn} + (U/2) sum_i n_i.

For states with total S'^z = 0 (all states reached from the Neel state) H'
has the same expectation values and dynamics as Eq. (FHM) with n_{i dn}
replaced by 1 - n'_{i dn}.

MPO channels (m-resolved, 6 components) in the order
[B, cd(+1/2), cd(-1/2), c(+1/2), c(-1/2), E]:

  W[B, cd(m)]  = -J a^dag_m F     W[cd(m), E] = a_m          (m=+1/2: up, -1/2: dn)
  W[B, c(+1/2)] = -J F a_dn       W[c(+1/2), E] = a^dag_dn
  W[B, c(-1/2)] = +J F a_up       W[c(-1/2), E] = -a^dag_up
  W[B, E] = -U n_up n_dn + (U/2)(n_up + n_dn),  W[B,B] = W[E,E] = 1.

The two doublets are the standard spherical components of the spin-1/2
tensor operators c^dag and (c_dn, -c_up), so in the reduced (W = 4) form the
channels are B (0,0), cd (+1, 1/2), c (-1, 1/2), E (0,0).
"""
from __future__ import annotations

import numpy as np

from . import cg as _cg
from .mps import D, local_ops

# site multiplets in the Shiba frame: (n, 2S) -> list of site states, m from +S down
SITE_MULTIPLETS_SU2 = [((0, 0), [0]), ((1, 1), [1, 2]), ((2, 0), [3])]
# U(1)xU(1): (n, 2S^z) -> single state
SITE_MULTIPLETS_U1 = [((0, 0), [0]), ((1, 1), [1]), ((1, -1), [2]), ((2, 0), [3])]
# MPO channel multiplets: (n, 2S) -> channel components, m from +S down
CHANNELS_SU2 = [((0, 0), [0]), ((1, 1), [1, 2]), ((-1, 1), [3, 4]), ((0, 0), [5])]
CHANNELS_U1 = [((0, 0), [0]), ((1, 1), [1]), ((1, -1), [2]), ((-1, 1), [3]), ((-1, -1), [4]), ((0, 0), [5])]


def shiba_mpo_tensor(J: float, U: float) -> np.ndarray:
    """m-resolved MPO W[w, w', s', s] of H' in the channel order documented above."""
    a_up, a_dn, F = local_ops()
    I = np.eye(D)
    n_up = a_up.T @ a_up
    n_dn = a_dn.T @ a_dn
    W = np.zeros((6, 6, D, D))
    W[0, 0] = I
    W[5, 5] = I
    W[0, 5] = -U * n_up @ n_dn + 0.5 * U * (n_up + n_dn)
    W[0, 1] = -J * a_up.T @ F
    W[1, 5] = a_up
    W[0, 2] = -J * a_dn.T @ F
    W[2, 5] = a_dn
    W[0, 3] = -J * F @ a_dn
    W[3, 5] = a_dn.T
    W[0, 4] = J * F @ a_up
    W[4, 5] = -a_up.T
    return W


def heff2_dense(Lenv, W1, W2, Renv, theta):
    """The two-site definition as four pairwise contractions in the stated order
    (L, then W1, then W2, then R); each pairwise contraction is handed to BLAS
    (``optimize=True`` only routes a two-operand einsum through tensordot)."""
    X = np.einsum("xwa,asqb->xwsqb", Lenv, theta, optimize=True)
    X = np.einsum("xwsqb,wuts->xutqb", X, W1, optimize=True)
    X = np.einsum("xutqb,uvrq->xvtrb", X, W2, optimize=True)
    return np.einsum("xvtrb,bvy->xtry", X, Renv, optimize=True)


def heff1_dense(Lenv, W, Renv, M):
    X = np.einsum("xwa,asb->xwsb", Lenv, M)
    X = np.einsum("xwsb,wvts->xvtb", X, W)
    return np.einsum("xvtb,bvy->xty", X, Renv)


def heff2_matrix(Lenv, W1, W2, Renv):
    """H_eff as an explicit matrix on vec(theta) (C order of [a,s1,s2,b]); tiny sizes only."""
    a, _, b = Lenv.shape[2], None, Renv.shape[0]
    n = a * D * D * b
    H = np.zeros((Lenv.shape[0] * D * D * Renv.shape[2], n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1.0
        H[:, k] = heff2_dense(Lenv, W1, W2, Renv, e.reshape(a, D, D, b)).reshape(-1)
    return H


# ---------------------------------------------------------------------------
# expansion of reduced tensors (Eq. symdecomp) into m-resolved dense arrays
# ---------------------------------------------------------------------------

class Bond:
    """A bond space given by sectors [(n, t, d)]; t = 2S (SU(2)) or 2S^z (U(1)xU(1)).

    Dense index of (sector k, degeneracy i, component alpha) is
    offset[k] + i * mult + alpha, with mult = t+1 (SU(2)) or 1 (U(1)xU(1)).
    """

    def __init__(self, sectors, su2: bool):
        self.sectors = [tuple(s) for s in sectors]
        self.su2 = su2
        self.offset, off = [], 0
        for (_, t, d) in self.sectors:
            self.offset.append(off)
            off += d * self.mult(t)
        self.dim = off
        self.index = {(n, t): k for k, (n, t, _) in enumerate(self.sectors)}

    def mult(self, t):
        return t + 1 if self.su2 else 1

    def rows(self, k):
        """dense indices of sector k as an array [d, mult]"""
        n, t, d = self.sectors[k]
        m = self.mult(t)
        return self.offset[k] + np.arange(d)[:, None] * m + np.arange(m)[None, :]


def _site(su2):
    return SITE_MULTIPLETS_SU2 if su2 else SITE_MULTIPLETS_U1


def _chan(su2):
    return CHANNELS_SU2 if su2 else CHANNELS_U1


def _c3(su2, t1, t2, t3):
    """<j1 m1; j2 m2 | j3 m3> as an array, or the U(1) coupling 1."""
    if su2:
        return _cg.cg_array(t1, t2, t3)
    return np.ones((1, 1, 1))


def expand_site(blocks, left: Bond, right: Bond):
    """blocks {(a, s, b): d_a x d_b} with a, b sector indices and s a site multiplet index."""
    su2 = left.su2
    A = np.zeros((left.dim, D, right.dim), dtype=complex)
    for (a, s, b), blk in blocks.items():
        ta, ts, tb = left.sectors[a][1], _site(su2)[s][0][1], right.sectors[b][1]
        C = _c3(su2, ta, ts, tb)
        ra, rb = left.rows(a), right.rows(b)
        for ia in range(blk.shape[0]):
            for ib in range(blk.shape[1]):
                for al in range(ra.shape[1]):
                    for si, sstate in enumerate(_site(su2)[s][1]):
                        for be in range(rb.shape[1]):
                            A[ra[ia, al], sstate, rb[ib, be]] += blk[ia, ib] * C[al, si, be]
    return A


def expand_theta(blocks, left: Bond, mid_t, right: Bond):
    """blocks {(a, s1, c, s2, b): d_a x d_b}; c is the (n, t) label of the coupled (a s1) channel."""
    su2 = left.su2
    T = np.zeros((left.dim, D, D, right.dim), dtype=complex)
    site = _site(su2)
    for (a, s1, c, s2, b), blk in blocks.items():
        ta, tb = left.sectors[a][1], right.sectors[b][1]
        t1, t2 = site[s1][0][1], site[s2][0][1]
        tc = c[1]
        C1 = _c3(su2, ta, t1, tc)
        C2 = _c3(su2, tc, t2, tb)
        X = np.einsum("xsg,gty->xsty", C1, C2)  # [alpha, sigma1, sigma2, beta]
        ra, rb = left.rows(a), right.rows(b)
        for al in range(ra.shape[1]):
            for i1, st1 in enumerate(site[s1][1]):
                for i2, st2 in enumerate(site[s2][1]):
                    for be in range(rb.shape[1]):
                        x = X[al, i1, i2, be]
                        if x != 0.0:
                            T[np.ix_(ra[:, al], [st1], [st2], rb[:, be])] += x * blk[:, None, None, :]
    return T


def expand_left_env(blocks, bra: Bond, ket: Bond):
    """blocks {(a', w, a): d_a' x d_a}, w a channel multiplet index -> L[a', 6, a]."""
    su2 = bra.su2
    chans = _chan(su2)
    E = np.zeros((bra.dim, 6, ket.dim), dtype=complex)
    for (ap, w, a), blk in blocks.items():
        tap, tw, ta = bra.sectors[ap][1], chans[w][0][1], ket.sectors[a][1]
        C = _c3(su2, ta, tw, tap)  # [alpha, mu, alpha']
        rap, ra = bra.rows(ap), ket.rows(a)
        for al in range(ra.shape[1]):
            for mi, comp in enumerate(chans[w][1]):
                for alp in range(rap.shape[1]):
                    x = C[al, mi, alp]
                    if x != 0.0:
                        E[np.ix_(rap[:, alp], [comp], ra[:, al])] += x * blk[:, None, :]
    return E


def expand_right_env(blocks, ket: Bond, bra: Bond):
    """blocks {(b, w, b'): d_b x d_b'} -> R[b, 6, b']."""
    su2 = ket.su2
    chans = _chan(su2)
    E = np.zeros((ket.dim, 6, bra.dim), dtype=complex)
    for (b, w, bp), blk in blocks.items():
        tb, tw, tbp = ket.sectors[b][1], chans[w][0][1], bra.sectors[bp][1]
        C = _c3(su2, tb, tw, tbp)  # [beta, mu, beta']
        rb, rbp = ket.rows(b), bra.rows(bp)
        for be in range(rb.shape[1]):
            for mi, comp in enumerate(chans[w][1]):
                for bep in range(rbp.shape[1]):
                    x = C[be, mi, bep]
                    if x != 0.0:
                        E[np.ix_(rb[:, be], [comp], rbp[:, bep])] += x * blk[:, None, :]
    return E


# ---------------------------------------------------------------------------
# enumeration of the blocks allowed by the selection rules (a1 bookkeeping)
# ---------------------------------------------------------------------------

def fuse(su2, q1, q2):
    """labels in q1 x q2: charges add; SU(2) spins |t1-t2|..t1+t2 step 2, or 2S^z adds."""
    n = q1[0] + q2[0]
    if su2:
        return [(n, t) for t in range(abs(q1[1] - q2[1]), q1[1] + q2[1] + 1, 2)]
    return [(n, q1[1] + q2[1])]


def theta_blocks(left: Bond, right: Bond):
    """All (a, s1, c, s2, b) allowed by fusion, in the enumeration order of the reduced format:
    a, then s1, then c ascending in t, then s2, then b (all ascending indices)."""
    su2 = left.su2
    site = _site(su2)
    out = []
    for a, (na, ta, _) in enumerate(left.sectors):
        for s1, (q1, _) in enumerate(site):
            for c in fuse(su2, (na, ta), q1):
                for s2, (q2, _) in enumerate(site):
                    for qb in fuse(su2, c, q2):
                        b = right.index.get(qb)
                        if b is not None:
                            out.append((a, s1, c, s2, b))
    return out


def left_env_blocks(bra: Bond, ket: Bond):
    """All (a', w, a) with a' in a x w."""
    su2 = bra.su2
    out = []
    for ap, (nap, tap, _) in enumerate(bra.sectors):
        for w, (qw, _) in enumerate(_chan(su2)):
            for a, (na, ta, _) in enumerate(ket.sectors):
                if (nap, tap) in fuse(su2, (na, ta), qw):
                    out.append((ap, w, a))
    return out


def right_env_blocks(ket: Bond, bra: Bond):
    """All (b, w, b') with b' in b x w."""
    su2 = ket.su2
    out = []
    for b, (nb, tb, _) in enumerate(ket.sectors):
        for w, (qw, _) in enumerate(_chan(su2)):
            for bp, (nbp, tbp, _) in enumerate(bra.sectors):
                if (nbp, tbp) in fuse(su2, (nb, tb), qw):
                    out.append((b, w, bp))
    return out


def reduce_theta(T, left: Bond, right: Bond, keys):
    """Project an m-resolved theta onto the reduced tree basis (inverse of expand_theta)."""
    su2 = left.su2
    site = _site(su2)
    out = {}
    for (a, s1, c, s2, b) in keys:
        ta, tb = left.sectors[a][1], right.sectors[b][1]
        t1, t2 = site[s1][0][1], site[s2][0][1]
        X = np.einsum("xsg,gty->xsty", _c3(su2, ta, t1, c[1]), _c3(su2, c[1], t2, tb))
        ra, rb = left.rows(a), right.rows(b)
        blk = np.zeros((ra.shape[0], rb.shape[0]), dtype=complex)
        for al in range(ra.shape[1]):
            for i1, st1 in enumerate(site[s1][1]):
                for i2, st2 in enumerate(site[s2][1]):
                    for be in range(rb.shape[1]):
                        x = X[al, i1, i2, be]
                        if x != 0.0:
                            blk += x * T[np.ix_(ra[:, al], [st1], [st2], rb[:, be])][:, 0, 0, :]
        out[(a, s1, c, s2, b)] = blk / np.sum(X * X)
    return out
