"""Pins for oracle O4 (brute-force H_eff) and the Clebsch-Gordan expansion.

* H_eff (two-site and one-site) built from environments equals the projection
  of H|psi> onto the MPS tangent space, computed from full state vectors of a
  random canonical MPS -- the definition in Sec. S2.2/S2.3.
* Clebsch-Gordan coefficients: textbook values (golden fixture), both
  orthogonality relations, and the raising-operator recursion.
* The reduced-tensor expansion (Eq. symdecomp): expanded tensors are SU(2)
  invariant, reduce(expand(x)) = x, and the particle-hole-frame MPO maps the
  reduced tree space into itself (which checks the channel doublet convention).
* Table S3 transcription: sum d = 12,288 = chi_SU(2), sum d (2j+1) = 30,842.
"""
import os

import numpy as np
import pytest

from oracle import cg, heff, mps

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return rows


def test_cg_textbook_values():
    for r in load("cg_textbook.txt"):
        args = tuple(int(x) for x in r[:6])
        assert abs(cg.cg(*args) - r[6]) < 1e-15, r


@pytest.mark.parametrize("tj1,tj2", [(1, 1), (2, 1), (4, 3), (6, 2), (12, 1), (5, 5)])
def test_cg_orthogonality(tj1, tj2):
    blocks = [cg.cg_array(tj1, tj2, tJ) for tJ in range(abs(tj1 - tj2), tj1 + tj2 + 1, 2)]
    # as a map from product basis to coupled basis: a real orthogonal matrix
    Q = np.concatenate([b.reshape((tj1 + 1) * (tj2 + 1), -1) for b in blocks], axis=1)
    assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-13
    assert np.abs(Q @ Q.T - np.eye(Q.shape[0])).max() < 1e-13


def spin_matrices(tj):
    """S^+ and S^z on the (2j+1) multiplet, basis m = j, j-1, ..., -j (Condon-Shortley)."""
    j = tj / 2
    m = j - np.arange(tj + 1)
    Sz = np.diag(m)
    Sp = np.zeros((tj + 1, tj + 1))
    for k in range(1, tj + 1):
        Sp[k - 1, k] = np.sqrt(j * (j + 1) - m[k] * (m[k] + 1))
    return Sp, Sz


@pytest.mark.parametrize("tj1,tj2,tJ", [(1, 1, 0), (2, 1, 3), (4, 2, 4), (3, 3, 2), (6, 1, 5)])
def test_cg_raising_recursion(tj1, tj2, tJ):
    """(S1+ + S2+) |J M> = S+ |J M>: the coupled states form a standard multiplet."""
    C = cg.cg_array(tj1, tj2, tJ)
    S1, _ = spin_matrices(tj1)
    S2, _ = spin_matrices(tj2)
    SJ, _ = spin_matrices(tJ)
    lhs = np.einsum("ab,bcM->acM", S1, C) + np.einsum("cd,adM->acM", S2, C)
    rhs = np.einsum("abN,NM->abM", C, SJ)
    assert np.abs(lhs - rhs).max() < 1e-13


def random_canonical_mps(dims, seed):
    g = np.random.default_rng(seed)
    out = []
    for k in range(len(dims) - 1):
        A = g.standard_normal((dims[k], 4, dims[k + 1])) + 1j * g.standard_normal((dims[k], 4, dims[k + 1]))
        out.append(A)
    return out


def left_canon(A):
    a, s, b = A.shape
    Q, _ = np.linalg.qr(A.reshape(a * s, b))
    return Q.reshape(a, s, b)


def right_canon(B):
    a, s, b = B.shape
    Q, _ = np.linalg.qr(B.reshape(a, s * b).T)
    return Q.T.reshape(a, s, b)


def chain_vectors(tensors):
    """Full vectors [bond_left, physical..., bond_right] of a product of site tensors."""
    X = tensors[0]
    for A in tensors[1:]:
        X = np.tensordot(X, A, axes=([-1], [0]))
    return X


@pytest.mark.parametrize("i", [0, 1, 2])
def test_heff_is_tangent_projection_of_H(i):
    L, J, U = 5, 1.0, 3.0
    dims = [1, 4, 6, 6, 4, 1]
    raw = random_canonical_mps(dims, 7 + i)
    A = [left_canon(raw[k]) for k in range(i)]
    B = [right_canon(raw[k]) for k in range(i + 2, L)]
    g = np.random.default_rng(11)
    theta = g.standard_normal((dims[i], 4, 4, dims[i + 2])) + 0j
    W = mps.mpo_tensor(J, U)
    H = mps.mpo_dense(L, J, U)  # C order of (s_0..s_4)
    # full state
    left = chain_vectors(A) if A else np.ones((1, 1))
    right = chain_vectors(B) if B else np.ones((1, 1))
    left = left.reshape(-1, dims[i])          # [phys_left, a]
    right = right.reshape(dims[i + 2], -1)    # [b, phys_right]
    psi = np.einsum("pa,astb,bq->pstq", left, theta, right).reshape(-1)
    Hpsi = (H @ psi).reshape(left.shape[0], 4, 4, right.shape[1])
    expected = np.einsum("pa,pstq,bq->astb", left.conj(), Hpsi, right.conj())
    Lenv = mps.left_edge(W)
    for X in A:
        Lenv = mps.update_left(Lenv, X, W)
    Renv = mps.right_edge(W)
    for X in reversed(B):
        Renv = mps.update_right(Renv, X, W)
    got = mps.heff2(Lenv, W, W, Renv, theta)
    assert np.abs(got - expected).max() < 1e-12
    assert np.abs(heff.heff2_dense(Lenv, W, W, Renv, theta) - expected).max() < 1e-12
    # one-site at site i with site i+1 right-canonical
    M = g.standard_normal((dims[i], 4, dims[i + 1])) + 0j
    Bi1 = right_canon(raw[i + 1])
    right1 = chain_vectors([Bi1] + B).reshape(dims[i + 1], -1)
    psi1 = np.einsum("pa,asb,bq->psq", left, M, right1).reshape(-1)
    H1 = (H @ psi1).reshape(left.shape[0], 4, right1.shape[1])
    expected1 = np.einsum("pa,psq,bq->asb", left.conj(), H1, right1.conj())
    R1 = mps.update_right(Renv, Bi1, W)
    assert np.abs(mps.heff1(Lenv, W, R1, M) - expected1).max() < 1e-12
    assert np.abs(heff.heff1_dense(Lenv, W, R1, M) - expected1).max() < 1e-12


def test_heff_matrix_is_hermitian_for_physical_envs():
    L, J, U = 4, 1.0, 2.0
    dims = [1, 4, 5, 4, 1]
    raw = random_canonical_mps(dims, 3)
    W = mps.mpo_tensor(J, U)
    Lenv = mps.update_left(mps.left_edge(W), left_canon(raw[0]), W)
    Renv = mps.update_right(mps.right_edge(W), right_canon(raw[3]), W)
    Hm = heff.heff2_matrix(Lenv, W, W, Renv)
    assert np.abs(Hm - Hm.conj().T).max() < 1e-12


# ---------------------------------------------------------------------------
# SU(2) expansion
# ---------------------------------------------------------------------------

def bond_spin(bond):
    """S^+ on the dense space of a Bond (replicated over degeneracy)."""
    S = np.zeros((bond.dim, bond.dim))
    for k, (_, t, d) in enumerate(bond.sectors):
        Sp, _ = spin_matrices(t)
        r = bond.rows(k)
        for i in range(d):
            S[np.ix_(r[i], r[i])] = Sp
    return S


def site_spin():
    a_up, a_dn, _ = mps.local_ops()
    return a_up.T @ a_dn  # S^+ = c^dag_up c_dn inside one site


def random_reduced(keys, shapes, seed):
    g = np.random.default_rng(seed)
    return {k: g.standard_normal(s) + 1j * g.standard_normal(s) for k, s in zip(keys, shapes)}


def small_bonds():
    left = heff.Bond([(3, 1, 2), (4, 0, 1), (4, 2, 2), (5, 1, 1), (2, 0, 1)], su2=True)
    right = heff.Bond([(5, 1, 2), (6, 0, 2), (6, 2, 1), (4, 0, 1), (5, 3, 1)], su2=True)
    return left, right


def test_expanded_theta_is_invariant_and_round_trips():
    left, right = small_bonds()
    keys = heff.theta_blocks(left, right)
    assert keys
    blocks = random_reduced(keys, [(left.sectors[k[0]][2], right.sectors[k[4]][2]) for k in keys], 5)
    T = heff.expand_theta(blocks, left, None, right)
    Sa, Sb, Ss = bond_spin(left), bond_spin(right), site_spin()
    # legs a, s1, s2 transform as kets, b as a bra
    gen = (np.einsum("xy,ystb->xstb", Sa, T) + np.einsum("st,xtub->xsub", Ss, T)
           + np.einsum("tu,xsub->xstb", Ss, T) - np.einsum("yb,xsty->xstb", Sb, T))
    assert np.abs(gen).max() < 1e-12
    back = heff.reduce_theta(T, left, right, keys)
    for k in keys:
        assert np.abs(back[k] - blocks[k]).max() < 1e-12


def test_su2_heff_stays_in_reduced_space():
    """With invariant environments and the particle-hole-frame MPO, H_eff maps the
    reduced tree space into itself: expand -> H_eff -> reduce -> expand is the identity
    on the result.  A wrong sign in a channel doublet breaks the invariance."""
    left, right = small_bonds()
    keys = heff.theta_blocks(left, right)
    th = random_reduced(keys, [(left.sectors[k[0]][2], right.sectors[k[4]][2]) for k in keys], 9)
    lk = heff.left_env_blocks(left, left)
    rk = heff.right_env_blocks(right, right)
    Lb = random_reduced(lk, [(left.sectors[k[0]][2], left.sectors[k[2]][2]) for k in lk], 10)
    Rb = random_reduced(rk, [(right.sectors[k[0]][2], right.sectors[k[2]][2]) for k in rk], 11)
    Lenv = heff.expand_left_env(Lb, left, left)
    Renv = heff.expand_right_env(Rb, right, right)
    W = heff.shiba_mpo_tensor(1.0, 4.0)
    out = heff.heff2_dense(Lenv, W, W, Renv, heff.expand_theta(th, left, None, right))
    red = heff.reduce_theta(out, left, right, keys)
    again = heff.expand_theta(red, left, None, right)
    assert np.abs(out).max() > 1.0
    assert np.abs(again - out).max() < 1e-11 * np.abs(out).max()
    # a flipped sign in the c doublet is caught
    Wbad = W.copy()
    Wbad[0, 4] *= -1
    out_bad = heff.heff2_dense(Lenv, Wbad, Wbad, Renv, heff.expand_theta(th, left, None, right))
    again_bad = heff.expand_theta(heff.reduce_theta(out_bad, left, right, keys), left, None, right)
    assert np.abs(again_bad - out_bad).max() > 1e-3


def test_table_s3_transcription():
    rows = load("table_s3_degeneracies.txt")
    assert len(rows) == 32
    d = [int(r[2]) for r in rows]
    tj = [int(r[1]) for r in rows]
    n = [int(r[0]) for r in rows]
    assert sum(d) == 12288  # chi_SU(2) of Table S3's caption
    assert sum(x * (t + 1) for x, t in zip(d, tj)) == 30842  # "chi ~ 30,000"
    assert max(d) == 1735
    # parity at a bond with 30 sites to its left: n even <-> j integer
    assert all((a + t) % 2 == 0 for a, t in zip(n, tj))


def test_blockwise_u1_matches_dense():
    """The benchmark-scale blockwise oracle equals the dense definition on a small problem."""
    from oracle import blockwise

    left = heff.Bond([(3, 1, 2), (3, -1, 2), (4, 0, 3), (4, 2, 1), (5, 1, 2)], su2=False)
    right = heff.Bond([(5, 1, 2), (5, -1, 1), (6, 0, 2), (6, 2, 1), (4, 0, 1)], su2=False)
    keys = heff.theta_blocks(left, right)
    lk, rk = heff.left_env_blocks(left, left), heff.right_env_blocks(right, right)
    th = random_reduced(keys, [(left.sectors[k[0]][2], right.sectors[k[4]][2]) for k in keys], 3)
    Lb = random_reduced(lk, [(left.sectors[k[0]][2], left.sectors[k[2]][2]) for k in lk], 4)
    Rb = random_reduced(rk, [(right.sectors[k[0]][2], right.sectors[k[2]][2]) for k in rk], 5)
    W = heff.shiba_mpo_tensor(1.0, 4.0)
    dense = heff.heff2_dense(heff.expand_left_env(Lb, left, left), W, W, heff.expand_right_env(Rb, right, right),
                             heff.expand_theta(th, left, None, right))
    ref = heff.reduce_theta(dense, left, right, keys)
    got, flops = blockwise.heff2_u1_blocks(left, right, keys, [th[k] for k in keys], lk, [Lb[k] for k in lk],
                                           rk, [Rb[k] for k in rk], W, keys)
    assert flops > 0
    for k in keys:
        assert np.abs(got[k] - ref[k]).max() < 1e-12
