"""GPU parity of the Krylov exponential (Sec. S2.2) through the C ABI.

The engine's Lanczos (full re-orthogonalisation twice, FP64) with its scaled
Taylor evaluation of exp(-i tau T_k) e_1 must reproduce the oracle's Lanczos
with an eigendecomposition of T_k, at a fixed Krylov dimension, on the same
seeded bond problem (1e-11 relative).  At adaptive dimension on the chain's
bond (0,1) the result must be the exact exp(-i tau H_eff) theta to the Krylov
tolerance (the oracle exponentiates the explicit H_eff matrix).
"""
import numpy as np
import pytest
import scipy.linalg

from gpu_helpers import fill_bond_problem
from oracle import heff, mps

pytestmark = pytest.mark.gpu


def oracle_apply(lb, rb, keys, Ld, Rd, W):
    Lenv = heff.expand_left_env(Ld, lb, lb)
    Renv = heff.expand_right_env(Rd, rb, rb)

    def apply(x):
        blocks, o = {}, 0
        for k in keys:
            r, c = lb.sectors[k[0]][2], rb.sectors[k[4]][2]
            blocks[k] = x[o:o + r * c].reshape(r, c)
            o += r * c
        out = heff.heff2_dense(Lenv, W, W, Renv, heff.expand_theta(blocks, lb, None, rb))
        red = heff.reduce_theta(out, lb, rb, keys)
        return np.concatenate([red[k].reshape(-1) for k in keys])

    return apply


@pytest.mark.parametrize("sym", ["su2", "u1u1"])
def test_krylov_fixed_dimension_matches_oracle(sym):
    from paper_2606_04771_b300 import BondProblem

    su2 = sym == "su2"
    left = [(3, 1, 2), (4, 0, 3), (4, 2, 2), (5, 1, 1)] if su2 else [(3, 1, 2), (3, -1, 2), (4, 0, 3), (5, 1, 1)]
    right = [(5, 1, 2), (6, 0, 2), (6, 2, 1), (4, 0, 1)] if su2 else [(5, 1, 2), (5, -1, 1), (6, 0, 2), (4, 0, 1)]
    kdim, tau = 8, 0.07
    bp = BondProblem(left, right, symmetry=sym, krylov_max=kdim, krylov_tol=1e-30)
    lb, rb, keys, theta, th, Ld, Rd, _ = fill_bond_problem(bp, left, right, su2, seed=99)
    theta = theta / np.linalg.norm(theta)
    got = bp.krylov_expm(theta, tau=tau)
    assert bp.last_krylov_dim() == kdim
    ref = mps.krylov_expm(oracle_apply(lb, rb, keys, Ld, Rd, heff.shiba_mpo_tensor(1.0, 4.0)), theta, tau,
                          kmax=kdim, tol=1e-30)
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()
    bp.close()


def test_krylov_adaptive_is_exact_exponential_on_chain():
    from paper_2606_04771_b300 import Chain

    ch = Chain(6, 1.0, 4.0, symmetry="su2")
    for _ in range(6):
        ch.step(0.05, 64, 1e-12)
    keys, dims, offs, n = ch.blocks(3)
    g = np.random.default_rng(5)
    x = g.standard_normal(n) + 1j * g.standard_normal(n)
    x /= np.linalg.norm(x)
    # explicit matrix of H_eff at bond (0,1) through the C ABI, column by column
    H = np.zeros((n, n), dtype=complex)
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1.0
        H[:, j] = ch.heff_apply(e)
    assert np.abs(H - H.conj().T).max() < 1e-12  # physical environments: Hermitian
    tau = 0.025
    got = ch.krylov_expm(x, tau=tau)
    ref = scipy.linalg.expm(-1j * tau * H) @ x
    assert np.abs(got - ref).max() < 1e-11
    assert ch.last_krylov_dim() < 20
    ch.close()
