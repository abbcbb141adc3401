"""Pins for oracle O1 (exact diagonalisation) and O3 (free fermions).

Each check is fixed by the paper's statements or by mathematics, not by the
oracle itself: the symmetry algebra of Sec. S2.1, the quantum numbers of the
Neel state, conservation laws, the U=0 closed form, lattice symmetries and a
short-time expansion derived by hand.
"""
import numpy as np
import pytest
from scipy.special import j0

from oracle import ed, free


def comm(a, b):
    return a @ b - b @ a


def test_sector_dimension_matches_config():
    # L=8 half filling, S^z=0: C(8,4)^2
    assert len(ed.sector_basis(8, 4, 4)) == 4900


def test_two_hamiltonian_constructions_agree():
    L, J, U = 4, 1.0, 3.0
    Hf = ed.fock_hamiltonian(L, J, U)
    basis = ed.sector_basis(L, 2, 2)
    Hs = ed.hamiltonian(L, J, U, basis)
    assert np.allclose(Hf[np.ix_(basis, basis)], Hs, atol=1e-14)
    # and the sector is closed under H
    others = [s for s in range(1 << 2 * L) if s not in set(basis)]
    assert np.abs(Hf[np.ix_(others, basis)]).max() == 0.0


@pytest.mark.parametrize("L", [3, 4])
def test_pseudospin_algebra_and_symmetry(L):
    """Sec. S2.1: [T+,T-]=2T^z, [T^z,T+-]=+-T+-, and the pseudospin commutes with H.

    Reading: the commutation [H, T+-] = 0 holds for the particle-hole symmetric
    interaction U (n_up - 1/2)(n_dn - 1/2); Eq. (FHM) as printed differs from it by
    (U/2) N - U L/4, so there [H, T+-] = +-U T+- while T^2 and T^z are conserved,
    which is all the dynamics at fixed N needs."""
    U = -2.0
    H = ed.fock_hamiltonian(L, 1.0, U)
    Tp, Tm, Tz = ed.fock_pseudospin(L)
    dim = H.shape[0]
    N = 2 * Tz + L * np.eye(dim)
    Hsym = H - 0.5 * U * N + 0.25 * U * L * np.eye(dim)
    assert np.allclose(comm(Tp, Tm), 2 * Tz)
    assert np.allclose(comm(Tz, Tp), Tp)
    assert np.allclose(comm(Tz, Tm), -Tm)
    for T in (Tp, Tm, Tz):
        assert np.abs(comm(Hsym, T)).max() < 1e-12
    assert np.abs(comm(H, Tp) - U * Tp).max() < 1e-12
    T2 = Tz @ Tz + 0.5 * (Tp @ Tm + Tm @ Tp)
    assert np.abs(comm(H, T2)).max() < 1e-12
    assert np.abs(comm(H, Tz)).max() < 1e-12
    Sp, Sm, Sz = ed.fock_spin(L)
    for S in (Sp, Sm, Sz):
        assert np.abs(comm(H, S)).max() < 1e-12


def test_pseudospin_needs_the_staggered_phase():
    """Without (-1)^i the operator does not commute with the hopping (Sec. S2.1)."""
    L = 4
    H = ed.fock_hamiltonian(L, 1.0, 0.0)  # U = 0: only the hopping matters
    c = [ed.fock_operator_c(L, p) for p in range(2 * L)]
    Tp_uniform = sum(c[ed.mode(i, 0)].T @ c[ed.mode(i, 1)].T for i in range(L))
    assert np.abs(comm(H, Tp_uniform)).max() > 0.5


def test_neel_quantum_numbers():
    """Sec. S2.1: the Neel state has S^z = 0, T_tot = 0, T^z = 0, but no definite S_tot."""
    L = 4
    psi = np.zeros(1 << 2 * L)
    basis = list(range(1 << 2 * L))
    psi = ed.neel_state(L, basis)
    Tp, Tm, Tz = ed.fock_pseudospin(L)
    Sp, Sm, Sz = ed.fock_spin(L)
    T2 = Tz @ Tz + 0.5 * (Tp @ Tm + Tm @ Tp)
    S2 = Sz @ Sz + 0.5 * (Sp @ Sm + Sm @ Sp)
    assert abs(np.vdot(psi, Sz @ psi)) < 1e-14
    assert abs(np.vdot(psi, Tz @ psi)) < 1e-14
    assert np.linalg.norm(T2 @ psi) < 1e-14  # T_tot = 0 exactly
    S2psi = S2 @ psi
    ev = np.vdot(psi, S2psi).real
    assert np.linalg.norm(S2psi - ev * psi) > 0.1  # not an eigenstate of S^2


@pytest.fixture(scope="module")
def ed_L6():
    L = 6
    basis = ed.sector_basis(L, 3, 3)
    out = {}
    for U in (4.0, -4.0, 0.0):
        H = ed.hamiltonian(L, 1.0, U, basis)
        psi0 = ed.neel_state(L, basis)
        times = [0.0, 0.3, 0.9, 2.0]
        out[U] = (H, [ed.observables(p, basis, L, H) for p in ed.evolve(H, psi0, times)], times)
    return L, basis, out


def test_conservation_and_exact_invariants(ed_L6):
    L, _, res = ed_L6
    for U, (H, obs, times) in res.items():
        E0 = obs[0]["energy"]
        for o in obs:
            assert abs(o["norm"] - 1) < 1e-12
            assert abs(o["energy"] - E0) < 1e-10 * max(1, abs(E0))
            # <n_i> = 1: T_tot = 0 and n_i - 1 is twice the local pseudospin z component
            assert np.abs(o["n"] - 1).max() < 1e-12
            assert abs(o["sz"].sum()) < 1e-12
            # reflection + spin flip maps the Neel state to itself
            assert np.abs(o["n_up"] - (1 - o["n_up"][::-1])).max() < 1e-12


def test_u_to_minus_u_invariance(ed_L6):
    _, _, res = ed_L6
    for a, b in zip(res[4.0][1], res[-4.0][1]):
        for key in ("n_up", "n_dn", "docc", "s_ent"):
            assert np.abs(a[key] - b[key]).max() < 1e-10


def test_u0_matches_free_fermions(ed_L6):
    L, _, res = ed_L6
    H, obs, times = res[0.0]
    for o, t in zip(obs, times):
        f = free.observables(L, 1.0, t)
        for key in ("n_up", "n_dn", "docc", "s_ent"):
            assert np.abs(o[key] - f[key]).max() < 1e-10, key
        assert abs(o["energy"] - f["energy"]) < 1e-10


def test_short_time_expansion():
    """n_{i up}(t) = 1 - z_i J^2 t^2 + O(t^4) on A sites, docc_i = z_i J^2 t^2 + O(t^4)
    (second-order expansion of exp(-iHt) on the Neel state; z_i = neighbour count)."""
    L, J, U = 6, 1.0, 4.0
    basis = ed.sector_basis(L, 3, 3)
    H = ed.hamiltonian(L, J, U, basis)
    psi0 = ed.neel_state(L, basis)
    t = 2e-3
    o = ed.observables(ed.evolve(H, psi0, [t])[0], basis, L)
    for i in range(0, L, 2):
        z = (i > 0) + (i < L - 1)
        assert abs((1 - o["n_up"][i]) / t ** 2 - z * J * J) < 1e-3
        assert abs(o["docc"][i] / t ** 2 - z * J * J) < 1e-3


def test_free_fermion_bulk_bessel_closed_form():
    """Infinite-chain limit: n_{i up}(t) = 1/2 + 1/2 J0(4 J t) on A sites before edge effects."""
    L, J = 240, 1.0
    for t in (0.5, 1.3, 3.0, 6.0):
        o = free.observables(L, J, t)
        i = L // 2
        assert abs(o["n_up"][i] - (0.5 + 0.5 * j0(4 * J * t))) < 1e-10
        assert abs(o["n_up"][i + 1] - (0.5 - 0.5 * j0(4 * J * t))) < 1e-10
