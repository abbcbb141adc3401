"""Pins for oracle O2 (dense MPS two-site TDVP).

The MPO is pinned to the Fock-space Hamiltonian built from operator products,
the Krylov exponential to scipy's expm, the truncation rule to hand-built
spectra, and the whole integrator to exact diagonalisation: at a bond
dimension that admits the exact state, two-site TDVP with negligible
truncation reproduces the exact dynamics (the projector-splitting integrator
is exact at full rank), and it conserves norm and energy.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import ed, heff, mps


def fock_permutation(L):
    """C-order index of (s_0..s_{L-1}) -> Fock integer sum_i s_i 4^i."""
    idx = np.arange(4 ** L).reshape((4,) * L)
    return idx.transpose(tuple(range(L - 1, -1, -1))).reshape(-1)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_mpo_equals_fock_hamiltonian(L):
    J, U = 0.7, 2.5
    Hm = mpo_dense_in_fock(mps.mpo_tensor(J, U), L)
    Hf = ed.fock_hamiltonian(L, J, U)
    assert np.abs(Hm - Hf).max() < 1e-13


def mpo_dense_in_fock(W, L):
    T = W[0]
    for _ in range(1, L):
        T = np.einsum("wxy,wvab->vxayb", T, W).reshape(W.shape[0], T.shape[1] * 4, T.shape[2] * 4)
    Hc = T[-1]
    p = fock_permutation(L)
    # Hc is indexed by C-order; entry (x, y) belongs to Fock states (p[x], p[y])
    Hf = np.zeros_like(Hc)
    Hf[np.ix_(p, p)] = Hc
    return Hf


@pytest.mark.parametrize("L", [2, 3, 4])
def test_shiba_mpo(L):
    """The particle-hole frame MPO equals -J hop - U n_up n_dn + U/2 n on the Fock space,
    and its channel doublets are standard spin-1/2 tensor operators (checked via the
    invariance of the whole operator under total spin)."""
    J, U = 1.3, 3.0
    Hm = mpo_dense_in_fock(heff.shiba_mpo_tensor(J, U), L)
    c = [ed.fock_operator_c(L, p) for p in range(2 * L)]
    cd = [m.T for m in c]
    dim = 4 ** L
    H = np.zeros((dim, dim))
    for i in range(L - 1):
        for s in (0, 1):
            a, b = ed.mode(i, s), ed.mode(i + 1, s)
            H += -J * (cd[a] @ c[b] + cd[b] @ c[a])
    for i in range(L):
        nu = cd[ed.mode(i, 0)] @ c[ed.mode(i, 0)]
        nd = cd[ed.mode(i, 1)] @ c[ed.mode(i, 1)]
        H += -U * nu @ nd + 0.5 * U * (nu + nd)
    assert np.abs(Hm - H).max() < 1e-13
    Sp, Sm, Sz = ed.fock_spin(L)
    assert np.abs(Hm @ Sp - Sp @ Hm).max() < 1e-12


def test_krylov_expm_matches_scipy():
    g = np.random.default_rng(3)
    n = 60
    A = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    H = (A + A.conj().T) / 2
    v = g.standard_normal(n) + 1j * g.standard_normal(n)
    for tau in (0.01, 0.05, -0.05):
        ref = scipy.linalg.expm(-1j * tau * H) @ v
        out = mps.krylov_expm(lambda x: H @ x, v, tau, kmax=40, tol=1e-13)
        assert np.abs(out - ref).max() < 1e-11 * np.linalg.norm(v)


def test_krylov_invariant_subspace_exact():
    H = np.diag([1.0, 2.0, 3.0])
    v = np.array([1.0, 0, 0], dtype=complex)
    info = {}
    out = mps.krylov_expm(lambda x: H @ x, v, 0.3, info=info)
    assert info["krylov_dim"] == 1
    assert np.allclose(out, [np.exp(-0.3j), 0, 0], atol=1e-15)


def test_truncation_rule():
    s = np.array([0.8, 0.5, 0.3, 1e-4, 1e-5])
    tot = np.sum(s ** 2)
    # eps admits dropping the last two (weights 1e-8 + 1e-10)
    assert mps.truncation_count(s, 10, 1.1e-8 / tot) == 3
    assert mps.truncation_count(s, 10, 0.9e-8 / tot) == 4
    assert mps.truncation_count(s, 2, 0.0) == 2
    assert mps.truncation_count(np.array([1.0]), 5, 1.0) == 1
    assert mps.truncation_count(np.array([1.0, 1.0]), 5, 0.9) == 1


@pytest.mark.parametrize("U", [4.0, 0.0])
def test_dense_tdvp_converges_to_ed(U):
    """Two-site TDVP at a bond dimension that admits the exact state is exact once
    the bonds have reached full rank; the only error is made while the rank grows
    from the product state, O(dt^3) per step over O(1) steps.  So the deviation from
    exact diagonalisation must fall by ~8x per halving of dt, while norm and energy
    are conserved to rounding."""
    L, J, T = 6, 1.0, 0.8
    basis = ed.sector_basis(L, 3, 3)
    H = ed.hamiltonian(L, J, U, basis)
    ex = ed.observables(ed.evolve(H, ed.neel_state(L, basis), [T])[0], basis, L, H)
    errs = []
    for dt in (0.1, 0.05):
        sim = mps.DenseTDVP(L, J, U)
        for _ in range(int(round(T / dt))):
            sim.step(dt, 64, 1e-14)
        o = sim.observables()
        errs.append(max(np.abs(o[k] - ex[k]).max() for k in ("n_up", "n_dn", "docc", "s_ent")))
        assert abs(o["norm"] - 1) < 1e-12
        assert abs(o["energy"] - ex["energy"]) < 1e-10
        assert np.abs(o["n"] - 1).max() < 1e-4  # exact only up to the integrator error
    assert errs[1] < 3e-5
    assert 5.0 < errs[0] / errs[1] < 11.0, errs


def test_dense_tdvp_full_rank_step_is_exact():
    """From an exact full-rank state, one TDVP step reproduces exact evolution (the
    exactness property of the projector-splitting integrator)."""
    L, J, U, dt = 4, 1.0, 4.0, 0.1
    sim = mps.DenseTDVP(L, J, U)
    for _ in range(10):
        sim.step(0.05, 16, 0.0)  # bonds grow to the full rank [4, 16, 4]
    assert sim.bond_dims() == [4, 16, 4]
    psi0 = mps.full_state(sim.mps)
    H = ed.fock_hamiltonian(L, J, U)
    ref = ed.evolve(H, psi0, [dt])[0]
    sim.step(dt, 16, 0.0)
    assert np.abs(mps.full_state(sim.mps) - ref).max() < 1e-10


def test_dense_tdvp_truncated_run_stays_physical():
    L = 6
    sim = mps.DenseTDVP(L, 1.0, 4.0)
    for _ in range(10):
        sim.step(0.05, 4, 1e-6)
    o = sim.observables()
    assert max(sim.bond_dims()) <= 4
    assert abs(o["norm"] - 1) < 1e-12
    assert np.abs(o["n"] - 1).max() < 1e-3


# ---------------------------------------------------------------------------
# one-site TDVP (Sec. S2.2, used once the bond dimension has saturated)
# ---------------------------------------------------------------------------

def _copy_sim(sim, L, J, U):
    c = mps.DenseTDVP(L, J, U, kmax=30, krylov_tol=1e-14)
    c.mps = [A.copy() for A in sim.mps]
    c._build_right_envs()
    return c


def test_dense_tdvp1_full_rank_is_exact():
    """At full bond dimension the one-site tangent space is the whole Hilbert space, so
    the one-site projector-splitting integrator reproduces exact evolution."""
    for L, steps in ((4, 10), (6, 12)):
        J, U = 1.0, 4.0
        sim = mps.DenseTDVP(L, J, U, kmax=30, krylov_tol=1e-14)
        for _ in range(steps):
            sim.step(0.05, 10**6, 0.0)
        full = [min(4 ** (i + 1), 4 ** (L - i - 1)) for i in range(L - 1)]
        assert sim.bond_dims() == full
        one = _copy_sim(sim, L, J, U)
        psi0 = mps.full_state(one.mps)
        ref = ed.evolve(ed.fock_hamiltonian(L, J, U), psi0, [0.4])[0]
        for _ in range(4):
            one.step1(0.1)
        assert np.abs(mps.full_state(one.mps) - ref).max() < 1e-11


def test_dense_tdvp1_conserves_energy_norm_and_bonds():
    """Below full rank the one-site integrator still conserves energy and norm exactly
    (up to the Krylov tolerance) and never changes a bond dimension."""
    L, J, U = 8, 1.0, 4.0
    sim = mps.DenseTDVP(L, J, U, kmax=30, krylov_tol=1e-14)
    for _ in range(6):
        sim.step(0.05, 16, 1e-12)
    dims = sim.bond_dims()
    assert max(dims) == 16
    one = _copy_sim(sim, L, J, U)
    E0 = one.observables()["energy"]
    for _ in range(4):
        one.step1(0.05)
    o = one.observables()
    assert abs(o["energy"] - E0) < 1e-11
    assert abs(np.linalg.norm(mps.full_state(one.mps)) - 1.0) < 1e-12
    assert one.bond_dims() == dims


def test_heff0_is_the_projected_hamiltonian():
    """H_eff^0 on the bond matrix equals <psi(C1)| H |psi(C2)> for the mixed-canonical
    embedding psi(C) = A_0..A_i C B_{i+1}..B_{L-1}, computed with the dense H."""
    L, J, U = 4, 1.0, 4.0
    rng = np.random.default_rng(5)
    sim = mps.DenseTDVP(L, J, U)
    for _ in range(3):
        sim.step(0.1, 16, 0.0)
    W = sim.W
    # left-orthonormal A_0, A_1 by QR sweeps; B_2, B_3 right-orthonormal already
    A = [x.copy() for x in sim.mps]
    for i in range(2):
        a, d, b = A[i].shape
        Q, R = np.linalg.qr(A[i].reshape(a * d, b))
        A[i] = Q.reshape(a, d, Q.shape[1])
        A[i + 1] = np.tensordot(R, A[i + 1], axes=([1], [0]))
    Le = mps.left_edge(W)
    for i in range(2):
        Le = mps.update_left(Le, A[i], W)
    Re = mps.right_edge(W)
    for i in (3, 2):
        a, d, b = A[i].shape
        if i == 2:  # make B_2 right-orthonormal (A[2] carries the centre after the QR sweep)
            Q, R = np.linalg.qr(A[2].reshape(a, d * b).conj().T)
            A[2] = Q.conj().T.reshape(Q.shape[1], d, b)
        Re = mps.update_right(Re, A[i], W)
    k = A[1].shape[2]
    C1 = rng.normal(size=(k, k)) + 1j * rng.normal(size=(k, k))
    C2 = rng.normal(size=(k, k)) + 1j * rng.normal(size=(k, k))

    def embed(C):
        t = [A[0], np.tensordot(A[1], C, axes=([2], [0])), A[2], A[3]]
        return mps.full_state(t)

    H = ed.fock_hamiltonian(L, J, U)
    want = np.vdot(embed(C1), H @ embed(C2))
    got = np.vdot(C1, mps.heff0(Le, Re, C2))
    assert abs(got - want) < 1e-10 * abs(want)


# ---------------------------------------------------------------------------
# the second initial state (Sec. S1): the Neel pattern with a central vacancy
# ---------------------------------------------------------------------------

def test_vacancy_state_and_full_rank_evolution():
    """The vacancy product state is the same in the ED and MPS oracles; once the
    bond dimensions are full, both integrators reproduce exact evolution, and the
    charge N = L - 1 and the S^z of the state are conserved."""
    L, J, U = 5, 1.0, 4.0
    occ = ed.vacancy_occupations(L)
    assert occ == [1, 2, 0, 2, 1]
    nu, nd = sum(o & 1 for o in occ), sum(o >> 1 & 1 for o in occ)
    basis = ed.sector_basis(L, nu, nd)
    H = ed.hamiltonian(L, J, U, basis)
    sim = mps.DenseTDVP(L, J, U, kmax=30, krylov_tol=1e-14, occ=occ)
    r0 = ed.observables(ed.product_state(L, occ, basis), basis, L, H)
    o0 = sim.observables()
    for key in ("n_up", "n_dn", "docc"):
        assert np.abs(o0[key] - r0[key]).max() < 1e-14
    for _ in range(12):
        sim.step(0.05, 10**6, 0.0)
    assert sim.bond_dims() == [4, 16, 16, 4]
    for method in ("two", "one"):
        c = _copy_sim(sim, L, J, U)
        psi0 = mps.full_state(c.mps)
        ref = ed.evolve(ed.fock_hamiltonian(L, J, U), psi0, [0.3])[0]
        for _ in range(3):
            c.step(0.1, 10**6, 0.0) if method == "two" else c.step1(0.1)
        assert np.abs(mps.full_state(c.mps) - ref).max() < 1e-10, method
        o = c.observables()
        assert abs(o["n"].sum() - (L - 1)) < 1e-10
        assert abs(0.5 * (o["n_up"] - o["n_dn"]).sum() - 0.5 * (nu - nd)) < 1e-10
