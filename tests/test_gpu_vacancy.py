"""The benchmark's second initial state (Sec. S1): the Neel pattern with a single
central vacancy, here L = 7 (N = 6, S^z = 1).  U(1)xU(1) engine against the dense
oracle from the same product state: two-site steps (dt=0.05, chi<=256, eps=1e-12)
to 1e-8 (same integrator); one-site steps on complete bond spaces against the exact
two-site steps (1e-8) and the oracle (1e-7); the energy is
that of Eq. (FHM) away from half filling; U(1)xSU(2) rejects the state; BF16x4 stays
within the observable bar of the FP64 path."""
import numpy as np
import pytest

from oracle import ed, mps

pytestmark = pytest.mark.gpu

L, J, U, DT = 7, 1.0, 4.0, 0.05


def _check(o, r, bar=1e-8):
    for key in ("n_up", "n_dn", "docc", "s_ent"):
        assert np.abs(o[key] - r[key]).max() < bar, (key, np.abs(o[key] - r[key]).max())
    assert abs(o["energy"] - r["energy"]) < bar


def test_vacancy_two_site_matches_oracle():
    from paper_2606_04771_b300 import Chain

    occ = ed.vacancy_occupations(L)
    sim = mps.DenseTDVP(L, J, U, occ=occ)
    ch = Chain(L, J, U, symmetry="u1u1", precision="fp64", occupations=occ)
    _check(ch.measure(), sim.observables(), 1e-14)
    for _ in range(10):
        sim.step(DT, 256, 1e-12)
        ch.step(DT, 256, 1e-12)
        _check(ch.measure(), sim.observables())
    o = ch.measure()
    assert abs(o["n"].sum() - (L - 1)) < 1e-10 and abs(o["sz"].sum() - 1.0) < 1e-10
    ch.close()


def test_vacancy_one_site_exact_on_complete_spaces():
    """Grown without truncation to the full capacity of every sector, the bond spaces
    are complete: one-site and two-site steps are then both exact, so two identical
    engine chains evolved with either must agree.  Bar 1e-8: eps = 0 keeps directions
    of zero weight, so some sectors' site matrices are rank-deficient and their gauge
    shift takes the shifted Cholesky QR, whose R^-1 magnifies rounding to ~1e-9
    (truncated states, eps > 0, have no such columns).  The dense oracle's one-site
    run is the secondary reference: its eps = 0 growth keeps noise-level directions
    that differ from the engine's and leaves ~1e-8 (bar 1e-7)."""
    from paper_2606_04771_b300 import Chain

    occ = ed.vacancy_occupations(L)
    sim = mps.DenseTDVP(L, J, U, occ=occ)
    a = Chain(L, J, U, symmetry="u1u1", precision="fp64", occupations=occ)
    b = Chain(L, J, U, symmetry="u1u1", precision="fp64", occupations=occ)
    for _ in range(14):
        sim.step(DT, 256, 0.0)
        a.step(DT, 256, 0.0)
        b.step(DT, 256, 0.0)
    chi, _ = a.bond_dims()
    assert list(chi[1:L]) == [4, 16, 46, 46, 16, 4]  # every bond at its sector capacity
    for _ in range(5):
        sim.step1(DT)
        assert a.step(DT, 256, 0.0, mode="one") == "one"
        b.step(DT, 256, 0.0)
        oa, ob, r = a.measure(), b.measure(), sim.observables()
        for key in ("n_up", "n_dn", "docc", "s_ent"):
            assert np.abs(oa[key] - ob[key]).max() < 1e-8, (key, np.abs(oa[key] - ob[key]).max())
            assert np.abs(oa[key] - r[key]).max() < 1e-7, (key, np.abs(oa[key] - r[key]).max())
        assert abs(oa["energy"] - r["energy"]) < 1e-11
    assert np.array_equal(a.bond_dims()[0], chi)
    a.close()
    b.close()


def test_vacancy_rejected_by_su2():
    from paper_2606_04771_b300 import Chain, TdvpError

    with pytest.raises(TdvpError) as e:
        Chain(L, J, U, symmetry="su2", occupations=ed.vacancy_occupations(L))
    assert e.value.code == -1


def test_vacancy_bf16x4_vs_fp64():
    from paper_2606_04771_b300 import Chain

    out = {}
    for p in ("fp64", "bf16x4"):
        ch = Chain(L, J, U, symmetry="u1u1", precision=p, occupations=ed.vacancy_occupations(L))
        for _ in range(12):
            ch.step(DT, 256, 1e-12)
        out[p] = ch.measure()
        ch.close()
    for key in ("n_up", "n_dn", "docc"):
        assert np.abs(out["bf16x4"][key] - out["fp64"][key]).max() < 1e-6, key
