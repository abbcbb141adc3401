"""GPU parity of single bond updates (the unit of the sweep) and of the synthetic
random states used by the sweep benchmark.

* tdvp_bond_update / tdvp_measure_center against the oracle performing the same
  sequence of two-site updates (with backward one-site steps) from the Neel state:
  local observables of the centre site and the entanglement entropy of each new
  bond (from the kept singular values) within 1e-9.
* tdvp_create_random: the synthetic state is normalised, has the requested bond
  dimension in the middle, conserves n_i = 1 on average (half filling), and a full
  time step on it keeps the norm (the centre site observables stay physical).
"""
import numpy as np
import pytest

from oracle import mps

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sym", ["su2", "u1u1"])
def test_bond_updates_match_oracle(sym):
    from paper_2606_04771_b300 import Chain

    L, J, U, dt = 6, 1.0, 4.0, 0.08
    ref = mps.DenseTDVP(L, J, U)
    ch = Chain(L, J, U, symmetry=sym)
    seq = [(0, 0), (1, 0), (2, 0), (3, 0), (3, 1), (2, 1), (1, 1)]
    for bond, direction in seq:
        s = ch.bond_update(bond, direction, dt, 256, 1e-12)
        if direction == 0:
            ref.bond_lr(bond, dt / 2, 256, 1e-12, True)
        else:
            ref.bond_rl(bond, dt / 2, 256, 1e-12, True)
        p = ref.last_s ** 2
        s_ref = float(-np.sum(p[p > 1e-300] * np.log(p[p > 1e-300])))
        assert abs(s - s_ref) < 1e-9, (bond, direction, s, s_ref)
    site, o = ch.measure_center()
    assert site == 1
    # oracle: full state, observables of the centre site
    r = mps.observables_full(mps.full_state(ref.mps), L)
    assert abs(o["n"] - r["n"][site]) < 1e-9
    assert abs(o["sz"] - r["sz"][site]) < 1e-9
    assert abs(o["docc"] - r["docc"][site]) < 1e-9
    ch.close()


@pytest.mark.parametrize("sym,chi", [("su2", 200), ("u1u1", 120)])
def test_random_state_is_normalised_and_steps(sym, chi):
    from paper_2606_04771_b300 import Chain

    L = 16
    ch = Chain(L, 1.0, 4.0, symmetry=sym, random_chi=chi, seed=3, precision="bf16x4")
    chis, _ = ch.bond_dims()
    assert chis[L // 2] >= chi and chis[0] == 1 and chis[L] == 1
    o = ch.measure(entropy=True)
    assert abs(np.mean(o["n"]) - 1.0) < 1e-6  # total particle number N = L
    assert np.all(o["s_ent"] >= -1e-12)
    ch.step(0.05, chi, 1e-9)
    o2 = ch.measure(entropy=False)
    assert abs(np.mean(o2["n"]) - 1.0) < 1e-6
    assert np.all((o2["docc"] >= -1e-9) & (o2["docc"] <= 1 + 1e-9))
    ch.close()
    # a random state with the centre in the middle supports bond updates there
    ch = Chain(L, 1.0, 4.0, symmetry=sym, random_chi=chi, seed=4, center=L // 2 - 1, precision="bf16x4")
    s1 = ch.bond_update(L // 2 - 1, 0, 0.05, chi, 1e-9)
    s2 = ch.bond_update(L // 2 - 1, 1, 0.05, chi, 1e-9)
    site, oc = ch.measure_center()
    assert site == L // 2 - 1 and s1 > 0 and s2 > 0
    assert 0 <= oc["docc"] <= 1
    ch.close()
