"""GPU parity of the one-site TDVP step and the adaptive two-site/one-site switch
(Sec. S2.2) against the oracle (L=8 open chain, J=1, U=4, Neel start, dt=0.05).

The chain first grows its bond dimensions with two-site steps that truncate
nothing (eps=0, cap above the largest Schmidt rank), so both sides end with the
complete sector-resolved bond spaces; then both run one-site steps: the same
integrator on the same bond spaces, so they agree to the Krylov tolerance (bar
1e-8, both FP64).  One-site TDVP
conserves energy and norm exactly and never changes a bond dimension; the
split-precision modes are compared with the FP64 path (BF16x4 at the observable bar
1e-6, 3xTF32 at 1e-4, the level its TF32 pieces allow).
"""
import numpy as np
import pytest

from oracle import mps

pytestmark = pytest.mark.gpu

L, J, U, DT = 8, 1.0, 4.0, 0.05
GROW, ONE = 8, 6


@pytest.fixture(scope="module")
def oracle_run():
    sim = mps.DenseTDVP(L, J, U)
    for _ in range(GROW):
        sim.step(DT, 256, 0.0)
    out = []
    for _ in range(ONE):
        sim.step1(DT)
        out.append((sim.observables(), sim.bond_dims()))
    return out


@pytest.mark.parametrize("sym", ["u1u1", "su2"])
def test_one_site_matches_dense_oracle(sym, oracle_run):
    from paper_2606_04771_b300 import Chain

    ch = Chain(L, J, U, symmetry=sym, precision="fp64")
    for _ in range(GROW):
        ch.step(DT, 256, 0.0)
    chi0, _ = ch.bond_dims()
    for k in range(ONE):
        assert ch.step(DT, 256, 1e-12, mode="one") == "one"
        o = ch.measure()
        r, dims = oracle_run[k]
        for key in ("n_up", "n_dn", "docc", "s_ent"):
            assert np.abs(o[key] - r[key]).max() < 1e-8, (sym, k, key, np.abs(o[key] - r[key]).max())
        assert abs(o["energy"] - r["energy"]) < 1e-8
        chi, _ = ch.bond_dims()
        assert np.array_equal(chi, chi0)  # one-site steps never change a bond dimension
        # the dense oracle spans the full 4^k spaces, the engine the complete spaces of
        # the half-filled sector: both are exact, so only the observables are compared
        assert all(c <= d for c, d in zip(chi[1:L], dims))
    assert ch.stats()["one_site_steps"] == ONE
    ch.close()


def test_one_site_conserves_energy_below_full_rank():
    from paper_2606_04771_b300 import Chain

    ch = Chain(L, J, U, symmetry="su2", precision="fp64")
    for _ in range(6):
        ch.step(DT, 16, 1e-12)  # the cap binds: a truncated state
    chi0, red0 = ch.bond_dims()
    e0 = ch.measure()["energy"]
    for _ in range(8):
        ch.step(DT, 16, 1e-12, mode="one")
    o = ch.measure()
    assert abs(o["energy"] - e0) < 1e-9
    assert np.abs(o["n"] - 1.0).max() < 1e-9  # U(1)xSU(2) keeps every site at half filling
    chi, red = ch.bond_dims()
    assert np.array_equal(chi, chi0) and np.array_equal(red, red0)
    ch.close()


def test_adaptive_switches_once_the_cap_binds():
    from paper_2606_04771_b300 import Chain

    ch = Chain(L, J, U, symmetry="su2", precision="fp64")
    used = [ch.step(DT, 24, 1e-12, mode="adaptive") for _ in range(12)]
    k = used.index("one")  # the step after the first one whose truncation hit the cap
    assert k >= 1 and all(u == "two" for u in used[:k]) and all(u == "one" for u in used[k:])
    chi_switch, _ = ch.bond_dims()
    assert chi_switch.max() <= 24
    ch.close()


@pytest.mark.parametrize("prec", ["3xtf32", "bf16x4"])
def test_one_site_split_precision_vs_fp64(prec):
    from paper_2606_04771_b300 import Chain

    out = {}
    for p in ("fp64", prec):
        ch = Chain(L, J, U, symmetry="su2", precision=p)
        for _ in range(GROW):
            ch.step(DT, 256, 1e-12)
        for _ in range(ONE):
            ch.step(DT, 256, 1e-12, mode="one")
        out[p] = ch.measure()
        ch.close()
    # BF16x4 products are exact to ~2^-30 of the row/column scales: the observable bar
    # 1e-6 holds with margin.  3xTF32 keeps ~2^-22 per product (matvec error ~1e-5),
    # which after 14 steps shows at the 1e-5 level: bar 1e-4.
    bar = 1e-6 if prec == "bf16x4" else 1e-4
    for key in ("n_up", "docc"):
        assert np.abs(out[prec][key] - out["fp64"][key]).max() < bar, key
