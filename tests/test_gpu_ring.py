"""The ring form of the split's FP32 Jacobi preconditioner.

Each sector's column pairs are held by a ring of warps inside one thread-block
cluster (two columns per warp, in registers); after every round each warp passes
its columns to its neighbours through shared memory (distributed shared memory
across the cluster's CTAs) instead of the whole grid meeting at a grid-wide
barrier.  The pairs, their order within each sweep, the arithmetic and the stopping
rule are the cooperative kernel's, so a bond update gives the same result bit for
bit whichever form ran (TDVP_JACOBI_RING=1 selects the ring form)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _with_env(env, fn):
    old = {k: os.environ.get(k) for k in env}
    os.environ.update({k: str(v) for k, v in env.items()})
    try:
        return fn()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _bond(env, chi, seed):
    from paper_2606_04771_b300 import Chain

    def run():
        ch = Chain(16, 1.0, 4.0, symmetry="su2", random_chi=chi, seed=seed, center=7, precision="bf16x4")
        s1 = ch.bond_update(7, 0, 0.05, chi, 1e-9)
        s2 = ch.bond_update(7, 1, 0.05, chi, 1e-9)
        o = ch.measure_center()
        chis, _ = ch.bond_dims()
        st = ch.stats()
        ch.close()
        return (s1, s2, o, chis), st

    return _with_env(env, run)


@pytest.mark.parametrize("chi,seed", [(512, 5), (2048, 7)])
def test_ring_and_cooperative_jacobi_agree(chi, seed):
    a, sa = _bond({"TDVP_JACOBI_RING": 1, "TDVP_JACOBI_RESIDENT_BYTES": 0}, chi, seed)
    b, sb = _bond({"TDVP_JACOBI_RING": 0, "TDVP_JACOBI_RESIDENT_BYTES": 0}, chi, seed)
    assert sa["jacobi_ring_calls"] > 0 and sb["jacobi_ring_calls"] == 0
    assert a[0] == b[0] and a[1] == b[1]  # bond entropies, bit for bit
    assert a[2] == b[2]
    assert np.array_equal(a[3], b[3])
    assert sa["sweeps32"] == sb["sweeps32"]


def test_ring_quench_matches_cooperative():
    from paper_2606_04771_b300 import Chain

    def run():
        ch = Chain(12, 1.0, 4.0, symmetry="u1u1", precision="bf16x4")
        for _ in range(6):
            ch.step(0.05, 64, 1e-10)
        o, st = ch.measure(), ch.stats()
        ch.close()
        return o, st

    a, sa = _with_env({"TDVP_JACOBI_RING": 1, "TDVP_JACOBI_RESIDENT_BYTES": 0}, run)
    b, sb = _with_env({"TDVP_JACOBI_RING": 0, "TDVP_JACOBI_RESIDENT_BYTES": 0}, run)
    assert sa["jacobi_ring_calls"] > 0
    for k in ("n", "sz", "docc", "s_ent"):
        assert np.array_equal(a[k], b[k]), k
    assert a["energy"] == b["energy"]
