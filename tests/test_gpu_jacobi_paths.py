"""The split's per-sector Jacobi has three launch forms: when every sector of a split
is small (at most 32 columns, working copy in shared memory) each sector runs inside
one CTA with CTA barriers; otherwise all sectors share the cooperative grid-wide
kernel, or, on request, each sector runs in one thread-block cluster (columns in
distributed shared memory, cluster barriers) when every sector fits in 8 CTAs.  All apply the same pairs in the same order with the
same arithmetic (explicit fma throughout), so the evolution is identical bit for
bit whichever form runs.  TDVP_JACOBI_RESIDENT_BYTES=0 switches the first form
off; the cluster form runs only with TDVP_JACOBI_CLUSTER=1."""
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


def _quench(precision, symmetry):
    from paper_2606_04771_b300 import Chain

    ch = Chain(10, 1.0, 4.0, symmetry=symmetry, precision=precision)
    for _ in range(6):
        ch.step(0.05, 48, 1e-10)
    o = ch.measure()
    st = ch.stats()
    ch.close()
    return o, st


@pytest.mark.parametrize("precision,symmetry", [("fp64", "su2"), ("bf16x4", "su2"), ("bf16x4", "u1u1")])
def test_resident_and_cooperative_jacobi_agree(precision, symmetry):
    a, sa = _with_env({"TDVP_JACOBI_RESIDENT_BYTES": 196608}, lambda: _quench(precision, symmetry))
    b, sb = _with_env({"TDVP_JACOBI_RESIDENT_BYTES": 0, "TDVP_JACOBI_CLUSTER": 0},
                      lambda: _quench(precision, symmetry))
    assert sa["jacobi_resident_calls"] > 0  # the small splits ran CTA-resident
    assert sb["jacobi_resident_calls"] == 0  # forced onto the cooperative kernel
    for k in ("n", "sz", "docc", "s_ent"):
        assert np.array_equal(a[k], b[k]), k
    assert a["energy"] == b["energy"]
    assert sa["sweeps32"] == sb["sweeps32"] and sa["sweeps64"] == sb["sweeps64"]


def _bond(precision, env):
    from paper_2606_04771_b300 import Chain

    def run():
        ch = Chain(16, 1.0, 4.0, symmetry="su2", random_chi=2048, seed=7, center=7, precision=precision)
        s1 = ch.bond_update(7, 0, 0.05, 2048, 1e-9)
        s2 = ch.bond_update(7, 1, 0.05, 2048, 1e-9)
        o = ch.measure_center()
        chis, _ = ch.bond_dims()
        st = ch.stats()
        ch.close()
        return (s1, s2, o, chis), st

    return _with_env(env, run)


@pytest.mark.parametrize("precision", ["fp64", "bf16x4"])
def test_cluster_and_cooperative_jacobi_agree(precision):
    a, sa = _bond(precision, {"TDVP_JACOBI_CLUSTER": 1})
    b, sb = _bond(precision, {"TDVP_JACOBI_CLUSTER": 0})
    assert sa["jacobi_cluster_calls"] > 0 and sb["jacobi_cluster_calls"] == 0
    assert sa["jacobi_resident_calls"] == 0  # sectors of more than 32 columns
    assert a[0] == b[0] and a[1] == b[1]  # bond entropies, bit for bit
    assert a[2] == b[2]
    assert np.array_equal(a[3], b[3])
    assert sa["sweeps32"] == sb["sweeps32"] and sa["sweeps64"] == sb["sweeps64"]
