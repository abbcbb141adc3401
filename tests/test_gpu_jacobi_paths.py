"""The split's per-sector Jacobi has two launch forms: when every sector of a split
is small (at most 32 columns, working copy in shared memory) each sector runs inside
one CTA with CTA barriers; otherwise all sectors share the cooperative grid-wide
kernel.  Both apply the same pairs in the same order with the same arithmetic
(explicit fma throughout), so the evolution is identical bit for bit whichever
form runs.  TDVP_JACOBI_RESIDENT_BYTES=0 forces the cooperative form."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _with_limit(limit, fn):
    old = os.environ.get("TDVP_JACOBI_RESIDENT_BYTES")
    os.environ["TDVP_JACOBI_RESIDENT_BYTES"] = str(limit)
    try:
        return fn()
    finally:
        if old is None:
            os.environ.pop("TDVP_JACOBI_RESIDENT_BYTES", None)
        else:
            os.environ["TDVP_JACOBI_RESIDENT_BYTES"] = old


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
    a, sa = _with_limit(196608, lambda: _quench(precision, symmetry))
    b, sb = _with_limit(0, lambda: _quench(precision, symmetry))
    assert sa["jacobi_resident_calls"] > 0  # the small splits ran CTA-resident
    assert sb["jacobi_resident_calls"] == 0  # forced onto the cooperative kernel
    for k in ("n", "sz", "docc", "s_ent"):
        assert np.array_equal(a[k], b[k]), k
    assert a["energy"] == b["energy"]
    assert sa["sweeps32"] == sb["sweeps32"] and sa["sweeps64"] == sb["sweeps64"]


def test_large_sectors_use_the_cooperative_kernel():
    from paper_2606_04771_b300 import Chain

    ch = Chain(16, 1.0, 4.0, symmetry="su2", random_chi=2048, seed=7, center=7, precision="bf16x4")
    ch.bond_update(7, 0, 0.05, 2048, 1e-9)
    st = ch.stats()
    ch.close()
    assert st["split_qmax"] > 32 and st["jacobi_calls"] > 0 and st["jacobi_resident_calls"] == 0
