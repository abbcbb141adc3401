"""Failure detection on the GPU without a fault: a bounded wait on an mbarrier that
nothing arrives at must give up, report TDVP_ETIMEOUT through the C ABI, and leave
the CUDA context usable for the next call."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_and_context_stays_usable():
    from paper_2606_04771_b300 import lib, svd

    rc = lib().tdvp_selftest_wait(1 << 16, None)
    assert rc == -7  # TDVP_ETIMEOUT
    assert b"expired" in lib().tdvp_last_error()
    a = np.random.default_rng(3).normal(size=(12, 9)) + 0j
    u, s, vh = svd(a)
    assert np.abs((u * s) @ vh - a).max() < 1e-12
