"""tdvp_svd_noalloc: the allocation-free SVD entry point.

Some callers cannot allocate device memory while they run (a serving process
whose own pool already holds nearly all of the GPU's memory, or code under a
memory budget frozen after start-up).  tdvp_svd_noalloc serves them: it keeps
its workspace in a static device array inside the library.  These tests call it
through the C ABI with device pointers and check that it returns what the
allocating entry point tdvp_svd returns, within the SVD tests' tolerance, on two
calls in a row (the second one smaller, so stale workspace contents from the
first would show), at the documented limit max(p, q) = 512 in both orientations,
that a call made after the first one takes no device memory (it does not lower
the device's free memory), and that it rejects sizes beyond its maximum.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(a, p, q):
    import torch

    from paper_2606_04771_b300._lib import check, lib

    r = min(p, q)
    u = torch.empty((p, r), dtype=torch.complex128, device=a.device)
    vh = torch.empty((r, q), dtype=torch.complex128, device=a.device)
    s = torch.empty(r, dtype=torch.float64, device=a.device)
    check(lib().tdvp_svd_noalloc(p, q, a.data_ptr(), s.data_ptr(), u.data_ptr(), vh.data_ptr(), None))
    return u.cpu().numpy(), s.cpu().numpy(), vh.cpu().numpy()


def test_noalloc_svd_matches_allocating_entry_point_twice():
    import torch

    from paper_2606_04771_b300._lib import svd

    for shape, seed in (((300, 180), 1), ((37, 129), 2)):
        g = np.random.default_rng(seed)
        a = g.standard_normal(shape) + 1j * g.standard_normal(shape)
        ad = torch.from_numpy(a).cuda()
        u0, s0, vh0 = (x.cpu().numpy() for x in svd(ad))
        u1, s1, vh1 = _noalloc(ad, *shape)
        tol = 1e-13 * s0[0]
        assert np.abs(s1 - s0).max() < tol
        assert np.abs(u1 - u0).max() < 1e-13 * max(shape)
        assert np.abs(vh1 - vh0).max() < 1e-13 * max(shape)
        assert np.abs((u1 * s1) @ vh1 - a).max() < 1e-13 * np.abs(a).max() * max(shape)


def test_noalloc_at_the_limit_and_without_device_allocation():
    import torch

    from paper_2606_04771_b300._lib import svd

    for shape, seed in (((512, 200), 3), ((200, 512), 4)):
        g = np.random.default_rng(seed)
        a = g.standard_normal(shape) + 1j * g.standard_normal(shape)
        ad = torch.from_numpy(a).cuda()
        u0, s0, vh0 = (x.cpu().numpy() for x in svd(ad))
        p, q = shape
        r = min(p, q)
        u = torch.empty((p, r), dtype=torch.complex128, device="cuda")
        vh = torch.empty((r, q), dtype=torch.complex128, device="cuda")
        s = torch.empty(r, dtype=torch.float64, device="cuda")
        from paper_2606_04771_b300._lib import check, lib

        check(lib().tdvp_svd_noalloc(p, q, ad.data_ptr(), s.data_ptr(), u.data_ptr(), vh.data_ptr(), None))
        torch.cuda.synchronize()
        free_before, _ = torch.cuda.mem_get_info()
        check(lib().tdvp_svd_noalloc(p, q, ad.data_ptr(), s.data_ptr(), u.data_ptr(), vh.data_ptr(), None))
        torch.cuda.synchronize()
        free_after, _ = torch.cuda.mem_get_info()
        assert free_after >= free_before, (free_before, free_after)
        s1, u1, vh1 = s.cpu().numpy(), u.cpu().numpy(), vh.cpu().numpy()
        assert np.abs(s1 - s0).max() < 1e-13 * s0[0]
        assert np.abs(u1 - u0).max() < 1e-13 * max(shape)
        assert np.abs(vh1 - vh0).max() < 1e-13 * max(shape)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch

    from paper_2606_04771_b300._lib import lib

    buf = torch.zeros(16, dtype=torch.complex128, device="cuda")
    p = buf.data_ptr()
    rc = lib().tdvp_svd_noalloc(513, 4, p, p, p, p, None)
    assert rc == -1
    assert b"TDVP_SVD_NOALLOC_MAX" in lib().tdvp_last_error()
