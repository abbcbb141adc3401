"""GPU parity of the per-sector SVD kernel (one-sided Jacobi, FP64) through tdvp_svd.

Singular values against LAPACK (numpy) within 1e-13 of the largest, the
reconstruction U diag(s) V^H within 1e-13 of ||A||, and orthonormal factors,
for tall, wide, square, ragged and rank-deficient matrices.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (1, 7), (9, 1), (37, 129), (300, 40), (64, 64), (65, 63), (200, 200)]


@pytest.mark.parametrize("shape", SHAPES)
def test_svd_matches_lapack(shape):
    from paper_2606_04771_b300._lib import svd

    g = np.random.default_rng(shape[0] * 1000 + shape[1])
    a = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    u, s, vh = svd(a)
    ref = np.linalg.svd(a, compute_uv=False)
    assert np.all(np.diff(s) <= 0)
    assert np.abs(s - ref).max() < 1e-13 * ref[0]
    assert np.abs((u * s) @ vh - a).max() < 1e-13 * np.abs(a).max() * max(shape)
    r = min(shape)
    assert np.abs(u.conj().T @ u - np.eye(r)).max() < 1e-13
    assert np.abs(vh @ vh.conj().T - np.eye(r)).max() < 1e-13


def test_svd_rank_deficient_and_device_path():
    import torch

    from paper_2606_04771_b300._lib import svd

    g = np.random.default_rng(3)
    b = g.standard_normal((50, 6)) + 1j * g.standard_normal((50, 6))
    a = b @ (g.standard_normal((6, 30)) + 1j * g.standard_normal((6, 30)))  # rank 6
    u, s, vh = svd(a)
    ref = np.linalg.svd(a, compute_uv=False)
    assert np.abs(s - ref).max() < 1e-13 * ref[0]
    assert np.all(s[6:] < 1e-12 * s[0])
    assert np.abs((u * s) @ vh - a).max() < 1e-12 * np.abs(a).max()
    ud, sd, vhd = svd(torch.from_numpy(a).cuda())
    assert np.array_equal(sd.cpu().numpy(), s)
    assert np.array_equal(ud.cpu().numpy(), u)
