"""Checkpoint / resume: a chain saved mid-run and resumed in a new context evolves
exactly as the uninterrupted run (bit for bit: the environments are rebuilt with
the same kernels in the same order), in FP64 and BF16x4, two-site and adaptive
(whose switch state is part of the checkpoint), U(1)xSU(2) and U(1)xU(1)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KEYS = ("n", "sz", "docc", "s_ent")


def _run(ch, steps, chi, mode):
    used = [ch.step(0.05, chi, 1e-10, mode=mode) for _ in range(steps)]
    return ch.measure(), used


@pytest.mark.parametrize("precision,mode,symmetry,vacancy,chi", [
    ("fp64", "two", "su2", False, 64),
    ("bf16x4", "adaptive", "su2", False, 12),
    ("fp64", "two", "u1u1", True, 64),
])
def test_resume_repeats_the_uninterrupted_run(tmp_path, precision, mode, symmetry, vacancy, chi):
    from paper_2606_04771_b300 import Chain
    from paper_2606_04771_b300._lib import vacancy_occupations

    L = 7 if vacancy else 10
    occ = vacancy_occupations(L) if vacancy else None
    path = str(tmp_path / "chain.ckpt")
    a = Chain(L, 1.0, 4.0, symmetry=symmetry, precision=precision, occupations=occ)
    _run(a, 5, chi, mode)
    a.save(path, t=0.25)
    oa, used_a = _run(a, 6, chi, mode)
    a.close()
    b, t = Chain.load(path, precision=precision)
    assert t == 0.25 and b.L == L and b.sym == symmetry
    ob, used_b = _run(b, 6, chi, mode)
    b.close()
    assert used_a == used_b
    if mode == "adaptive":
        assert "one" in used_a  # the cap bound before the checkpoint or after it
    for k in KEYS:
        assert np.array_equal(oa[k], ob[k]), k
    assert oa["energy"] == ob["energy"]


def test_bond_problem_cannot_be_saved(tmp_path):
    from paper_2606_04771_b300 import BondProblem
    from paper_2606_04771_b300._lib import lib

    bp = BondProblem([(3, 1, 2), (4, 0, 1)], [(5, 1, 2), (4, 0, 1)], symmetry="su2")
    assert lib().tdvp_save(bp.h, str(tmp_path / "x").encode(), 0.0) == -2
    bp.close()


def test_quench_driver_resumes_from_its_checkpoint(tmp_path):
    from paper_2606_04771_b300 import quench

    ck = str(tmp_path / "q.ckpt")
    kw = dict(L=8, U=4.0, dt=0.05, chi=64, eps=1e-10, mode="two", precision="fp64", measure_every=2, log=None)
    full = quench.run(t_final=0.4, **kw)
    quench.run(t_final=0.2, checkpoint=ck, **kw)
    rest = quench.run(t_final=0.4, resume=ck, **kw)
    assert rest["t"][0] == pytest.approx(0.2) and rest["t"][-1] == pytest.approx(0.4)
    assert np.array_equal(rest["n_up"][-1], full["n_up"][-1])
    assert np.array_equal(rest["s_ent"][-1], full["s_ent"][-1])
