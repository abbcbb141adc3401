"""CPU FP64 oracle for two-site TDVP of the open Fermi-Hubbard chain.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import,
call or execute anything in this package.  The product path (the CUDA engine
behind ``include/tdvp.h``) never calls it, and this package never imports the
product package: the two share no code.  Inputs that both sides consume come
from the seeded generators in ``synth/``, which hold none of the method's
arithmetic.

Everything here is plain and slow on purpose: numpy/scipy library primitives
(matmul, eigh, svd) used as single steps, FP64 / complex128 throughout,
Python loops where the size is small.

Parts (each module cites the passage of the paper it restates):

* ``ed``    -- O1, exact diagonalisation of Eq. (FHM) in a fixed (N, S^z)
               sector, the Neel state of Eq. (neel), exact time evolution and
               the observables n_{i sigma}, double occupancy, entanglement.
* ``free``  -- O3, U = 0 closed form by propagating the one-body correlation
               matrix of each spin species.
* ``mps``   -- O2, dense (unblocked) MPS with the Jordan-Wigner MPO of
               Eq. (FHM), two-site TDVP sweeps (Sec. S2.2) with a Lanczos
               Krylov exponential and SVD truncation on the truncated weight
               (Sec. S2.4).
* ``heff``  -- O4, brute-force effective-Hamiltonian application
               (Sec. S2.3): dense einsum, explicit matrix, and the expansion
               of U(1)xSU(2) reduced tensors (Eq. symdecomp) into the
               m-resolved basis with Clebsch-Gordan coefficients.
* ``cg``    -- exact Clebsch-Gordan coefficients (Racah's closed form, in
               rational arithmetic) used by ``heff`` for the expansion.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants, brute force or values printed in the paper.  The
absolute curves of the paper's figures are not printed in it, so the
long-time L=60 observables themselves are "parity unpinned".
"""
