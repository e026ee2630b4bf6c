"""Plain FP64 CPU oracle for Multipolynomial Monte Carlo (arXiv:2306.09559).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA path (``paper_2306_09559_gb300``); the only
thing both sides consume is the seeded input generator
``paper_2306_09559_gb300.synth`` (gauge fields and starting vectors), which
holds none of the method's arithmetic.

Everything here is written for a reader checking it against the paper by
eye: numpy in complex128, full 4x4 gamma matrices (no half-spinor
projection), products formed in the order the paper states them, and no
blocking or fusion.

Modules
-------
lattice     Wilson-Dirac matrix A = I - kappa*H, gamma matrices, dense A.
philox      Philox-4x32-10 counter generator and Z4 noise (Sec. 1).
polynomial  GMRES polynomials in product (root) form, power basis,
            composite "double" polynomial, scalar values, Leja order
            (Secs. 2.3, 2.4, 3.1, 3.2).
krylov      Arnoldi / GMRES, harmonic Ritz values, PP-GMRES, PP-Arnoldi,
            gamma5 left eigenvectors, eigen selection (Secs. 2.1, 3.1, 4, 5).
mpmc        Deflated level samples, exact corrections, statistics,
            deflated polynomial, multilevel cost formula
            (Secs. 2.2, 3.1, 4.1, 4.3, 5; Eqs. (2), (3)).

Pins: every function is checked by ``tests/test_oracle_*.py`` against
mathematics that does not come from this package (closed forms, dense
linear algebra, invariants, printed numbers).  Functions without such a
pin say "parity unpinned" in their docstring; at present that is only the
bit pattern of Philox (no published known-answer vector is available
offline), see ``oracle/philox.py``.
"""
