"""CPU FP64 oracle for the RAS-PML Helmholtz hot path.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import anything under oracle/. The product
path (the CUDA library and its Python binding) never imports it, and the
oracle imports nothing from the product package: the two share no code. The
only common module is `workloads`, which holds seeded inputs and no method
arithmetic.

Contents, each following the paper (Xie, Gong, Graham, Spence, Zhang,
"Massively parallel Schwarz methods for the high frequency Helmholtz
equation"):

  fem.py     Section 1: PML stretching, the truncated weak form on P1
             triangles (the complex-symmetric gamma_1 gamma_2 form, or
             eq. weak as printed), global matrix and load vector, direct solve.
  ras.py     Section 2 and Section 3 (ii): Cartesian covering, local PML
             stretching, local operators A_j with impedance closure,
             partition of unity chi_j, and the preconditioner
             B^-1 = sum_j R~_j^T A_j^-1 R_j.
  krylov.py  Algorithm 1 (Richardson), and GMRES / FGMRES with B^-1 as a right
             preconditioner (Section 4.1).

Every function is plain NumPy/SciPy in complex128. Pins against values fixed
by the paper and by mathematics live in tests/test_oracle_*.py.
"""
