"""CPU oracle for the SYK matrix-free Krylov correlators (TEST INFRASTRUCTURE).

A plain, slow, fp64 restatement of what the paper computes, written from its
definitions and shared with no part of the CUDA path.  Only the test suite,
the package smoke check and the benchmark's CPU-baseline leg may import it;
the product path never calls it.

Modules
-------
jw           Majorana operators by the Jordan-Wigner map (Supp. Sec. I.A) as
             dense matrices and as their action on basis states.
hamiltonian  Eq. 1: term list, Pauli-string table of each term, the sector
             restriction of H (Supp. Sec. I.A, parity), brute-force rows.
evolve       exact e^{zH} psi (dense eigendecomposition, or scipy's
             Al-Mohy-Higham expm_multiply for larger sectors) and the m x m
             tridiagonal exponential (Supp. Sec. I.B).
correlators  G(t) (Eq. G) and the regularized OTOC F(t) (Eq. F_reg) estimated
             with one random state (Eq. q_typicality), plus trace forms for
             small N.
capply       ctypes wrapper of c/apply_terms.c: a term-at-a-time fp64 H|psi>
             loop (OpenMP), used to time the CPU baseline.

Parity pins: every function is checked in tests/test_oracle_pins.py against
closed forms, invariants or library routines; none is marked unpinned.
"""
