"""CPU oracle for the Pfaffian-sign hot path (test infrastructure only).

A plain, slow, FP64 restatement of what the GPU library computes, written from
the paper (arXiv:2108.11989, Sec. 2 and Sec. 3).  Only the test-suite, the
smoke check and the CPU-baseline leg of the benchmark may import it; the
product path never does.  It shares no code with the CUDA library: the only
common module is ``synth_inputs`` (seeded random numbers, no arithmetic of the
method).

Modules
  gamma     chiral-basis Dirac matrices, C = i g0 g2, sigma_{mu nu}   (Sec. 3)
  lattice   orientifold-doubled lattice for C* boundaries, mirror links (Sec. 3, eq. for T)
  dirac     O(a)-improved Wilson-Dirac operator D and Q = g5 D, as 12x12 site
            blocks (matrix-free, sparse, dense)                         (Sec. 2, Sec. 3)
  pfaffian  Pfaffian by Parlett-Reid elimination (log-modulus + phase),
            brute force for tiny matrices; pfaffian_c.c for large n     (eq. power1/4)
  sign      the Pfaffian sign by its definition (dense pf ratio) and by the
            eigenvalue count, the step-A mass scan and the step-B flow  (Sec. 3)
  lowmodes  smallest eigenvalues of |Q| by library Lanczos (scipy)     (Sec. 3)

Parity status of each function is stated in its docstring; every function is
pinned by a test in tests/test_oracle_*.py against closed forms, invariants
or brute force, except where a docstring says "parity unpinned".
"""
