"""CPU oracle for the ABAC-preconditioned MINRES all-at-once wave solver.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
FP64 restatement of what the paper (Lin & Hon, "A block alpha-circulant based
preconditioned MINRES method for wave equations") computes.  Only the test
suite, the smoke check and the CPU-baseline leg of the benchmark may import
it; the product path (the C-ABI library and its Python binding) never does.
It shares no code with the GPU path: the only module both use is the seeded
input generator `workloads`, which holds no arithmetic of the method.

Modules
  system    -- Delta_h, L, the all-at-once matrix T (eq. main_matrix), Y, C_alpha
               (def. matrix_C_alpha and its Kronecker split eqn C_decom), the
               right-hand side, Y*T applied as a stencil, the error E_{tau,h}
  fast      -- P_alpha^{-1} by the three-step procedure of Section 2.3 with
               explicit DFT / DST matrices (no FFT)
  dense     -- tiny-size dense forms: sqrtm(C_alpha), P_alpha, Cholesky solves,
               the ideal preconditioner, the alpha = 1 (ABC) case
  minres    -- textbook preconditioned MINRES
  stepping  -- sequential time stepping of the same scheme

Parity status: every function is pinned by a `-m "not gpu"` test in
tests/test_oracle_*.py against closed forms, invariants, the paper's
Table 2 values, library special cases or brute force.  No function is
"parity unpinned".
"""
