"""CPU oracle for the LRE hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct CPU restatements of the linear regression
estimation (LRE) of Qi et al. as used in "Full reconstruction of a 14-qubit
state within four hours" (arXiv:1602.08604):

  explicit.py  Sec. II, Eqs. (1)-(5): build the 6^n x 4^n design matrix X
               from the Pauli eigenprojectors and solve the normal equations
               (X^T X) theta = sum_j p_j Gamma^(j) by Cholesky (n <= 5); build
               mu = sum_i theta_i Omega_i by explicit Kronecker products.
  direct.c     Sec. III-IV: the paper's zero-dropped direct sums.  Step (i):
               per basis group, the 2^n x 2^n nonzero matrix times the group's
               outcome counts, added into the 2^n compatible coefficients,
               then divided by the X^T X diagonal.  Step (ii): mu assembled
               per group of Omega_i sharing nonzero locations (x-mask).
  project.py   Sec. II step (iii): the Smolin-Gambetta-Smith closest-density-
               matrix algorithm, plus an independent sort-based simplex
               projection used only to cross-check it.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
arm may import, call, link or run anything in this package.  It shares no
code with the CUDA path in paper_1602_08604_gb300/.

Parity status: every function here is pinned by tests/test_oracle_*.py
(hand-checked n=1 fixtures, the X^T X diagonal the paper states, infinite-
shot counts of known states, explicit-vs-direct agreement, projection
optimality and the maximally-mixed mean-squared-error law of Sec. V).
"""
