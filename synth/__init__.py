"""Seeded synthetic inputs for the LRE hot path.

This package holds only input synthesis: quantum states, their Born
probabilities under the 3^n Pauli product bases, and multinomial count
samplers driven by a counter-based random generator (Philox4x32-10).
It is shared by the CPU oracle's tests and by the GPU benchmarks and holds
none of the estimator's arithmetic (no least squares, no fold, no assembly,
no projection).

Conventions (fixed for the whole project):
  * n qubits, d = 2**n; qubit 1 is the most significant digit of every index.
  * basis index   b = sum_q a_q 3**(n-q),  a_q in {0:X, 1:Y, 2:Z}
  * outcome index o = sum_q o_q 2**(n-q),  o_q = 0 is the +1 eigenvalue
  * Pauli index   i = sum_q p_q 4**(n-q),  p_q in {0:I, 1:X, 2:Y, 3:Z}
  * counts[b][o] row-major, int32 or int16.
"""
