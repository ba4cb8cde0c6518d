"""CPU oracle for the TNS amplitude method (test infrastructure only).

Plain, slow, complex128 NumPy code written from the paper (Guo, Zhao, Huang,
"Verifying Random Quantum Circuits with Arbitrary Geometry Using Tensor
Network States Algorithm"). It exists to check the CUDA path and is used only
by the tests, by ``__graft_entry__.smoke()`` and by the benchmark's CPU
baseline leg. Nothing in the product library imports it and it imports
nothing from the product library.

Modules:

* ``statevector``  brute-force Schroedinger simulation: the definition
  a(s) = <s|U|0...0> that the untruncated method reaches exactly.
* ``tns``          the method step by step: gate split (Eq. gatesplit), gate
  application (Eqs. result1/result2), SVD compression (Eqs. svd/svd2, and a
  two-sided QR + SVD variant of them),
  two-sided evolution (Fig. 2a), overlap network (Eq. overlap), cutting and
  a contraction by the oracle's own greedy pairwise order; the same sums
  grouped as the double-layer network (ket and bra tensors as separate nodes).
* ``path``         the path score of the supplement (score recursion and
  Eq. optscore) by brute force over orders and by subset dynamic programming.
"""
