"""CPU oracle for the CAP-terminated Landauer transmission T(E, k).

THIS PACKAGE IS TEST INFRASTRUCTURE.  It is a plain, slow, complex128 restatement of
what the GPU library computes, written from the paper (Zhu, Feldman & Dunham,
"Highly parallelizable electronic transport calculations in periodic Rhodium and
Copper nanostructures", arXiv 2208.02783) so that the CUDA path can be checked
against it.  Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline
leg may import it; the library never does, and it shares no code with the library
(its only shared dependency is the seeded input package ``workloads``).

Modules
-------
fd           central finite-difference coefficients (exact rationals)
hamiltonian  H_k with Bloch-phased lateral faces and A(E, k) in CSR form
transmission T(E, k) by dense LU, sparse LU or plain COCG / transpose BiCG; k-average
closed_form  separable V = 0 transmission and open-channel (mode) counting
unet         NumPy forward/backward of the learned preconditioner's network
eigen        the paper's eigen route: eigenpairs of H_k - i Gamma, transformed CAPs, eigen-sum
sketch       the two-sided randomized sketch of T with the library's splitmix64 draws

Every function is pinned by tests/test_oracle_*.py against facts fixed by the paper
or by mathematics (polynomial exactness, Hermiticity, separable closed form, the
long-CAP limit T -> number of open channels, T_LR = T_RL, T(k) = T(-k), the Ward
identity); none is pinned only against itself.
"""
