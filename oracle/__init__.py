"""Plain FP64 CPU oracle for closed-shell CD-CCSD energies, Lambda amplitudes,
Cholesky-basis densities and gradients.

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
benchmark's CPU-baseline / reference arm may import it.  The product path
(the CUDA library and its Python binding) never calls into it, and it shares
no code with that path: it reads inputs produced by `synth` only.

Modules
  model       the model Hamiltonian built from orbital energies and L^P_pq
  ccsd        T1-dressed closed-shell CCSD residual, energy, DIIS solver
  lagrangian  Lambda equations and Gamma^P = dL/dL^P (reverse-mode AD)
  fci2        exact two-electron singlet FCI (pin for o = 1)
  brute       determinant-space projection <mu|exp(-T) H exp(T)|0> (pin)
  mp2         closed-form MP2 energy (pin for the first iteration)
  rows        energy and residual rows at given amplitudes, no full ladder
              (checks at sizes where the full residual is too slow)

Parity status of each function is stated in its docstring; every function
used by the GPU parity tests is pinned by a `-m "not gpu"` test.
"""
