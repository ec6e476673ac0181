"""FP64 CPU oracle for the two-site update of MPS algorithms (DMRG and TEBD).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of the package entry module
and the CPU-baseline leg of the benchmark may import this package.  The product path
(the CUDA library and its Python binding) never imports, calls or falls back to it.

Everything here is plain, slow and written to be checked by eye against the paper
(arXiv:1610.02244, "The Tensor Network Theory Library"): complex128 arithmetic, numpy
einsum / linalg as the only library primitives, no blocking or fusion beyond what the
definitions state.  Each function names the passage it follows.  The oracle shares no
code with the CUDA path; both receive their inputs from the seeded generators in
``paper_1610_02244_gb300.synth`` (random draws and integer structure only), which this
package itself never imports.

Modules
  bose_hubbard  local operators, Hamiltonian MPO, Trotter bond terms and gates (Sec. 5)
  ed            exact diagonalisation in a fixed boson-number sector (the pin)
  contract      theta formation, gate application, H_eff.theta, environments (Sec. 4.2,
                App. B.1.1, Listing 1)
  lanczos       Lanczos eigensolver with full re-orthogonalisation (Sec. 4.3)
  svd           truncated SVD with the four truncation rules (App. B.1.2, Eq. 3)
  dmrg          two-site DMRG sweeps (Sec. 4.3, Listing 2, in two-site form)
  tebd          second-order Trotter TEBD (Sec. 3, Sec. 5)

Parity status: every function is pinned by a test under tests/ against exact
diagonalisation, closed forms, library routines on special cases, brute force or
invariants; none is "parity unpinned".
"""
