"""CPU oracle for the D^3M hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct fp64 NumPy/SciPy restatement of what the
paper computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import it; the product path (the CUDA
library and its Python binding) never does, and this package imports nothing
from the product except the seeded input generator
``paper_2002_05018_gb300.workloads``.

Modules
  fem       lowest-order Nedelec brick elements, curl-curl - k^2 eps_r with a
            first-order ABC, plane-wave RHS (Theory section, decomposed BVP)
  decomp    subdomains with interface loss/gain, signed Lagrange-multiplier
            map D and interface blocks (Theory section, Eq. (1))
  ordering  nested dissection inside each subdomain, block nested dissection
            of the clique graph of K, supernodal symbolic factorisation by the
            elimination game (main steps 3-4)
  bk        dense Bunch-Kaufman LDL^T restricted to a pivot block (ref. [6])
  d3m       the seven main steps: domain matrices K_D, assembly of K,
            Algorithm 1 block LDL^T, substitution, recovery of E
  adjoint   gradient of J = sum |x_probe|^2 w.r.t. per-cell eps_r
  gmres_ir  plain and GMRES-based iterative refinement with a low-precision
            factorisation (the mixed path's refinement step and its
            GMRES-IR variant)

Parity status per function is stated in each module header.
"""
