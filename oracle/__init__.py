"""CPU oracle for the nodal DG acoustic solver on vertically mapped wedges and
tetrahedra (Chan, Wang, Hewett, Warburton, "Reduced storage nodal
discontinuous Galerkin methods on semi-structured prismatic meshes").

TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64 NumPy.  Only tests/,
__graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may
import it; the library never does, and this package imports nothing from the
library (it shares no code with the CUDA path).

Modules
  reference  -- 1D GLL line, triangle and tetrahedron reference elements
                (Section 3.1), built from their definitions by quadrature.
  mesh       -- connectivity and face-node matching by coordinates.
  dg         -- Lemma 3.1 geometry, the Kronecker (method) form of
                Section 4.2, the brute-force quadrature form of Section 2.1,
                LSRK45, discrete energy (Section 4.1), dense RHS matrix,
                GLL mass-lumped variant (Section 4.1) and L2 errors.
"""
