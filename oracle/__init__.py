"""Plain FP64 CPU oracle for the SIMP hot path of arXiv 2012.08208.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the CPU
baseline / reference arm of `bench.py` may import or run anything in this
package.  The product path (the CUDA library and its Python binding) never
imports it, and this package imports nothing from the product.  The two share no
code; they share only the seeded problem data in `workloads`.

Modules (each function cites the passage of the paper it follows):
  element  unit Q4 / H8 element stiffness K0 (Gauss quadrature and exact rational)
  mesh     structured-grid numbering and element centres
  fem      assembled sparse K(rho), direct / CG solve, matrix-free reference product
  sens     compliance and element sensitivities
  filt     mesh-independency sensitivity filter (dense EDM and sparse forms)
  oc       optimality-criteria update with bisection, and the exact multiplier
  simp     the SIMP loop
  nn       reference 3D conv network (FP64) for the learned warm start
  helm     Helmholtz (PDE) filter of the paper's parallel runs
  p1       the paper's own elements: vector P1 on triangulated / tetrahedralised
           structured grids, DG0 density, one SIMP iteration

Parity status: every function here is pinned by `-m "not gpu"` tests
(closed forms, invariants, exact arithmetic, brute force, finite differences),
except the whole-loop trajectory, which the paper prints no numbers for
("parity unpinned" against the paper itself; pinned per step).
"""
