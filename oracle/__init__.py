"""Plain, slow FP64 CPU oracle of the paper's discrete method (test infrastructure).

ONLY tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may
import this package.  The product path (the CUDA library and its Python binding)
never imports, calls or links anything here, and this package imports nothing from
the product path.  The two share only the seeded input generators in `workloads`.

Everything is numpy float64, vectorised over elements and quadrature points, with
the steps in the order the paper states them:

  q1.py        Q1 hexahedra, 2x2x2 Gauss quadrature, interpolation and weak-form
               assembly (Section 2.1.2 discretisation on uniform hexes).
  galpha.py    generalized-alpha parameters and the n+alpha / n+alpha_m states
               (Section 2.1.2, generalized-alpha equations).
  bc.py        Dirichlet node sets and values from a problem description.
  ns.py        momentum/continuity residual (Eq. PG_NS with the Newtonian stress of
               Section 2.2 and the Neo-Hookean stress of Section 2.3) and its
               Jacobian-vector product incl. the solid-stress linearization of
               Section 2.4 / Appendix B.
  ac.py        Allen-Cahn residual and JVP (Eq. Allen-Cahn, Eq. PPV_AC).
  cgt.py       left Cauchy-Green transport residual and JVP (Eq. semiCGT).
  mobility.py  time-dependent mobility gamma (Section 2.2.2, Appendix A) and the
               Lagrange multiplier beta (Section 2.2.1).
  diag.py      Jacobi diagonal by probing (definition e_i^T J e_i).
  gmres.py     restarted right-preconditioned GMRES with modified Gram-Schmidt.
  assemble.py  sparse block Jacobians by 27-colour probing and the exact (sparse LU)
               linear solve.
  tet.py       linear tetrahedra (six per box cell, optionally jittered nodes) with
               the same interface, so the weak forms above evaluate on them.
  step.py      partitioned block Newton time step (Section 2.5).
  gridcell.py  grid-cell distance and ray-casting sign with non-duplicated plane
               partitioning (Section 3, Algorithms 1 and 2).
  diagnostics.py  solid centre of mass (Section 5.2) and point tracking (Appendix C).
  pcnet.py     the learned right preconditioner of the NS block (not in the paper): the
               3D convolutional U-Net, its loss, weight gradients, Adam, and the
               flexible-GMRES apply, with the bfloat16 roundings of the GPU network
               emulated where asked.
  fields.py    the nodal state layout and the quadrature-point fields the operators
               share.
  blocks.py    block bookkeeping of the partitioned solve (Section 2.5): the NS, AC
               and B blocks and their unknowns.

Parity pins for every function live in tests/test_oracle_*.py.  Where a function is
not pinned to something outside itself, its docstring says "parity unpinned".
"""
