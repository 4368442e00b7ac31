"""Plain FP64 CPU oracle for the coupling-aware Vanka (CAV) multigrid method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link or
execute this package: only the tests, the smoke check and the bench's CPU
baseline use it.  It shares no code with the CUDA library; the two meet only in
the seeded inputs of `ib_workloads`.

Each module restates one part of the paper, in the paper's order and notation,
with library primitives (sparse products, dense solves, eigenvalues) as steps
and no blocking, fusion or reordering:

  grid       MAC grid, D, G, L, A0 and the reduced operator K_E   (Sec. 2, Eq. intro_saddle)
  ib         Peskin 4-point kernel, spreading S, interpolation J,
             force matrices E and E_E = S E J                     (Sec. 2, Sec. 5.1, 5.2)
  patches    Vanka, box B(b,o) and CAV patch sets                   (Sec. 3.1, 3.2, Eq. cav_patch_set)
  smoother   local matrices, equilibration, LU, multiplicative and
             weighted additive sweeps                             (Sec. 3.3, Eq. additive_cav_saddle)
  colouring  classes of mutually independent patches and the
             multiplicative sweep visiting them class by class     (Sec. 3.3)
  multigrid  RT0 / bilinear transfers, Galerkin E_E, hierarchy,
             coarsest bordered solve, V-cycle                      (Sec. 4)
  fgmres     right-preconditioned flexible GMRES                    (Sec. 5)
  twogrid    two-grid iteration matrix and its spectrum            (Sec. 5.1, Table 1)
  fiber      nonlinear fiber energies, force and Newton tangent    (Sec. 5.3)
  newton     Newton's method for one semi-implicit step            (Sec. 5.3)
  channel    the inflow / traction-outflow channel: MAC operators, multigrid, the
             fiber's linear systems and its Newton time step          (Sec. 5.3)
"""
from . import grid, ib, patches, smoother, colouring, multigrid, fgmres, twogrid, fiber, newton  # noqa: F401
from . import channel  # noqa: F401
