"""CPU FP64 reference implementation of the MRCM pressure solve (the ORACLE).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the paper's method used to check the CUDA path.  Only the test
suite, the package smoke check and the bench's CPU-baseline leg may import or
run it; the product path (the C-ABI library and its Python binding) never
touches it and shares no code with it.

Modules:
  problem    - geometry, decomposition, interface space V_H, Eq. dof_PH
  tpfa       - Eq. aijk / Eq. darcy-discrete and the global fine solver
  mrcm       - Alg. MRCM: local problems, interface system, reconstruction
  monolithic - the monolithic system solved densely (tiny grids)
  conv3d     - the learned warm-start network's reference forward/backward
"""
from .problem import Problem, from_workload, build_bases, count_interface_dofs, interior_rhs_count
from .tpfa import solve_fine, fine_system
from .mrcm import solve_mrcm, relative_errors, mass_residual
from .monolithic import solve_monolithic
