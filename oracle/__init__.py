"""FP64 CPU oracle of the C-AMS pressure solver (Tene, Wang & Hajibeygi,
"Adaptive Algebraic Multiscale Solver for Compressible Flow in Heterogeneous
Porous Media").

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
GPU path is checked against.  Only the test-suite, the smoke check of the
package entry point and the CPU-baseline leg of the benchmark may import it;
the library itself never does, and it shares no code with the CUDA path.

Layout (one module per part of the method):
  problem     Sec. 2: grid, fluid, TPFA transmissibilities, nonlinear
              residual, Eq. 19 error, linearised system of Eqs. 3-6 (and
              the full-Jacobian variant of that linearisation)
  wirebasket  Sec. 3: primal/dual-coarse grids, vertex/edge/face/interior
              classification of fine cells and the local entities
  basis       Sec. 3, Eqs. 8-11: basis operators, the staged
              reduced-problem construction of the prolongation P and the
              correction functions
  coarse      Sec. 3, Eqs. 7, 13-15: MSFE/MSFV restriction, R A P and
              the coarse direct solve
  ilu         the ILU(0) second-stage smoother of Sec. 3 / Table 1
  solver      Table 1 iteration inside the Newton loop of Sec. 4.1.1 with
              the adaptive operator updates of Sec. 4.1.2
  net         the learned basis surrogate's network (convolutions, ReLU,
              masked MSE, Adam) for checking the GPU layer kernels

Every floating-point quantity is float64.  Readings of points the paper
leaves open are marked "Reading R<n>" at the place they are used.
"""
from .problem import Grid, Fluid, BC, Problem, transmissibilities, assemble  # noqa: F401
from .wirebasket import Wirebasket, build_wirebasket  # noqa: F401
from .basis import basis_operator, prolongation, prolongation_global  # noqa: F401
from .coarse import restriction, coarse_operator  # noqa: F401
from .ilu import ilu0, ilu_apply  # noqa: F401
from .solver import Options, BasisState, cams_iteration, solve_step, run  # noqa: F401
