"""CPU FP64 oracle for homogeneous diffusion inpainting and data optimisation.

TEST INFRASTRUCTURE ONLY. Nothing in the product package may import, call or
execute this package; only the tests, the graft smoke check and the CPU
baseline leg of the benchmark do. It shares no code with the CUDA path: it
restates the paper's definitions in plain NumPy/SciPy (FP64) so that a reader
can check each function against the paper by eye.

Modules
  laplace   -- the discrete model of Sec. 2.1: L, A = C + (I-C)L, b = Cf,
               the inpainting solve and its general-right-hand-side variant.
  tonal     -- tonal optimisation (Sec. 5): B = A^{-1}C, B^T via the
               symmetrised system, CG on the normal equations, CGNR with the
               MSE-gain stopping rule, and an
               independent projection formulation used as a cross-check.
  ras       -- restricted additive Schwarz for tonal optimisation (Alg. 2)
               with exact local solves, and the overlapping decomposition.
  vi        -- Voronoi initialisation of tonal optimisation (Sec. 5.3):
               influence-zone weights, the average-interpolation Richardson
               iteration with its stop-on-rise rule.
  densify   -- one Delaunay densification step (Sec. 4, Alg. 1) with exact
               integer geometry, and the random-dithering initial mask.
  splitmix  -- SplitMix64 counter-based generator (Steele, Lea, Flood 2014).

Parity status: every function is pinned by tests in tests/test_oracle_*.py
except where a module header says "parity unpinned".
"""

from .laplace import (  # noqa: F401
    laplacian,
    apply_A,
    inpaint,
    solve_A,
    inpaint_residual,
    rel_residual,
)
from .tonal import (  # noqa: F401
    B_apply,
    Bt_apply,
    tonal,
    tonal_projection,
    normal_residual,
    mse,
    tonal_cgnr,
    mse_gain_stop,
)
