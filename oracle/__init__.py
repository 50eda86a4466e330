"""Plain FP64 CPU oracle for the MLMC multigrid hot path.

TEST INFRASTRUCTURE ONLY. Only tests/, the smoke check and the CPU-baseline leg of
bench.py may import this package. It shares no code with the CUDA library
(paper_1607_03252_gb300) and never imports it.

Contents:
  mlmc_oracle.c  the solver, field and sample pipeline in plain C (FP64), each
                 function citing the passage of Gmeiner et al. it follows;
  core.py        ctypes wrapper around it;
  stats.py       MLMC estimator statistics (Sec. 2: Eqs. 6, 8, 10, 11, 14, 15) from
                 their plain definitions with exactly rounded sums, and the rate fit of
                 the alpha, beta, gamma exponents (Eqs. 12, 14);
  adaptive.py    Algorithm 2 (adaptive MLMC with level growth by the bias test) over
                 any sampler of the level differences;
  schedule.py    the performance model and scheduling rules of Secs. 4-5, with the
                 heterogeneous optimum by exhaustive search;
  fe.py          P1 finite elements on the tetrahedral mesh (four-vertex quadrature of
                 k), P1 transfers, FMG-2V(4,4) and the point and flux QoIs (Secs. 3.1, 7).

Parity status (each item's pin lives in tests/test_oracle_*.py):
  Philox4x32-10 words  round structure pinned through the 64-bit variant against
                       numpy's Philox4x64-10; the 32-bit constants are pinned only by
                       statistical tests (no published test vector is available offline);
  field                pinned by its mean, variance and covariance closed forms, for the
                       Gaussian covariance and for the exponential one of Sec. 3.2 (the
                       multivariate Cauchy radial law, isotropy, the characteristic function);
  operator, smoother,  pinned by the exact discrete eigenfunction, the O(h^2)
  transfer, V-cycle    manufactured-solution rate, a dense direct solve, the transfer
                       adjoint and exactness identities, and h-independent convergence;
  QoI                  pinned by trapezoid exactness on multilinear functions;
  statistics           pinned by math.fsum and a hand-evaluated Eq. 11 case;
  SPDE sampler         pinned by the FP32 log's error bound, the normals' law, an
                       independent aggregation of the octant noise (fine and coupled
                       coarse cells), the operator by hand, the exact solve against the
                       operator, the sampled covariance against the discrete model's
                       exact covariance, and that model against Whittle's closed form;
  rate fit             pinned by exact geometric data and an independent polynomial fit;
  P1 FE / FMG          pinned by symmetry, conservation, the seven-point structure on
                       this mesh, the constant-k Laplacian, the patch test, O(h^2)
                       manufactured convergence, exact linear prolongation, FMG's algebraic
                       error far below the discretisation error, and closed-form QoIs;
  scheduling model     pinned by the paper's worked examples (716 s; 684 s with the
                       allocation (1031, 172, 36, 6) on 7783 processors; two sequential
                       steps at 524288 processors and Sec. 5.2's 75% / below-1% chances of
                       the slow run) and closed forms of the Amdahl surrogate;
  Algorithm 2          pinned by hand-worked level counts of synthetic samplers (the
                       eps_b / eps and alpha choices each change them) and by the
                       stopping invariants (Eq. 10 sampling variance <= eps_s^2, the bias
                       test met at L and failed at L - 1).
"""
from .core import *  # noqa: F401,F403
from . import adaptive, fe, schedule, stats  # noqa: F401
