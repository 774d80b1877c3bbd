"""FP64 CPU oracle for the agent-based optimal-control image solver (arXiv 2510.16154).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite, the smoke check in
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import or run
anything in this package.  The CUDA library never calls it and has no fallback to it.

The oracle is a plain, slow, obviously-correct NumPy/SciPy float64 restatement of what
the paper defines, written from the paper's equations:

* ``model``  -- the alignment ODE (Eq. MAsystem) with the anisotropic distance
  (Eq. ellipsoid) and the C2 Wendland kernel (Eq. kernel), explicit Euler in time
  (Section 3.2), the Jacobians of Section 3.1 and the exact discrete adjoint of Euler.
* ``tv``     -- the discrete gradient with reflective boundaries (Definition 3.1,
  Eq. reflective_boundary), its exact transpose, the costs J (Eq. cost_functional),
  K (Eq. cost_TV), L (Eq. cost_tv_regular) and L~ (Eq. complete_square), the terminal
  adjoint (Eq. admm_terminal), the shrinkage (Eq. soft_threshold) and the dual ascent
  (Eq. dual_ascent).
* ``solve``  -- Algorithm 1 (DAL with projected two-way Armijo) and Algorithm 2 (ADMM).
* ``labels`` -- connected-component cluster labels of a colour field (threshold 0.02,
  the watershed threshold of Section 5).
* ``rof``    -- Chambolle-Pock and exact-c-step ADMM loops on the ROF problem, used only
  as pins for the TV operators.

Every reading of a garbled, ambiguous or silent passage is listed in the module that
takes it and gathered in the design notes of the repository.
"""
from .model import (Params, phi, dphi, window_offsets, norm_constant, velocity, forward,
                    forward_final, jacobian_transpose_apply, control_derivative, velocity_at,
                    jacobian_transpose_apply_at,
                    adjoint_step, adjoint, project)
from .tv import (grad, grad_T, grad_matrix, shrink, project_ball, cost_J, cost_K, cost_L,
                 cost_Ltilde, dLtilde_dc, dJ_dc, terminal_adjoint, dual_ascent, alm_stats)
from .solve import SolveOpts, dal_iteration, admm_solve, dal_solve, free_components
from .labels import cluster_labels, cluster_labels_bfs, label_agreement

__all__ = [n for n in dir() if not n.startswith("_")]
