"""Plain CPU FP64 oracle for the Rotne-Prager-Blake Brownian-dynamics hot path.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
reference that the CUDA library is checked against.  Only tests/, the smoke
check in __graft_entry__.py and the CPU-baseline leg of bench.py may import,
call, link or execute anything under oracle/.  The product path never does: it
fails loudly when its CUDA library is missing.  The oracle shares no code,
header, helper or constant table with the CUDA path, and neither imports the
other; only the seeded input generator (paper_1612_00474_gb300/inputs.py, no
method arithmetic in it) serves both.

Pieces and the passages they follow:
  rpb_oracle.c   free-space RPY tt/tr blocks with their overlap branches (Sec. II.B,
                 Sec. III), regularisation M = B Mtilde B (Appendix A), matvec and
                 dense assembly, soft steric + gravity forces (Sec. III).
  wall_image.c   generated by derive_wall.py: Faxen operators applied to Blake's
                 image system (Eq. mobilityDifferential, Eq. mobilityDifferentialTR).
  core.py        Lanczos M^{1/2} W (Sec. II.C; optionally with the block-diagonal
                 preconditioner that section reports trying), RFD drift (Sec. II.A), AB step (Eq. AB).
  philox.py      Philox4x32-10 Gaussian noise (generator of Salmon et al., SC'11).

  equilibrium.py Metropolis Monte Carlo of the Gibbs-Boltzmann distribution (mcmc.c) and
                 the height density and pair correlation of Appendix B (test statistics).

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, invariants, library routines or brute force; Philox4x32-10 is
pinned against the independent implementation in the Triton library (run on
the CPU by its interpreter) and its 4x64 round structure against numpy's
Philox (see philox.py).
"""
from .core import (ab_step, blake_image_raw, blake_image_raw_batch, dense, forces, freespace_tr, freespace_tt, lanczos_sqrt,  # noqa: F401
                   mobility_apply, noise, pair_blocks, rel_err, rfd_drift, self_diagonal, wall_image_tr,
                   wall_image_tt)
