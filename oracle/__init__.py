"""CPU oracle for the matrix-free FAS multigrid V-cycle with X-MCGS smoothing.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call or execute this package:
only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs use it. It shares
no code with the CUDA path (paper_2510_11152_gb300/); the two meet only through the seeded input
generators in workloads/.

The oracle is plain float64 numpy, written step by step from the paper:
  - cell_centred.py : discrete operator (Sec. 2.2, Eq. PDE_discret with ghost relations),
                      X-MCGS smoother (Sec. 2.3 Eqs. FCGS-1..4; 3D sets of Appendix B),
                      restriction / prolongation (Appendix C), FAS two-grid Algorithm 1 with the
                      recursive multilevel remark, the residual norm of Eq. residual,
                      backward-Euler heat stepping, mixed-precision iterative refinement;
                      periodic axes (reading A17).
  - staggered.py    : MAC face grids and the first- and second-order projection steps (Sec. 4).
  - grain_growth.py : the grain-growth example's multi-order-parameter Allen-Cahn step (Sec. 3.3.1),
                      one periodic solve per order parameter.
Each function's docstring names the passage it follows, and every reading taken where the paper is
silent or garbled is stated where it is used.
"""
from . import cell_centred  # noqa: F401
