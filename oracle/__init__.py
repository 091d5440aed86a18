"""Oracle: a plain, slow, FP64 CPU restatement of the flux-reconstruction (FR) method.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's CPU-baseline
leg may import this package.  The CUDA library never calls it, and it shares no code with the
library: it has its own Gauss-Legendre nodes (Newton on P_N), its own Lagrange/derivative and
correction construction, its own mesh connectivity (centroid and flux-point coordinate
matching instead of vertex-id sorting) and its own dense per-element operators.

What it computes (arXiv 2308.06605, Section "FR Algorithm"):
  * Eq. 1: the conservation law mapped to the reference hexahedron, Q^ = |J| Q,
    F^ = |J| J^-1 F with J_ij = dx_i/dxi_j.
  * Eq. 2a-c: nodal Lagrange representation of Q, F, G on N^3 Gauss-Legendre solution points.
  * Eq. 3: the semi-discrete residual dQ/dt = -|J|^-1 [div_xi F^ + sum over faces and flux
    points of div(g_ij) (F^I_perp - F_perp)] + S, with the correction g chosen so the scheme is
    nodal collocated DG (VCJH c = 0, Huynh 2007), an approximate Riemann solver (Rusanov) for the
    common normal flux, and the BR2 viscous treatment.
  * The explicit RK time integration (classical four-stage RK).

Modules: `basis` (1D nodes, Lagrange, derivative, correction), `fr1d` (1D linear advection, used
to pin DG equivalence), `hexfr` (3D hexahedral Navier-Stokes residual and RK44), `gas`
(ideal-gas fluxes).  Pins live in tests/ (marked "not gpu").
"""
