"""Plain FP64 CPU oracle of the MRT-LB method of Shi, Yuan & Chai (arXiv 2512.16230).

TEST INFRASTRUCTURE ONLY. The oracle is the slow, obviously correct statement of what the CUDA
library computes, written from the paper (Sec. 2, Sec. 4, Sec. 5, App. A, C, D) with numpy in FP64.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it. It shares no code, tables, constants or pre/post-processing with the CUDA path, and the
product path never routes through it.

Parity status of each function (pins live in ``tests/test_oracle_*.py``):

* weights (Eq. (WeightQ25), (Q13lattice), App. D): pinned by the printed worked examples of
  App. C (D2Q17 cases 1-5) and by the brute-force lattice-moment identities Eq. (Cont1-5);
* Hermite rows and their rectangular correction (Eq. (CorrectQ25), App. D): pinned by the
  printed closed-form correction coefficients (special D2Q21, rD3Q53, rD3Q33), the printed
  monomial matrices (Eq. (TransM), Eq. (TransM33)) and HWH^T being diagonal;
* equilibrium (Eq. (feq-1)): pinned by the continuous moments up to third order and f^eq(rho,0)
  = w rho;
* collision (Eq. (2-3), Eq. (H-MRT-LB)): pinned by exact mass and momentum conservation, the
  block form Eq. (H-MRT-LB-1), S = I and the BGK special case; distinct rates of the orders >= 4
  by projectors built independently from all monomials of each degree; the bulk block of
  Eq. (4-27) by the sound-wave damping of Eq. (4-29) and its diagonal special case;
* streaming (Eq. (2-2b)): pinned by delta transport and reversibility;
* dynamics: pinned by Taylor-Green decay at nu = cs2 (1/s - 1/2), Kolmogorov steady flow, and
  Gaussian-hill diffusion of the linear NCDE.
"""
from . import lattice, mrt  # noqa: F401
