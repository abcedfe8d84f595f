"""FP64 CPU oracle for one domain-decomposed PINN training step.

This package is TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product path (the CUDA
library and its Python binding) never does, and shares no code with it.

It restates the method in plain double-precision PyTorch CPU ops:
  * the network of Sec. 3 (tanh hidden layers, slope n*a^k = 1, identity or
    softplus last layer);
  * input derivatives by reverse-mode automatic differentiation, as the paper
    computes them (Sec. 4.1);
  * the PDE residuals of Sec. 7 (Eqs. BE, NSEq, heq) and the Poisson problem;
  * the cPINN loss (Eq. cPINNLoss) and the XPINN loss (Eq. XPINNLoss) with the
    neighbour's interface values treated as constants (Algorithm 1 receives
    them by message passing and optimises each subdomain on its own);
  * per-subdomain Adam (Sec. 6) and the stitched prediction (Eq. FSol).

Every function is pinned by tests that do not reuse it (closed forms, finite
differences, invariants and special cases); see tests/test_oracle_pins.py.
"""
from .xpinn_oracle import (  # noqa: F401
    Oracle, network, jets, residual, flux_normal, adam_update, route_rect, route_voronoi,
    K_RES, K_IFACE, n_eq, n_out_total,
)
