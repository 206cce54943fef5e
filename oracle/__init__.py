"""FP64 CPU oracle for the split (I1 + I2) nonlocal potential solver.

TEST INFRASTRUCTURE ONLY. Nothing in the product package imports this
directory; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code, tables or constants with the
CUDA path.

What it computes (Mauser, Stimming, Zhang, "A novel nonlocal potential solver
based on nonuniform FFT ...", Sec. 2.1):

  Phi = I1 + I2                                   (eqs. PotSplitWhoSpace/SubInt1/SubInt2)
  I1  = zero-padded trapezoid/FFT evaluation of the (1-p) part  (Sec. 2.1, kappa >= 2)
  I2  = polar Gauss quadrature of the p part     (eq. I2PolarDisc)
        with rho_hat at the polar nodes from the trapezoid rule written
        as a direct sum (the exact value a type-2 NUFFT approximates, eq. 2.2)
        and the weighted sum back onto the grid written as a direct sum
        (the exact value a type-1 NUFFT approximates, eq. 2.1).

Parity status of each function is stated in its module docstring; every
function here is pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*``.
"""

from .potential import (  # noqa: F401
    OracleParams,
    grid_axis,
    polar_nodes,
    radial_rule,
    polar_weights,
    partition,
    multiplier,
    multiplier_high,
    DS_MULTIPLIER,
    i1_padded_fft,
    i1_padded_fft_adjoint,
    rho_hat_direct,
    i2_direct_from_coeffs,
    i2_direct,
    solve,
    solve_adjoint,
    standard_fft_solve,
)
from .closed_forms import (  # noqa: F401
    gaussian_potential,
    gaussian_i2_exact,
    gaussian_potential_alpha0,
    gaussian_coulomb,
    gaussian_abs_k,
    paper_gaussian_density,
    paper_gaussian_potential,
    arkadiev_density,
    arkadiev_potential,
)
