"""FP64 CPU oracle of the time-splitting spectral DS step (Sec. 2.3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* linear flow (eqs. 1st_tssp, 1st_tssp_more), exact in Fourier space on the
  periodic grid: v_hat <- exp(-i tau (k_x^2 - alpha k_y^2)) v_hat;
* nonlinear flow (eqs. 2nd_tssp, 2nd_tssp_more) with |w| and Phi frozen:
  w <- w exp(i tau (2 beta |w|^2 + 4 beta Phi)), Phi from ``oracle.solve``;
* Strang composition L(tau/2) N(tau) L(tau/2) (the paper composes the two
  flows; Sec. 2.3 uses a fourth-order composition, the symmetric second-order
  one is the simplest of that family).
"""

from __future__ import annotations

import numpy as np

from .potential import OracleParams, solve


def wave_numbers(n: int, half_width: float) -> np.ndarray:
    h = 2.0 * half_width / n
    return 2.0 * np.pi * np.fft.fftfreq(n, d=h)


def linear_flow(u: np.ndarray, lx: float, ly: float, tau: float, alpha: float) -> np.ndarray:
    ny, nx = u.shape
    kx = wave_numbers(nx, lx)[None, :]
    ky = wave_numbers(ny, ly)[:, None]
    return np.fft.ifft2(np.exp(-1j * tau * (kx * kx - alpha * ky * ky)) * np.fft.fft2(u))


def nonlinear_flow(u: np.ndarray, phi: np.ndarray, tau: float, beta: float) -> np.ndarray:
    return u * np.exp(1j * tau * (2.0 * beta * np.abs(u) ** 2 + 4.0 * beta * phi))


def strang_step(u: np.ndarray, p: OracleParams, tau: float, alpha: float, beta: float) -> np.ndarray:
    u = linear_flow(u, p.lx, p.ly, 0.5 * tau, alpha)
    phi = solve(np.abs(u) ** 2, p)
    u = nonlinear_flow(u, phi, tau, beta)
    return linear_flow(u, p.lx, p.ly, 0.5 * tau, alpha)


def arkadiev_lump(x: np.ndarray, y: np.ndarray, t: float) -> np.ndarray:
    """Case I of Example 3 (Sec. 3.2): the exact moving lump of the
    hyperbolic-elliptic DS equation with alpha = 1, beta = -1."""
    return 2.0 * np.exp(1j * (2.0 * y + 4.0 * t)) / ((x + 1.0) ** 2 + (y + 4.0 * t) ** 2 + 1.0)
