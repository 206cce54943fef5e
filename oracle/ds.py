"""FP64 CPU oracle of the time-splitting spectral DS step (Sec. 2.3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* linear flow (eqs. 1st_tssp, 1st_tssp_more), exact in Fourier space on the
  periodic grid: v_hat <- exp(-i tau (k_x^2 - alpha k_y^2)) v_hat;
* nonlinear flow (eqs. 2nd_tssp, 2nd_tssp_more) with |w| and Phi frozen:
  w <- w exp(i tau (2 beta |w|^2 + 4 beta Phi)), Phi from ``oracle.solve``;
* Strang composition L(tau/2) N(tau) L(tau/2), the symmetric second-order
  member of the family of compositions of the two flows;
* Yoshida's fourth-order composition, the integrator the paper uses (Sec. 2.3):
  seven sub-flows A(a1 t) B(b1 t) A(a2 t) B(b2 t) A(a3 t) B(b3 t) A(a4 t).
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


def yoshida_coefficients():
    """Sec. 2.3: b1 = b3 = 1/(2 - 2^(1/3)), b2 = -2^(1/3) b3, a1 = a4 = b3/2,
    a2 = a3 = (b3 + b2)/2.  Returns (a1, a2, a3, a4), (b1, b2, b3)."""
    cbrt2 = 2.0 ** (1.0 / 3.0)
    b3 = 1.0 / (2.0 - cbrt2)
    b1 = b3
    b2 = -cbrt2 * b3
    a1 = a4 = 0.5 * b3
    a2 = a3 = 0.5 * (b3 + b2)
    return (a1, a2, a3, a4), (b1, b2, b3)


def yoshida_step(u: np.ndarray, p: OracleParams, tau: float, alpha: float, beta: float) -> np.ndarray:
    """u^{n+1} = e^{A a1 tau} e^{B b1 tau} e^{A a2 tau} e^{B b2 tau} e^{A a3 tau}
    e^{B b3 tau} e^{A a4 tau} u^n (Sec. 2.3): the rightmost factor acts first.
    Each B sub-flow freezes Phi = A(|w|^2) of the field it starts from."""
    a, b = yoshida_coefficients()
    u = linear_flow(u, p.lx, p.ly, a[3] * tau, alpha)
    for j in (2, 1, 0):
        phi = solve(np.abs(u) ** 2, p)
        u = nonlinear_flow(u, phi, b[j] * tau, beta)
        u = linear_flow(u, p.lx, p.ly, a[j] * tau, alpha)
    return u


def arkadiev_lump(x: np.ndarray, y: np.ndarray, t: float) -> np.ndarray:
    """Case I of Example 3 (Sec. 3.2): the exact moving lump of the
    hyperbolic-elliptic DS equation with alpha = 1, beta = -1."""
    return 2.0 * np.exp(1j * (2.0 * y + 4.0 * t)) / ((x + 1.0) ** 2 + (y + 4.0 * t) ** 2 + 1.0)
