"""Closed-form densities and potentials used to pin the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Gaussian rho = exp(-r^2): the paper's Example 1 (Sec. 3.1) prints the
  potential of rho_p = pi exp(-pi^2 r^2).  Because the multiplier
  -k_x^2/|k|^2 is homogeneous of degree 0, Phi[rho(a .)](x) = Phi[rho](a x);
  with rho_p(x) = pi rho(pi x) this gives
      Phi(r, phi) = -1/2 [ e^{-r^2} + cos(2 phi) (e^{-r^2}(1 + r^2) - 1) / r^2 ]
  for rho = exp(-r^2), Phi(0) = -1/2.
* I2 of the Gaussian with the Gaussian partition p = exp(-|w|^2/sigma^2):
  p rho_hat = pi exp(-l^2 |w|^2 / 4) with l^2 = 1 + 4/sigma^2, which is
  rho_hat of exp(-r^2/l^2) divided by l^2, so I2 = Phi(x/l) / l^2 (for the
  untruncated disk; the disk |w| <= P drops a part of relative size
  exp(-l^2 P^2 / 4)).
* Arkadiev's rational pair of Example 2 (Sec. 3.1).
* Other multipliers of the family |w|^alpha (a0 + ac cos 2theta + as sin 2theta)
  (the Remark of Sec. 2.2), for rho = exp(-r^2), rho_hat = pi exp(-|w|^2/4):
  - alpha = 0: a0 rho + (ac cos 2phi + as sin 2phi) f(r), where f is the
    cos 2phi part above (a rotation by 45 degrees turns cos 2theta into
    sin 2theta in both spaces);
  - 2 pi/|w| (the 2D transform of the 3D Coulomb kernel 1/|x|):
    Phi = (2 pi)^-2 int 2 pi^2 e^{-k^2/4}/k e^{i w.x} dw = pi int_0^inf e^{-k^2/4} J0(k r) dk
        = pi^{3/2} e^{-r^2/2} I0(r^2/2);
  - |w|: Phi = 1/2 int_0^inf k^2 e^{-k^2/4} J0(k r) dk
        = sqrt(pi) e^{-r^2/2} [(1 - r^2) I0(r^2/2) + r^2 I1(r^2/2)]
  (both integrals from int_0^inf e^{-a k^2} J0(b k) dk = (1/2) sqrt(pi/a)
  e^{-b^2/(8a)} I0(b^2/(8a)) and its derivative in a).
"""

from __future__ import annotations

import math

import numpy as np
import scipy.special


def _f2(s: np.ndarray) -> np.ndarray:
    """(e^{-s}(1 + s) - 1) / s^2, with its Taylor series
    sum_{k>=2} (-1)^k (1 - k) / k! s^{k-2} where the direct form cancels."""
    s = np.asarray(s, dtype=np.float64)
    out = np.empty_like(s)
    small = s < 1.0
    ss = s[small]
    acc = np.zeros_like(ss)
    term_pow = np.ones_like(ss)
    for k in range(2, 40):
        coef = (-1.0) ** k * (1.0 - k) / math.factorial(k)
        acc += coef * term_pow
        term_pow = term_pow * ss
    out[small] = acc
    sb = s[~small]
    out[~small] = (np.exp(-sb) * (1.0 + sb) - 1.0) / (sb * sb)
    return out


def gaussian_potential(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Phi for rho = exp(-(x^2 + y^2)); cos(2 phi) r^-2 = (x^2 - y^2) r^-4."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    s = x * x + y * y
    return -0.5 * (np.exp(-s) + (x * x - y * y) * _f2(s))


def gaussian_potential_alpha0(x: np.ndarray, y: np.ndarray, a0: float, ac: float, as_: float) -> np.ndarray:
    """Phi for rho = exp(-r^2) and m = a0 + ac cos 2theta + as sin 2theta."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    s = x * x + y * y
    return a0 * np.exp(-s) + (ac * (x * x - y * y) + as_ * 2.0 * x * y) * _f2(s)


def gaussian_coulomb(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Phi for rho = exp(-r^2) and m = 2 pi/|w|: pi^{3/2} e^{-r^2/2} I0(r^2/2)."""
    s = np.asarray(x, dtype=np.float64) ** 2 + np.asarray(y, dtype=np.float64) ** 2
    return math.pi ** 1.5 * scipy.special.i0e(0.5 * s)


def gaussian_abs_k(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Phi for rho = exp(-r^2) and m = |w|."""
    s = np.asarray(x, dtype=np.float64) ** 2 + np.asarray(y, dtype=np.float64) ** 2
    return math.sqrt(math.pi) * ((1.0 - s) * scipy.special.i0e(0.5 * s) + s * scipy.special.i1e(0.5 * s))


def gaussian_i2_exact(x: np.ndarray, y: np.ndarray, sigma: float) -> np.ndarray:
    """I2 (untruncated) of rho = exp(-r^2) with p = exp(-|w|^2/sigma^2)."""
    l2 = 1.0 + 4.0 / (sigma * sigma)
    l = math.sqrt(l2)
    return gaussian_potential(np.asarray(x) / l, np.asarray(y) / l) / l2


def paper_gaussian_density(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """rho = pi exp(-pi^2 (x^2 + y^2)) (Example 1, Sec. 3.1)."""
    return math.pi * np.exp(-math.pi**2 * (x * x + y * y))


def paper_gaussian_potential(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Example 1's printed potential, in polar coordinates:
    -(pi/2 e^{-pi^2 r^2} + cos(2 theta) e^{-pi^2 r^2} (2 pi r^2)^-1
      (1 + pi^2 r^2 - e^{pi^2 r^2})),
    evaluated with the same small-r series (s = pi^2 r^2)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    r2 = x * x + y * y
    s = math.pi**2 * r2
    # cos(2 theta) e^{-s}(1 + s - e^{s}) / (2 pi r^2)
    #   = (x^2 - y^2)/r^2 * (e^{-s}(1+s) - 1) / (2 pi r^2)
    #   = (x^2 - y^2) * f2(s) * s^2 / (2 pi r^4)
    #   = (x^2 - y^2) * f2(s) * pi^3 / 2                [s^2 = pi^4 r^4]
    aniso = (x * x - y * y) * _f2(s) * math.pi**3 / 2.0
    return -(0.5 * math.pi * np.exp(-s) + aniso)


def arkadiev_density(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """rho = 4 / ((x+1)^2 + y^2 + 1)^2 (Example 2, Sec. 3.1)."""
    d = (x + 1.0) ** 2 + y * y + 1.0
    return 4.0 / (d * d)


def arkadiev_potential(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Phi = -2 (y^2 - (x+1)^2 + 1) / ((x+1)^2 + y^2 + 1)^2 (Example 2)."""
    d = (x + 1.0) ** 2 + y * y + 1.0
    return -2.0 * (y * y - (x + 1.0) ** 2 + 1.0) / (d * d)
