"""Plain FP64 CPU oracle of the split nonlocal potential solver.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Mauser, Stimming, Zhang, "A novel nonlocal potential solver based on
nonuniform FFT for efficient simulation of the Davey-Stewartson equations",
Sec. 2.1 (the split solver) and Sec. 2.2 (type-1 / type-2 sums).

Conventions (each one is a reading of the paper; all are pinned by tests):

* Grid (Sec. 2.1 and Sec. 3): x_n = -L + n h, n = 0..N-1, h = 2L/N, periodic
  N points per axis.  Arrays are row-major ``[ny][nx]`` (x fastest).
* Angular frequencies throughout: rho_hat(w) = int rho(x) e^{-i w.x} dx and
  Phi = (2 pi)^-2 int m(w) rho_hat(w) e^{i w.x} dw with m = -w_x^2/|w|^2
  (eqs. Def_Fourier / FourTransDef with k = w / (2 pi); Phi itself does not
  depend on the convention because m is homogeneous of degree 0).
* Partition p(w) = exp(-|w|^2 / sigma^2) (Sec. 2.1, after eq. SubInt2).
  ``partition="sharp"`` is the indicator of the disk |w| <= P;
  ``partition="none"`` is p = 0 (the standard periodic FFT solver of Sec. 2.1
  / Table 1, used with pad=1).
* I1 (eq. SubInt1): trapezoid rule on the padded square, i.e. an FFT of the
  zero-padded density on the kappa N grid, multiplication by
  m1 = (1 - p) m with m1(0) = 0, inverse FFT, restriction to the physical
  N x N points.
* I2 (eq. I2PolarDisc): radial Gauss-Legendre nodes on [0, P] (the Jacobian r
  folded into the weight), or the Gauss-Jacobi rule whose weight function is
  that Jacobian (Sec. 2.1), times the uniform angular rule theta_j = 2 pi j /
  N_theta; weights D = -(2 pi)^-2 W_r (2 pi / N_theta) cos^2(theta) p(r).
  rho_hat at the nodes is the trapezoid sum h_x h_y sum_n rho_n e^{-i k.x_n}
  (the exact sum that a type-2 NUFFT approximates, eq. 2.2); I2 is
  Re sum_j D_j rho_hat_j e^{+i k_j.x_n} (the exact sum a type-1 NUFFT
  approximates, eq. 2.1).  Both sums are evaluated directly; the only
  library primitives are FFTs (I1), a Gauss-Legendre table and dense matrix
  products that evaluate the nested sums over x and y.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.special
import scipy.fft as sfft

TWO_PI = 2.0 * math.pi


@dataclasses.dataclass(frozen=True)
class OracleParams:
    """Parameters of one solve.  ``cut_radius`` is the disk radius P of Sec.
    2.1 ("c" there) in angular frequency; ``sigma`` = 0 selects P/6."""

    nx: int
    ny: int
    lx: float
    ly: float
    cut_radius: float
    n_r: int
    n_theta: int
    sigma: float = 0.0
    pad: int = 2
    partition: str = "gauss"
    radial: str = "legendre"  # "legendre" (Jacobian r in the weight) or "jacobi" (weight (1+t), Sec. 2.1)
    # Fourier multiplier m(k) = |k|^alpha (a0 + ac cos 2theta + as sin 2theta), theta = arg k, as
    # (alpha, a0, ac, as); the default (0, -1/2, -1/2, 0) is -cos^2 theta = -k_x^2/|k|^2 (eq. Disct_Fourier)
    multiplier: tuple = (0, -0.5, -0.5, 0.0)

    @property
    def hx(self) -> float:
        return 2.0 * self.lx / self.nx

    @property
    def hy(self) -> float:
        return 2.0 * self.ly / self.ny

    @property
    def sigma_eff(self) -> float:
        return self.sigma if self.sigma > 0 else self.cut_radius / 6.0


def grid_axis(n: int, half_width: float) -> np.ndarray:
    """x_n = -L + n h, n = 0..N-1, h = 2L/N (Sec. 2.1; Sec. 3 grid)."""
    h = 2.0 * half_width / n
    return -half_width + h * np.arange(n, dtype=np.float64)


def partition(w2: np.ndarray, p: OracleParams) -> np.ndarray:
    """p(w) of Sec. 2.1 evaluated at |w|^2 = w2."""
    if p.partition == "gauss":
        return np.exp(-w2 / p.sigma_eff**2)
    if p.partition == "sharp":
        return (w2 <= p.cut_radius**2).astype(np.float64)
    if p.partition == "none":
        return np.zeros_like(w2)
    raise ValueError(f"unknown partition {p.partition!r}")


DS_MULTIPLIER = (0, -0.5, -0.5, 0.0)


def multiplier(wx: np.ndarray, wy: np.ndarray, p: OracleParams) -> np.ndarray:
    """m(w) with m(0) = 0 (the rho_hat(0) = 0 convention of Sec. 2.1).  The DS
    multiplier is -w_x^2/|w|^2 (eq. Disct_Fourier); the Remark of Sec. 2.2
    applies the method to any multiplier known analytically, here
    |w|^alpha (a0 + ac cos 2theta + as sin 2theta) with
    cos 2theta = (w_x^2 - w_y^2)/|w|^2 and sin 2theta = 2 w_x w_y/|w|^2."""
    w2 = wx * wx + wy * wy
    with np.errstate(divide="ignore", invalid="ignore"):
        if tuple(p.multiplier) == DS_MULTIPLIER:
            m = -(wx * wx) / w2
        else:
            alpha, a0, ac, as_ = p.multiplier
            # the Nyquist frequency of an axis stands for both +K and -K: the
            # odd sin 2theta term is averaged over the aliases, i.e. dropped there
            nyq = np.isclose(np.abs(wx), math.pi / p.hx, rtol=1e-12, atol=0.0) | \
                np.isclose(np.abs(wy), math.pi / p.hy, rtol=1e-12, atol=0.0)
            odd = np.where(nyq, 0.0, as_ * 2.0 * wx * wy)
            ang = a0 + (ac * (wx * wx - wy * wy) + odd) / w2
            m = np.power(w2, 0.5 * alpha) * ang
        return np.where(w2 > 0, m, 0.0)


def multiplier_high(wx: np.ndarray, wy: np.ndarray, p: OracleParams) -> np.ndarray:
    """m1 = m (1 - p(w)) (eq. SubInt1), m1(0) = 0."""
    w2 = wx * wx + wy * wy
    return multiplier(wx, wy, p) * (1.0 - partition(w2, p))


def _omega_axis(m_pts: int, h: float) -> np.ndarray:
    """Angular frequencies of an m_pts-point FFT on spacing h: 2 pi q / (m h),
    q in [-m/2, m/2) in FFT order."""
    return TWO_PI * np.fft.fftfreq(m_pts, d=h)


def i1_padded_fft(rho: np.ndarray, p: OracleParams) -> np.ndarray:
    """I1 of eq. SubInt1 by the padded trapezoid rule (Sec. 2.1).

    rho is zero-padded to the (pad*ny, pad*nx) grid (indices >= N are zero),
    transformed, multiplied by m1 and transformed back; the physical N x N
    block is returned."""
    ny, nx = rho.shape
    my, mx = p.pad * ny, p.pad * nx
    buf = np.zeros((my, mx), dtype=np.float64)
    buf[:ny, :nx] = rho
    spec = sfft.fft2(buf, workers=-1)
    del buf
    wx = _omega_axis(mx, p.hx)[None, :]
    wy = _omega_axis(my, p.hy)[:, None]
    spec *= multiplier_high(wx, wy, p)
    out = sfft.ifft2(spec, workers=-1)
    return np.ascontiguousarray(out[:ny, :nx].real)


def i1_padded_fft_adjoint(g: np.ndarray, p: OracleParams) -> np.ndarray:
    """Transpose of ``i1_padded_fft`` written out: restrict^T = pad,
    ifft^T, m1, fft^T, pad^T = restrict (the matrix of I1 is
    K[n, n'] = M^-2 sum_q m1(q) e^{2 pi i q (n - n')/M})."""
    ny, nx = g.shape
    my, mx = p.pad * ny, p.pad * nx
    buf = np.zeros((my, mx), dtype=np.float64)
    buf[:ny, :nx] = g
    spec = sfft.ifft2(buf, workers=-1)
    del buf
    wx = _omega_axis(mx, p.hx)[None, :]
    wy = _omega_axis(my, p.hy)[:, None]
    spec *= multiplier_high(wx, wy, p)
    out = sfft.fft2(spec, workers=-1)
    return np.ascontiguousarray(out[:ny, :nx].real)


def radial_rule(p: OracleParams):
    """Nodes r_i in (0, P) and weights W_i with sum_i W_i f(r_i) ~ int_0^P f(r) r dr.

    "legendre": Gauss-Legendre on [0, P] (numpy's table mapped affinely) with
    the Jacobian r multiplied into the weight.  "jacobi": the Gauss-Jacobi rule
    the paper names (Sec. 2.1) for the weight (1 - t)^0 (1 + t)^1 on [-1, 1]
    (scipy's table), which is the Jacobian itself: with r = P (1 + t)/2,
    r dr = (P/2)^2 (1 + t) dt."""
    if p.radial == "legendre":
        t, v = np.polynomial.legendre.leggauss(p.n_r)
        r = 0.5 * p.cut_radius * (t + 1.0)
        return r, r * (0.5 * p.cut_radius * v)
    if p.radial == "jacobi":
        t, v = scipy.special.roots_jacobi(p.n_r, 0.0, 1.0)
        return 0.5 * p.cut_radius * (t + 1.0), (0.5 * p.cut_radius) ** 2 * v
    raise ValueError(f"unknown radial rule {p.radial!r}")


def polar_nodes(p: OracleParams):
    """Polar quadrature nodes of eq. I2PolarDisc.

    Radial: ``radial_rule`` (weights for int f(r) r dr).  Angular: theta_j =
    2 pi j / N_theta with weight 2 pi / N_theta (trapezoid rule on the circle).
    Node order: radial index major, angular index minor.
    Returns (kx, ky, r, W_r, theta)."""
    r, w_rad = radial_rule(p)
    theta = TWO_PI * np.arange(p.n_theta, dtype=np.float64) / p.n_theta
    kx = (r[:, None] * np.cos(theta)[None, :]).ravel()
    ky = (r[:, None] * np.sin(theta)[None, :]).ravel()
    return kx, ky, r, w_rad, theta


def polar_weights(p: OracleParams) -> np.ndarray:
    """D_j = -(2 pi)^-2 W_r (2 pi/N_theta) cos^2(theta) p(r): the weights of
    eq. I2PolarDisc with the Jacobian r (inside W_r) and the (2 pi)^-2 of the
    angular frequency convention written in.  For another multiplier
    r^alpha (a0 + ac cos 2theta + as sin 2theta) replaces -cos^2(theta)."""
    _, _, r, w_rad, theta = polar_nodes(p)
    w_theta = TWO_PI / p.n_theta
    if tuple(p.multiplier) == DS_MULTIPLIER:
        radial = w_rad * partition(r * r, p)
        ang = -np.cos(theta) ** 2 * w_theta
    else:
        alpha, a0, ac, as_ = p.multiplier
        radial = w_rad * np.power(r, float(alpha)) * partition(r * r, p)
        ang = (a0 + ac * np.cos(2.0 * theta) + as_ * np.sin(2.0 * theta)) * w_theta
    return ((radial[:, None] * ang[None, :]) / TWO_PI**2).ravel()


def _node_chunks(n_nodes: int, width: int, chunk: int):
    step = max(1, chunk // max(1, width))
    for s in range(0, n_nodes, step):
        yield slice(s, min(n_nodes, s + step))


def rho_hat_direct(f: np.ndarray, x: np.ndarray, y: np.ndarray,
                   kx: np.ndarray, ky: np.ndarray, sign: float = -1.0,
                   chunk: int = 1 << 24) -> np.ndarray:
    """h_x h_y sum_n f_n exp(sign * i k_j.x_n) for every node j.

    With sign = -1 this is the trapezoid rule for rho_hat(k_j) (eq.
    FourTransDef discretised as in Sec. 2.1), i.e. the exact value of the
    type-2 sum eq. 2.2.  The double sum over (y, x) is written as the inner
    sum over x (a dense matrix product) followed by the sum over y."""
    ny, nx = f.shape
    hx = x[1] - x[0]
    hy = y[1] - y[0]
    out = np.empty(kx.size, dtype=np.complex128)
    for sl in _node_chunks(kx.size, max(nx, ny), chunk):
        ax = np.outer(kx[sl], x)                       # (J, nx)
        inner_c = f @ np.cos(ax).T                     # (ny, J)
        inner_s = f @ np.sin(ax).T
        inner = inner_c + (sign * 1j) * inner_s        # sum_x f e^{sign i kx x}
        ay = np.outer(ky[sl], y)                       # (J, ny)
        ey = np.exp((sign * 1j) * ay)                  # (J, ny)
        out[sl] = np.einsum("jy,yj->j", ey, inner)
    return out * (hx * hy)


def i2_direct_from_coeffs(c: np.ndarray, kx: np.ndarray, ky: np.ndarray,
                          x: np.ndarray, y: np.ndarray, sign: float = 1.0,
                          chunk: int = 1 << 24) -> np.ndarray:
    """Re sum_j c_j exp(sign * i k_j.x) on the tensor grid (y, x): the exact
    value of the type-1 sum eq. 2.1 (real part).  Returns [len(y)][len(x)]."""
    out = np.zeros((y.size, x.size), dtype=np.float64)
    for sl in _node_chunks(kx.size, max(x.size, y.size), chunk):
        ey = np.exp((sign * 1j) * np.outer(y, ky[sl])) * c[sl][None, :]  # (ny, J)
        ex = np.exp((sign * 1j) * np.outer(kx[sl], x))                  # (J, nx)
        out += ey.real @ ex.real - ey.imag @ ex.imag
    return out


def _axes(p: OracleParams):
    return grid_axis(p.nx, p.lx), grid_axis(p.ny, p.ly)


def i2_direct(rho: np.ndarray, p: OracleParams, rows=None, cols=None) -> np.ndarray:
    """I2 of eq. I2PolarDisc with both nonuniform sums evaluated directly.
    ``rows`` / ``cols`` select output grid indices (default: all)."""
    x, y = _axes(p)
    kx, ky, *_ = polar_nodes(p)
    rh = rho_hat_direct(rho, x, y, kx, ky, sign=-1.0)
    c = polar_weights(p) * rh
    xo = x if cols is None else x[np.asarray(cols)]
    yo = y if rows is None else y[np.asarray(rows)]
    return i2_direct_from_coeffs(c, kx, ky, xo, yo, sign=1.0)


def solve(rho: np.ndarray, p: OracleParams, rows=None, cols=None,
          return_parts: bool = False):
    """Phi = I1 + I2 (eq. PotSplitWhoSpace), FP64.  ``rows``/``cols`` select
    a sub-grid of outputs (I1 is still computed on the whole grid)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    if rho.shape != (p.ny, p.nx):
        raise ValueError("rho must have shape (ny, nx)")
    i1 = i1_padded_fft(rho, p)
    if rows is not None:
        i1 = i1[np.asarray(rows), :]
    if cols is not None:
        i1 = i1[:, np.asarray(cols)]
    i2 = i2_direct(rho, p, rows=rows, cols=cols)
    if return_parts:
        return i1 + i2, i1, i2
    return i1 + i2


def solve_adjoint(g: np.ndarray, p: OracleParams) -> np.ndarray:
    """Transpose of ``solve`` written out term by term: I1^T (see
    ``i1_padded_fft_adjoint``) plus I2^T g = Re sum_j D_j g_hat_j
    e^{-i k_j.x_n} with g_hat_j = h^2 sum_n g_n e^{+i k_j.x_n}."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    x, y = _axes(p)
    kx, ky, *_ = polar_nodes(p)
    gh = rho_hat_direct(g, x, y, kx, ky, sign=+1.0)
    c = polar_weights(p) * gh
    i2t = i2_direct_from_coeffs(c, kx, ky, x, y, sign=-1.0)
    return i1_padded_fft_adjoint(g, p) + i2t


def standard_fft_solve(rho: np.ndarray, lx: float, ly: float, multiplier=DS_MULTIPLIER) -> np.ndarray:
    """The standard periodic FFT solver of Sec. 2.1 (no split, no padding,
    Phi_hat(0) = 0), i.e. I1 with p = 0 and kappa = 1.  Used for Table 1."""
    ny, nx = rho.shape
    p = OracleParams(nx=nx, ny=ny, lx=lx, ly=ly, cut_radius=1.0, n_r=1,
                     n_theta=4, pad=1, partition="none", multiplier=tuple(multiplier))
    return i1_padded_fft(rho, p)
