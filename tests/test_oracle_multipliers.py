"""Pins of the oracle for multipliers other than the DS one (the Remark of
Sec. 2.2: the split applies to any multiplier known analytically), in the
family |k|^alpha (a0 + ac cos 2theta + as sin 2theta)."""

import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special

import oracle as O
from oracle import OracleParams


def _grid(n, L):
    x = O.grid_axis(n, L)
    return np.meshgrid(x, x)


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("a0,ac,as_", [(0.0, 0.0, -0.5), (0.3, 0.7, -0.2), (-0.5, -0.5, 0.0)])
def test_alpha0_family_matches_the_rotated_closed_form(a0, ac, as_):
    """Degree-0 multipliers: Phi = a0 rho + (ac cos 2phi + as sin 2phi) f(r) for
    rho = exp(-r^2); the (-1/2, -1/2, 0) case is the DS closed form itself."""
    n, L = 128, 16.0
    X, Y = _grid(n, L)
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=4.0, sigma=2 / 3, n_r=48, n_theta=96,
                     multiplier=(0, a0, ac, as_))
    phi = O.solve(np.exp(-(X * X + Y * Y)), p)
    assert _rel(phi, O.gaussian_potential_alpha0(X, Y, a0, ac, as_)) < 1e-14
    if (a0, ac, as_) == (-0.5, -0.5, 0.0):
        assert _rel(O.gaussian_potential_alpha0(X, Y, a0, ac, as_), O.gaussian_potential(X, Y)) < 1e-15


@pytest.mark.parametrize("x,y", [(0.0, 0.0), (0.7, -0.3), (2.5, 1.0), (6.0, 0.0)])
def test_coulomb_closed_form_by_real_space_quadrature(x, y):
    """pi^{3/2} e^{-r^2/2} I0(r^2/2) = int exp(-|z|^2)/|x - z| dz, the integral
    taken in polar coordinates around x (the 1/|x - z| cancels the Jacobian)."""
    f = lambda t, rho: math.exp(-((x + rho * math.cos(t)) ** 2 + (y + rho * math.sin(t)) ** 2))
    val, _ = scipy.integrate.dblquad(f, 0.0, 30.0, 0.0, 2 * math.pi, epsabs=1e-13, epsrel=1e-12)
    assert abs(O.gaussian_coulomb(np.array(x), np.array(y)) / val - 1.0) < 1e-10


@pytest.mark.parametrize("r", [0.0, 0.4, 1.3, 3.0])
def test_abs_k_closed_form_by_hankel_quadrature(r):
    """sqrt(pi) e^{-r^2/2} [(1 - r^2) I0 + r^2 I1](r^2/2) = 1/2 int k^2 e^{-k^2/4} J0(k r) dk."""
    val, _ = scipy.integrate.quad(lambda k: 0.5 * k * k * math.exp(-k * k / 4) * scipy.special.j0(k * r),
                                  0.0, 40.0, limit=400, epsabs=1e-14, epsrel=1e-13)
    assert abs(float(O.gaussian_abs_k(np.array(r), np.array(0.0))) - val) < 1e-11


def test_coulomb_split_halves():
    """m = 2 pi/|k| (the 2D transform of 1/|x|), sigma fixed: I2 alone equals
    its closed form Phi_C(x/l)/l (l^2 = 1 + 4/sigma^2) to rounding; I1 carries
    the trapezoid error of the kink of m (1 - p) ~ 2 pi |k|/sigma^2 at k = 0,
    third order in dk (a factor 8 per halving of dk)."""
    sig, mult = 0.75, (-1, 2 * math.pi, 0.0, 0.0)
    l = math.sqrt(1.0 + 4.0 / sig ** 2)
    errs = []
    for L, n in ((16.0, 128), (32.0, 256)):
        X, Y = _grid(n, L)
        p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=6 * sig, sigma=sig, n_r=64, n_theta=192,
                         multiplier=mult)
        phi, i1, i2 = O.solve(np.exp(-(X * X + Y * Y)), p, return_parts=True)
        ex = O.gaussian_coulomb(X, Y)
        i2ex = O.gaussian_coulomb(X / l, Y / l) / l
        if L == 16.0:
            assert np.abs(i2 - i2ex).max() / np.abs(ex).max() < 1e-14
        errs.append(np.abs(i1 - (ex - i2ex)).max() / np.abs(ex).max())
        assert _rel(phi, ex) < 5e-5
    assert 7.0 < errs[0] / errs[1] < 9.0, errs


def test_abs_k_multiplier_closed_form():
    """m = |k| (the half Laplacian (-Delta)^{1/2}): m (1 - p) ~ |k|^3 at k = 0."""
    n, L = 128, 16.0
    X, Y = _grid(n, L)
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=4.0, sigma=2 / 3, n_r=48, n_theta=96,
                     multiplier=(1, 1.0, 0.0, 0.0))
    assert _rel(O.solve(np.exp(-(X * X + Y * Y)), p), O.gaussian_abs_k(X, Y)) < 1e-7


def test_generic_operator_is_symmetric():
    """<g, A rho> = <A g, rho> for a multiplier with all three angular terms."""
    n, L = 32, 8.0
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=3.0, sigma=0.5, n_r=16, n_theta=32,
                     multiplier=(-1, 1.3, 0.4, -0.7))
    lhs = float(np.sum(b * O.solve(a, p)))
    rhs = float(np.sum(O.solve(b, p) * a))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert _rel(O.solve_adjoint(a, p), O.solve(a, p)) < 1e-12


def test_nyquist_alias_average_keeps_the_multiplier_even():
    """With the sin 2theta term averaged over the +-K aliases of the Nyquist row
    and column, m(-k) = m(k) on the whole discrete grid, so the full complex
    inverse transform of m (1 - p) rho_hat of a real density is real (the
    reading that fixes the otherwise ambiguous Nyquist value)."""
    import oracle.potential as OP

    n, L = 32, 8.0
    rho = np.random.default_rng(5).standard_normal((n, n))
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=3.0, sigma=0.5, n_r=8, n_theta=16,
                     multiplier=(0, 0.3, 0.7, -0.2))
    buf = np.zeros((2 * n, 2 * n))
    buf[:n, :n] = rho
    wx = OP._omega_axis(2 * n, p.hx)[None, :]
    wy = OP._omega_axis(2 * n, p.hy)[:, None]
    out = np.fft.ifft2(np.fft.fft2(buf) * O.multiplier_high(wx, wy, p))
    assert np.abs(out.imag).max() <= 1e-15 * np.abs(out.real).max()
