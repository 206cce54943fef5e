"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test compares the oracle with something other than itself: the paper's
printed tables (tests/golden/), closed-form potentials (Examples 1 and 2 of
Sec. 3.1 and the Gaussian-partition closed form of I2), exactness of the
Gauss-Legendre rule, and operator identities (symmetry, linearity, the
x<->y transposition identity cos^2 + sin^2 = 1, reflection parity).
"""

import math

import numpy as np
import pytest

import oracle as O
from oracle import OracleParams
from conftest import read_golden
import synth


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _grid(n, L):
    x = O.grid_axis(n, L)
    return np.meshgrid(x, x)


def _split_params(n, L, h):
    """Split-solver parameters used for the paper's examples: sigma L = 12,
    P = 6 sigma (p(P) = e^-36), P below the grid's Nyquist, 64 x 128 nodes."""
    sig = 12.0 / L
    P = min(6.0 * sig, 0.9 * math.pi / h)
    return OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=P, sigma=P / 6.0,
                        n_r=64, n_theta=128)


def _matches_printed(value, printed, rel):
    return abs(value / printed - 1.0) <= rel


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("rule", ["legendre", "jacobi"])
def test_gaussian_closed_form_resolved(rule):
    """rho = exp(-r^2) on [-16,16)^2, N = 128, P = 4, sigma = 2/3 with a
    resolved polar rule (either radial rule): Phi matches the closed form to
    rounding."""
    p = OracleParams(nx=128, ny=128, lx=16, ly=16, cut_radius=4.0, sigma=2 / 3,
                     n_r=48, n_theta=96, radial=rule)
    X, Y = _grid(128, 16)
    phi, i1, i2 = O.solve(np.exp(-(X**2 + Y**2)), p, return_parts=True)
    ex = O.gaussian_potential(X, Y)
    i2ex = O.gaussian_i2_exact(X, Y, p.sigma_eff)
    assert rel_linf(phi, ex) < 1e-14
    # each half separately: I2 = Phi(x/l)/l^2, I1 = Phi - I2
    assert np.abs(i2 - i2ex).max() / np.abs(ex).max() < 1e-14
    assert np.abs(i1 - (ex - i2ex)).max() / np.abs(ex).max() < 1e-14


def test_gaussian_closed_form_config1_rule():
    """The 32 x 64 polar rule at P = 4 is quadrature-limited: ~3e-7."""
    p = OracleParams(nx=128, ny=128, lx=16, ly=16, cut_radius=4.0, sigma=2 / 3,
                     n_r=32, n_theta=64)
    X, Y = _grid(128, 16)
    phi = O.solve(np.exp(-(X**2 + Y**2)), p)
    err = rel_linf(phi, O.gaussian_potential(X, Y))
    assert 1e-8 < err < 1e-6


def test_paper_gaussian_is_scaled_unit_gaussian():
    """Example 1's printed potential equals pi Phi_1(pi x) (scale covariance of
    a degree-0 multiplier), including the small-r series region."""
    x = np.linspace(-3, 3, 241)
    X, Y = np.meshgrid(x, x + 1e-3)
    a = O.paper_gaussian_potential(X, Y)
    b = math.pi * O.gaussian_potential(math.pi * X, math.pi * Y)
    assert np.abs(a - b).max() < 1e-14
    assert abs(O.gaussian_potential(np.array([0.0]), np.array([0.0]))[0] + 0.5) < 1e-16


def test_closed_forms_solve_the_pde():
    """-Lap Phi = d_xx rho (eq. DSII_exact_pot) for both printed closed forms,
    checked symbolically."""
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y", real=True)
    r2 = x**2 + y**2
    rho_g = sp.exp(-r2)
    phi_g = -sp.Rational(1, 2) * (sp.exp(-r2) + (x**2 - y**2) * (sp.exp(-r2) * (1 + r2) - 1) / r2**2)
    res = -(sp.diff(phi_g, x, 2) + sp.diff(phi_g, y, 2)) - sp.diff(rho_g, x, 2)
    for pt in [(3, 7), (11, -4), (-20, 5)]:
        val = res.subs({x: sp.Rational(pt[0], 10), y: sp.Rational(pt[1], 10)}).evalf(40)
        assert abs(float(val)) < 1e-30
    d = (x + 1) ** 2 + y**2 + 1
    rho_a = 4 / d**2
    phi_a = -2 * (y**2 - (x + 1) ** 2 + 1) / d**2
    res_a = sp.simplify(-(sp.diff(phi_a, x, 2) + sp.diff(phi_a, y, 2)) - sp.diff(rho_a, x, 2))
    assert res_a == 0
    # the numeric closed forms agree with the symbolic ones
    fa = sp.lambdify((x, y), phi_a, "numpy")
    fg = sp.lambdify((x, y), phi_g, "numpy")
    pts = np.array([[0.3, 0.7], [1.1, -0.4], [-2.0, 0.5], [3.0, 3.0]])
    assert np.allclose(O.arkadiev_potential(pts[:, 0], pts[:, 1]), fa(pts[:, 0], pts[:, 1]), rtol=1e-14)
    assert np.allclose(O.gaussian_potential(pts[:, 0], pts[:, 1]), fg(pts[:, 0], pts[:, 1]), rtol=1e-12)


# ---------------------------------------------------------------- paper tables

@pytest.mark.parametrize("L,h,printed", read_golden("table1_std_fft_gaussian.txt"))
def test_table1_standard_fft(L, h, printed):
    n = int(round(2 * L / h))
    X, Y = _grid(n, L)
    phi = O.standard_fft_solve(O.paper_gaussian_density(X, Y), L, L)
    err = rel_linf(phi, O.paper_gaussian_potential(X, Y))
    assert _matches_printed(err, printed, 0.005), err


@pytest.mark.parametrize("L,h,printed", read_golden("table2_nufft_gaussian.txt"))
def test_table2_split_solver(L, h, printed):
    n = int(round(2 * L / h))
    X, Y = _grid(n, L)
    phi = O.solve(O.paper_gaussian_density(X, Y), _split_params(n, L, h))
    err = rel_linf(phi, O.paper_gaussian_potential(X, Y))
    if h < 0.1:
        assert err <= printed  # the paper's NUFFT tolerance floor
    else:
        assert _matches_printed(err, printed, 0.01), err


@pytest.mark.parametrize("L,h,printed", read_golden("table4_std_fft_arkadiev.txt"))
def test_table4_standard_fft_arkadiev(L, h, printed):
    n = int(round(2 * L / h))
    X, Y = _grid(n, L)
    phi = O.standard_fft_solve(O.arkadiev_density(X, Y), L, L)
    err = rel_linf(phi, O.arkadiev_potential(X, Y))
    assert _matches_printed(err, printed, 0.005), err


@pytest.mark.parametrize("L,h,printed", read_golden("table5_nufft_arkadiev.txt"))
def test_table5_split_solver_arkadiev(L, h, printed):
    n = int(round(2 * L / h))
    X, Y = _grid(n, L)
    phi = O.solve(O.arkadiev_density(X, Y), _split_params(n, L, h))
    err = rel_linf(phi, O.arkadiev_potential(X, Y))
    assert _matches_printed(err, printed, 0.01), err


# ---------------------------------------------------------------- quadrature

@pytest.mark.parametrize("rule,extra", [("legendre", 0), ("jacobi", 1)])
@pytest.mark.parametrize("n_r", [1, 7, 32, 64])
def test_radial_rule_exact_for_polynomials(n_r, rule, extra):
    """The radial weights W integrate f(r) r dr on [0, P]: exactly for
    f = r^k with k <= 2 n_r - 2 (Gauss-Legendre times r) and k <= 2 n_r - 1
    (Gauss-Jacobi, whose weight function is r itself)."""
    P = 3.7
    p = OracleParams(nx=8, ny=8, lx=1, ly=1, cut_radius=P, n_r=n_r, n_theta=4, radial=rule)
    r, w = O.radial_rule(p)
    for k in range(0, 2 * n_r - 1 + extra):
        exact = P ** (k + 2) / (k + 2)
        assert abs(np.sum(w * r**k) / exact - 1.0) < 1e-13, k
    assert np.all((r > 0) & (r < P)) and np.all(np.diff(r) > 0)
    if n_r <= 7:  # one degree more is not integrated exactly (not over-specified)
        k = 2 * n_r - 1 + extra
        assert abs(np.sum(w * r**k) / (P ** (k + 2) / (k + 2)) - 1.0) > 1e-8


def test_angular_rule_and_weights():
    """Trapezoid on the circle: sum of D over the disk equals
    -(2 pi)^-2 int_0^P r p(r) dr int cos^2 = -(2 pi)^-2 pi sigma^2/2 (1 - e^{-P^2/s^2})."""
    P, s = 5.0, 1.3
    p = OracleParams(nx=8, ny=8, lx=1, ly=1, cut_radius=P, sigma=s, n_r=40, n_theta=64)
    D = O.polar_weights(p)
    exact = -(1.0 / (2 * math.pi) ** 2) * math.pi * (s * s / 2.0) * (1.0 - math.exp(-P * P / (s * s)))
    assert abs(D.sum() / exact - 1.0) < 1e-13
    kx, ky, *_ = O.polar_nodes(p)
    # node set symmetric under k -> -k (N_theta even)
    d2 = (kx[:, None] + kx[None, :]) ** 2 + (ky[:, None] + ky[None, :]) ** 2
    assert d2.min(axis=1).max() < 1e-24


# ---------------------------------------------------------------- operator identities

def _small_params(n=32, L=8.0):
    return OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=4.0, sigma=2 / 3, n_r=24, n_theta=48)


def test_symmetry_and_adjoint():
    """<g, A rho> = <A g, rho>, and the written-out transpose equals A."""
    p = _small_params()
    g = np.random.Generator(np.random.PCG64(11))
    rho = g.standard_normal((32, 32))
    w = g.standard_normal((32, 32))
    a_rho = O.solve(rho, p)
    a_w = O.solve(w, p)
    lhs = float(np.sum(w * a_rho))
    rhs = float(np.sum(a_w * rho))
    assert abs(lhs - rhs) < 1e-13 * max(abs(lhs), 1.0) * 32
    at_w = O.solve_adjoint(w, p)
    assert np.abs(at_w - a_w).max() < 1e-13 * np.abs(a_w).max()


def test_linearity():
    p = _small_params()
    g = np.random.Generator(np.random.PCG64(12))
    a, b = g.standard_normal((2, 32, 32))
    lhs = O.solve(2.5 * a - 0.75 * b, p)
    rhs = 2.5 * O.solve(a, p) - 0.75 * O.solve(b, p)
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max()


def test_transpose_identity():
    """Phi[rho] + (Phi[rho^T])^T = -rho (cos^2 + sin^2 = 1; N_theta % 4 == 0),
    to discretisation accuracy for a decayed density."""
    n, L = 128, 16.0
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=4.0, sigma=2 / 3, n_r=48, n_theta=96)
    rho = synth.density_sum(n, n, L, L, seed=7, count=4)
    rho_t = np.ascontiguousarray(rho.T)
    lhs = O.solve(rho, p) + O.solve(rho_t, p).T
    assert np.abs(lhs + rho).max() < 1e-11 * np.abs(rho).max()


def test_reflection_parity():
    """Reflecting rho in x (index n -> (N - n) mod N, with rho = 0 on the first
    row and column) reflects Phi exactly, for I1 and I2 alike."""
    n, L = 64, 8.0
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=4.0, sigma=2 / 3, n_r=32, n_theta=64)
    rho = synth.density_sum(n, n, L, L, seed=3, count=3)
    rho[:, 0] = 0.0
    rho[0, :] = 0.0
    idx = (-np.arange(n)) % n
    phi = O.solve(rho, p)
    # x_0 = -L has no mirror point on the periodic grid: compare n = 1..N-1
    phi_r = O.solve(rho[:, idx], p)
    assert np.abs(phi_r - phi[:, idx])[:, 1:].max() < 1e-13 * np.abs(phi).max()
    phi_ry = O.solve(rho[idx, :], p)
    assert np.abs(phi_ry - phi[idx, :])[1:, :].max() < 1e-13 * np.abs(phi).max()


def test_subsample_outputs_match_full():
    p = _small_params()
    rho = synth.density_sum(32, 32, 8.0, 8.0, seed=5, count=3)
    full = O.solve(rho, p)
    rows, cols = np.arange(1, 32, 3), np.arange(0, 32, 5)
    sub = O.solve(rho, p, rows=rows, cols=cols)
    assert np.abs(sub - full[np.ix_(rows, cols)]).max() < 1e-15 * 32 * np.abs(full).max()


def test_rectangular_grid_closed_form():
    """nx != ny, lx != ly, hx != hy: still the closed form."""
    p = OracleParams(nx=128, ny=64, lx=16.0, ly=8.0, cut_radius=4.0, sigma=2 / 3,
                     n_r=48, n_theta=96)
    x = O.grid_axis(128, 16.0)
    y = O.grid_axis(64, 8.0)
    X, Y = np.meshgrid(x, y)
    phi = O.solve(np.exp(-(X**2 + Y**2)), p)
    assert rel_linf(phi, O.gaussian_potential(X, Y)) < 1e-13


def test_sharp_partition_with_a_decayed_tail_reduces_to_the_polar_quadrature():
    """Sharp split (p = 1 on |k| <= P) for rho = exp(-r^2), whose transform
    pi exp(-|k|^2/4) integrates to e^{-P^2/4} (= 1.4e-11 at P = 10) outside the
    disk: I1 then vanishes to that level, and I2 alone, with the polar rule
    resolved (n_theta > P R, R the half-diagonal), carries the closed form."""
    n, L = 128, 16.0
    X, Y = _grid(n, L)
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=10.0, n_r=120, n_theta=244, partition="sharp")
    phi, i1, i2 = O.solve(np.exp(-(X**2 + Y**2)), p, return_parts=True)
    ex = O.gaussian_potential(X, Y)
    scale = np.abs(ex).max()
    assert np.abs(i1).max() / scale < 5e-11
    assert np.abs(i2 - ex).max() / scale < 5e-11
    assert rel_linf(phi, ex) < 1e-12


def _naive_dft2(x, sign):
    """Literal 2D DFT: X[k, l] = sum_m sum_n x[m, n] e^{sign 2 pi i (k m / M_y + l n / M_x)}."""
    my, mx = x.shape
    out = np.zeros((my, mx), dtype=np.complex128)
    for k in range(my):
        for l in range(mx):
            acc = 0j
            for m in range(my):
                for n in range(mx):
                    acc += x[m, n] * complex(math.cos(sign * 2 * math.pi * (k * m / my + l * n / mx)),
                                             math.sin(sign * 2 * math.pi * (k * m / my + l * n / mx)))
            out[k, l] = acc
    return out


@pytest.mark.parametrize("nx,ny", [(16, 16), (16, 8)])
def test_i1_against_a_literal_dft_on_small_grids(nx, ny):
    """I1 (eq. SubInt1) with its padded FFT replaced by the literal double sum of
    the DFT definition (kappa = 2: a 32 x 32 or 16 x 32 sum), written here
    without the oracle's FFT library or frequency helpers: the angular
    frequency of index q on M points of spacing h is 2 pi qbar / (M h), qbar
    the signed index."""
    lx, ly, P = 4.0, 2.0 * ny / nx * 2.0, 2.5
    rho = synth.density_sum(nx, ny, lx, ly, seed=21, count=3)
    p = OracleParams(nx=nx, ny=ny, lx=lx, ly=ly, cut_radius=P, n_r=8, n_theta=16)
    my, mx = 2 * ny, 2 * nx
    pad = np.zeros((my, mx))
    pad[:ny, :nx] = rho
    R = _naive_dft2(pad, -1.0)
    hx, hy = 2 * lx / nx, 2 * ly / ny
    sig2 = (P / 6.0) ** 2
    for k in range(my):
        for l in range(mx):
            kb = k if k < my // 2 else k - my
            lb = l if l < mx // 2 else l - mx
            wy, wx = 2 * math.pi * kb / (my * hy), 2 * math.pi * lb / (mx * hx)
            s = wx * wx + wy * wy
            R[k, l] *= 0.0 if s == 0 else -(wx * wx / s) * (1.0 - math.exp(-s / sig2))
    back = _naive_dft2(R, +1.0) / (mx * my)
    want = back[:ny, :nx].real
    got = O.i1_padded_fft(rho, p)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    assert np.abs(back[:ny, :nx].imag).max() <= 1e-13 * np.abs(want).max()
