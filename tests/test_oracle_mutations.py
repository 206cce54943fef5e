"""Planted mistakes in the oracle (on the CPU) must trip at least one pin.

Each mutation monkeypatches one step of ``oracle.potential`` with a plausible
error (a dropped term, a wrong sign, a transposed operand, a shifted index)
and runs a small battery of the pins from ``test_oracle_pins``: the Gaussian
closed form, one Table 5 entry (Arkadiev, an off-centre density) and one
Table 1 entry.  The unmutated oracle passes the battery.
"""

import math

import numpy as np
import pytest

import oracle as O
import oracle.potential as OP
from oracle import OracleParams


def _battery():
    """True when every pin of the battery passes."""
    ok = True
    # Gaussian closed form, resolved polar rule
    p = OracleParams(nx=64, ny=64, lx=8, ly=8, cut_radius=4.0, sigma=2 / 3, n_r=48, n_theta=96)
    x = O.grid_axis(64, 8)
    X, Y = np.meshgrid(x, x)
    phi = O.solve(np.exp(-(X**2 + Y**2)), p)
    ex = O.gaussian_potential(X, Y)
    ok &= np.abs(phi - ex).max() / np.abs(ex).max() < 1e-12
    # Table 5, L = 16, h = 1/4: 4.28E-06
    L, h = 16.0, 0.25
    n = int(2 * L / h)
    x = O.grid_axis(n, L)
    X, Y = np.meshgrid(x, x)
    P = min(6 * 12 / L, 0.9 * math.pi / h)
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=P, sigma=P / 6, n_r=64, n_theta=128)
    phi = O.solve(O.arkadiev_density(X, Y), p)
    ex = O.arkadiev_potential(X, Y)
    ok &= abs((np.abs(phi - ex).max() / np.abs(ex).max()) / 4.28e-6 - 1) < 0.01
    # Table 1, L = 8, h = 1/4: 2.38E-03
    n = 64
    x = O.grid_axis(n, 8.0)
    X, Y = np.meshgrid(x, x)
    phi = O.standard_fft_solve(O.paper_gaussian_density(X, Y), 8.0, 8.0)
    ex = O.paper_gaussian_potential(X, Y)
    ok &= abs((np.abs(phi - ex).max() / np.abs(ex).max()) / 2.38e-3 - 1) < 0.005
    return bool(ok)


def test_unmutated_oracle_passes_battery():
    assert _battery()


def _mut_drop_one_minus_p(monkeypatch):
    def m1(wx, wy, p):
        w2 = wx * wx + wy * wy
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(w2 > 0, -(wx * wx) / w2, 0.0)
    monkeypatch.setattr(OP, "multiplier_high", m1)


def _mut_drop_jacobian(monkeypatch):
    orig = OP.polar_weights

    def w(p):
        _, _, r, _, _ = OP.polar_nodes(p)
        return orig(p) / np.repeat(r, p.n_theta)
    monkeypatch.setattr(OP, "polar_weights", w)


def _mut_sin_for_cos(monkeypatch):
    orig = OP.polar_nodes

    def nodes(p):
        kx, ky, r, w_r, theta = orig(p)
        return ky, kx, r, w_r, theta    # transposed operand: cos^2 -> sin^2
    monkeypatch.setattr(OP, "polar_nodes", nodes)


def _mut_type1_sign(monkeypatch):
    orig = OP.i2_direct_from_coeffs

    def t1(c, kx, ky, x, y, sign=1.0, chunk=1 << 24):
        return orig(c, kx, ky, x, y, sign=-sign, chunk=chunk)
    monkeypatch.setattr(OP, "i2_direct_from_coeffs", t1)


def _mut_type2_index_shift(monkeypatch):
    orig = OP.rho_hat_direct

    def t2(f, x, y, kx, ky, sign=-1.0, chunk=1 << 24):
        return orig(f, x + (x[1] - x[0]), y, kx, ky, sign=sign, chunk=chunk)
    monkeypatch.setattr(OP, "rho_hat_direct", t2)


def _mut_missing_two_pi(monkeypatch):
    orig = OP.polar_weights
    monkeypatch.setattr(OP, "polar_weights", lambda p: orig(p) * (2 * math.pi) ** 2)


def _mut_zero_mode(monkeypatch):
    orig = OP.multiplier_high

    def m1(wx, wy, p):
        m = orig(wx, wy, p)
        return np.where((wx == 0) & (wy == 0), -1.0, m)
    monkeypatch.setattr(OP, "multiplier_high", m1)


def _mut_no_padding(monkeypatch):
    orig = OP.i1_padded_fft

    def i1(rho, p):
        import dataclasses
        return orig(rho, dataclasses.replace(p, pad=1))
    monkeypatch.setattr(OP, "i1_padded_fft", i1)


@pytest.mark.parametrize("mutation", [
    _mut_drop_one_minus_p, _mut_drop_jacobian, _mut_sin_for_cos, _mut_type1_sign,
    _mut_type2_index_shift, _mut_missing_two_pi, _mut_zero_mode, _mut_no_padding,
])
def test_mutation_is_caught(monkeypatch, mutation):
    mutation(monkeypatch)
    assert not _battery()


def test_reversed_sharp_indicator_is_caught(monkeypatch):
    """The sharp partition's pin (a decayed tail: I1 vanishes, I2 carries the
    closed form) catches an indicator taken outside the disk instead of
    inside; the total alone would not, the split being exact for any p."""
    orig = OP.partition

    def part(w2, p):
        if p.partition == "sharp":
            return (w2 > p.cut_radius ** 2).astype(float)
        return orig(w2, p)
    monkeypatch.setattr(OP, "partition", part)
    n, L = 128, 16.0
    x = O.grid_axis(n, L)
    X, Y = np.meshgrid(x, x)
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=10.0, n_r=120, n_theta=244, partition="sharp")
    phi, i1, i2 = O.solve(np.exp(-(X**2 + Y**2)), p, return_parts=True)
    scale = np.abs(O.gaussian_potential(X, Y)).max()
    assert np.abs(i1).max() / scale > 5e-11
