"""Planted mistakes in the oracle's generic multiplier family (on the CPU) must
trip at least one of its pins.

The family |k|^alpha (a0 + ac cos 2theta + as sin 2theta) enters twice: as the
high-frequency multiplier of I1 (``multiplier``) and in the polar weights of
I2 (``polar_weights``).  Each mutation plants one plausible error there (a
flipped sign, cos^2 for cos 2theta, a dropped or doubled power of |k|, swapped
coefficients) and runs a battery of the closed-form pins of
``test_oracle_multipliers``: the degree-0 family with all three angular terms,
the half Laplacian |k| and the 2D Coulomb multiplier 2 pi/|k|.  The unmutated
oracle passes the battery.
"""

import math

import numpy as np
import pytest

import oracle as O
import oracle.potential as OP
from oracle import OracleParams


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _battery():
    """True when every pin of the battery passes."""
    ok = True
    n, L = 128, 16.0
    x = O.grid_axis(n, L)
    X, Y = np.meshgrid(x, x)
    rho = np.exp(-(X * X + Y * Y))
    # degree 0, all three angular terms
    a0, ac, as_ = 0.3, 0.7, -0.2
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=4.0, sigma=2 / 3, n_r=48, n_theta=96,
                     multiplier=(0, a0, ac, as_))
    ok &= _rel(O.solve(rho, p), O.gaussian_potential_alpha0(X, Y, a0, ac, as_)) < 1e-12
    # |k|
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=4.0, sigma=2 / 3, n_r=48, n_theta=96,
                     multiplier=(1, 1.0, 0.0, 0.0))
    ok &= _rel(O.solve(rho, p), O.gaussian_abs_k(X, Y)) < 1e-7
    # 2 pi / |k|
    sig = 0.75
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=6 * sig, sigma=sig, n_r=64, n_theta=192,
                     multiplier=(-1, 2 * math.pi, 0.0, 0.0))
    ok &= _rel(O.solve(rho, p), O.gaussian_coulomb(X, Y)) < 5e-5
    return bool(ok)


def test_unmutated_oracle_passes_battery():
    assert _battery()


def _generic_weights(p, ang_fn, radial_power=lambda alpha: float(alpha)):
    """polar_weights for the generic family with the angular factor and the
    radial power supplied (the planted mistakes go there)."""
    _, _, r, w_rad, theta = OP.polar_nodes(p)
    alpha, a0, ac, as_ = p.multiplier
    radial = w_rad * np.power(r, radial_power(alpha)) * OP.partition(r * r, p)
    ang = ang_fn(theta, a0, ac, as_) * (2 * math.pi / p.n_theta)
    return ((radial[:, None] * ang[None, :]) / (2 * math.pi) ** 2).ravel()


def _patch_weights(monkeypatch, **kw):
    orig = OP.polar_weights

    def w(p):
        if tuple(p.multiplier) == OP.DS_MULTIPLIER:
            return orig(p)
        return _generic_weights(p, **kw)
    monkeypatch.setattr(OP, "polar_weights", w)


def test_unmutated_restatement_of_the_weights_passes_battery(monkeypatch):
    """Control: the restatement the weight mutations start from, unmutated,
    passes (so a caught mutation is caught for its planted error)."""
    _patch_weights(monkeypatch, ang_fn=lambda t, a0, ac, as_: a0 + ac * np.cos(2 * t) + as_ * np.sin(2 * t))
    assert _battery()


def _mut_weights_sin_sign(monkeypatch):
    _patch_weights(monkeypatch, ang_fn=lambda t, a0, ac, as_: a0 + ac * np.cos(2 * t) - as_ * np.sin(2 * t))


def _mut_weights_cos_squared(monkeypatch):
    _patch_weights(monkeypatch, ang_fn=lambda t, a0, ac, as_: a0 + ac * np.cos(t) ** 2 + as_ * np.sin(2 * t))


def _mut_weights_swapped_coefficients(monkeypatch):
    _patch_weights(monkeypatch, ang_fn=lambda t, a0, ac, as_: a0 + as_ * np.cos(2 * t) + ac * np.sin(2 * t))


def _mut_weights_drop_radial_power(monkeypatch):
    _patch_weights(monkeypatch, ang_fn=lambda t, a0, ac, as_: a0 + ac * np.cos(2 * t) + as_ * np.sin(2 * t),
                   radial_power=lambda alpha: 0.0)


def _patch_multiplier(monkeypatch, fn):
    orig = OP.multiplier

    def m(wx, wy, p):
        if tuple(p.multiplier) == OP.DS_MULTIPLIER:
            return orig(wx, wy, p)
        return fn(wx, wy, p)
    monkeypatch.setattr(OP, "multiplier", m)


def _mut_multiplier_sin_sign(monkeypatch):
    def fn(wx, wy, p):
        alpha, a0, ac, as_ = p.multiplier
        w2 = wx * wx + wy * wy
        with np.errstate(divide="ignore", invalid="ignore"):
            m = np.power(w2, 0.5 * alpha) * (a0 + (ac * (wx * wx - wy * wy) - as_ * 2 * wx * wy) / w2)
        return np.where(w2 > 0, m, 0.0)
    _patch_multiplier(monkeypatch, fn)


def _mut_multiplier_doubled_power(monkeypatch):
    def fn(wx, wy, p):
        alpha, a0, ac, as_ = p.multiplier
        w2 = wx * wx + wy * wy
        with np.errstate(divide="ignore", invalid="ignore"):
            m = np.power(w2, float(alpha)) * (a0 + (ac * (wx * wx - wy * wy) + as_ * 2 * wx * wy) / w2)
        return np.where(w2 > 0, m, 0.0)
    _patch_multiplier(monkeypatch, fn)


@pytest.mark.parametrize("mutation", [
    _mut_weights_sin_sign, _mut_weights_cos_squared, _mut_weights_swapped_coefficients,
    _mut_weights_drop_radial_power, _mut_multiplier_sin_sign, _mut_multiplier_doubled_power,
])
def test_mutation_is_caught(monkeypatch, mutation):
    mutation(monkeypatch)
    assert not _battery()
