"""Pins of the CPU oracle of the split-step DS loop (Sec. 2.3, Example 3)."""

import math

import numpy as np
import pytest

import oracle
from oracle import OracleParams
from oracle import ds as D
from conftest import read_golden
import synth


def test_linear_flow_is_exact_on_a_fourier_mode():
    n, L, tau, alpha = 32, 4.0, 0.37, 1.0
    x = oracle.grid_axis(n, L)
    X, Y = np.meshgrid(x, x)
    kx = 2 * math.pi * 3 / (2 * L)
    ky = 2 * math.pi * -5 / (2 * L)
    u = np.exp(1j * (kx * X + ky * Y))
    out = D.linear_flow(u, L, L, tau, alpha)
    assert np.abs(out - np.exp(-1j * tau * (kx * kx - alpha * ky * ky)) * u).max() < 1e-13


def _small():
    n, L = 64, 8.0
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=4.0, sigma=2 / 3, n_r=24, n_theta=48)
    u = synth.wavefunction_sum(n, n, L, L, seed=4, count=3)
    return p, u


def test_strang_step_conserves_mass_and_is_reversible():
    p, u0 = _small()
    u = u0.copy()
    for _ in range(5):
        u = D.strang_step(u, p, 1e-2, 1.0, 1.0)
    assert abs(np.sum(np.abs(u) ** 2) / np.sum(np.abs(u0) ** 2) - 1.0) < 1e-13
    for _ in range(5):
        u = D.strang_step(u, p, -1e-2, 1.0, 1.0)
    # the symmetric composition is time-reversible up to the change of |u|
    # inside the nonlinear flow, which is exactly zero: back to u0 to rounding
    assert np.abs(u - u0).max() < 1e-12 * np.abs(u0).max()


@pytest.mark.parametrize("L,h,printed", read_golden("table8_ds_case1_nufft.txt"))
def test_table8_moving_lump(L, h, printed):
    n = int(round(2 * L / h))
    x = oracle.grid_axis(n, L)
    X, Y = np.meshgrid(x, x)
    P = min(6 * 12 / L, 0.9 * math.pi / h)
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=P, sigma=P / 6, n_r=64, n_theta=128)
    u = D.arkadiev_lump(X, Y, 0.0)
    tau, T = 0.01, 0.4
    for _ in range(int(round(T / tau))):
        u = D.strang_step(u, p, tau, 1.0, -1.0)
    ex = D.arkadiev_lump(X, Y, T)
    err = float(np.linalg.norm(u - ex) / np.linalg.norm(ex))
    assert abs(err / printed - 1.0) < 0.01, err


# ---------------------------------------------------------------- Yoshida (Sec. 2.3)

def test_yoshida_coefficients_satisfy_the_order_conditions():
    """Consistency (sum a = sum b = 1), symmetry, and the third-order condition
    of the triple jump, b1^3 + b2^3 + b3^3 = 0, that makes the symmetric
    composition fourth order."""
    a, b = D.yoshida_coefficients()
    assert abs(sum(a) - 1.0) < 1e-15 and abs(sum(b) - 1.0) < 1e-15
    assert a[0] == a[3] and a[1] == a[2] and b[0] == b[2]
    assert abs(sum(x ** 3 for x in b)) < 1e-14
    assert b[1] < 0 and a[1] < 0  # the backward sub-steps of the triple jump


def _order_case():
    n, L = 32, 8.0
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=4.0, sigma=2 / 3, n_r=16, n_theta=32)
    return p, synth.wavefunction_sum(n, n, L, L, seed=4, count=3)


def _evolve(step, u, p, tau, T, alpha=1.0, beta=1.0):
    for _ in range(int(round(abs(T / tau)))):
        u = step(u, p, tau, alpha, beta)
    return u


def test_yoshida_is_fourth_order_and_strang_second_order():
    """Global error at T = 0.16 against a Yoshida run with tau = 0.0025: halving
    tau divides the Yoshida error by ~16 and the Strang error by ~4."""
    p, u0 = _order_case()
    ref = _evolve(D.yoshida_step, u0, p, 0.0025, 0.16)
    for step, lo, hi in ((D.yoshida_step, 13.0, 19.0), (D.strang_step, 3.5, 4.5)):
        e = [np.abs(_evolve(step, u0, p, tau, 0.16) - ref).max() for tau in (0.04, 0.02, 0.01)]
        for k in range(2):
            assert lo < e[k] / e[k + 1] < hi, (step.__name__, e)


def test_yoshida_conserves_mass_and_is_reversible():
    p, u0 = _order_case()
    u = _evolve(D.yoshida_step, u0, p, 0.02, 0.1)
    assert abs(np.sum(np.abs(u) ** 2) / np.sum(np.abs(u0) ** 2) - 1.0) < 1e-13
    u = _evolve(D.yoshida_step, u, p, -0.02, 0.1)
    assert np.abs(u - u0).max() < 1e-12 * np.abs(u0).max()
