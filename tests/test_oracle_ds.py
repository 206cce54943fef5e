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
