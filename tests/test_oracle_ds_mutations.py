"""Planted mistakes in the oracle of the split-step DS loop (on the CPU) must
trip at least one of its pins.

Each mutation replaces one piece of ``oracle.ds`` with a plausible error (a
sign or factor in a flow, a lost half step, a wrong Yoshida coefficient) and
runs a battery of pins that do not re-use the oracle's own formulas: a plane
wave under the linear flow, a short run of the exact moving lump of Example 3
(Case I, Sec. 3.2), and the measured orders of the Strang and Yoshida
compositions (Sec. 2.3).  The unmutated oracle passes the battery.
"""

import math

import numpy as np
import pytest

import oracle as O
import oracle.ds as D
import synth
from oracle import OracleParams


def _battery():
    """True when every pin of the battery passes."""
    ok = True
    # a plane wave with grid frequencies is an eigenfunction of the linear flow
    n, L, tau, alpha = 32, 4.0, 0.37, 0.5
    x = O.grid_axis(n, L)
    X, Y = np.meshgrid(x, x)
    kx, ky = 2 * math.pi * 3 / (2 * L), 2 * math.pi * -5 / (2 * L)
    u = np.exp(1j * (kx * X + ky * Y))
    out = D.linear_flow(u, L, L, tau, alpha)
    ok &= np.abs(out - np.exp(-1j * tau * (kx * kx - alpha * ky * ky)) * u).max() < 1e-13
    # the exact moving lump (alpha = 1, beta = -1), ten Strang steps to T = 0.1:
    # the unmutated relative L-inf error is 3.2e-3 (splitting and quadrature)
    L, h = 16.0, 0.25
    n = int(2 * L / h)
    x = O.grid_axis(n, L)
    X, Y = np.meshgrid(x, x)
    P = min(72 / L, 0.5 * math.pi / h)
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=P, sigma=P / 6, n_r=32, n_theta=64)
    u = D.arkadiev_lump(X, Y, 0.0)
    for _ in range(10):
        u = D.strang_step(u, p, 0.01, 1.0, -1.0)
    ex = D.arkadiev_lump(X, Y, 0.1)
    ok &= np.abs(u - ex).max() / np.abs(ex).max() < 4e-3
    # measured orders: halving tau divides the error by ~4 (Strang), ~16 (Yoshida)
    n, L = 32, 8.0
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=4.0, sigma=2 / 3, n_r=16, n_theta=32)
    u0 = synth.wavefunction_sum(n, n, L, L, seed=4, count=3)

    def run(step, tau, T=0.16):
        u = u0
        for _ in range(int(round(T / tau))):
            u = step(u, p, tau, 1.0, 1.0)
        return u

    ref = run(D.yoshida_step, 0.005)
    for step, lo, hi in ((D.yoshida_step, 13.0, 19.0), (D.strang_step, 3.5, 4.5)):
        e = [np.abs(run(step, tau) - ref).max() for tau in (0.04, 0.02)]
        ok &= lo < e[0] / e[1] < hi
    return bool(ok)


def test_unmutated_oracle_passes_battery():
    assert _battery()


def _mut_linear_sign(monkeypatch):
    def lf(u, lx, ly, tau, alpha):
        ny, nx = u.shape
        kx = D.wave_numbers(nx, lx)[None, :]
        ky = D.wave_numbers(ny, ly)[:, None]
        return np.fft.ifft2(np.exp(1j * tau * (kx * kx - alpha * ky * ky)) * np.fft.fft2(u))
    monkeypatch.setattr(D, "linear_flow", lf)


def _mut_linear_alpha_sign(monkeypatch):
    def lf(u, lx, ly, tau, alpha):
        ny, nx = u.shape
        kx = D.wave_numbers(nx, lx)[None, :]
        ky = D.wave_numbers(ny, ly)[:, None]
        return np.fft.ifft2(np.exp(-1j * tau * (kx * kx + alpha * ky * ky)) * np.fft.fft2(u))
    monkeypatch.setattr(D, "linear_flow", lf)


def _mut_nonlinear_self_factor(monkeypatch):
    monkeypatch.setattr(D, "nonlinear_flow",
                        lambda u, phi, tau, beta: u * np.exp(1j * tau * (beta * np.abs(u) ** 2 + 4.0 * beta * phi)))


def _mut_nonlinear_potential_factor(monkeypatch):
    monkeypatch.setattr(D, "nonlinear_flow",
                        lambda u, phi, tau, beta: u * np.exp(1j * tau * (2.0 * beta * np.abs(u) ** 2 + 2.0 * beta * phi)))


def _mut_strang_without_half_steps(monkeypatch):
    def step(u, p, tau, alpha, beta):
        u = D.linear_flow(u, p.lx, p.ly, tau, alpha)
        phi = O.solve(np.abs(u) ** 2, p)
        return D.nonlinear_flow(u, phi, tau, beta)
    monkeypatch.setattr(D, "strang_step", step)


def _mut_yoshida_a_middle(monkeypatch):
    orig = D.yoshida_coefficients

    def coeffs():
        (a1, _, _, a4), b = orig()
        return (a1, 0.5 * b[1], 0.5 * b[1], a4), b
    monkeypatch.setattr(D, "yoshida_coefficients", coeffs)


def _mut_yoshida_b_middle(monkeypatch):
    orig = D.yoshida_coefficients

    def coeffs():
        a, (b1, _, b3) = orig()
        return a, (b1, -(2.0 ** (1.0 / 3.0)), b3)
    monkeypatch.setattr(D, "yoshida_coefficients", coeffs)


@pytest.mark.parametrize("mutation", [
    _mut_linear_sign, _mut_linear_alpha_sign, _mut_nonlinear_self_factor, _mut_nonlinear_potential_factor,
    _mut_strang_without_half_steps, _mut_yoshida_a_middle, _mut_yoshida_b_middle,
])
def test_mutation_is_caught(monkeypatch, mutation):
    mutation(monkeypatch)
    assert not _battery()
