"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the potential solver: it only draws
parameters from a seeded generator and evaluates sums of Gaussians on the
uniform grid x_n = -L + n h.  The densities mimic the paper's workloads
(Sec. 3.1: smooth, rapidly decaying densities on a square domain; Sec. 3.2:
rho = |u|^2 of a Gaussian-type wave function).
"""

from __future__ import annotations

import dataclasses

import numpy as np


def axis(n: int, half_width: float) -> np.ndarray:
    h = 2.0 * half_width / n
    return -half_width + h * np.arange(n, dtype=np.float64)


@dataclasses.dataclass(frozen=True)
class GaussianSum:
    """sum_k A_k e^{i phi_k} exp(-((x-cx_k)^2/(2 sx_k^2) + (y-cy_k)^2/(2 sy_k^2)))."""

    cx: np.ndarray
    cy: np.ndarray
    sx: np.ndarray
    sy: np.ndarray
    amp: np.ndarray
    phase: np.ndarray

    def evaluate(self, nx: int, ny: int, lx: float, ly: float,
                 complex_valued: bool = False, dtype=np.float64) -> np.ndarray:
        x = axis(nx, lx)
        y = axis(ny, ly)
        cdt = np.complex128 if complex_valued else np.float64
        out = np.zeros((ny, nx), dtype=cdt)
        for k in range(self.cx.size):
            gx = np.exp(-((x - self.cx[k]) ** 2) / (2.0 * self.sx[k] ** 2))
            gy = np.exp(-((y - self.cy[k]) ** 2) / (2.0 * self.sy[k] ** 2))
            coef = self.amp[k] * (np.exp(1j * self.phase[k]) if complex_valued else 1.0)
            out += coef * np.outer(gy, gx)
        if complex_valued:
            return out.astype(np.complex64 if dtype in (np.float32, np.complex64) else np.complex128)
        return out.astype(dtype)


def gaussian_sum(seed: int, count: int, center=(-4.0, 4.0), width=(0.5, 2.0),
                 amplitude=(0.5, 1.5)) -> GaussianSum:
    """Draw ``count`` axis-aligned Gaussians: centers U(center)^2, standard
    deviations U(width)^2, amplitudes U(amplitude), phases U[0, 2 pi)."""
    g = np.random.Generator(np.random.PCG64(seed))
    cx = g.uniform(*center, count)
    cy = g.uniform(*center, count)
    sx = g.uniform(*width, count)
    sy = g.uniform(*width, count)
    amp = g.uniform(*amplitude, count)
    phase = g.uniform(0.0, 2.0 * np.pi, count)
    return GaussianSum(cx, cy, sx, sy, amp, phase)


def isotropic_gaussian(nx: int, ny: int, lx: float, ly: float) -> np.ndarray:
    """rho = exp(-(x^2 + y^2))."""
    x = axis(nx, lx)
    y = axis(ny, ly)
    return np.outer(np.exp(-y * y), np.exp(-x * x))


def density_sum(nx: int, ny: int, lx: float, ly: float, seed: int, count: int) -> np.ndarray:
    """Real density: a sum of ``count`` seeded Gaussians (FP64, [ny][nx])."""
    return gaussian_sum(seed, count).evaluate(nx, ny, lx, ly)


def wavefunction_sum(nx: int, ny: int, lx: float, ly: float, seed: int, count: int,
                     single: bool = False) -> np.ndarray:
    """Complex wave function u: a sum of ``count`` seeded complex Gaussians."""
    return gaussian_sum(seed, count).evaluate(
        nx, ny, lx, ly, complex_valued=True,
        dtype=np.complex64 if single else np.complex128)


def density_abs2(nx: int, ny: int, lx: float, ly: float, seed: int, count: int) -> np.ndarray:
    """rho = |u|^2 with u = ``wavefunction_sum`` (FP64)."""
    u = wavefunction_sum(nx, ny, lx, ly, seed, count)
    return (u.real * u.real + u.imag * u.imag).astype(np.float64)


def normal_field(nx: int, ny: int, seed: int) -> np.ndarray:
    """Seeded N(0, 1) field (FP64, [ny][nx]), e.g. loss weights w(x)."""
    g = np.random.Generator(np.random.PCG64(seed))
    return g.standard_normal((ny, nx))


def batch_members(seed: int, count: int, sizes=(256, 512, 1024, 2048),
                  kmin: int = 4, kmax: int = 16):
    """(n, n_gaussians, member_seed) for a ragged batch of densities."""
    g = np.random.Generator(np.random.PCG64(seed))
    ns = g.choice(np.asarray(sizes), size=count)
    ks = g.integers(kmin, kmax + 1, size=count)
    seeds = g.integers(0, 2**31 - 1, size=count)
    return [(int(n), int(k), int(s)) for n, k, s in zip(ns, ks, seeds)]
