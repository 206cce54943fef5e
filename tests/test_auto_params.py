"""Automatic choice of the split solver's polar parameters for a target
accuracy (dsnu_params_auto): the rule's properties on the host, the oracle
meeting the target on the closed-form Gaussian with the chosen parameters,
and the GPU solver doing the same."""

import math

import numpy as np
import pytest

import oracle as O
from paper_1409_2014_gb300 import _abi
from paper_1409_2014_gb300.build import build


@pytest.fixture(scope="module")
def lib():
    build()
    return _abi.load()


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-10, 1e-14])
@pytest.mark.parametrize("n,lx,ly", [(128, 8.0, 8.0), (256, 16.0, 8.0), (1024, 32.0, 32.0)])
def test_rule_properties(lib, n, lx, ly, eps):
    p = _abi.dsnu_params_auto(n, n, lx, ly, eps, _abi.DSNU_FP64)
    assert abs(p.sigma * min(lx, ly) - 12.0) < 1e-12
    assert abs(math.exp(-(p.cut_radius / p.sigma) ** 2) / eps - 1.0) < 1e-9  # p(P) = eps
    assert p.n_theta % 4 == 0 and p.n_r % 8 == 0
    cR = p.cut_radius * math.hypot(lx, ly)
    assert p.n_theta >= cR + 16 > p.n_theta - 4
    assert p.n_r >= cR / 2 + 4 > p.n_r - 8
    assert p.radial_rule == _abi.DSNU_RADIAL_JACOBI and p.partition == _abi.DSNU_PARTITION_GAUSS
    assert p.pad_factor == 2 and p.kernel_width == 0


def test_rule_is_monotone_and_clamped(lib):
    prev = None
    for eps in (1e-2, 1e-4, 1e-8, 1e-12, 1e-15, 1e-20):
        p = _abi.dsnu_params_auto(256, 256, 16.0, 16.0, eps, _abi.DSNU_FP64)
        if prev is not None:
            assert p.cut_radius >= prev.cut_radius and p.n_r >= prev.n_r and p.n_theta >= prev.n_theta
        prev = p
    a = _abi.dsnu_params_auto(256, 256, 16.0, 16.0, 1e-20, _abi.DSNU_FP64)
    b = _abi.dsnu_params_auto(256, 256, 16.0, 16.0, 1e-15, _abi.DSNU_FP64)
    assert a.cut_radius == b.cut_radius  # clamped at 1e-15
    m = _abi.dsnu_params_auto(256, 256, 16.0, 16.0, 1e-12, _abi.DSNU_MIXED)
    c = _abi.dsnu_params_auto(256, 256, 16.0, 16.0, 1e-7, _abi.DSNU_MIXED)
    assert m.cut_radius == c.cut_radius  # MIXED: clamped at 1e-7


@pytest.mark.parametrize("args", [(100, 128, 8.0, 8.0, 1e-6, 0), (128, 128, 0.0, 8.0, 1e-6, 0),
                                  (128, 128, 8.0, 8.0, 0.0, 0), (128, 128, 8.0, 8.0, 1.5, 0),
                                  (128, 128, 8.0, 8.0, 1e-6, 7), (16, 16, 0.25, 0.25, 1e-14, 0)])
def test_rule_rejects_bad_input(lib, args):
    with pytest.raises(_abi.DsnuError):
        _abi.dsnu_params_auto(*args)


def test_oracle_meets_the_target_with_the_chosen_parameters(lib):
    """rho = exp(-r^2) on [-8,8)^2, N = 128, eps = 1e-10: the oracle with the
    chosen parameters matches the closed form to within eps."""
    n, L, eps = 128, 8.0, 1e-10
    p = _abi.dsnu_params_auto(n, n, L, L, eps, _abi.DSNU_FP64)
    op = O.OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=p.cut_radius, sigma=p.sigma, n_r=p.n_r,
                        n_theta=p.n_theta, radial="jacobi")
    x = O.grid_axis(n, L)
    X, Y = np.meshgrid(x, x)
    phi = O.solve(np.exp(-(X * X + Y * Y)), op)
    ex = O.gaussian_potential(X, Y)
    assert np.abs(phi - ex).max() / np.abs(ex).max() <= eps


@pytest.mark.gpu
@pytest.mark.parametrize("prec,eps", [("fp64", 1e-6), ("fp64", 1e-10), ("fp64", 1e-14), ("mixed", 1e-6)])
@pytest.mark.parametrize("n,L", [(128, 8.0), (256, 16.0), (1024, 64.0)])
def test_gpu_meets_the_target(n, L, prec, eps):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_2014_gb300 import Plan

    plan = Plan.auto(n, lx=L, eps=eps, precision=prec)
    x = O.grid_axis(n, L)
    X, Y = np.meshgrid(x, x)
    phi = plan.solve(torch.from_numpy(np.exp(-(X * X + Y * Y))).cuda()).cpu().numpy()
    plan.close()
    ex = O.gaussian_potential(X, Y)
    assert np.abs(phi - ex).max() / np.abs(ex).max() <= max(eps, 2e-15)
