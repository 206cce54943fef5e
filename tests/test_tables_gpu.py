"""Tables 2 and 5 of the paper (Sec. 3.1; their error columns are repeated in
Tables 3 and 6) reproduced by the split solver on the GPU: the relative
discrete l-infinity error against the closed-form potential of Example 1 (the
Gaussian) and Example 2 (Arkadiev's density), with the parameters the oracle
pins use (sigma L = 12, P = 6 sigma capped below the grid's Nyquist, 64 x 128
polar nodes).  FP64 plans match every printed value to 1 %, except the h = 1/16
entries of Table 2 (printed 2.7e-15, the paper's NUFFT tolerance floor), which
must stay below 1e-13; mixed plans are checked where the printed error is far
above FP32 rounding.  Entries whose disk plus ES stencil does not fit the
padded grid (the coarsest h) are skipped: the plan refuses them."""

import math

import numpy as np
import pytest

import oracle as O
from conftest import read_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_2014_gb300.build import build

    build()


def _error(L, h, prec, density, potential):
    from paper_1409_2014_gb300 import Plan, _abi

    n = int(round(2 * L / h))
    sig = 12.0 / L
    P = min(6.0 * sig, 0.9 * math.pi / h)
    try:
        plan = Plan(n, lx=L, cut_radius=P, sigma=P / 6.0, n_r=64, n_theta=128, precision=prec)
    except _abi.DsnuError as e:
        assert e.status == _abi.DSNU_EINVAL
        pytest.skip(f"disk plus ES stencil outside the padded grid at L={L}, h={h}")
    x = O.grid_axis(n, L)
    X, Y = np.meshgrid(x, x)
    phi = plan.solve(torch.from_numpy(density(X, Y)).cuda()).cpu().numpy()
    plan.close()
    ex = potential(X, Y)
    return float(np.abs(phi - ex).max() / np.abs(ex).max())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,h,printed", read_golden("table2_nufft_gaussian.txt"))
def test_table2_on_gpu(L, h, printed, prec):
    if prec == "mixed" and printed < 1e-4:
        pytest.skip("printed error below what FP32 transforms resolve")
    err = _error(L, h, prec, O.paper_gaussian_density, O.paper_gaussian_potential)
    if h < 0.1:
        assert err < 1e-13, err
    else:
        assert abs(err / printed - 1.0) <= 0.01, err


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("L,h,printed", read_golden("table5_nufft_arkadiev.txt"))
def test_table5_on_gpu(L, h, printed, prec):
    if prec == "mixed" and printed < 1e-4:
        pytest.skip("printed error below what FP32 transforms resolve")
    err = _error(L, h, prec, O.arkadiev_density, O.arkadiev_potential)
    assert abs(err / printed - 1.0) <= 0.01, err
