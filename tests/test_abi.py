"""The C-ABI library loads, exports every declared symbol, and rejects
invalid parameters before touching the GPU (no compute calls here)."""

import ctypes
import os
import re

import pytest

import paper_1409_2014_gb300 as pkg
from paper_1409_2014_gb300 import _abi
from paper_1409_2014_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return _abi.load()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"\b(dsnu_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "dsnu_solve" in names and "dsnu_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(_abi.EXPORTED) <= set(names)


def test_struct_layout_matches_header():
    assert ctypes.sizeof(_abi.dsnu_params) == 64
    assert _abi.dsnu_params.lx.offset == 8
    assert _abi.dsnu_params.n_r.offset == 40
    assert _abi.dsnu_params.partition.offset == 60
    assert ctypes.sizeof(_abi.dsnu_plan_info) == 56


def _params(**kw):
    base = dict(nx=128, ny=128, lx=16.0, ly=16.0, cut_radius=4.0, n_r=32, n_theta=64)
    base.update(kw)
    return pkg.make_params(**base)


@pytest.mark.parametrize("bad", [
    dict(nx=100), dict(ny=8), dict(nx=8192), dict(lx=0.0), dict(ly=-1.0), dict(cut_radius=0.0),
    dict(n_theta=63), dict(n_r=0), dict(kernel_width=1), dict(kernel_width=17),
    dict(sigma=-1.0), dict(cut_radius=40.0),
])
def test_invalid_params_are_rejected(lib, bad):
    with pytest.raises(_abi.DsnuError) as ei:
        _abi.dsnu_plan_create(_params(**bad), 0)
    assert ei.value.status in (_abi.DSNU_EINVAL, _abi.DSNU_EUNSUPPORTED)
    assert _abi.dsnu_last_error()


def test_unsupported_padding(lib):
    p = _params()
    p.pad_factor = 3
    with pytest.raises(_abi.DsnuError) as ei:
        _abi.dsnu_plan_create(p, 0)
    assert ei.value.status == _abi.DSNU_EUNSUPPORTED


def test_standard_solver_needs_pad_factor_one(lib):
    """partition NONE is the unpadded standard solver: pad_factor must be 1,
    and pad_factor 1 is accepted only with partition NONE."""
    p = _params(partition="none")
    assert p.pad_factor == 1 and p.partition == _abi.DSNU_PARTITION_NONE
    for part, pad in ((_abi.DSNU_PARTITION_NONE, 2), (_abi.DSNU_PARTITION_NONE, 0),
                      (_abi.DSNU_PARTITION_GAUSS, 1), (_abi.DSNU_PARTITION_SHARP, 1), (3, 1)):
        q = _params()
        q.partition, q.pad_factor = part, pad
        with pytest.raises(_abi.DsnuError) as ei:
            _abi.dsnu_plan_create(q, 0)
        assert ei.value.status == _abi.DSNU_EINVAL


def test_null_plan_calls(lib):
    assert lib.dsnu_workspace_bytes(None) == 0
    assert lib.dsnu_solve(None, None, None, None) == _abi.DSNU_EINVAL
    assert lib.dsnu_solve_adjoint(None, None, None, None) == _abi.DSNU_EINVAL
    assert lib.dsnu_set_workspace(None, None, 0) == _abi.DSNU_EINVAL
    assert lib.dsnu_plan_destroy(None) == _abi.DSNU_OK
    assert lib.dsnu_status_poll(None, None) == _abi.DSNU_EINVAL
