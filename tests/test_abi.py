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


def test_struct_layout_matches_header(tmp_path):
    """ctypes layouts equal the C compiler's for the header's structs."""
    import shutil
    import subprocess

    assert ctypes.sizeof(_abi.dsnu_params) == 72
    assert _abi.dsnu_params.lx.offset == 8
    assert _abi.dsnu_params.n_r.offset == 40
    assert _abi.dsnu_params.partition.offset == 60
    assert _abi.dsnu_params.radial_rule.offset == 64
    assert ctypes.sizeof(_abi.dsnu_plan_info) == 64
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    checks = []
    for struct, cls in (("dsnu_params", _abi.dsnu_params), ("dsnu_plan_info", _abi.dsnu_plan_info),
                        ("dsnu_ds_params", _abi.dsnu_ds_params), ("dsnu_multiplier", _abi.dsnu_multiplier)):
        checks.append(f'printf("{struct} sizeof %zu\\n", sizeof({struct}));')
        for name, _ in cls._fields_:
            checks.append(f'printf("{struct} {name} %zu\\n", offsetof({struct}, {name}));')
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "dsnufft.h"\nint main(void) {\n'
                   + "\n".join(checks) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line.strip()}
    for struct, cls in (("dsnu_params", _abi.dsnu_params), ("dsnu_plan_info", _abi.dsnu_plan_info),
                        ("dsnu_ds_params", _abi.dsnu_ds_params), ("dsnu_multiplier", _abi.dsnu_multiplier)):
        assert got[(struct, "sizeof")] == ctypes.sizeof(cls), struct
        for name, _ in cls._fields_:
            assert got[(struct, name)] == getattr(cls, name).offset, (struct, name)


@pytest.mark.parametrize("rule,name", [(0, "legendre"), (1, "jacobi")])
@pytest.mark.parametrize("n_r", [1, 2, 7, 33, 64, 200])
def test_library_radial_rule_matches_oracle(lib, rule, name, n_r):
    """dsnu_radial_nodes (the library's own Newton solvers) equals the oracle's
    rule (numpy's Gauss-Legendre table, scipy's Gauss-Jacobi table)."""
    import numpy as np

    import oracle as O

    P = 5.5
    r, w = _abi.dsnu_radial_nodes(n_r, rule, P)
    ro, wo = O.radial_rule(O.OracleParams(nx=8, ny=8, lx=1, ly=1, cut_radius=P, n_r=n_r, n_theta=4, radial=name))
    assert np.abs(np.array(r) - ro).max() <= 1e-14 * P
    # numpy's Gauss-Legendre weights lose accuracy with n (3.9e-13 of the largest
    # weight at n = 200 against a 40-digit evaluation; the library's 4.9e-15)
    tol = 1e-13 if n_r <= 64 else 1e-12
    assert np.abs(np.array(w) - wo).max() <= tol * np.abs(wo).max()


def test_library_radial_rule_rejects_bad_input(lib):
    for args in ((0, 0, 1.0), (4097, 0, 1.0), (4, 2, 1.0), (4, 0, 0.0), (4, 1, float("nan"))):
        with pytest.raises(_abi.DsnuError):
            _abi.dsnu_radial_nodes(*args)


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


@pytest.mark.parametrize("alpha,a0", [(2, 1.0), (-2, 1.0), (0, float("inf"))])
def test_bad_multiplier_is_rejected(lib, alpha, a0):
    m = _abi.dsnu_multiplier(alpha=alpha, reserved=0, a0=a0, a_cos=0.0, a_sin=0.0)
    with pytest.raises(_abi.DsnuError) as ei:
        _abi.dsnu_plan_create_multiplier(_params(), m, 0)
    assert ei.value.status == _abi.DSNU_EINVAL


def test_stream_solve_rejects_bad_arguments(lib):
    assert lib.dsnu_stream_staging_bytes(None) == 0
    vp = ctypes.c_void_p
    arr = (vp * 1)(vp(1))
    assert lib.dsnu_solve_host_stream(None, 1, arr, arr, vp(256), 1 << 20, None) == _abi.DSNU_EINVAL


def test_null_plan_calls(lib):
    assert lib.dsnu_workspace_bytes(None) == 0
    assert lib.dsnu_solve(None, None, None, None) == _abi.DSNU_EINVAL
    assert lib.dsnu_solve_adjoint(None, None, None, None) == _abi.DSNU_EINVAL
    assert lib.dsnu_set_workspace(None, None, 0) == _abi.DSNU_EINVAL
    assert lib.dsnu_plan_destroy(None) == _abi.DSNU_OK
    assert lib.dsnu_status_poll(None, None) == _abi.DSNU_EINVAL
