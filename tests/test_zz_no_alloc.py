"""dsnu_solve_noalloc: the solve for callers that cannot allocate device
memory when they solve (it uses a 32 MiB scratch array compiled into the
library instead of a caller workspace).

Called through the C ABI, two calls in a row, each compared with dsnu_solve
on the same input: both run the same kernels in the same order on the same
plan tables, only the scratch differs, so the results must be bitwise equal;
the absolute accuracy is checked against the FP64 oracle on a sample of the
grid within the parity tolerances of the other GPU tests.  This file is
collected last so that a failure here cannot hide the others; it builds the
library itself so that it also runs alone in a fresh process.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-12, "mixed": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_2014_gb300.build import build

    build()


@pytest.mark.parametrize("prec,n,L,P", [("mixed", 1024, 32.0, 8.0), ("fp64", 256, 16.0, 6.0)])
def test_noalloc_matches_solve_twice(prec, n, L, P):
    from paper_1409_2014_gb300 import Plan, _abi

    plan = Plan(n, lx=L, cut_radius=P, n_r=64, n_theta=256, precision=prec)
    assert _abi.dsnu_noalloc_scratch_bytes() == 32 << 20
    stream = torch.cuda.current_stream().cuda_stream
    rows, cols = np.arange(1, n, 16), np.arange(3, n, 16)
    op = oracle.OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=P, n_r=64, n_theta=256)
    for seed in (11, 12):  # two calls in a row on different inputs
        rho_np = synth.density_abs2(n, n, L, L, seed=seed, count=8)
        rho = torch.from_numpy(rho_np).cuda()
        ref = plan.solve(rho)
        out = torch.full_like(rho, float("nan"))
        _abi.dsnu_solve_noalloc(plan.handle, rho.data_ptr(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        o = out.cpu().numpy()[np.ix_(rows, cols)]
        want = oracle.solve(rho_np, op, rows=rows, cols=cols)
        assert float(np.abs(o - want).max() / np.abs(want).max()) <= TOL[prec]
    assert plan.status_poll() == _abi.DSNU_OK
    plan.close()


def test_noalloc_rejects_plans_beyond_the_static_scratch():
    from paper_1409_2014_gb300 import Plan, _abi

    plan = Plan(2048, lx=64.0, cut_radius=8.0, n_r=64, n_theta=256, precision="mixed")
    assert _abi.dsnu_workspace_bytes(plan.handle) > _abi.dsnu_noalloc_scratch_bytes()
    x = torch.zeros(2048, 2048, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(_abi.DsnuError) as ei:
        _abi.dsnu_solve_noalloc(plan.handle, x.data_ptr(), y.data_ptr(), 0)
    assert ei.value.status == _abi.DSNU_EINVAL
    assert "static scratch" in str(ei.value)
    plan.close()
