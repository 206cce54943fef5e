"""Batched solves (ragged grid sizes, shared plans, CUDA graph replay) through
the C ABI.  With one launch sequence per plan on forked streams every member
equals its own dsnu_solve bit for bit (the same kernels); with one launch per
pipeline stage for all grid sizes (the same kernel bodies compiled into other
kernels, where the compiler may contract multiply-adds differently) every
member equals it to FP32 rounding, and repeated batch solves are bitwise
reproducible.  One member of each grid size matches the FP64 oracle on a
sample of its grid."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_2014_gb300.build import build

    build()


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


# the one-launch-per-stage kernels against the single-plan ones: FP32 rounding
STAGE_TOL = 1e-6


def _plan(n, prec):
    from paper_1409_2014_gb300 import Plan

    return Plan(n, lx=32.0, cut_radius=8.0 if n >= 256 else 2.0, n_r=64, n_theta=256, precision=prec)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_ragged_batch_equals_single_solves(prec):
    from paper_1409_2014_gb300 import Batch

    sizes = [128, 256, 128, 512, 256, 128]
    plans = {n: _plan(n, prec) for n in set(sizes)}
    rhos = [torch.from_numpy(synth.density_sum(n, n, 32.0, 32.0, seed=100 + i, count=4 + i)).cuda()
            for i, n in enumerate(sizes)]
    phis = [torch.empty_like(r) for r in rhos]
    b = Batch([plans[n] for n in sizes], rhos, phis)
    b.solve()
    for n, r, f in zip(sizes, rhos, phis):
        assert torch.equal(f, plans[n].solve(r))
    # graph capture and replay, with new inputs written in place
    b.capture_graph()
    for i, r in enumerate(rhos):
        r.mul_(0.5 + 0.1 * i)
    b.solve()
    torch.cuda.synchronize()
    for n, r, f in zip(sizes, rhos, phis):
        assert torch.equal(f, plans[n].solve(r))
    b.close()
    for p in plans.values():
        p.close()


def test_config5_batch_of_64():
    """64 seeded densities (4-16 Gaussians) on {256, 512, 1024, 2048}^2, mixed:
    one launch per pipeline stage for all four grid sizes, in a CUDA graph."""
    from paper_1409_2014_gb300 import Batch

    members = synth.batch_members(seed=5, count=64)
    plans = {n: _plan(n, "mixed") for n in {m[0] for m in members}}
    rhos = [torch.from_numpy(synth.density_sum(n, n, 32.0, 32.0, seed=s, count=k)).cuda()
            for n, k, s in members]
    phis = [torch.empty_like(r) for r in rhos]
    b = Batch([plans[m[0]] for m in members], rhos, phis, schedule="stage_launches")
    assert b.schedule_in_use == "stage_launches"
    assert b.launches == 8  # the plans share one spreading configuration (same disk, nodes, spacing)
    b.capture_graph()
    b.solve()
    torch.cuda.synchronize()
    first = [f.clone() for f in phis]
    for (n, _, _), r, f in zip(members, rhos, phis):
        assert _rel(f, plans[n].solve(r)) <= STAGE_TOL
    b.solve()
    torch.cuda.synchronize()
    assert all(torch.equal(a, f) for a, f in zip(first, phis))  # reproducible
    for p in plans.values():
        assert p.status_poll() == 0
    # the first member of each size against the oracle (stride-n/128 sample)
    seen = set()
    for (n, k, s), f in zip(members, phis):
        if n in seen:
            continue
        seen.add(n)
        rows, cols = np.arange(1, n, n // 128), np.arange(2, n, n // 128)
        op = oracle.OracleParams(nx=n, ny=n, lx=32.0, ly=32.0, cut_radius=8.0, n_r=64, n_theta=256)
        ref = oracle.solve(synth.density_sum(n, n, 32.0, 32.0, seed=s, count=k), op, rows=rows, cols=cols)
        got = f.cpu().numpy()[np.ix_(rows, cols)]
        assert float(np.abs(got - ref).max() / np.abs(ref).max()) <= 1e-6, n
    assert len(seen) == 4
    b.close()
    for p in plans.values():
        p.close()


@pytest.mark.parametrize("schedule", ["stage_launches", "forked_streams"])
def test_ragged_schedules_equal_single_solves(schedule):
    """Square and rectangular grids of 256 .. 2048 points per axis (one plan
    with a single member), both schedules, direct launches and graph replay:
    every member bitwise equal to its own dsnu_solve."""
    from paper_1409_2014_gb300 import Batch, Plan

    shapes = [(256, 256), (2048, 2048), (512, 256), (256, 256), (1024, 1024), (2048, 2048), (1024, 512)]
    plans = {sh: Plan(sh[0], sh[1], lx=32.0, ly=32.0 * sh[1] / sh[0], cut_radius=8.0, n_r=32, n_theta=128,
                      precision="mixed") for sh in set(shapes)}
    rhos = [torch.from_numpy(synth.density_sum(nx, ny, 32.0, 32.0 * ny / nx, seed=200 + i, count=5)).cuda()
            for i, (nx, ny) in enumerate(shapes)]
    phis = [torch.full_like(r, float("nan")) for r in rhos]
    b = Batch([plans[sh] for sh in shapes], rhos, phis, schedule=schedule)
    assert b.schedule_in_use == schedule

    def check():
        for sh, r, f in zip(shapes, rhos, phis):
            want = plans[sh].solve(r)
            if schedule == "forked_streams":
                assert torch.equal(f, want), sh
            else:
                assert _rel(f, want) <= STAGE_TOL, (sh, _rel(f, want))

    b.solve()
    torch.cuda.synchronize()
    check()
    b.capture_graph()
    for i, r in enumerate(rhos):
        r.mul_(1.5 - 0.1 * i)
    b.solve()
    torch.cuda.synchronize()
    check()
    b.close()
    for p in plans.values():
        p.close()


def test_stage_launches_refused_outside_their_sizes():
    from paper_1409_2014_gb300 import Batch, _abi

    plans = [_plan(128, "mixed"), _plan(256, "mixed")]
    rhos = [torch.zeros(p.shape, dtype=torch.float64, device="cuda") for p in plans]
    phis = [torch.empty_like(r) for r in rhos]
    with pytest.raises(_abi.DsnuError) as ei:
        Batch(plans, rhos, phis, schedule="stage_launches")
    assert ei.value.status == _abi.DSNU_EUNSUPPORTED
    b = Batch(plans, rhos, phis)  # auto
    assert b.schedule_in_use == "forked_streams"
    b.close()
    for p in plans:
        p.close()
