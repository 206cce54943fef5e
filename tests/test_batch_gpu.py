"""Batched solves (ragged grid sizes, shared plans, CUDA graph replay) through
the C ABI: every member equals its own dsnu_solve bit for bit, and one member
of each grid size matches the FP64 oracle on a sample of its grid."""

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
    """64 seeded densities (4-16 Gaussians) on {256, 512, 1024, 2048}^2, mixed."""
    from paper_1409_2014_gb300 import Batch

    members = synth.batch_members(seed=5, count=64)
    plans = {n: _plan(n, "mixed") for n in {m[0] for m in members}}
    rhos = [torch.from_numpy(synth.density_sum(n, n, 32.0, 32.0, seed=s, count=k)).cuda()
            for n, k, s in members]
    phis = [torch.empty_like(r) for r in rhos]
    b = Batch([plans[m[0]] for m in members], rhos, phis)
    b.capture_graph()
    b.solve()
    torch.cuda.synchronize()
    for (n, _, _), r, f in zip(members, rhos, phis):
        assert torch.equal(f, plans[n].solve(r))
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
