"""GPU differentiation and split-step DS loop (through the C ABI) against the
CPU oracle, finite differences and invariants."""

import math

import numpy as np
import pytest

import oracle
from oracle import OracleParams
from oracle import ds as D
import synth
from conftest import read_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_2014_gb300.build import build

    build()


def _plans(n, L, prec, P=4.0, n_r=24, n_theta=48, sigma=2 / 3):
    from paper_1409_2014_gb300 import Plan
    from paper_1409_2014_gb300.ds import DSPlan

    solver = Plan(n, lx=L, cut_radius=P, n_r=n_r, n_theta=n_theta, sigma=sigma, precision=prec)
    ds = DSPlan(n, lx=L, precision=prec)
    return solver, ds


TOL = {"fp64": 1e-12, "mixed": 2e-5}
CDT = {"fp64": torch.complex128, "mixed": torch.complex64}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_flows_match_oracle(prec):
    n, L, tau, alpha, beta = 64, 8.0, 0.01, 1.0, 1.0
    solver, ds = _plans(n, L, prec)
    u_np = synth.wavefunction_sum(n, n, L, L, seed=4, count=3)
    u = torch.from_numpy(u_np).to(CDT[prec]).cuda()
    ds.set_linear_step(tau, alpha)
    lin = ds.linear_(u.clone()).cpu().numpy()
    ref = D.linear_flow(u_np, L, L, tau, alpha)
    assert np.abs(lin - ref).max() <= TOL[prec] * np.abs(ref).max()
    back = ds.linear_(torch.from_numpy(lin).to(CDT[prec]).cuda(), adjoint=True).cpu().numpy()
    assert np.abs(back - u_np).max() <= 10 * TOL[prec] * np.abs(u_np).max()
    rho = ds.abs2(u)
    assert np.abs(rho.cpu().numpy() - np.abs(u_np) ** 2).max() <= TOL[prec] * np.abs(u_np).max() ** 2
    phi = solver.solve(rho)
    nl = ds.nonlinear_(u.clone(), phi, tau, beta).cpu().numpy()
    ref_nl = D.nonlinear_flow(u_np, phi.cpu().numpy(), tau, beta)
    assert np.abs(nl - ref_nl).max() <= TOL[prec] * np.abs(u_np).max()
    solver.close()
    ds.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_strang_steps_match_oracle(prec):
    from paper_1409_2014_gb300.ds import evolve

    n, L, tau = 64, 8.0, 0.01
    solver, ds = _plans(n, L, prec)
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=4.0, sigma=2 / 3, n_r=24, n_theta=48)
    u_np = synth.wavefunction_sum(n, n, L, L, seed=4, count=3)
    ref = u_np.copy()
    for _ in range(3):
        ref = D.strang_step(ref, p, tau, 1.0, 1.0)
    with torch.no_grad():
        out = evolve(torch.from_numpy(u_np).to(CDT[prec]).cuda(), 3, ds, solver, tau, 1.0, 1.0)
    out = out.cpu().numpy()
    assert np.abs(out - ref).max() <= 3 * TOL[prec] * np.abs(ref).max()
    solver.close()
    ds.close()


def _loss_grad(u, w, solver):
    from paper_1409_2014_gb300.ds import potential

    u = u.detach().clone().requires_grad_(True)
    rho = (u.real ** 2 + u.imag ** 2).to(torch.float64)
    loss = (w * potential(rho, solver)).sum()
    loss.backward()
    return float(loss.detach()), u.grad


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_potential_gradient_matches_oracle_transpose(prec):
    """dL/du for L = sum w Phi(|u|^2) equals 2 (A^T w) u (oracle's transposed sums)."""
    n, L = 128, 16.0
    solver, ds = _plans(n, L, prec, P=4.0, n_r=32, n_theta=64)
    u_np = synth.wavefunction_sum(n, n, L, L, seed=4, count=6)
    w_np = synth.normal_field(n, n, seed=44)
    _, g = _loss_grad(torch.from_numpy(u_np).to(CDT[prec]).cuda(), torch.from_numpy(w_np).cuda(), solver)
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=4.0, n_r=32, n_theta=64)
    ref = 2.0 * oracle.solve_adjoint(w_np, p) * u_np
    g = g.cpu().numpy()
    assert np.abs(g - ref).max() <= 5 * TOL[prec] * np.abs(ref).max()
    solver.close()
    ds.close()


def test_potential_gradient_central_differences_1024():
    """complex128 u on 1024^2: directional derivatives vs central differences (h = 1e-6)."""
    n, L = 1024, 32.0
    solver, ds = _plans(n, L, "fp64", P=8.0, n_r=64, n_theta=256, sigma=0.0)
    u = torch.from_numpy(synth.wavefunction_sum(n, n, L, L, seed=3, count=16)).cuda()
    w = torch.from_numpy(synth.normal_field(n, n, seed=4)).cuda()
    _, g = _loss_grad(u, w, solver)
    gen = torch.Generator(device="cpu").manual_seed(7)
    from paper_1409_2014_gb300.ds import potential

    def L_of(v):
        with torch.no_grad():
            return float((w * potential((v.real ** 2 + v.imag ** 2), solver)).sum())

    h = 1e-6
    for _ in range(4):
        d = torch.complex(torch.randn(n, n, generator=gen, dtype=torch.float64),
                          torch.randn(n, n, generator=gen, dtype=torch.float64)).cuda()
        fd = (L_of(u + h * d) - L_of(u - h * d)) / (2 * h)
        an = float((g.real * d.real + g.imag * d.imag).sum())
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3)
    solver.close()
    ds.close()


def test_ds_loop_200_steps_checkpointed_gradient():
    """1024^2 complex128, 200 Strang steps (alpha = 1, beta = 1, dt = 1e-3): mass
    is conserved, and the gradient through checkpointed recomputation equals the
    full-tape gradient and a central difference."""
    from paper_1409_2014_gb300.ds import evolve, mass

    n, L, tau, steps = 1024, 32.0, 1e-3, 200
    solver, ds = _plans(n, L, "fp64", P=8.0, n_r=64, n_theta=256, sigma=0.0)
    u0 = torch.from_numpy(synth.wavefunction_sum(n, n, L, L, seed=3, count=16)).cuda()
    w = torch.from_numpy(synth.normal_field(n, n, seed=4)).cuda()

    def loss_of(u):
        return (w * (u.real ** 2 + u.imag ** 2)).sum()

    grads = []
    for ck in (14, 0):
        u = u0.clone().requires_grad_(True)
        out = evolve(u, steps, ds, solver, tau, 1.0, 1.0, checkpoint_every=ck)
        if ck:
            m0, m1 = mass(u0, L, L), mass(out.detach(), L, L)
            assert abs(m1 / m0 - 1.0) < 1e-12
        loss_of(out).backward()
        grads.append(u.grad.clone())
    assert torch.allclose(grads[0], grads[1], rtol=0, atol=1e-12 * float(grads[1].abs().max()))
    # central difference along one direction (fewer steps keep it quick)
    gen = torch.Generator(device="cpu").manual_seed(9)
    d = torch.complex(torch.randn(n, n, generator=gen, dtype=torch.float64),
                      torch.randn(n, n, generator=gen, dtype=torch.float64)).cuda()
    k = 10
    u = u0.clone().requires_grad_(True)
    loss_of(evolve(u, k, ds, solver, tau, 1.0, 1.0, checkpoint_every=4)).backward()
    an = float((u.grad.real * d.real + u.grad.imag * d.imag).sum())
    h = 1e-6
    with torch.no_grad():
        fp = float(loss_of(evolve(u0 + h * d, k, ds, solver, tau, 1.0, 1.0)))
        fm = float(loss_of(evolve(u0 - h * d, k, ds, solver, tau, 1.0, 1.0)))
    fd = (fp - fm) / (2 * h)
    assert abs(fd - an) <= 1e-6 * abs(an)
    solver.close()
    ds.close()


def test_ds_loop_complex64_gradient_vs_complex128():
    """complex64 (mixed plans) gradient agrees with the complex128 one."""
    from paper_1409_2014_gb300.ds import evolve

    n, L, tau, steps = 256, 16.0, 1e-3, 20
    grads = {}
    for prec in ("fp64", "mixed"):
        solver, ds = _plans(n, L, prec, P=6.0, n_r=32, n_theta=64, sigma=1.0)
        u0 = torch.from_numpy(synth.wavefunction_sum(n, n, L, L, seed=3, count=8)).to(CDT[prec]).cuda()
        w = torch.from_numpy(synth.normal_field(n, n, seed=4)).cuda()
        u = u0.clone().requires_grad_(True)
        out = evolve(u, steps, ds, solver, tau, 1.0, 1.0, checkpoint_every=5)
        (w * (out.real.double() ** 2 + out.imag.double() ** 2)).sum().backward()
        grads[prec] = u.grad.to(torch.complex128).cpu().numpy()
        solver.close()
        ds.close()
    ref = grads["fp64"]
    assert np.abs(grads["mixed"] - ref).max() <= 1e-4 * np.abs(ref).max()


# ---------------------------------------------------------------- Yoshida (Sec. 2.3)

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_yoshida_steps_match_oracle(prec):
    from paper_1409_2014_gb300.ds import evolve

    n, L, tau = 64, 8.0, 0.01
    solver, ds = _plans(n, L, prec)
    p = OracleParams(nx=n, ny=n, lx=L, ly=L, cut_radius=4.0, sigma=2 / 3, n_r=24, n_theta=48)
    u_np = synth.wavefunction_sum(n, n, L, L, seed=4, count=3)
    ref = u_np.copy()
    for _ in range(3):
        ref = D.yoshida_step(ref, p, tau, 1.0, -1.0)
    with torch.no_grad():
        out = evolve(torch.from_numpy(u_np).to(CDT[prec]).cuda(), 3, ds, solver, tau, 1.0, -1.0,
                     scheme="yoshida")
    out = out.cpu().numpy()
    assert np.abs(out - ref).max() <= 10 * TOL[prec] * np.abs(ref).max()
    solver.close()
    ds.close()


def test_yoshida_gradient_checkpointed_equals_full_tape_and_fd():
    from paper_1409_2014_gb300.ds import evolve

    n, L, tau, steps = 256, 16.0, 2e-3, 12
    solver, ds = _plans(n, L, "fp64", P=6.0, n_r=32, n_theta=64, sigma=1.0)
    u0 = torch.from_numpy(synth.wavefunction_sum(n, n, L, L, seed=3, count=8)).cuda()
    w = torch.from_numpy(synth.normal_field(n, n, seed=4)).cuda()

    def loss_of(u):
        return (w * (u.real ** 2 + u.imag ** 2)).sum() + (w * u.real).sum()

    grads = []
    for ck in (5, 0):
        u = u0.clone().requires_grad_(True)
        loss_of(evolve(u, steps, ds, solver, tau, 1.0, -1.0, checkpoint_every=ck, scheme="yoshida")).backward()
        grads.append(u.grad.clone())
    assert torch.allclose(grads[0], grads[1], rtol=0, atol=1e-12 * float(grads[1].abs().max()))
    gen = torch.Generator(device="cpu").manual_seed(11)
    d = torch.complex(torch.randn(n, n, generator=gen, dtype=torch.float64),
                      torch.randn(n, n, generator=gen, dtype=torch.float64)).cuda()
    an = float((grads[1].real * d.real + grads[1].imag * d.imag).sum())
    h = 1e-6
    with torch.no_grad():
        fp = float(loss_of(evolve(u0 + h * d, steps, ds, solver, tau, 1.0, -1.0, scheme="yoshida")))
        fm = float(loss_of(evolve(u0 - h * d, steps, ds, solver, tau, 1.0, -1.0, scheme="yoshida")))
    assert abs((fp - fm) / (2 * h) - an) <= 1e-6 * abs(an)
    solver.close()
    ds.close()


def _lump_phi(X, Y, t):
    """Case I of Example 3: the exact potential of the moving lump."""
    d = (X + 1.0) ** 2 + (Y + 4.0 * t) ** 2 + 1.0
    return -2.0 * ((Y + 4.0 * t) ** 2 - X * (X + 2.0)) / (d * d)


def _lump_errors(L, h, standard):
    """Arkadiev's moving lump (alpha = 1, beta = -1) from t = 0 to T = 0.4 with
    Yoshida steps of 1e-3 (the paper's integrator and step); relative l2 errors
    of u(T) and of Phi computed from |u(T)|^2."""
    from paper_1409_2014_gb300 import Plan
    from paper_1409_2014_gb300.ds import DSPlan, evolve

    n = int(round(2 * L / h))
    x = oracle.grid_axis(n, L)
    X, Y = np.meshgrid(x, x)
    if standard:
        solver = Plan(n, lx=L, partition="none", precision="fp64")
    else:
        P = min(6.0 * 12.0 / L, 0.5 * math.pi / h)
        solver = Plan(n, lx=L, cut_radius=P, sigma=P / 6.0, n_r=64, n_theta=128, precision="fp64")
    ds = DSPlan(n, lx=L, precision="fp64")
    with torch.no_grad():
        u = evolve(torch.from_numpy(D.arkadiev_lump(X, Y, 0.0)).cuda(), 400, ds, solver, 1e-3, 1.0, -1.0,
                   scheme="yoshida")
        phi = solver.solve(ds.abs2(u)).cpu().numpy()
    u = u.cpu().numpy()
    solver.close()
    ds.close()
    ex_u, ex_phi = D.arkadiev_lump(X, Y, 0.4), _lump_phi(X, Y, 0.4)
    return (float(np.linalg.norm(u - ex_u) / np.linalg.norm(ex_u)),
            float(np.linalg.norm(phi - ex_phi) / np.linalg.norm(ex_phi)))


@pytest.mark.parametrize("L,h,pu,pphi", read_golden("table7_ds_case1_fft.txt"))
def test_table7_moving_lump_standard_fft_solver(L, h, pu, pphi):
    eu, ephi = _lump_errors(L, h, standard=True)
    assert abs(eu / pu - 1.0) <= 0.006 and abs(ephi / pphi - 1.0) <= 0.006, (eu, ephi)


@pytest.mark.parametrize("L,h,pu,pphi", read_golden("table8_ds_case1_nufft_full.txt"))
def test_table8_moving_lump_split_solver(L, h, pu, pphi):
    eu, ephi = _lump_errors(L, h, standard=False)
    assert abs(eu / pu - 1.0) <= 0.006 and abs(ephi / pphi - 1.0) <= 0.006, (eu, ephi)


# ------------------------------------------------- config 4 at its stated sizes
# u on 1024^2, [-32, 32)^2, the u-generator of the 4096^2 workload (16 complex
# Gaussians), P = 8, 64 x 256 polar nodes; loss L = sum w Phi(|u|^2) with
# seeded Gaussian-random w; gradients through the hand-written adjoint chain
# (dsnu_solve_adjoint, then dsnu_ds_abs2_vjp).

def _config4(prec):
    n, L = 1024, 32.0
    solver, ds = _plans(n, L, prec, P=8.0, n_r=64, n_theta=256, sigma=0.0)
    u_np = synth.wavefunction_sum(n, n, L, L, seed=3, count=16)
    w_np = synth.normal_field(n, n, seed=4)
    return n, L, solver, ds, u_np, w_np


def _wave_loss_grad(u, w, ds, solver):
    from paper_1409_2014_gb300.ds import potential_of_wave

    u = u.detach().clone().requires_grad_(True)
    loss = (w * potential_of_wave(u, ds, solver)).sum()
    loss.backward()
    return float(loss.detach()), u.grad


_ADJ_1024 = {}


def _oracle_adjoint_1024(w_np):
    if "a" not in _ADJ_1024:
        p = OracleParams(nx=1024, ny=1024, lx=32.0, ly=32.0, cut_radius=8.0, n_r=64, n_theta=256)
        _ADJ_1024["a"] = oracle.solve_adjoint(w_np, p)  # the transposed direct sums on the full grid
    return _ADJ_1024["a"]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_config4_gradient_vs_oracle_transposed_sums_1024(prec):
    """dL/du = 2 (A^T w) u on the whole 1024^2 grid: complex128 u with FP64
    plans to <= 1e-12, complex64 u with mixed plans to <= 2e-5 (relative L-inf)."""
    n, L, solver, ds, u_np, w_np = _config4(prec)
    _, g = _wave_loss_grad(torch.from_numpy(u_np).to(CDT[prec]).cuda(), torch.from_numpy(w_np).cuda(), ds, solver)
    ref = 2.0 * _oracle_adjoint_1024(w_np) * u_np.astype(np.complex64 if prec == "mixed" else np.complex128)
    g = g.to(torch.complex128).cpu().numpy()
    assert np.abs(g - ref).max() <= TOL[prec] * np.abs(ref).max()
    solver.close()
    ds.close()


def test_config4_central_differences_16_directions_64_entries():
    """complex128 on 1024^2, h = 1e-6: 16 seeded random directions and 64
    single entries (real and imaginary parts of seeded grid points where the
    gradient is not negligible) against the adjoint's directional derivatives."""
    from paper_1409_2014_gb300.ds import potential_of_wave

    n, L, solver, ds, u_np, w_np = _config4("fp64")
    u = torch.from_numpy(u_np).cuda()
    w = torch.from_numpy(w_np).cuda()
    _, g = _wave_loss_grad(u, w, ds, solver)

    def L_of(v):
        with torch.no_grad():
            return float((w * potential_of_wave(v, ds, solver)).sum())

    h = 1e-6
    # rounding noise of a loss difference: the two evaluations' rounding errors
    # (a few ulps per term, random signs) add up like the L2 norm of the terms
    scale = float(torch.linalg.vector_norm(w * potential_of_wave(u, ds, solver)))
    noise = 16 * np.finfo(np.float64).eps * scale / h
    gen = torch.Generator(device="cpu").manual_seed(16)
    for _ in range(16):
        d = torch.complex(torch.randn(n, n, generator=gen, dtype=torch.float64),
                          torch.randn(n, n, generator=gen, dtype=torch.float64)).cuda()
        fd = (L_of(u + h * d) - L_of(u - h * d)) / (2 * h)
        an = float((g.real * d.real + g.imag * d.imag).sum())
        assert abs(fd - an) <= 1e-7 * abs(an) + noise, (fd, an)
    gmag = g.abs().cpu().numpy()
    cand = np.flatnonzero(gmag.ravel() > 0.05 * gmag.max())
    pick = np.random.Generator(np.random.PCG64(64)).choice(cand, size=64, replace=False)
    for k, idx in enumerate(pick):
        iy, ix = divmod(int(idx), n)
        unit = 1.0 if k % 2 == 0 else 1j
        d = torch.zeros(n, n, dtype=torch.complex128, device="cuda")
        d[iy, ix] = unit
        fd = (L_of(u + h * d) - L_of(u - h * d)) / (2 * h)
        an = float(g[iy, ix].real) if k % 2 == 0 else float(g[iy, ix].imag)
        assert abs(fd - an) <= 1e-6 * abs(an) + noise, (iy, ix, fd, an)
    solver.close()
    ds.close()


def test_config4_complex64_gradient_vs_fp64_adjoint_1024():
    """The complex64 / mixed-precision gradient against the FP64 adjoint
    (complex128 / FP64 plans) on the same u (FD is meaningless in FP32)."""
    grads = {}
    for prec in ("fp64", "mixed"):
        n, L, solver, ds, u_np, w_np = _config4(prec)
        _, g = _wave_loss_grad(torch.from_numpy(u_np).to(CDT[prec]).cuda(), torch.from_numpy(w_np).cuda(), ds,
                               solver)
        grads[prec] = g.to(torch.complex128).cpu().numpy()
        solver.close()
        ds.close()
    ref = grads["fp64"]
    assert np.abs(grads["mixed"] - ref).max() <= 2e-5 * np.abs(ref).max()


def test_config4_200_steps_complex64_checkpointed():
    """complex64 u on 1024^2, 200 Strang steps (alpha = beta = 1, dt = 1e-3):
    mass conserved to FP32 rounding, the checkpointed gradient equals the
    full-tape gradient, and it follows the complex128 gradient."""
    from paper_1409_2014_gb300.ds import evolve, mass

    steps, tau = 200, 1e-3
    out_grads = {}
    for prec in ("mixed", "fp64"):
        n, L, solver, ds, u_np, w_np = _config4(prec)
        u0 = torch.from_numpy(u_np).to(CDT[prec]).cuda()
        w = torch.from_numpy(w_np).cuda()
        gs = []
        for ck in ((14, 0) if prec == "mixed" else (14,)):
            u = u0.clone().requires_grad_(True)
            out = evolve(u, steps, ds, solver, tau, 1.0, 1.0, checkpoint_every=ck)
            if prec == "mixed" and ck:
                m0, m1 = mass(u0.to(torch.complex128), L, L), mass(out.detach().to(torch.complex128), L, L)
                assert abs(m1 / m0 - 1.0) < 1e-4
            (w * (out.real.double() ** 2 + out.imag.double() ** 2)).sum().backward()
            gs.append(u.grad.to(torch.complex128).clone())
        if prec == "mixed":
            assert torch.allclose(gs[0], gs[1], rtol=0, atol=1e-5 * float(gs[1].abs().max()))
        out_grads[prec] = gs[0].cpu().numpy()
        solver.close()
        ds.close()
    ref = out_grads["fp64"]
    assert np.abs(out_grads["mixed"] - ref).max() <= 1e-3 * np.abs(ref).max()
