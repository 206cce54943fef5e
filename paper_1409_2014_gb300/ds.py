"""Differentiable potential and split-step DS time loop on the GPU.

* ``potential(rho, plan)``: Phi = A rho through the C ABI, differentiable; its
  backward is ``dsnu_solve_adjoint`` (the transposed pipeline).
* ``potential_of_wave(u, ds, plan)``: Phi(|u|^2) as a function of the wave
  function u, differentiable; its backward is the hand-written adjoint chain
  A^T (``dsnu_solve_adjoint``) then 2 g u (``dsnu_ds_abs2_vjp``).
* ``strang_step(u, ...)``: one Strang step of the time-splitting spectral
  method (Sec. 2.3 of the paper, in its symmetric form): half a linear flow,
  a full nonlinear flow with Phi = A |u|^2 frozen, half a linear flow.  Both
  flows and their vector-Jacobian products run in the library's kernels.
* ``yoshida_step(u, ...)``: one step of the fourth-order composition the paper
  integrates with (Sec. 2.3): four linear and three nonlinear sub-flows.
* ``evolve(u0, steps, ...)``: many steps of either scheme, optionally with
  checkpointed recomputation (torch.utils.checkpoint) every
  ``checkpoint_every`` steps.

Gradients follow PyTorch's convention for complex inputs of a real loss:
dL/dRe + i dL/dIm.
"""

from __future__ import annotations

import torch
import torch.utils.checkpoint as _ckpt

from . import _abi
from . import Plan

_PREC = {"fp64": _abi.DSNU_FP64, "mixed": _abi.DSNU_MIXED}


def _stream(dev):
    return torch.cuda.current_stream(dev).cuda_stream


class DSPlan:
    """Unpadded periodic transform and pointwise kernels for u on [-lx,lx) x [-ly,ly).

    precision "fp64" works on complex128 fields, "mixed" on complex64."""

    def __init__(self, nx, ny=None, lx=None, ly=None, precision="fp64", device=None):
        ny = nx if ny is None else ny
        ly = lx if ly is None else ly
        dev = torch.device(device if device is not None else "cuda")
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.shape = (int(ny), int(nx))
        self.precision = precision
        self.cdtype = torch.complex128 if precision == "fp64" else torch.complex64
        prm = _abi.dsnu_ds_params(nx=int(nx), ny=int(ny), lx=float(lx), ly=float(ly),
                                  precision=_PREC[precision], reserved=0)
        with torch.cuda.device(dev):
            self._h = _abi.dsnu_ds_plan_create(prm, _stream(dev))

    def _chk(self, u):
        if u.dtype != self.cdtype or tuple(u.shape) != self.shape or not u.is_contiguous() \
                or u.device != self.device:
            raise ValueError(f"expected a contiguous {self.cdtype} tensor of shape {self.shape} on "
                             f"{self.device}")

    def set_linear_step(self, tau, alpha):
        _abi.dsnu_ds_set_linear_step(self._h, tau, alpha, _stream(self.device))

    def linear_(self, u, adjoint=False):
        self._chk(u)
        _abi.dsnu_ds_linear(self._h, u.data_ptr(), 1 if adjoint else 0, _stream(self.device))
        return u

    def abs2(self, u):
        self._chk(u)
        rho = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        _abi.dsnu_ds_abs2(self._h, u.data_ptr(), rho.data_ptr(), _stream(self.device))
        return rho

    def abs2_vjp(self, u, g_rho):
        """2 g_rho u: the gradient with respect to u through rho = |u|^2."""
        self._chk(u)
        grad = torch.empty_like(u)
        _abi.dsnu_ds_abs2_vjp(self._h, u.data_ptr(), g_rho.contiguous().data_ptr(), grad.data_ptr(),
                              _stream(self.device))
        return grad

    def nonlinear_(self, u, phi, tau, beta):
        self._chk(u)
        _abi.dsnu_ds_nonlinear(self._h, u.data_ptr(), phi.data_ptr(), tau, beta, _stream(self.device))
        return u

    def nonlinear_vjp(self, u, phi, g, tau, beta):
        self._chk(u)
        self._chk(g)
        s = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        part = torch.empty_like(u)
        _abi.dsnu_ds_nonlinear_vjp(self._h, u.data_ptr(), phi.data_ptr(), g.data_ptr(), tau, beta,
                                   s.data_ptr(), part.data_ptr(), _stream(self.device))
        return s, part

    def nonlinear_vjp_finish_(self, u, s, ats, tau, beta, part):
        _abi.dsnu_ds_nonlinear_vjp_finish(self._h, u.data_ptr(), s.data_ptr(), ats.data_ptr(), tau, beta,
                                          part.data_ptr(), _stream(self.device))
        return part

    def close(self):
        if getattr(self, "_h", None):
            torch.cuda.synchronize(self.device)
            _abi.dsnu_ds_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- potential

class PotentialFn(torch.autograd.Function):
    """Phi = A rho; backward: A^T g by the transposed pipeline."""

    @staticmethod
    def forward(ctx, rho, plan: Plan):
        ctx.plan = plan
        return plan.solve(rho.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.solve_adjoint(g.contiguous()), None


def potential(rho, plan: Plan):
    return PotentialFn.apply(rho, plan)


class PotentialOfWaveFn(torch.autograd.Function):
    """Phi = A |u|^2; backward: grad_u = 2 (A^T g) u, both steps in the library's kernels."""

    @staticmethod
    def forward(ctx, u, ds: DSPlan, plan: Plan):
        u = u.contiguous()
        ctx.save_for_backward(u)
        ctx.ds, ctx.plan = ds, plan
        return plan.solve(ds.abs2(u))

    @staticmethod
    def backward(ctx, g):
        (u,) = ctx.saved_tensors
        return ctx.ds.abs2_vjp(u, ctx.plan.solve_adjoint(g.contiguous())), None, None


def potential_of_wave(u, ds: DSPlan, plan: Plan):
    return PotentialOfWaveFn.apply(u, ds, plan)


# --------------------------------------------------------------------------- DS flows

class LinearFlow(torch.autograd.Function):
    """u -> F^-1[e^{-i tau (k_x^2 - alpha k_y^2)} F u]; backward: the inverse flow."""

    @staticmethod
    def forward(ctx, u, ds: DSPlan, tau, alpha):
        ctx.ds, ctx.tau, ctx.alpha = ds, tau, alpha
        ds.set_linear_step(tau, alpha)
        return ds.linear_(u.contiguous().clone())

    @staticmethod
    def backward(ctx, g):
        ctx.ds.set_linear_step(ctx.tau, ctx.alpha)
        return ctx.ds.linear_(g.contiguous().clone(), adjoint=True), None, None, None


class NonlinearFlow(torch.autograd.Function):
    """u -> u e^{i tau (2 beta |u|^2 + 4 beta Phi(|u|^2))}."""

    @staticmethod
    def forward(ctx, u, ds: DSPlan, solver: Plan, tau, beta):
        u = u.contiguous()
        phi = solver.solve(ds.abs2(u))
        ctx.save_for_backward(u, phi)
        ctx.ds, ctx.solver, ctx.tau, ctx.beta = ds, solver, tau, beta
        return ds.nonlinear_(u.clone(), phi, tau, beta)

    @staticmethod
    def backward(ctx, g):
        u, phi = ctx.saved_tensors
        ds, solver = ctx.ds, ctx.solver
        s, part = ds.nonlinear_vjp(u, phi, g.contiguous(), ctx.tau, ctx.beta)
        ats = solver.solve_adjoint(s)
        return ds.nonlinear_vjp_finish_(u, s, ats, ctx.tau, ctx.beta, part), None, None, None, None


def strang_step(u, ds: DSPlan, solver: Plan, tau, alpha, beta):
    """One Strang step: L(tau/2) N(tau) L(tau/2) (Sec. 2.3)."""
    u = LinearFlow.apply(u, ds, 0.5 * tau, alpha)
    u = NonlinearFlow.apply(u, ds, solver, tau, beta)
    return LinearFlow.apply(u, ds, 0.5 * tau, alpha)


_CBRT2 = 2.0 ** (1.0 / 3.0)
# Sec. 2.3: b1 = b3 = 1/(2 - 2^(1/3)), b2 = -2^(1/3) b3, a1 = a4 = b3/2,
# a2 = a3 = (b3 + b2)/2
YOSHIDA_B = (1.0 / (2.0 - _CBRT2), -_CBRT2 / (2.0 - _CBRT2), 1.0 / (2.0 - _CBRT2))
YOSHIDA_A = (0.5 * YOSHIDA_B[0], 0.5 * (YOSHIDA_B[0] + YOSHIDA_B[1]),
             0.5 * (YOSHIDA_B[0] + YOSHIDA_B[1]), 0.5 * YOSHIDA_B[0])


def yoshida_step(u, ds: DSPlan, solver: Plan, tau, alpha, beta):
    """u <- A(a1 tau) B(b1 tau) A(a2 tau) B(b2 tau) A(a3 tau) B(b3 tau) A(a4 tau) u
    (Sec. 2.3; the rightmost sub-flow acts first).  Each nonlinear sub-flow
    freezes Phi of the field it starts from."""
    u = LinearFlow.apply(u, ds, YOSHIDA_A[3] * tau, alpha)
    for j in (2, 1, 0):
        u = NonlinearFlow.apply(u, ds, solver, YOSHIDA_B[j] * tau, beta)
        u = LinearFlow.apply(u, ds, YOSHIDA_A[j] * tau, alpha)
    return u


_SCHEMES = {"strang": strang_step, "yoshida": yoshida_step}


def evolve(u0, steps, ds: DSPlan, solver: Plan, tau, alpha, beta, checkpoint_every=0, scheme="strang"):
    """``steps`` steps of ``scheme`` ("strang" or "yoshida"); with
    checkpoint_every > 0 only the input of every segment of that many steps is
    kept for the backward pass, and each segment is recomputed during backward."""
    step = _SCHEMES[scheme]

    def segment(u, n):
        for _ in range(n):
            u = step(u, ds, solver, tau, alpha, beta)
        return u

    u = u0
    if checkpoint_every and checkpoint_every > 0:
        done = 0
        while done < steps:
            n = min(checkpoint_every, steps - done)
            u = _ckpt.checkpoint(segment, u, n, use_reentrant=False)
            done += n
        return u
    return segment(u, steps)


def mass(u, lx, ly):
    """sum |u|^2 h_x h_y (conserved by both flows)."""
    ny, nx = u.shape
    return float((u.abs() ** 2).sum()) * (2 * lx / nx) * (2 * ly / ny)
