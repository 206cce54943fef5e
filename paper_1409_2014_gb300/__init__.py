"""GB300 (sm_103a) split nonlocal potential solver for the Davey-Stewartson
equations: Phi = F^-1[-k_x^2/|k|^2 rho_hat] evaluated as I1 (zero-padded FFT,
high frequencies) + I2 (polar Gauss quadrature via type-2 / type-1 NUFFTs),
after Mauser, Stimming, Zhang (Sec. 2.1).

The compute runs in the C-ABI library ``libdsnufft.so`` (include/dsnufft.h);
this module only marshals arguments.  PyTorch supplies device memory and
streams.
"""

from __future__ import annotations

from . import _abi
from ._abi import (  # noqa: F401
    DSNU_FP64, DSNU_MIXED, DSNU_PARTITION_GAUSS, DSNU_PARTITION_SHARP, DSNU_PARTITION_NONE, DsnuError,
    dsnu_last_error, dsnu_params, dsnu_plan_create, dsnu_plan_destroy, dsnu_plan_get_info,
    dsnu_set_workspace, dsnu_solve, dsnu_solve_adjoint, dsnu_status_poll, dsnu_workspace_bytes,
    dsnu_solve_host, dsnu_profile_begin, dsnu_profile_end, dsnu_stage_count, dsnu_stage_name,
)

_PREC = {"fp64": DSNU_FP64, "mixed": DSNU_MIXED}
_PART = {"gauss": DSNU_PARTITION_GAUSS, "sharp": DSNU_PARTITION_SHARP, "none": DSNU_PARTITION_NONE}
_RADIAL = {"legendre": _abi.DSNU_RADIAL_LEGENDRE, "jacobi": _abi.DSNU_RADIAL_JACOBI}
_ACCUM = {"fp64": _abi.DSNU_ACCUM_FP64, "working": _abi.DSNU_ACCUM_WORKING}


def make_params(nx, ny, lx, ly, cut_radius, n_r, n_theta, sigma=0.0, kernel_width=0,
                precision="fp64", partition="gauss", radial="legendre", accumulation="fp64") -> dsnu_params:
    """partition "none" selects the standard periodic FFT solver (no split, no
    padding: pad_factor 1); the polar parameters are then ignored.  radial:
    "legendre" or "jacobi" (the radial rule of the polar quadrature).
    accumulation: how a mixed plan adds Phi = I1 + I2, "fp64" (each FP32 term
    widened and added in FP64) or "working" (added in FP32)."""
    standard = partition == "none"
    return dsnu_params(nx=int(nx), ny=int(ny), lx=float(lx), ly=float(ly),
                       cut_radius=float(cut_radius or 0.0), sigma=float(sigma), n_r=int(n_r or 0),
                       n_theta=int(n_theta or 0), kernel_width=int(kernel_width),
                       pad_factor=1 if standard else 2,
                       precision=_PREC[precision], partition=_PART[partition],
                       radial_rule=_RADIAL[radial], accumulation=_ACCUM[accumulation])


class Plan:
    """A solver plan on one CUDA device with a torch-owned workspace.

    ``solve(rho)`` takes a contiguous float64 (ny, nx) CUDA tensor and returns
    Phi (float64, same shape), enqueued on the current torch stream.
    ``multiplier=(alpha, a0, a_cos, a_sin)`` selects m(k) = |k|^alpha (a0 +
    a_cos cos 2theta + a_sin sin 2theta) instead of the DS -k_x^2/|k|^2."""

    def __init__(self, nx, ny=None, lx=None, ly=None, cut_radius=None, n_r=None, n_theta=None,
                 sigma=0.0, kernel_width=0, precision="fp64", partition="gauss", radial="legendre",
                 device=None, params=None, multiplier=None, accumulation="fp64"):
        import torch

        ny = nx if ny is None else ny
        ly = lx if ly is None else ly
        dev = torch.device(device if device is not None else "cuda")
        if dev.type != "cuda":
            raise ValueError("the solver runs on CUDA devices only")
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.params = params if params is not None else make_params(
            nx, ny, lx, ly, cut_radius, n_r, n_theta, sigma, kernel_width, precision, partition, radial,
            accumulation)
        self.shape = (int(ny), int(nx))
        self._handle = None
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            if multiplier is None:
                self._handle = dsnu_plan_create(self.params, stream)
            else:
                alpha, a0, a_cos, a_sin = multiplier
                self.multiplier = _abi.dsnu_multiplier(alpha=int(alpha), reserved=0, a0=float(a0),
                                                       a_cos=float(a_cos), a_sin=float(a_sin))
                self._handle = _abi.dsnu_plan_create_multiplier(self.params, self.multiplier, stream)
            nbytes = dsnu_workspace_bytes(self._handle)
            self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
            dsnu_set_workspace(self._handle, self.workspace.data_ptr(), self.workspace.numel())
        self.info = dsnu_plan_get_info(self._handle)

    @classmethod
    def auto(cls, nx, ny=None, lx=None, ly=None, eps=1e-12, precision="fp64", device=None):
        """A plan whose polar part is chosen for the target accuracy eps
        (dsnu_params_auto: sigma = 12/min(l), P = sigma sqrt(ln 1/eps),
        Gauss-Jacobi radial rule, node counts from P sqrt(lx^2 + ly^2))."""
        ny = nx if ny is None else ny
        ly = lx if ly is None else ly
        prm = _abi.dsnu_params_auto(nx, ny, lx, ly, eps, _PREC[precision])
        return cls(nx, ny, lx, ly, precision=precision, device=device, params=prm)

    @property
    def handle(self) -> int:
        return self._handle

    def _check_input(self, x):
        import torch

        if not isinstance(x, torch.Tensor) or x.dtype != torch.float64:
            raise TypeError("expected a float64 torch tensor")
        if x.device != self.device:
            raise ValueError(f"tensor on {x.device}, plan on {self.device}")
        if tuple(x.shape) != self.shape:
            raise ValueError(f"expected shape {self.shape}, got {tuple(x.shape)}")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")

    def _run(self, fn, x, out):
        import torch

        self._check_input(x)
        if out is None:
            out = torch.empty_like(x)
        else:
            self._check_input(out)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        fn(self._handle, x.data_ptr(), out.data_ptr(), stream)
        return out

    def solve(self, rho, out=None):
        return self._run(dsnu_solve, rho, out)

    def solve_adjoint(self, g, out=None):
        return self._run(dsnu_solve_adjoint, g, out)

    def solve_host(self, rho_host, phi_host, rho_dev, phi_dev):
        """Host-buffer solve: rho_host/phi_host are (pinned) CPU float64
        tensors, rho_dev/phi_dev device staging tensors; asynchronous on the
        current stream (synchronise before reading phi_host)."""
        import torch

        for t in (rho_host, phi_host):
            if t.device.type != "cpu" or t.dtype != torch.float64 or tuple(t.shape) != self.shape \
                    or not t.is_contiguous():
                raise ValueError("host buffers must be contiguous float64 CPU tensors of the grid shape")
        self._check_input(rho_dev)
        self._check_input(phi_dev)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        dsnu_solve_host(self._handle, rho_host.data_ptr(), phi_host.data_ptr(), rho_dev.data_ptr(),
                        phi_dev.data_ptr(), stream)
        return phi_host

    def solve_host_stream(self, rho_hosts, phi_hosts):
        """Streams host densities through the plan with overlapped copies
        (dsnu_solve_host_stream): rho_hosts[i] -> phi_hosts[i], contiguous
        float64 CPU tensors of the grid shape (pinned for asynchronous copies);
        a tensor may appear several times.  Asynchronous on the current stream
        (synchronise before reading the results).  The device staging (four
        grid-sized slots) is allocated once and kept by the plan object."""
        import torch

        if len(rho_hosts) != len(phi_hosts) or not rho_hosts:
            raise ValueError("rho_hosts and phi_hosts must have the same, non-zero length")
        for t in list(rho_hosts) + list(phi_hosts):
            if t.device.type != "cpu" or t.dtype != torch.float64 or tuple(t.shape) != self.shape \
                    or not t.is_contiguous():
                raise ValueError("host buffers must be contiguous float64 CPU tensors of the grid shape")
        nbytes = _abi.dsnu_stream_staging_bytes(self._handle)
        if getattr(self, "_staging", None) is None or self._staging.numel() < nbytes:
            self._staging = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        _abi.dsnu_solve_host_stream(self._handle, [t.data_ptr() for t in rho_hosts],
                                    [t.data_ptr() for t in phi_hosts], self._staging.data_ptr(),
                                    self._staging.numel(), stream)
        return phi_hosts

    def profile_begin(self, max_solves: int) -> None:
        dsnu_profile_begin(self._handle, max_solves)

    def profile_end(self):
        """{stage name: total ms} over the recorded solves, and their count."""
        ms, n = dsnu_profile_end(self._handle)
        return {dsnu_stage_name(i): ms[i] for i in range(len(ms))}, n

    def status_poll(self) -> int:
        import torch

        return dsnu_status_poll(self._handle, torch.cuda.current_stream(self.device).cuda_stream)

    def close(self):
        if self._handle is not None:
            import torch

            torch.cuda.synchronize(self.device)
            dsnu_plan_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_SCHEDULE = {"auto": _abi.DSNU_BATCH_AUTO, "stage_launches": _abi.DSNU_BATCH_STAGE_LAUNCHES,
             "forked_streams": _abi.DSNU_BATCH_FORKED_STREAMS}


class Batch:
    """Many densities per launch sequence (members may use different plans).

    ``Batch(plans, rhos, phis)`` binds device tensors; ``solve()`` runs every
    member; ``capture_graph()`` records the launch sequence as a CUDA graph
    that ``solve()`` then replays.  ``schedule``: "stage_launches" (one launch
    per pipeline stage for all grid sizes), "forked_streams" (one launch
    sequence per plan on forked streams) or "auto" (the faster on this GPU:
    forked streams); ``schedule_in_use`` and ``launches`` report the result."""

    def __init__(self, plans, rhos, phis, schedule="auto"):
        import torch

        if not (len(plans) == len(rhos) == len(phis)) or not plans:
            raise ValueError("plans, rhos and phis must have the same, non-zero length")
        for p, r, f in zip(plans, rhos, phis):
            p._check_input(r)
            p._check_input(f)
        self.plans, self.rhos, self.phis = list(plans), list(rhos), list(phis)
        self.device = plans[0].device
        self._h = _abi.dsnu_batch_create([p.handle for p in plans])
        _abi.dsnu_batch_set_schedule(self._h, _SCHEDULE[schedule])
        nbytes = _abi.dsnu_batch_workspace_bytes(self._h)
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        _abi.dsnu_batch_bind(self._h, [r.data_ptr() for r in rhos], [f.data_ptr() for f in phis],
                             self.workspace.data_ptr(), self.workspace.numel(),
                             torch.cuda.current_stream(self.device).cuda_stream)

    @property
    def schedule_in_use(self) -> str:
        return {_abi.DSNU_BATCH_STAGE_LAUNCHES: "stage_launches",
                _abi.DSNU_BATCH_FORKED_STREAMS: "forked_streams"}[_abi.dsnu_batch_schedule(self._h)]

    @property
    def launches(self) -> int:
        """Kernel launches of one batch solve."""
        return _abi.dsnu_batch_launches(self._h)

    def capture_graph(self):
        import torch

        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        _abi.dsnu_batch_capture_graph(self._h, s.cuda_stream)
        torch.cuda.current_stream(self.device).wait_stream(s)

    def solve(self):
        import torch

        _abi.dsnu_batch_solve(self._h, torch.cuda.current_stream(self.device).cuda_stream)
        return self.phis

    def close(self):
        if getattr(self, "_h", None):
            import torch

            torch.cuda.synchronize(self.device)
            _abi.dsnu_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
