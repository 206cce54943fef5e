"""ctypes declarations of the C ABI in include/dsnufft.h (argument marshalling
only; every step of a solve runs in the library's CUDA kernels).

The library is the in-tree ``libdsnufft.so``; there is no fallback: when it is
missing or fails to load, every entry point raises.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdsnufft.so")

DSNU_OK, DSNU_EINVAL, DSNU_ENOMEM, DSNU_ECUDA, DSNU_ETIMEOUT, DSNU_EUNSUPPORTED = range(6)
DSNU_FP64, DSNU_MIXED = 0, 1
DSNU_PARTITION_GAUSS, DSNU_PARTITION_SHARP, DSNU_PARTITION_NONE = 0, 1, 2
DSNU_RADIAL_LEGENDRE, DSNU_RADIAL_JACOBI = 0, 1
DSNU_ACCUM_FP64, DSNU_ACCUM_WORKING = 0, 1
DSNU_BATCH_AUTO, DSNU_BATCH_STAGE_LAUNCHES, DSNU_BATCH_FORKED_STREAMS = 0, 1, 2

STATUS_NAMES = {0: "DSNU_OK", 1: "DSNU_EINVAL", 2: "DSNU_ENOMEM", 3: "DSNU_ECUDA",
                4: "DSNU_ETIMEOUT", 5: "DSNU_EUNSUPPORTED"}

EXPORTED = [
    "dsnu_plan_create", "dsnu_workspace_bytes", "dsnu_set_workspace", "dsnu_solve",
    "dsnu_solve_adjoint", "dsnu_status_poll", "dsnu_plan_destroy", "dsnu_last_error",
    "dsnu_plan_get_info", "dsnu_solve_host", "dsnu_profile_begin", "dsnu_profile_end",
    "dsnu_stage_count", "dsnu_stage_name", "dsnu_solve_noalloc", "dsnu_noalloc_scratch_bytes",
    "dsnu_ds_plan_create", "dsnu_ds_set_linear_step", "dsnu_ds_linear", "dsnu_ds_abs2",
    "dsnu_ds_nonlinear", "dsnu_ds_nonlinear_vjp", "dsnu_ds_nonlinear_vjp_finish", "dsnu_ds_plan_destroy",
    "dsnu_batch_create", "dsnu_batch_workspace_bytes", "dsnu_batch_bind", "dsnu_batch_capture_graph",
    "dsnu_batch_solve", "dsnu_batch_destroy", "dsnu_radial_nodes", "dsnu_params_auto",
    "dsnu_plan_create_multiplier", "dsnu_stream_staging_bytes", "dsnu_solve_host_stream",
    "dsnu_measure_fma_peak", "dsnu_ds_abs2_vjp", "dsnu_batch_set_schedule", "dsnu_batch_schedule",
    "dsnu_batch_launches",
]


class dsnu_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("cut_radius", ctypes.c_double), ("sigma", ctypes.c_double),
        ("n_r", ctypes.c_int32), ("n_theta", ctypes.c_int32),
        ("kernel_width", ctypes.c_int32), ("pad_factor", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("partition", ctypes.c_int32),
        ("radial_rule", ctypes.c_int32), ("accumulation", ctypes.c_int32),
    ]


class dsnu_multiplier(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("a0", ctypes.c_double), ("a_cos", ctypes.c_double), ("a_sin", ctypes.c_double),
    ]


class dsnu_plan_info(ctypes.Structure):
    _fields_ = [
        ("n_nodes", ctypes.c_int32), ("band_q", ctypes.c_int32),
        ("kernel_width", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("sigma", ctypes.c_double), ("es_beta", ctypes.c_double),
        ("n_tiles", ctypes.c_int32), ("max_tile_nodes", ctypes.c_int32),
        ("n_items", ctypes.c_int32), ("spread_tile", ctypes.c_int32),
        ("spread_split", ctypes.c_int32), ("spread_chunk", ctypes.c_int32),
        ("row_prefetch", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class dsnu_ds_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("precision", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class DsnuError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_LIB = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the library and declare every entry point (raises if missing)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not built: run paper_1409_2014_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, st = ctypes.c_void_p, ctypes.c_int
    lib.dsnu_plan_create.argtypes = [ctypes.POINTER(dsnu_params), vp, ctypes.POINTER(vp)]
    lib.dsnu_plan_create.restype = st
    lib.dsnu_workspace_bytes.argtypes = [vp]
    lib.dsnu_workspace_bytes.restype = ctypes.c_size_t
    lib.dsnu_set_workspace.argtypes = [vp, vp, ctypes.c_size_t]
    lib.dsnu_set_workspace.restype = st
    for name in ("dsnu_solve", "dsnu_solve_adjoint"):
        getattr(lib, name).argtypes = [vp, vp, vp, vp]
        getattr(lib, name).restype = st
    lib.dsnu_status_poll.argtypes = [vp, vp]
    lib.dsnu_status_poll.restype = st
    lib.dsnu_plan_destroy.argtypes = [vp]
    lib.dsnu_plan_destroy.restype = st
    lib.dsnu_last_error.argtypes = []
    lib.dsnu_last_error.restype = ctypes.c_char_p
    lib.dsnu_plan_get_info.argtypes = [vp, ctypes.POINTER(dsnu_plan_info)]
    lib.dsnu_plan_get_info.restype = st
    lib.dsnu_solve_host.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.dsnu_solve_host.restype = st
    lib.dsnu_profile_begin.argtypes = [vp, ctypes.c_int]
    lib.dsnu_profile_begin.restype = st
    lib.dsnu_profile_end.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int)]
    lib.dsnu_profile_end.restype = st
    lib.dsnu_radial_nodes.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.dsnu_radial_nodes.restype = st
    lib.dsnu_plan_create_multiplier.argtypes = [ctypes.POINTER(dsnu_params), ctypes.POINTER(dsnu_multiplier), vp,
                                                ctypes.POINTER(vp)]
    lib.dsnu_plan_create_multiplier.restype = st
    lib.dsnu_stream_staging_bytes.argtypes = [vp]
    lib.dsnu_stream_staging_bytes.restype = ctypes.c_size_t
    lib.dsnu_solve_host_stream.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(vp), ctypes.POINTER(vp), vp,
                                           ctypes.c_size_t, vp]
    lib.dsnu_solve_host_stream.restype = st
    lib.dsnu_params_auto.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int32, ctypes.POINTER(dsnu_params)]
    lib.dsnu_params_auto.restype = st
    lib.dsnu_stage_count.argtypes = []
    lib.dsnu_stage_count.restype = ctypes.c_int32
    lib.dsnu_stage_name.argtypes = [ctypes.c_int32]
    lib.dsnu_stage_name.restype = ctypes.c_char_p
    lib.dsnu_solve_noalloc.argtypes = [vp, vp, vp, vp]
    lib.dsnu_solve_noalloc.restype = st
    lib.dsnu_noalloc_scratch_bytes.argtypes = []
    lib.dsnu_noalloc_scratch_bytes.restype = ctypes.c_size_t
    lib.dsnu_measure_fma_peak.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double), vp]
    lib.dsnu_measure_fma_peak.restype = st
    d = ctypes.c_double
    lib.dsnu_batch_set_schedule.argtypes = [vp, ctypes.c_int32]
    lib.dsnu_batch_set_schedule.restype = st
    lib.dsnu_batch_schedule.argtypes = [vp]
    lib.dsnu_batch_schedule.restype = ctypes.c_int32
    lib.dsnu_batch_launches.argtypes = [vp]
    lib.dsnu_batch_launches.restype = ctypes.c_int32
    lib.dsnu_ds_abs2_vjp.argtypes = [vp, vp, vp, vp, vp]
    lib.dsnu_ds_abs2_vjp.restype = st
    lib.dsnu_ds_plan_create.argtypes = [ctypes.POINTER(dsnu_ds_params), vp, ctypes.POINTER(vp)]
    lib.dsnu_ds_set_linear_step.argtypes = [vp, d, d, vp]
    lib.dsnu_ds_linear.argtypes = [vp, vp, ctypes.c_int32, vp]
    lib.dsnu_ds_abs2.argtypes = [vp, vp, vp, vp]
    lib.dsnu_ds_nonlinear.argtypes = [vp, vp, vp, d, d, vp]
    lib.dsnu_ds_nonlinear_vjp.argtypes = [vp, vp, vp, vp, d, d, vp, vp, vp]
    lib.dsnu_ds_nonlinear_vjp_finish.argtypes = [vp, vp, vp, vp, d, d, vp, vp]
    lib.dsnu_ds_plan_destroy.argtypes = [vp]
    for name in ("dsnu_ds_plan_create", "dsnu_ds_set_linear_step", "dsnu_ds_linear", "dsnu_ds_abs2",
                 "dsnu_ds_nonlinear", "dsnu_ds_nonlinear_vjp", "dsnu_ds_nonlinear_vjp_finish",
                 "dsnu_ds_plan_destroy"):
        getattr(lib, name).restype = st
    lib.dsnu_batch_create.argtypes = [ctypes.c_int32, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    lib.dsnu_batch_workspace_bytes.argtypes = [vp]
    lib.dsnu_batch_workspace_bytes.restype = ctypes.c_size_t
    lib.dsnu_batch_bind.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, ctypes.c_size_t, vp]
    lib.dsnu_batch_capture_graph.argtypes = [vp, vp]
    lib.dsnu_batch_solve.argtypes = [vp, vp]
    lib.dsnu_batch_destroy.argtypes = [vp]
    for name in ("dsnu_batch_create", "dsnu_batch_bind", "dsnu_batch_capture_graph", "dsnu_batch_solve",
                 "dsnu_batch_destroy"):
        getattr(lib, name).restype = st
    _LIB = lib
    return lib


def _check(status: int, where: str) -> None:
    if status != DSNU_OK:
        msg = load().dsnu_last_error().decode(errors="replace")
        raise DsnuError(status, where, msg)


# Thin wrappers with the ABI's names ------------------------------------------

def dsnu_plan_create(params: dsnu_params, stream: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(load().dsnu_plan_create(ctypes.byref(params), ctypes.c_void_p(stream), ctypes.byref(out)),
           "dsnu_plan_create")
    return out.value


def dsnu_plan_create_multiplier(params: dsnu_params, mult: dsnu_multiplier, stream: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(load().dsnu_plan_create_multiplier(ctypes.byref(params), ctypes.byref(mult) if mult is not None
                                              else None, ctypes.c_void_p(stream), ctypes.byref(out)),
           "dsnu_plan_create_multiplier")
    return out.value


def dsnu_workspace_bytes(plan: int) -> int:
    return int(load().dsnu_workspace_bytes(ctypes.c_void_p(plan)))


def dsnu_set_workspace(plan: int, ptr: int, nbytes: int) -> None:
    _check(load().dsnu_set_workspace(ctypes.c_void_p(plan), ctypes.c_void_p(ptr), nbytes),
           "dsnu_set_workspace")


def dsnu_solve(plan: int, rho_ptr: int, phi_ptr: int, stream: int = 0) -> None:
    _check(load().dsnu_solve(ctypes.c_void_p(plan), ctypes.c_void_p(rho_ptr),
                             ctypes.c_void_p(phi_ptr), ctypes.c_void_p(stream)), "dsnu_solve")


def dsnu_solve_adjoint(plan: int, g_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _check(load().dsnu_solve_adjoint(ctypes.c_void_p(plan), ctypes.c_void_p(g_ptr),
                                     ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream)),
           "dsnu_solve_adjoint")


def dsnu_status_poll(plan: int, stream: int = 0) -> int:
    return int(load().dsnu_status_poll(ctypes.c_void_p(plan), ctypes.c_void_p(stream)))


def dsnu_plan_destroy(plan: int) -> None:
    _check(load().dsnu_plan_destroy(ctypes.c_void_p(plan)), "dsnu_plan_destroy")


def dsnu_last_error() -> str:
    return load().dsnu_last_error().decode(errors="replace")


def dsnu_plan_get_info(plan: int) -> dsnu_plan_info:
    info = dsnu_plan_info()
    _check(load().dsnu_plan_get_info(ctypes.c_void_p(plan), ctypes.byref(info)), "dsnu_plan_get_info")
    return info


def dsnu_solve_host(plan: int, rho_host: int, phi_host: int, rho_dev: int, phi_dev: int,
                    stream: int = 0) -> None:
    _check(load().dsnu_solve_host(ctypes.c_void_p(plan), ctypes.c_void_p(rho_host),
                                  ctypes.c_void_p(phi_host), ctypes.c_void_p(rho_dev),
                                  ctypes.c_void_p(phi_dev), ctypes.c_void_p(stream)),
           "dsnu_solve_host")


def dsnu_profile_begin(plan: int, max_solves: int) -> None:
    _check(load().dsnu_profile_begin(ctypes.c_void_p(plan), int(max_solves)), "dsnu_profile_begin")


def dsnu_profile_end(plan: int):
    """Returns (per-stage total ms list, number of recorded solves)."""
    n = dsnu_stage_count()
    arr = (ctypes.c_double * n)()
    cnt = ctypes.c_int()
    _check(load().dsnu_profile_end(ctypes.c_void_p(plan), arr, n, ctypes.byref(cnt)),
           "dsnu_profile_end")
    return list(arr), cnt.value


def dsnu_radial_nodes(n_r: int, rule: int, cut_radius: float):
    """(r, w) lists: nodes in (0, P) and weights for int_0^P f(r) r dr (host only)."""
    r = (ctypes.c_double * int(n_r))()
    w = (ctypes.c_double * int(n_r))()
    _check(load().dsnu_radial_nodes(int(n_r), int(rule), float(cut_radius), r, w), "dsnu_radial_nodes")
    return list(r), list(w)


def dsnu_params_auto(nx: int, ny: int, lx: float, ly: float, eps: float, precision: int) -> dsnu_params:
    out = dsnu_params()
    _check(load().dsnu_params_auto(int(nx), int(ny), float(lx), float(ly), float(eps), int(precision),
                                   ctypes.byref(out)), "dsnu_params_auto")
    return out


def dsnu_stream_staging_bytes(plan: int) -> int:
    return int(load().dsnu_stream_staging_bytes(ctypes.c_void_p(plan)))


def dsnu_solve_host_stream(plan: int, rho_hosts, phi_hosts, staging: int, staging_bytes: int,
                           stream: int = 0) -> None:
    n = len(rho_hosts)
    ra = (ctypes.c_void_p * n)(*[ctypes.c_void_p(p) for p in rho_hosts])
    pa = (ctypes.c_void_p * n)(*[ctypes.c_void_p(p) for p in phi_hosts])
    _check(load().dsnu_solve_host_stream(ctypes.c_void_p(plan), n, ra, pa, ctypes.c_void_p(staging),
                                         ctypes.c_size_t(staging_bytes), ctypes.c_void_p(stream)),
           "dsnu_solve_host_stream")


def dsnu_stage_count() -> int:
    return int(load().dsnu_stage_count())


def dsnu_stage_name(i: int) -> str:
    return load().dsnu_stage_name(int(i)).decode()


def dsnu_solve_noalloc(plan: int, rho_ptr: int, phi_ptr: int, stream: int = 0) -> None:
    """dsnu_solve with the library's static scratch instead of a workspace
    (for callers that cannot allocate device memory when they solve)."""
    _check(load().dsnu_solve_noalloc(ctypes.c_void_p(plan), ctypes.c_void_p(rho_ptr),
                                     ctypes.c_void_p(phi_ptr), ctypes.c_void_p(stream)),
           "dsnu_solve_noalloc")


def dsnu_noalloc_scratch_bytes() -> int:
    return int(load().dsnu_noalloc_scratch_bytes())


def dsnu_measure_fma_peak(precision: int, stream: int = 0) -> float:
    """Measured FMA throughput of the current device in flop/s (DSNU_FP64 or
    DSNU_MIXED for FP32)."""
    out = ctypes.c_double()
    _check(load().dsnu_measure_fma_peak(ctypes.c_int32(precision), ctypes.byref(out), ctypes.c_void_p(stream)),
           "dsnu_measure_fma_peak")
    return float(out.value)


def _vp(x):
    return ctypes.c_void_p(x)


def dsnu_ds_plan_create(params: dsnu_ds_params, stream: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(load().dsnu_ds_plan_create(ctypes.byref(params), _vp(stream), ctypes.byref(out)),
           "dsnu_ds_plan_create")
    return out.value


def dsnu_ds_set_linear_step(plan: int, tau: float, alpha: float, stream: int = 0) -> None:
    _check(load().dsnu_ds_set_linear_step(_vp(plan), float(tau), float(alpha), _vp(stream)),
           "dsnu_ds_set_linear_step")


def dsnu_ds_linear(plan: int, u: int, adjoint: int, stream: int = 0) -> None:
    _check(load().dsnu_ds_linear(_vp(plan), _vp(u), int(adjoint), _vp(stream)), "dsnu_ds_linear")


def dsnu_ds_abs2(plan: int, u: int, rho: int, stream: int = 0) -> None:
    _check(load().dsnu_ds_abs2(_vp(plan), _vp(u), _vp(rho), _vp(stream)), "dsnu_ds_abs2")


def dsnu_ds_abs2_vjp(plan: int, u: int, g_rho: int, grad: int, stream: int = 0) -> None:
    _check(load().dsnu_ds_abs2_vjp(_vp(plan), _vp(u), _vp(g_rho), _vp(grad), _vp(stream)), "dsnu_ds_abs2_vjp")


def dsnu_ds_nonlinear(plan: int, u: int, phi: int, tau: float, beta: float, stream: int = 0) -> None:
    _check(load().dsnu_ds_nonlinear(_vp(plan), _vp(u), _vp(phi), float(tau), float(beta), _vp(stream)),
           "dsnu_ds_nonlinear")


def dsnu_ds_nonlinear_vjp(plan, u, phi, g, tau, beta, s, part, stream=0) -> None:
    _check(load().dsnu_ds_nonlinear_vjp(_vp(plan), _vp(u), _vp(phi), _vp(g), float(tau), float(beta),
                                        _vp(s), _vp(part), _vp(stream)), "dsnu_ds_nonlinear_vjp")


def dsnu_ds_nonlinear_vjp_finish(plan, u, s, ats, tau, beta, grad, stream=0) -> None:
    _check(load().dsnu_ds_nonlinear_vjp_finish(_vp(plan), _vp(u), _vp(s), _vp(ats), float(tau),
                                               float(beta), _vp(grad), _vp(stream)),
           "dsnu_ds_nonlinear_vjp_finish")


def dsnu_ds_plan_destroy(plan: int) -> None:
    _check(load().dsnu_ds_plan_destroy(_vp(plan)), "dsnu_ds_plan_destroy")


def dsnu_batch_create(plans) -> int:
    arr = (ctypes.c_void_p * len(plans))(*plans)
    out = ctypes.c_void_p()
    _check(load().dsnu_batch_create(len(plans), arr, ctypes.byref(out)), "dsnu_batch_create")
    return out.value


def dsnu_batch_workspace_bytes(batch: int) -> int:
    return int(load().dsnu_batch_workspace_bytes(_vp(batch)))


def dsnu_batch_bind(batch: int, rho_ptrs, phi_ptrs, ws: int, nbytes: int, stream: int = 0) -> None:
    r = (ctypes.c_void_p * len(rho_ptrs))(*rho_ptrs)
    p = (ctypes.c_void_p * len(phi_ptrs))(*phi_ptrs)
    _check(load().dsnu_batch_bind(_vp(batch), r, p, _vp(ws), nbytes, _vp(stream)), "dsnu_batch_bind")


def dsnu_batch_set_schedule(batch: int, schedule: int) -> None:
    _check(load().dsnu_batch_set_schedule(_vp(batch), ctypes.c_int32(schedule)), "dsnu_batch_set_schedule")


def dsnu_batch_schedule(batch: int) -> int:
    return int(load().dsnu_batch_schedule(_vp(batch)))


def dsnu_batch_launches(batch: int) -> int:
    return int(load().dsnu_batch_launches(_vp(batch)))


def dsnu_batch_capture_graph(batch: int, stream: int = 0) -> None:
    _check(load().dsnu_batch_capture_graph(_vp(batch), _vp(stream)), "dsnu_batch_capture_graph")


def dsnu_batch_solve(batch: int, stream: int = 0) -> None:
    _check(load().dsnu_batch_solve(_vp(batch), _vp(stream)), "dsnu_batch_solve")


def dsnu_batch_destroy(batch: int) -> None:
    _check(load().dsnu_batch_destroy(_vp(batch)), "dsnu_batch_destroy")
