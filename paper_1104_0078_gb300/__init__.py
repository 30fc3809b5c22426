"""GB300 library for the hybrid model-H solver of arXiv:1104.0078 -- Python binding.

Thin ctypes marshalling over the C ABI declared in ``include/flb.h``: every
function keeps its C name (``flb_init``, ``flb_step``, ``flb_moments``,
``flb_structure_factor`` ...).  PyTorch only provides the device workspace
(a uint8 tensor) and the CUDA stream; every step of the solver runs in the
library's own CUDA kernels.  There is no CPU fallback: on a machine without the
built library or without a GPU the compute calls raise.

``Solver`` is a convenience owner of one handle, its workspace and stream.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libflb.so")

FLB_OK, FLB_EINVAL, FLB_ENOSPC, FLB_ECUDA, FLB_ENONFINITE, FLB_ETIMEOUT, FLB_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
FLB_FD, FLB_FV, FLB_NAIVE = 0, 1, 2
FLB_LAP_SO, FLB_LAP_CD, FLB_LAP_PK, FLB_LAP_LB = 0, 1, 2, 3
FLB_EULER, FLB_HEUN, FLB_RK4 = 1, 2, 4
FLB_F32_DEV, FLB_F16_DEV = 0, 1
FLB_COUPLE_FORCE, FLB_COUPLE_ADVECT = 1, 2
FLB_FORCE_MATCHED, FLB_FORCE_CD, FLB_FORCE_FV, FLB_FORCE_STRESS = 0, 1, 2, 3
FLB_SQ_PSI, FLB_SQ_HEIGHT, FLB_SQ_DYNAMIC = 0, 1, 2
FLB_MODE_PLAIN, FLB_MODE_BATCHED, FLB_MODE_PERSISTENT = 0, 1, 2
FLB_TUNE_FORCE = 1
FLB_INIT_REST, FLB_INIT_EQUILIBRIUM, FLB_INIT_USER = 0, 1, 2


class FlbParams(ctypes.Structure):
    """Mirror of ``flb_params`` (include/flb.h)."""
    _fields_ = [
        ("dim", ctypes.c_int32), ("q", ctypes.c_int32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("rho0", ctypes.c_double), ("tau", ctypes.c_double),
        ("gamma_bulk", ctypes.c_double), ("gamma_ghost", ctypes.c_double),
        ("kT", ctypes.c_double), ("A", ctypes.c_double), ("B", ctypes.c_double),
        ("K", ctypes.c_double), ("M", ctypes.c_double),
        ("psi_scheme", ctypes.c_int32), ("integrator", ctypes.c_int32),
        ("storage", ctypes.c_int32), ("coupling", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("sq_kmax", ctypes.c_int32), ("force_grad", ctypes.c_int32),
        ("sq_lags", ctypes.c_int32), ("laplacian", ctypes.c_int32),
        ("init", ctypes.c_int32),
    ]


class FlbError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {flb_strerror(code)} ({code})")


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libflb.so (built by ``build_lib.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"the CUDA library {path} is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P, c_int, c_i64, c_sz, vp = ctypes.POINTER, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p
    dp = P(ctypes.c_double)
    H = vp
    sig = {
        "flb_params_default": (None, [P(FlbParams)]),
        "flb_workspace_bytes": (c_sz, [P(FlbParams), ctypes.c_int32]),
        "flb_init": (c_int, [P(FlbParams), ctypes.c_int32, vp, c_sz, vp, P(vp)]),
        "flb_set_fields": (c_int, [H, ctypes.c_int32, dp, dp, dp]),
        "flb_get_populations": (c_int, [H, ctypes.c_int32, dp]),
        "flb_set_populations": (c_int, [H, ctypes.c_int32, dp]),
        "flb_get_psi_u": (c_int, [H, ctypes.c_int32, dp, dp]),
        "flb_get_window": (c_int, [H, ctypes.c_int32] + [ctypes.c_int32] * 6 + [dp, dp]),
        "flb_step": (c_int, [H, c_i64]),
        "flb_get_step": (c_int, [H, ctypes.c_int32, P(c_i64)]),
        "flb_moments": (c_int, [H, ctypes.c_int32, dp, dp]),
        "flb_mode_variances": (c_int, [H, ctypes.c_int32, dp]),
        "flb_set_sampling": (c_int, [H, ctypes.c_int32, ctypes.c_int32]),
        "flb_sample": (c_int, [H, ctypes.c_int32]),
        "flb_structure_factor": (c_int, [H, ctypes.c_int32, ctypes.c_int32, dp, P(c_i64)]),
        "flb_structure_factor_size": (c_i64, [H, ctypes.c_int32, ctypes.c_int32]),
        "flb_sq_reset": (c_int, [H, ctypes.c_int32]),
        "flb_set_mode": (c_int, [H, ctypes.c_int32]),
        "flb_get_tuning": (c_int, [H, ctypes.c_int32, P(ctypes.c_int32)]),
        "flb_set_tuning": (c_int, [H, ctypes.c_int32, ctypes.c_int32]),
        "flb_set_psi_fused": (c_int, [H, ctypes.c_int32]),
        "flb_autotune": (c_int, [H, ctypes.c_char_p, ctypes.c_int32]),
        "flb_set_wait_limit": (c_int, [H, ctypes.c_double]),
        "flb_state_bytes": (c_sz, [H, ctypes.c_int32]),
        "flb_get_state": (c_int, [H, ctypes.c_int32, vp, c_sz]),
        "flb_set_state": (c_int, [H, ctypes.c_int32, vp, c_sz]),
        "flb_synchronize": (c_int, [H]),
        "flb_launch_count": (c_i64, [H]),
        "flb_set_profiling": (c_int, [H, ctypes.c_int32]),
        "flb_kernel_times": (c_int, [H, dp, P(c_i64)]),
        "flb_structure_factor_noalloc": (c_int, [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_int32, vp, vp]),
        "flb_gaussians": (c_int, [ctypes.c_uint64, c_i64, ctypes.c_uint32, ctypes.c_uint32, c_i64, ctypes.c_int32,
                                  vp, vp]),
        "flb_strerror": (ctypes.c_char_p, [c_int]),
        "flb_destroy": (None, [H]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def flb_strerror(code: int) -> str:
    return load_library().flb_strerror(code).decode()


def _check(code: int, where: str):
    if code != FLB_OK:
        raise FlbError(code, where)


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---- functions with the C names (argument marshalling only) -----------------
def flb_params_default(**overrides) -> FlbParams:
    p = FlbParams()
    load_library().flb_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def flb_workspace_bytes(params) -> int:
    arr = _param_array(params)
    return int(load_library().flb_workspace_bytes(arr, len(arr)))


def _param_array(params):
    if isinstance(params, FlbParams):
        params = [params]
    arr = (FlbParams * len(params))(*params)
    return arr


def flb_init(params, workspace_ptr: int, workspace_bytes: int, stream_ptr: int):
    arr = _param_array(params)
    h = ctypes.c_void_p()
    _check(load_library().flb_init(arr, len(arr), ctypes.c_void_p(workspace_ptr), workspace_bytes,
                                   ctypes.c_void_p(stream_ptr), ctypes.byref(h)), "flb_init")
    return h


def flb_step(h, n: int):
    _check(load_library().flb_step(h, n), "flb_step")


def flb_moments(h, rep: int, dim: int):
    tot = np.zeros(2 + dim)
    u2 = np.zeros(dim)
    rc = load_library().flb_moments(h, rep, _dp(tot), _dp(u2))
    if rc not in (FLB_OK, FLB_ENONFINITE):
        _check(rc, "flb_moments")
    return tot, u2, rc


def flb_structure_factor(h, rep: int, which: int):
    n = int(load_library().flb_structure_factor_size(h, rep, which))
    if n < 0:
        raise FlbError(FLB_EINVAL, "flb_structure_factor_size")
    out = np.zeros(max(n, 1))
    ns = ctypes.c_int64()
    _check(load_library().flb_structure_factor(h, rep, which, _dp(out), ctypes.byref(ns)), "flb_structure_factor")
    return out[:n], int(ns.value)


# ---- convenience owner ------------------------------------------------------
def gaussians(seed: int, step: int, stream: int, site0: int, nsites: int, nblocks: int, device="cuda"):
    """The standard normals the kernels draw (flb_gaussians) as a torch tensor
    (nsites, 8*nblocks) on `device`, computed on that device's current stream."""
    import torch
    out = torch.empty((nsites, 8 * nblocks), dtype=torch.float32, device=device)
    st = torch.cuda.current_stream(out.device).cuda_stream
    _check(load_library().flb_gaussians(seed, step, stream, site0, nsites, nblocks, out.data_ptr(), st),
           "flb_gaussians")
    return out


class Solver:
    """One handle over nrep replicas, with its torch-owned workspace and stream."""

    def __init__(self, params, device: str = "cuda:0", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("flb needs a CUDA device; there is no CPU path")
        self.lib = load_library()
        self.params = [params] if isinstance(params, FlbParams) else list(params)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        nbytes = flb_workspace_bytes(self.params)
        if nbytes == 0:
            raise FlbError(FLB_EINVAL, "flb_workspace_bytes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.h = flb_init(self.params, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)

    # geometry helpers
    def n(self, rep=0):
        p = self.params[rep]
        return p.nx * p.ny * (p.nz if p.dim == 3 else 1)

    def shape(self, rep=0):
        p = self.params[rep]
        return (p.nz if p.dim == 3 else 1, p.ny, p.nx)

    def set_fields(self, rep=0, rho=None, u=None, psi=None):
        f = lambda a, shp: None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(shp)
        N, d = self.n(rep), self.params[rep].dim
        _check(self.lib.flb_set_fields(self.h, rep, _dp(f(rho, N)), _dp(f(u, (d, N))), _dp(f(psi, N))),
               "flb_set_fields")

    def get_populations(self, rep=0):
        out = np.zeros((self.params[rep].q, self.n(rep)))
        _check(self.lib.flb_get_populations(self.h, rep, _dp(out)), "flb_get_populations")
        return out

    def set_populations(self, f, rep=0):
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(self.params[rep].q, self.n(rep))
        _check(self.lib.flb_set_populations(self.h, rep, _dp(a)), "flb_set_populations")

    def get_psi_u(self, rep=0):
        psi = np.zeros(self.n(rep))
        u = np.zeros((self.params[rep].dim, self.n(rep)))
        _check(self.lib.flb_get_psi_u(self.h, rep, _dp(psi), _dp(u)), "flb_get_psi_u")
        return psi, u

    def get_psi(self, rep=0):
        """psi [N] alone (flb_get_psi_u with no velocity)."""
        psi = np.zeros(self.n(rep))
        _check(self.lib.flb_get_psi_u(self.h, rep, _dp(psi), None), "flb_get_psi_u")
        return psi

    def get_window(self, origin, size, rep=0):
        W = size[0] * size[1] * size[2]
        f = np.zeros((self.params[rep].q, W))
        psi = np.zeros(W)
        _check(self.lib.flb_get_window(self.h, rep, *origin, *size, _dp(f), _dp(psi)), "flb_get_window")
        return f, psi

    def step(self, n=1):
        flb_step(self.h, n)

    def get_step(self, rep=0):
        s = ctypes.c_int64()
        _check(self.lib.flb_get_step(self.h, rep, ctypes.byref(s)), "flb_get_step")
        return s.value

    def moments(self, rep=0):
        return flb_moments(self.h, rep, self.params[rep].dim)

    def mode_variances(self, rep=0):
        """(1/N) sum_r m_k(r)^2 of every moment mode k (flb_mode_variances), FP64 [q]."""
        out = np.zeros(self.params[rep].q)
        _check(self.lib.flb_mode_variances(self.h, rep, _dp(out)), "flb_mode_variances")
        return out

    def set_sampling(self, every_m, mask=1):
        _check(self.lib.flb_set_sampling(self.h, every_m, mask), "flb_set_sampling")

    def sample(self, mask=1):
        _check(self.lib.flb_sample(self.h, mask), "flb_sample")

    def structure_factor(self, rep=0, which=FLB_SQ_PSI):
        return flb_structure_factor(self.h, rep, which)

    def sq_reset(self, rep=-1):
        _check(self.lib.flb_sq_reset(self.h, rep), "flb_sq_reset")

    def set_mode(self, mode):
        _check(self.lib.flb_set_mode(self.h, mode), "flb_set_mode")

    def set_wait_limit(self, seconds: float):
        _check(self.lib.flb_set_wait_limit(self.h, float(seconds)), "flb_set_wait_limit")

    def get_tuning(self, rep=0) -> int:
        """Planes per psi block (the z chunk) of replica rep."""
        v = ctypes.c_int32()
        _check(self.lib.flb_get_tuning(self.h, rep, ctypes.byref(v)), "flb_get_tuning")
        return int(v.value)

    def set_tuning(self, psi_zchunk: int, rep: int = -1):
        _check(self.lib.flb_set_tuning(self.h, rep, int(psi_zchunk)), "flb_set_tuning")

    def set_psi_fused(self, on=True):
        """Single-pass Heun psi step (flb_set_psi_fused)."""
        _check(self.lib.flb_set_psi_fused(self.h, 1 if on else 0), "flb_set_psi_fused")

    def autotune(self, cache=None, force=False):
        """Time the psi z-chunk candidates on this handle (see flb_autotune); returns
        the chosen value of every replica."""
        path = os.fsencode(cache) if cache is not None else None
        _check(self.lib.flb_autotune(self.h, path, FLB_TUNE_FORCE if force else 0), "flb_autotune")
        return [self.get_tuning(r) for r in range(len(self.params))]

    def get_state(self, rep=0) -> bytes:
        n = int(self.lib.flb_state_bytes(self.h, rep))
        buf = ctypes.create_string_buffer(n)
        _check(self.lib.flb_get_state(self.h, rep, buf, n), "flb_get_state")
        return buf.raw

    def set_state(self, data: bytes, rep=0):
        buf = ctypes.create_string_buffer(data, len(data))
        _check(self.lib.flb_set_state(self.h, rep, buf, len(data)), "flb_set_state")

    def synchronize(self):
        _check(self.lib.flb_synchronize(self.h), "flb_synchronize")

    def launch_count(self) -> int:
        return int(self.lib.flb_launch_count(self.h))

    def set_profiling(self, on: bool):
        _check(self.lib.flb_set_profiling(self.h, int(on)), "flb_set_profiling")

    def kernel_times(self):
        """({'lb','psi','sample'} ms, launch counts) since profiling was switched on."""
        ms = np.zeros(3)
        cnt = (ctypes.c_int64 * 3)()
        _check(self.lib.flb_kernel_times(self.h, _dp(ms), cnt), "flb_kernel_times")
        keys = ("lb", "psi", "sample")
        return dict(zip(keys, ms.tolist())), dict(zip(keys, list(cnt)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.flb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
