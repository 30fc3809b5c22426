"""CPU checks of the C ABI: the library loads, exports every function that
include/flb.h declares, the ctypes mirror of flb_params has the C layout, and
the host-only entry points validate their arguments (no device calls here)."""
import ctypes
import math
import os
import re
import subprocess
import tempfile

import pytest

import paper_1104_0078_gb300 as F
from paper_1104_0078_gb300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(flb_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return F.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", F.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = sorted(n for n in names if n not in exported)
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_params_layout_matches_c():
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "flb.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(flb_params), offsetof(flb_params, rho0),
             offsetof(flb_params, kT), offsetof(flb_params, psi_scheme), offsetof(flb_params, seed),
             offsetof(flb_params, sq_kmax), offsetof(flb_params, force_grad), offsetof(flb_params, sq_lags));
      return 0; }
    """
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = list(map(int, subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()))
    P = F.FlbParams
    assert vals == [ctypes.sizeof(P), P.rho0.offset, P.kT.offset, P.psi_scheme.offset, P.seed.offset,
                    P.sq_kmax.offset, P.force_grad.offset, P.sq_lags.offset]


def test_defaults_and_workspace_sizing(lib):
    p = F.flb_params_default()
    assert (p.dim, p.q, p.nx, p.psi_scheme, p.integrator, p.coupling) == (3, 19, 32, F.FLB_FV, F.FLB_HEUN, 3)
    assert p.force_grad == F.FLB_FORCE_MATCHED
    assert math.isnan(p.gamma_bulk)
    n32 = F.flb_workspace_bytes(p)
    N = 32 ** 3
    assert n32 > 2 * 19 * N * 4           # two population buffers at least
    p16 = F.flb_params_default(storage=F.FLB_F16_DEV)
    assert F.flb_workspace_bytes(p16) < n32
    # replicas of different sizes share one workspace
    ps = [F.flb_params_default(nx=n, ny=n, nz=n) for n in (16, 24)]
    assert F.flb_workspace_bytes(ps) > F.flb_workspace_bytes(ps[:1])


@pytest.mark.parametrize("field,value", [("nx", 3), ("q", 17), ("q", 27), ("tau", 0.0), ("gamma_ghost", 1.0), ("kT", -1.0),
                                         ("psi_scheme", 3), ("integrator", 3), ("storage", 2), ("coupling", 4),
                                         ("M", -0.1), ("sq_kmax", -1), ("force_grad", 4), ("force_grad", -1),
                                         ("sq_lags", -1), ("sq_lags", 5000), ("laplacian", 4),
                                         ("laplacian", -1), ("psi_scheme", -1)])
def test_invalid_parameters_rejected(lib, field, value):
    p = F.flb_params_default(**{field: value})
    assert F.flb_workspace_bytes(p) == 0


def test_d3q15_and_stencil_options(lib):
    fd = dict(q=15, psi_scheme=F.FLB_FD)
    assert F.flb_workspace_bytes(F.flb_params_default(**fd)) > 2 * 15 * 32 ** 3 * 4
    assert F.flb_workspace_bytes(F.flb_params_default(**fd, force_grad=F.FLB_FORCE_STRESS)) > 0
    assert F.flb_workspace_bytes(F.flb_params_default(**fd, integrator=F.FLB_RK4)) > 0
    assert F.flb_workspace_bytes(F.flb_params_default(**fd, force_grad=F.FLB_FORCE_FV)) > 0
    assert F.flb_workspace_bytes(F.flb_params_default(q=15)) > 0             # FV on D3Q15: per-site kernels
    assert F.flb_workspace_bytes(F.flb_params_default(**fd, dim=2, nz=1)) == 0
    # every App. A Laplacian in 3D, SO and CD in 2D; the naive scheme in both
    for lap in (F.FLB_LAP_CD, F.FLB_LAP_PK, F.FLB_LAP_LB):
        assert F.flb_workspace_bytes(F.flb_params_default(laplacian=lap)) > 0
    d2 = dict(dim=2, q=9, nz=1)
    assert F.flb_workspace_bytes(F.flb_params_default(**d2, laplacian=F.FLB_LAP_CD)) > 0
    assert F.flb_workspace_bytes(F.flb_params_default(**d2, laplacian=F.FLB_LAP_PK)) == 0
    assert F.flb_workspace_bytes(F.flb_params_default(**d2, psi_scheme=F.FLB_NAIVE)) > 0
    assert F.flb_workspace_bytes(F.flb_params_default(psi_scheme=F.FLB_NAIVE, laplacian=F.FLB_LAP_CD)) > 0
    # the stress kernels use the SO stencil
    assert F.flb_workspace_bytes(F.flb_params_default(force_grad=F.FLB_FORCE_STRESS, laplacian=F.FLB_LAP_CD)) == 0
    # D3Q15 needs fewer population planes than D3Q19
    assert F.flb_workspace_bytes(F.flb_params_default(**fd)) < \
        F.flb_workspace_bytes(F.flb_params_default(psi_scheme=F.FLB_FD))


def test_mixed_replica_structure_rejected(lib):
    a = F.flb_params_default()
    b = F.flb_params_default(psi_scheme=F.FLB_FD)
    assert F.flb_workspace_bytes([a, b]) == 0


def test_init_argument_checks_without_device(lib):
    p = F.flb_params_default()
    h = ctypes.c_void_p()
    arr = (F.FlbParams * 1)(p)
    assert lib.flb_init(arr, 1, None, 1 << 30, None, ctypes.byref(h)) == F.FLB_EINVAL
    assert lib.flb_init(arr, 1, ctypes.c_void_p(0x1001), 1 << 30, None, ctypes.byref(h)) == F.FLB_EINVAL
    assert lib.flb_init(arr, 1, ctypes.c_void_p(0x100000), 16, None, ctypes.byref(h)) == F.FLB_ENOSPC
    assert lib.flb_step(None, 1) == F.FLB_EINVAL
    assert F.flb_strerror(F.FLB_ENONFINITE).startswith("non-finite")


def test_init_field_defaults_and_validation(lib):
    # flb_params.init: REST by default; EQUILIBRIUM needs the Gaussian free energy
    # to be stable (A > 0, K >= 0), checked before any device work
    p = F.flb_params_default(nx=8, ny=8, nz=8)
    assert p.init == F.FLB_INIT_REST
    assert F.flb_workspace_bytes(p) > 0
    for init, A, ok in [(F.FLB_INIT_EQUILIBRIUM, 0.05, True), (F.FLB_INIT_EQUILIBRIUM, -0.0625, False),
                        (F.FLB_INIT_EQUILIBRIUM, 0.0, False), (F.FLB_INIT_USER, -0.0625, True), (3, 0.05, False),
                        (-1, 0.05, False)]:
        q = F.flb_params_default(nx=8, ny=8, nz=8, A=A, init=init)
        assert (F.flb_workspace_bytes(q) > 0) == ok, (init, A)
