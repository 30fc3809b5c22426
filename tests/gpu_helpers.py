"""Shared helpers of the GPU tests: build a Solver and an oracle State from the
same seeded inputs, and the field-error metric used throughout.

Error metric: err(x) = max_r |x_gpu - x_oracle| / RMS_r(x_oracle - x_eq), with
x_eq = w_i rho0 for populations and 0 for psi and u."""
import numpy as np

import oracle as O
import paper_1104_0078_gb300 as F


def flb_params(d: dict, **kw) -> F.FlbParams:
    d = {**d, **kw}
    p = F.flb_params_default()
    p.dim, p.q = d["dim"], d["q"]
    p.nx, p.ny, p.nz = d["nx"], d["ny"], d.get("nz", 1) if d["dim"] == 3 else 1
    p.rho0, p.tau = d.get("rho0", 1.0), d["tau"]
    p.gamma_bulk = d.get("gamma_bulk", float("nan"))
    p.gamma_ghost = d.get("gamma_ghost", 0.0)
    p.kT, p.A, p.B, p.K, p.M = d["kT"], d["A"], d["B"], d["K"], d["M"]
    p.psi_scheme = d.get("scheme", 1)
    p.integrator = d.get("integrator", 2)
    p.storage = d.get("storage", F.FLB_F32_DEV)
    p.laplacian = d.get("laplacian", 0)
    p.coupling = d.get("coupling", 3)
    p.seed = d.get("seed", 1)
    p.sq_kmax = d.get("sq_kmax", 0)
    p.sq_lags = d.get("sq_lags", 0)
    p.force_grad = d.get("force_grad", 0)
    p.init = d.get("init", 0)
    return p


def oracle_params(d: dict, **kw) -> O.Params:
    d = {**d, **kw}
    return O.Params(dim=d["dim"], q=d["q"], nx=d["nx"], ny=d["ny"], nz=d.get("nz", 1) if d["dim"] == 3 else 1,
                    rho0=d.get("rho0", 1.0), tau=d["tau"], gamma_bulk=d.get("gamma_bulk", float("nan")),
                    gamma_ghost=d.get("gamma_ghost", 0.0), kT=d["kT"], A=d["A"], B=d["B"], K=d["K"], M=d["M"],
                    scheme=d.get("scheme", 1), integrator=d.get("integrator", 2), coupling=d.get("coupling", 3),
                    seed=d.get("seed", 1), force_grad=d.get("force_grad", 0), laplacian=d.get("laplacian", 0))


def field_error(gpu, ora, eq=0.0):
    gpu = np.asarray(gpu, dtype=np.float64)
    ora = np.asarray(ora, dtype=np.float64)
    dev = ora - eq
    rms = np.sqrt(np.mean(dev ** 2))
    return float(np.max(np.abs(gpu - ora)) / max(rms, 1e-300))


def weights_column(q):
    _, w = O.lattice(2 if q == 9 else 3, q)
    return w[:, None]
