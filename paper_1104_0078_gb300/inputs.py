"""Seeded synthetic inputs shaped like the paper's workloads (Sec. VI).

This module only draws numbers and lays out parameter sets; it holds none of
the solver's arithmetic.  Both the CUDA path and the FP64 checker start from
what it returns: every floating-point field it produces is exactly
representable in binary32 (population deviations, psi), so the library's FP32
storage and the checker's FP64 arrays begin from the same real numbers.

Workloads (lattice units, periodic):
  bulk_2d    D2Q9 64x64, rho0 1, tau 1, kT 1e-4, A 0.05, B 0, K 0.04, M 0.1, FD,
             psi0 = 0, u0 = 0 (equilibrium fluctuations, Eqs. test1/test2).
  bulk_3d    D3Q19 64^3, tau 0.8, kT 1e-5, A 0.05, B 0, K 0.04, M 0.1, FV.
  slab       D3Q19 256x256x64, A -0.0625, B 0.0625, K 0.04, M 0.1, kT 2e-5, two
             flat interfaces normal to z at z = 16 and 48 (capillary waves).
  ensemble   256 D3Q19 replicas, 64 each of 16^3, 24^3, 32^3, 48^3, kT uniform in
             [1e-5, 1e-4], seeds 1 + r, A 0.05, B 0, K 0.04, M 0.1.
  quench     D3Q19 512^3 spinodal quench, A -0.0625, B 0.0625, K 0.04, M 0.1,
             kT 1e-5, psi0 uniform in [-0.01, 0.01], u0 = 0.
  fluct_d3q15  D3Q15 32^3, tau 1.1, kT 1/3000, A 0.625, B = K = 0, M 0.095, FD:
             the lattice and parameters of the paper's own order-parameter
             fluctuation test (Sec. VI), a Gaussian free energy with
             S(q) = kT/A at every q.
"""
from __future__ import annotations

import math

import numpy as np

WORKLOADS = {
    "bulk_2d": dict(dim=2, q=9, nx=64, ny=64, nz=1, rho0=1.0, tau=1.0, kT=1e-4, A=0.05, B=0.0, K=0.04, M=0.1,
                    scheme=0, seed=1),
    "bulk_3d": dict(dim=3, q=19, nx=64, ny=64, nz=64, rho0=1.0, tau=0.8, kT=1e-5, A=0.05, B=0.0, K=0.04, M=0.1,
                    scheme=1, seed=1),
    "slab": dict(dim=3, q=19, nx=256, ny=256, nz=64, rho0=1.0, tau=0.8, kT=2e-5, A=-0.0625, B=0.0625, K=0.04,
                 M=0.1, scheme=1, seed=1),
    "fluct_d3q15": dict(dim=3, q=15, nx=32, ny=32, nz=32, rho0=1.0, tau=1.1, kT=1.0 / 3000.0, A=0.625, B=0.0,
                        K=0.0, M=0.095, scheme=0, seed=1),
    "quench": dict(dim=3, q=19, nx=512, ny=512, nz=512, rho0=1.0, tau=0.8, kT=1e-5, A=-0.0625, B=0.0625,
                   K=0.04, M=0.1, scheme=1, seed=1),
}

ENSEMBLE_SIZES = (16, 24, 32, 48)


def f32(a) -> np.ndarray:
    """Round to binary32 and return as float64 (exactly representable values)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def random_deviations(q: int, n: int, amp: float, seed: int) -> np.ndarray:
    """Population deviations fbar_i - w_i rho0, shape (q, n), binary32-exact."""
    rng = np.random.default_rng(seed)
    return f32(amp * rng.standard_normal((q, n)))


def random_field(n: int, amp: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return f32(amp * rng.standard_normal(n))


def uniform_field(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """psi0 uniform in [lo, hi] (the quench's initial condition), binary32-exact."""
    rng = np.random.default_rng(seed)
    return f32(rng.uniform(lo, hi, size=n))


def slab_profile(nx: int, ny: int, nz: int, A: float, B: float, K: float, z1: float, z2: float) -> np.ndarray:
    """Two flat interfaces: psi = psi_b tanh((z - z1)/l) tanh((z2 - z)/l) with
    psi_b = sqrt(|A|/B), l = sqrt(2K/|A|) (Eqs. tanh, intthick); +psi_b inside
    (z1, z2), -psi_b outside, continuous across the periodic wrap.  Site order
    x fastest; binary32-exact."""
    l = math.sqrt(2.0 * K / abs(A))
    pb = math.sqrt(abs(A) / B)
    z = np.arange(nz, dtype=np.float64)
    prof = pb * np.tanh((z - z1) / l) * np.tanh((z2 - z) / l)
    return f32(np.broadcast_to(prof[:, None, None], (nz, ny, nx)).reshape(-1))


def ensemble(seed: int = 1000, per_size: int = 64):
    """The uneven replica set: 64 each of 16^3, 24^3, 32^3, 48^3 (256 in all),
    kT_r uniform in [1e-5, 1e-4] (seeded), seed_r = 1 + r."""
    rng = np.random.default_rng(seed)
    out = []
    r = 0
    for n in ENSEMBLE_SIZES:
        for _ in range(per_size):
            out.append(dict(dim=3, q=19, nx=n, ny=n, nz=n, rho0=1.0, tau=0.8, kT=float(1e-5 + 9e-5 * rng.random()),
                            A=0.05, B=0.0, K=0.04, M=0.1, scheme=1, seed=1 + r))
            r += 1
    return out
