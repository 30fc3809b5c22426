"""Plain FP64 CPU oracle for the hybrid model-H time step (arXiv:1104.0078).

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  It shares no code with
the CUDA library: the arithmetic lives in ``flb_oracle.c`` (plain loops, double
precision) and in the closed forms of ``theory.py``; this module only marshals
numpy arrays into the C functions and adds the observables that are a library
primitive away (an FFT) or plain loops (interface heights).

Array layout: value k of site s at ``a[k, s]`` with s = x + nx*(y + ny*z).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flb_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_flb_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, OpenMP over sites, no FMA contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(os.path.join(_HERE, "flb_oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OraParams(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("q", ctypes.c_int32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("rho0", ctypes.c_double), ("tau", ctypes.c_double),
        ("gamma_bulk", ctypes.c_double), ("gamma_ghost", ctypes.c_double),
        ("kT", ctypes.c_double), ("A", ctypes.c_double), ("B", ctypes.c_double),
        ("K", ctypes.c_double), ("M", ctypes.c_double),
        ("scheme", ctypes.c_int32), ("integrator", ctypes.c_int32),
        ("coupling", ctypes.c_int32), ("lb_on", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("gext", ctypes.c_double * 3),
        ("gnx", ctypes.c_int32), ("gny", ctypes.c_int32), ("gnz", ctypes.c_int32),
        ("ox", ctypes.c_int32), ("oy", ctypes.c_int32), ("oz", ctypes.c_int32),
        ("force_grad", ctypes.c_int32),
        ("laplacian", ctypes.c_int32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        dp = P(ctypes.c_double)
        L.ora_threads.restype = ctypes.c_int
        L.ora_set_threads.argtypes = [ctypes.c_int32]
        L.ora_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        L.ora_gaussians.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_int32, dp]
        L.ora_gaussians_sites.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int64,
                                          ctypes.c_uint32, ctypes.c_int32, dp]
        L.ora_lattice.argtypes = [ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32), dp]
        L.ora_moment_basis.argtypes = [ctypes.c_int32, ctypes.c_int32, dp, dp]
        L.ora_laplacian_so.argtypes = [ctypes.c_int32] * 4 + [dp, dp]
        L.ora_laplacian.argtypes = [ctypes.c_int32] * 5 + [dp, dp]
        L.ora_fv_laplacian.argtypes = [ctypes.c_int32] * 5 + [dp, dp]
        L.ora_mu.argtypes = [P(OraParams), dp, dp]
        L.ora_force.argtypes = [P(OraParams), dp, dp, dp]
        L.ora_fd_noise.argtypes = [P(OraParams), ctypes.c_int64, dp]
        L.ora_psi_rhs.argtypes = [P(OraParams), dp, dp, ctypes.c_int64, ctypes.c_int32, dp]
        L.ora_step.argtypes = [P(OraParams), dp, dp, dp, ctypes.c_int64, ctypes.c_int64]
        L.ora_moments.argtypes = [P(OraParams), dp, dp, dp, dp]
        L.ora_equilibrium.argtypes = [P(OraParams), dp, dp, dp]
        for name in ("ora_lattice", "ora_moment_basis", "ora_laplacian", "ora_fv_laplacian", "ora_psi_rhs", "ora_step",
                     "ora_moments", "ora_equilibrium"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Params:
    """Physical and numerical parameters of one lattice (names follow the paper)."""
    dim: int = 3
    q: int = 19
    nx: int = 16
    ny: int = 16
    nz: int = 16
    rho0: float = 1.0
    tau: float = 0.8
    gamma_bulk: float = float("nan")
    gamma_ghost: float = 0.0
    kT: float = 0.0
    A: float = 0.05
    B: float = 0.0
    K: float = 0.04
    M: float = 0.1
    scheme: int = 1          # 0 FD, 1 FV, 2 the naive contrast scheme (Sec. III)
    integrator: int = 2      # 1 Euler, 2 Heun
    coupling: int = 3
    lb_on: int = 1
    seed: int = 1
    gext: tuple = (0.0, 0.0, 0.0)
    gdims: tuple = (0, 0, 0)
    origin: tuple = (0, 0, 0)
    force_grad: int = 0      # 1 central difference (Sec. IV), 2 FV gradient (Eq. fvgrad), 0 matched to scheme
    laplacian: int = 0       # App. A stencil: 0 SO, 1 CD, 2 PK, 3 LB

    @property
    def n(self) -> int:
        return self.nx * self.ny * (self.nz if self.dim == 3 else 1)

    @property
    def shape(self) -> tuple:
        """numpy shape of one field plane, (nz, ny, nx) (nz = 1 in 2D)."""
        return (self.nz if self.dim == 3 else 1, self.ny, self.nx)

    def c(self) -> OraParams:
        p = OraParams()
        p.dim, p.q, p.nx, p.ny = self.dim, self.q, self.nx, self.ny
        p.nz = self.nz if self.dim == 3 else 1
        p.rho0, p.tau, p.gamma_bulk, p.gamma_ghost = self.rho0, self.tau, self.gamma_bulk, self.gamma_ghost
        p.kT, p.A, p.B, p.K, p.M = self.kT, self.A, self.B, self.K, self.M
        p.scheme, p.integrator, p.coupling, p.lb_on = self.scheme, self.integrator, self.coupling, self.lb_on
        p.seed = self.seed
        for a in range(3):
            p.gext[a] = self.gext[a]
        p.gnx, p.gny, p.gnz = self.gdims
        p.ox, p.oy, p.oz = self.origin
        p.force_grad = self.force_grad
        p.laplacian = self.laplacian
        return p


def threads() -> int:
    """OpenMP threads the oracle's site loops use."""
    return int(lib().ora_threads())


def set_threads(n: int) -> None:
    """Threads the oracle's site loops use from now on."""
    lib().ora_set_threads(int(n))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().ora_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def gaussians(seed: int, step: int, site: int, stream: int, nblocks: int) -> np.ndarray:
    g = np.zeros(8 * nblocks)
    lib().ora_gaussians(seed, step, site, stream, nblocks, _dp(g))
    return g


def gaussians_sites(seed: int, step: int, site0: int, nsites: int, stream: int, nblocks: int) -> np.ndarray:
    """The normals of `gaussians` for counter sites site0 .. site0 + nsites - 1, shape (nsites, 8 nblocks)."""
    g = np.zeros(nsites * 8 * nblocks)
    lib().ora_gaussians_sites(seed, step, site0, nsites, stream, nblocks, _dp(g))
    return g.reshape(nsites, 8 * nblocks)


def lattice(dim: int, q: int):
    c = (ctypes.c_int32 * (3 * q))()
    w = np.zeros(q)
    if lib().ora_lattice(dim, q, c, _dp(w)):
        raise ValueError("unsupported lattice")
    return np.array(list(c), dtype=np.int64).reshape(q, 3), w


def moment_basis(dim: int, q: int):
    E = np.zeros(q * q)
    b = np.zeros(q)
    if lib().ora_moment_basis(dim, q, _dp(E), _dp(b)):
        raise ValueError("unsupported lattice")
    return E.reshape(q, q), b


def laplacian_so(dim: int, field_: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(field_, dtype=np.float64)
    nz, ny, nx = a.shape if a.ndim == 3 else (1,) + a.shape
    out = np.zeros_like(a)
    lib().ora_laplacian_so(dim, nx, ny, nz, _dp(a), _dp(out))
    return out


def laplacian(dim: int, kind: int, field_: np.ndarray) -> np.ndarray:
    """The App. A stencil `kind` (0 SO, 1 CD, 2 PK, 3 LB) applied to a periodic field."""
    a = np.ascontiguousarray(field_, dtype=np.float64)
    nz, ny, nx = a.shape if a.ndim == 3 else (1,) + a.shape
    out = np.zeros_like(a)
    if lib().ora_laplacian(dim, kind, nx, ny, nz, _dp(a), _dp(out)):
        raise ValueError("no such stencil in this dimension")
    return out


def fv_laplacian(dim: int, q: int, field_: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(field_, dtype=np.float64)
    nz, ny, nx = a.shape if a.ndim == 3 else (1,) + a.shape
    out = np.zeros_like(a)
    if lib().ora_fv_laplacian(dim, q, nx, ny, nz, _dp(a), _dp(out)):
        raise ValueError("unsupported lattice")
    return out


def mu(p: Params, psi: np.ndarray) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.float64).reshape(-1)
    out = np.zeros(p.n)
    cp = p.c()
    lib().ora_mu(ctypes.byref(cp), _dp(psi), _dp(out))
    return out


def force(p: Params, psi: np.ndarray) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.float64).reshape(-1)
    m = mu(p, psi)
    F = np.zeros((3, p.n))
    cp = p.c()
    lib().ora_force(ctypes.byref(cp), _dp(psi), _dp(m), _dp(F))
    return F


def fd_noise(p: Params, step: int) -> np.ndarray:
    eta = np.zeros(p.n)
    cp = p.c()
    lib().ora_fd_noise(ctypes.byref(cp), step, _dp(eta))
    return eta


def psi_rhs(p: Params, psi: np.ndarray, u: np.ndarray, step: int = 0, with_noise: bool = False) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.float64).reshape(-1)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(3, -1) if u is not None else np.zeros((3, p.n))
    R = np.zeros(p.n)
    cp = p.c()
    lib().ora_psi_rhs(ctypes.byref(cp), _dp(psi), _dp(u), step, int(with_noise), _dp(R))
    return R


def equilibrium(p: Params, rho=None, u=None) -> np.ndarray:
    rho_a = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1) if rho is not None else None
    u_a = np.ascontiguousarray(u, dtype=np.float64).reshape(3, -1) if u is not None else None
    f = np.zeros((p.q, p.n))
    cp = p.c()
    rc = lib().ora_equilibrium(ctypes.byref(cp), _dp(rho_a) if rho_a is not None else None,
                               _dp(u_a) if u_a is not None else None, _dp(f))
    if rc:
        raise ValueError("unsupported lattice")
    return f


def moments(p: Params, f: np.ndarray):
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho = np.zeros(p.n)
    j = np.zeros((3, p.n))
    m = np.zeros((p.q, p.n))
    cp = p.c()
    lib().ora_moments(ctypes.byref(cp), _dp(f), _dp(rho), _dp(j), _dp(m))
    return rho, j, m


@dataclass
class State:
    """Oracle state: fbar after streaming (q x N), psi (N), last velocity u (3 x N), step."""
    p: Params
    f: np.ndarray
    psi: np.ndarray
    u: np.ndarray
    step: int = 0

    @classmethod
    def rest(cls, p: Params, psi=None, rho=None, u=None) -> "State":
        f = equilibrium(p, rho, u)
        ps = np.zeros(p.n) if psi is None else np.ascontiguousarray(psi, dtype=np.float64).reshape(-1).copy()
        uu = np.zeros((3, p.n))
        if u is not None:
            uu[:] = np.asarray(u, dtype=np.float64).reshape(3, -1)
        return cls(p, f, ps, uu, 0)

    @classmethod
    def equilibrium(cls, p: Params) -> "State":
        """The equilibrium start of the Gaussian model (Sec. VI's runs start from
        equilibrium; B is not part of it).
        Fluid: the stationary law of the linearised fluctuating LB is independent
        normal population deviations of variance mu_n w_i, mu_n = rho0 kT / c_s^2
        (Sec. III); the stored post-collision deviation of population i at site s
        is sqrt(mu_n w_i) g_i(s), with g_0..g_{q-1} the normals of Philox stream 3,
        step 0, counter site s; after streaming f_i(r) = w_i rho0 + that value at
        r - c_i.
        Order parameter: the Gibbs law of the Gaussian free energy A/2 psi^2 +
        K/2 |grad psi|^2 on the lattice gives S(q) = kT/(A - K L(q)) with L the
        symbol of the Laplacian in mu (Eq. test2).  psi = Re W with W(r) = sum_q
        X(q) e^{iq.r}, X(q) = sqrt(S(q)/N) (a + i b) for q != 0 and X(0) = 0
        (the conserved mean), (a, b) the first two normals of Philox stream 4,
        step 0, counter = the mode's index kx + nx (ky + ny kz) in FFT order; then
        <|psi~(q)|^2> = N S(q) on every q != 0.
        u: the velocity sum fbar c / rho of those populations."""
        from . import theory as T
        c, w = lattice(p.dim, p.q)
        shape = p.shape
        nb = (p.q + 7) // 8
        G = gaussians_sites(p.seed, 0, 0, p.n, 3, nb)[:, :p.q].T          # (q, N)
        dev = np.sqrt(p.rho0 * p.kT * 3.0 * w)[:, None] * G
        f = np.empty((p.q, p.n))
        for i in range(p.q):
            d = dev[i].reshape(shape)
            f[i] = w[i] * p.rho0 + np.roll(d, shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2)).reshape(-1)
        qg = T.q_grid(shape)
        if p.dim == 2:
            qg[..., 2] = 0.0
        L = T.L_kind(qg, p.dim, p.laplacian)
        S = p.kT / (p.A - p.K * L)
        Gq = gaussians_sites(p.seed, 0, 0, p.n, 4, 1)
        X = np.sqrt(S / p.n) * (Gq[:, 0] + 1j * Gq[:, 1]).reshape(shape)
        X[0, 0, 0] = 0.0
        psi = np.real(np.fft.ifftn(X) * p.n).reshape(-1)
        rho, j, _ = moments(p, f)
        u = j / rho[None, :]
        return cls(p, f, psi, u, 0)

    def advance(self, nsteps: int) -> "State":
        cp = self.p.c()
        rc = lib().ora_step(ctypes.byref(cp), _dp(self.f), _dp(self.psi), _dp(self.u), self.step, nsteps)
        if rc:
            raise ValueError(f"ora_step rejected the parameters ({rc})")
        self.step += nsteps
        return self

    def copy(self) -> "State":
        return State(self.p, self.f.copy(), self.psi.copy(), self.u.copy(), self.step)


# --------------------------------------------------------------------------
# Observables (Sec. VI): conserved totals, structure factor, interface heights
# --------------------------------------------------------------------------
def totals(p: Params, f: np.ndarray, psi: np.ndarray) -> dict:
    """Sum of rho, of j = sum fbar c and of psi over the lattice (conservation, Sec. I)."""
    rho, j, _ = moments(p, f)
    return {"mass": float(rho.sum()), "momentum": j.sum(axis=1), "psi": float(np.sum(psi))}


def structure_factor(p: Params, psi: np.ndarray) -> np.ndarray:
    """|psi~(q)|^2 / N on the full FFT grid, shape (nz, ny, nx) (Eqs. test1, test2)."""
    a = np.asarray(psi, dtype=np.float64).reshape(p.shape)
    return np.abs(np.fft.fftn(a)) ** 2 / p.n


def structure_factor_at(p: Params, psi: np.ndarray, ks) -> np.ndarray:
    """|psi~(q)|^2 / N at the integer wavevectors ks = [(kx, ky, kz), ...],
    q_a = 2 pi k_a / n_a, straight from the definition psi~(q) = sum_r psi(r)
    e^{-i q.r} (Eqs. test1, test2), summed axis by axis in FP64 -- for fields too
    large for a full FFT, where only some wavevectors are wanted."""
    a = np.asarray(psi, dtype=np.float64).reshape(p.shape)   # (nz, ny, nx)
    nz, ny, nx = p.shape
    out = []
    cache = {}
    for kx, ky, kz in ks:
        if kx not in cache:   # sum over x: (nz, ny) complex
            ph = 2.0 * math.pi * kx * np.arange(nx) / nx
            cache[kx] = a @ np.cos(ph) - 1j * (a @ np.sin(ph))
        t = cache[kx]
        ey = np.exp(-2j * math.pi * ky * np.arange(ny) / ny)
        ez = np.exp(-2j * math.pi * kz * np.arange(nz) / nz)
        v = ez @ (t @ ey)
        out.append(abs(v) ** 2 / p.n)
    return np.array(out)


def dynamic_structure_factor(p: Params, psis, nlags: int) -> np.ndarray:
    """S(q, l) = mean over samples t with t >= l of Re[psi~(q, t) conj(psi~(q, t - l))],
    psi~(q) = N^-1/2 sum_r psi(r) e^{-iq.r}: the paper's S(q, tau) of Sec. VI.A
    (Eq. strf) for the lag tau = l sampling intervals, from the sampled fields
    psis (oldest first).  Full FFT grid, shape (nlags, nz, ny, nx)."""
    F = [np.fft.fftn(np.asarray(s, dtype=np.float64).reshape(p.shape)) for s in psis]
    out = np.zeros((nlags,) + tuple(p.shape))
    for l in range(nlags):
        terms = [np.real(F[t] * np.conj(F[t - l])) for t in range(l, len(F))]
        if terms:
            out[l] = np.mean(terms, axis=0) / p.n
    return out


def interface_heights(p: Params, psi: np.ndarray):
    """Heights of the two psi = 0 surfaces of a slab normal to z (Sec. VI.C).

    In every column the first sign change of psi in z in [0, nz/2) and in
    [nz/2, nz) is located by linear interpolation between the two bracketing
    nodes (the paper's "simple linear interpolation").  Returns (h1, h2), each
    (ny, nx); NaN where a half-column has no crossing."""
    a = np.asarray(psi, dtype=np.float64).reshape(p.shape)
    nz = a.shape[0]
    out = []
    for lo, hi in ((0, nz // 2), (nz // 2, nz)):
        h = np.full(a.shape[1:], np.nan)
        for y in range(a.shape[1]):
            for x in range(a.shape[2]):
                for z in range(lo, hi):
                    v0, v1 = a[z, y, x], a[(z + 1) % nz, y, x]
                    if (v0 < 0.0) != (v1 < 0.0):
                        h[y, x] = z + v0 / (v0 - v1)
                        break
        out.append(h)
    return out[0], out[1]


def height_spectrum(h: np.ndarray) -> np.ndarray:
    """|h~(q)|^2 with h~ = N2^-1/2 sum (h - <h>) e^{-iqx} (Eq. flucinterf normalisation)."""
    d = h - h.mean()
    return np.abs(np.fft.fft2(d)) ** 2 / d.size


def free_energy(p: Params, psi: np.ndarray) -> float:
    """Discrete Landau free energy whose variation is mu (Eqs. Feng, feng):
    sum_r [A psi^2/2 + B psi^4/4 - (K/2) psi lap psi], lap the stencil of mu."""
    a = np.asarray(psi, dtype=np.float64).reshape(p.shape)
    lap = laplacian(p.dim, p.laplacian, a if p.dim == 3 else a[0]).reshape(p.shape)
    return float(np.sum(0.5 * p.A * a ** 2 + 0.25 * p.B * a ** 4 - 0.5 * p.K * a * lap))


def kinetic_energy(p: Params, f: np.ndarray) -> float:
    rho, j, _ = moments(p, f)
    return float(np.sum(0.5 * (j ** 2).sum(axis=0) / rho))
