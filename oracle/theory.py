"""Closed forms the paper fixes, used to pin the oracle (TEST INFRASTRUCTURE).

Each function states the passage it restates.  Wavevectors q are arrays with
a trailing axis of length 3 (q_x, q_y, q_z); in 2D q_z is ignored.
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0


def _cs(q):
    q = np.asarray(q, dtype=np.float64)
    return np.cos(q[..., 0]), np.cos(q[..., 1]), np.cos(q[..., 2])


def _sn(q):
    q = np.asarray(q, dtype=np.float64)
    return np.sin(q[..., 0]), np.sin(q[..., 1]), np.sin(q[..., 2])


# ---- App. A: Fourier symbols of the Laplacian stencils ----------------------
def L_cd(q):
    """Eq. (fdlapft): 2{[c_x + c_y + c_z] - 3}."""
    cx, cy, cz = _cs(q)
    return 2.0 * ((cx + cy + cz) - 3.0)


def L_pk(q):
    """Eq. (pklapft)."""
    cx, cy, cz = _cs(q)
    return (28 * (cx + cy + cz) + 12 * (cx * cy + cx * cz + cy * cz) + 8 * cx * cy * cz - 128) / 30.0


def L_so(q):
    """Eq. (solapft): (12[c_x+c_y+c_z] + 12[c_x c_y + c_x c_z + c_y c_z] + 8 c_x c_y c_z - 80)/22."""
    cx, cy, cz = _cs(q)
    return (12 * (cx + cy + cz) + 12 * (cx * cy + cx * cz + cy * cz) + 8 * cx * cy * cz - 80) / 22.0


def L_lb(q):
    """Eq. (lblapft)."""
    cx, cy, cz = _cs(q)
    return (2 * (cx + cy + cz) + 4 * (cx * cy + cx * cz + cy * cz) + 8 * cx * cy * cz - 26) / 9.0


def L_so_2d(q):
    """Symbol of the planar stencil 1/4[2 sum N1 + sum N2 - 12 psi] (2D reading of Eq. solap):
    c_x + c_y + c_x c_y - 3."""
    cx, cy, _ = _cs(q)
    return cx + cy + cx * cy - 3.0


def L_cd_2d(q):
    """5-point planar stencil (2D reading of Eq. fdlap): 2(c_x + c_y) - 4."""
    cx, cy, _ = _cs(q)
    return 2.0 * (cx + cy) - 4.0


def L_kind(q, dim, kind):
    """Symbol of the App. A stencil `kind` (0 SO, 1 CD, 2 PK, 3 LB) in dimension dim."""
    if dim == 2:
        return (L_so_2d, L_cd_2d)[kind](q)
    return (L_so, L_cd, L_pk, L_lb)[kind](q)


def cd_divergence_power(q, dim):
    """|Gamma(q)|^2 of the central-difference divergence of Sec. III (omega_i = +-1/2
    on the nearest neighbours, Gamma_a = i sin q_a): sum_a sin^2 q_a."""
    sx, sy, sz = _sn(q)
    return sx * sx + sy * sy + (sz * sz if dim == 3 else 0.0)


def L_fv_d3q15(q):
    """Eq. (fvlapft), printed for the paper's D3Q15 lattice:
    -(1/9){[2 s_x + s_x c_y c_z]^2 + [2 s_y + s_y c_x c_z]^2 + [2 s_z + s_z c_x c_y]^2}."""
    cx, cy, cz = _cs(q)
    sx, sy, sz = _sn(q)
    return -((2 * sx + sx * cy * cz) ** 2 + (2 * sy + sy * cx * cz) ** 2 + (2 * sz + sz * cx * cy) ** 2) / 9.0


def fv_gradient_symbol(q, c, w):
    """Gamma(q)/c_s^2 of Eq. (fvft) with the imaginary unit removed:
    G_alpha(q) = (1/c_s^2) sum_i w_i c_i,alpha sin(q . c_i)."""
    q = np.asarray(q, dtype=np.float64)
    phase = q @ np.asarray(c, dtype=np.float64).T                      # (..., Q)
    return np.einsum("...i,i,ia->...a", np.sin(phase), np.asarray(w), np.asarray(c, dtype=np.float64)) / CS2


def L_fv(q, c, w):
    """[L(q)]_FV = Gamma.Gamma / c_s^4 = -|G(q)|^2 for any velocity set (Sec. V.B)."""
    G = fv_gradient_symbol(q, c, w)
    return -np.sum(G ** 2, axis=-1)


# ---- Sec. V: linearised psi dynamics ----------------------------------------
def lam(q, p, L_mob):
    """Decay rate per step of a Fourier mode for B = 0 (Eq. strf):
    lambda = M (-L_mob(q)) (A - K L_mu(q)) dt, L_mu the stencil of mu (SO unless
    p.laplacian says otherwise)."""
    Lmu = L_kind(q, p.dim, getattr(p, "laplacian", 0))
    return p.M * (-L_mob) * (p.A - p.K * Lmu)


def amplification(z, integrator):
    """Exact one-step amplification of dpsi/dt = z psi: Euler 1 + z, Heun 1 + z + z^2/2,
    RK4 1 + z + z^2/2 + z^3/6 + z^4/24."""
    if integrator == 1:
        return 1.0 + z
    if integrator == 4:
        return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0 + z ** 4 / 24.0
    return 1.0 + z + 0.5 * z * z


def discrete_variance_factor(lmb, integrator):
    """Stationary variance of psi_{n+1} = R psi_n + S eta_n divided by the
    continuous-time value, with the noise held fixed over the step (for
    dpsi/dt = -lambda psi + noise, R the amplification and S = (R - 1)/z the
    noise gain at z = -lambda): 2 lambda S^2 / (1 - R^2).  This is Euler
    1/(1 - lambda/2) and Heun (2 - lambda)/(2 - lambda + lambda^2/2)."""
    lmb = np.asarray(lmb, dtype=np.float64)
    if integrator == 1:
        return 1.0 / (1.0 - 0.5 * lmb)
    if integrator == 2:
        return (2.0 - lmb) / (2.0 - lmb + 0.5 * lmb * lmb)
    z = -lmb
    R = amplification(z, integrator)
    S = 1.0 + z / 2.0 + z * z / 6.0 + z ** 3 / 24.0
    den = 1.0 - R * R
    small = np.abs(lmb) < 1e-12          # a mode that does not decay: the limit lambda -> 0 is 1
    return np.where(small, 1.0, 2.0 * lmb * S * S / np.where(small, 1.0, den))


def noise_gain(z, integrator):
    """Gain S of the step psi_{n+1} = R psi_n + S eta for dpsi/dt = z psi + eta with
    eta held fixed over the step: S = (R - 1)/z, i.e. 1 (Euler), 1 + z/2 (Heun),
    1 + z/2 + z^2/6 + z^3/24 (RK4)."""
    if integrator == 1:
        return np.ones_like(z)
    if integrator == 4:
        return 1.0 + z / 2.0 + z * z / 6.0 + z ** 3 / 24.0
    return 1.0 + z / 2.0


def advected_variance_factor(lmb, theta, integrator):
    """Stationary variance of a mode with z = -lambda - i theta (decay lambda,
    advection phase theta = u . Gamma(q) per step in a uniform flow, Sec. VI.B)
    over the continuous-time equilibrium value: 2 lambda |S|^2 / (1 - |R|^2).
    theta = 0 gives discrete_variance_factor; theta != 0 makes the factor depend
    on the direction of q relative to the flow -- the anisotropy of the
    high-Mach runs of Sec. VI.B."""
    lmb = np.asarray(lmb, dtype=np.float64)
    z = -lmb - 1j * np.asarray(theta, dtype=np.float64)
    R = amplification(z, integrator)
    S = noise_gain(z, integrator)
    den = 1.0 - np.abs(R) ** 2
    small = np.abs(lmb) < 1e-12
    return np.where(small, 1.0, 2.0 * lmb * np.abs(S) ** 2 / np.where(small, 1.0, den))


def static_structure_factor(q, p, L_mob, steps=None, noise_power=None):
    """<|psi~(q)|^2> = kT/(A - K L_mu(q)) (Eq. test2 with the lattice Laplacian),
    times the discrete-time factor of the integrator; with a start from psi = 0
    after `steps` steps, times (1 - g^(2 steps)).  noise_power: the symbol P(q)
    of a noise whose spectrum is 2 kT M P(q) rather than the -2 kT M L_mob(q)
    that the fluctuation-dissipation theorem asks for (Sec. III, Eq.
    FTorderpara); the spectrum then carries the equilibrium ratio P/(-L_mob)."""
    Lmu = L_kind(q, p.dim, getattr(p, "laplacian", 0))
    S = p.kT / (p.A - p.K * Lmu)
    if noise_power is not None:
        S = S * noise_power / np.where(L_mob == 0, 1.0, -L_mob)
    lmb = lam(q, p, L_mob)
    S = S * discrete_variance_factor(lmb, p.integrator)
    if steps is not None:
        g = amplification(-lmb, p.integrator)
        S = S * (1.0 - g ** (2 * steps))
    return S


def q_grid(shape):
    """Wavevectors of np.fft.fftn on a (nz, ny, nx) lattice, as (nz, ny, nx, 3) (q_x, q_y, q_z)."""
    nz, ny, nx = shape
    kz = 2 * np.pi * np.fft.fftfreq(nz)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    kx = 2 * np.pi * np.fft.fftfreq(nx)
    Z, Y, X = np.meshgrid(kz, ky, kx, indexing="ij")
    return np.stack([X, Y, Z], axis=-1)


# ---- Sec. II.A: planar interface -------------------------------------------
def interface_width(A, K):
    """l = sqrt(2K/|A|) (Eq. intthick with |A|: the printed sqrt(2K/A) is imaginary for A < 0)."""
    return np.sqrt(2.0 * K / abs(A))


def interfacial_tension(A, B, K):
    """gamma = (2/3) sqrt(2 K |A|^3 / B^2) (Eq. st with |A|)."""
    return (2.0 / 3.0) * np.sqrt(2.0 * K * abs(A) ** 3 / B ** 2)


def bulk_order_parameter(A, B):
    """psi_+- = +-sqrt(|A|/B) (Eq. tanh with |A|)."""
    return np.sqrt(abs(A) / B)
