"""Pins of the oracle's equilibrium start (State.equilibrium): the construction
checked point by point against independently drawn normals and a brute-force
inverse DFT, and its statistics against the closed forms it must reach -- the
population law N(0, rho0 kT w_i / c_s^2) of the linearised fluctuating LB
(Sec. III), S(q) = kT/(A - K L(q)) of the Gaussian free energy (Eq. test2) and
<u_a^2> = kT/rho0."""
import numpy as np
import pytest

import oracle as O
from oracle import theory as T


def _p(dim=3, q=19, n=(6, 5, 4), **kw):
    d = dict(dim=dim, q=q, nx=n[0], ny=n[1], nz=n[2] if dim == 3 else 1, tau=0.8, kT=2e-4, A=0.05, B=0.0,
             K=0.04, M=0.1, seed=7)
    d.update(kw)
    return O.Params(**d)


@pytest.mark.parametrize("dim,q", [(3, 19), (3, 15), (2, 9)])
def test_equilibrium_populations_are_the_streamed_draws(dim, q):
    p = _p(dim, q)
    st = O.State.equilibrium(p)
    c, w = O.lattice(dim, q)
    nb = (q + 7) // 8
    nz, ny, nx = p.shape
    for (x, y, z) in [(0, 0, 0), (5, 4, nz - 1), (2, 1, 0), (3, 2, nz // 2)]:
        r = x + nx * (y + ny * z)
        for i in range(q):
            xs, ys, zs = (x - c[i, 0]) % nx, (y - c[i, 1]) % ny, (z - c[i, 2]) % nz
            g = O.gaussians(p.seed, 0, xs + nx * (ys + ny * zs), 3, nb)[i]
            assert abs(st.f[i, r] - (w[i] * p.rho0 + np.sqrt(3 * p.rho0 * p.kT * w[i]) * g)) < 1e-14
    rho, j, _ = O.moments(p, st.f)
    assert np.allclose(st.u, j / rho, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim,lap", [(3, 0), (3, 2), (2, 0), (2, 1)])
def test_equilibrium_psi_is_the_real_part_of_the_mode_sum(dim, lap):
    # W(r) = sum_q X(q) e^{iq.r} by brute force over every mode of a small box
    p = _p(dim, 19 if dim == 3 else 9, n=(4, 3, 5), laplacian=lap)
    st = O.State.equilibrium(p)
    nz, ny, nx = p.shape
    qg = T.q_grid(p.shape)
    if dim == 2:
        qg[..., 2] = 0.0
    S = p.kT / (p.A - p.K * T.L_kind(qg, dim, lap))
    W = np.zeros(p.n, dtype=complex)
    r = np.array([[x, y, z] for z in range(nz) for y in range(ny) for x in range(nx)], dtype=float)
    for kz in range(nz):
        for ky in range(ny):
            for kx in range(nx):
                t = kx + nx * (ky + ny * kz)
                if t == 0:
                    continue
                a, b = O.gaussians(p.seed, 0, t, 4, 1)[:2]
                X = np.sqrt(S[kz, ky, kx] / p.n) * (a + 1j * b)
                W += X * np.exp(1j * (r @ qg[kz, ky, kx]))
    assert np.allclose(st.psi, W.real, rtol=0, atol=1e-14)
    assert abs(st.psi.sum()) < 1e-13


def test_equilibrium_statistics():
    # four seeds of a 32^3 box: S(q)/theory per |q| shell within 3% (each shell
    # holds >= 2000 modes x 4 seeds: s.d. <= 1.2%), population variances within
    # 1.5% of rho0 kT w_i / c_s^2 (s.d. 0.4%), <u_a^2> within 1.5% of kT/rho0
    p = _p(3, 19, n=(32, 32, 32))
    c, w = O.lattice(3, 19)
    qg = T.q_grid(p.shape)
    th = p.kT / (p.A - p.K * T.L_so(qg))
    qm = np.sqrt((qg ** 2).sum(-1))
    acc = np.zeros(p.shape)
    var = np.zeros(19)
    u2 = np.zeros(3)
    for seed in (1, 2, 3, 4):
        p.seed = seed
        st = O.State.equilibrium(p)
        acc += O.structure_factor(p, st.psi) / 4
        var += ((st.f - w[:, None] * p.rho0) ** 2).mean(axis=1) / 4
        u2 += (st.u ** 2).mean(axis=1) / 4
    edges = np.linspace(1e-9, qm.max() + 1e-9, 9)
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (qm >= lo) & (qm < hi)
        if sel.sum() >= 2000:
            assert abs((acc[sel] / th[sel]).mean() - 1) < 0.03, (lo, hi)
    assert acc[0, 0, 0] < 1e-20
    assert np.all(np.abs(var / (3 * p.rho0 * p.kT * w) - 1) < 0.015)
    assert np.all(np.abs(u2 / p.kT - 1) < 0.015)
