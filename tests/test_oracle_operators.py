"""Pins of the oracle's lattice operators against the Fourier symbols printed in
App. A and Sec. V.B, and of the finite-difference noise against Eq. (etafdt)."""
import numpy as np
import pytest

import oracle as O
from oracle import theory as T


def _plane_waves(shape):
    """Yield (q, cos(q.r)) for every wavevector of the lattice (nz, ny, nx)."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    qg = T.q_grid(shape)
    for idx in np.ndindex(shape):
        qv = qg[idx]
        yield qv, np.cos(qv[0] * x + qv[1] * y + qv[2] * z)


def test_so_laplacian_symbol_3d():
    # Eq. (solap) applied to cos(q.r) multiplies it by Eq. (solapft)
    shape = (4, 6, 8)
    for qv, wave in _plane_waves(shape):
        out = O.laplacian_so(3, wave)
        assert np.allclose(out, T.L_so(qv) * wave, atol=1e-13)


def test_so_laplacian_symbol_2d():
    shape = (1, 6, 8)
    for qv, wave in _plane_waves(shape):
        out = O.laplacian_so(2, wave[0])
        assert np.allclose(out, T.L_so_2d(qv) * wave[0], atol=1e-13)


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_app_a_laplacian_symbols_3d(kind):
    # each stencil of App. A (SO, CD, PK, LB) applied to cos(q.r) multiplies it by its
    # printed Fourier transform, Eqs. (solapft), (fdlapft), (pklapft), (lblapft)
    shape = (4, 6, 8)
    for qv, wave in _plane_waves(shape):
        out = O.laplacian(3, kind, wave)
        assert np.allclose(out, T.L_kind(qv, 3, kind) * wave, atol=1e-13)


@pytest.mark.parametrize("kind", [0, 1])
def test_planar_laplacian_symbols(kind):
    # 2D readings: the planar SO stencil and the 5-point CD stencil
    shape = (1, 6, 8)
    for qv, wave in _plane_waves(shape):
        out = O.laplacian(2, kind, wave[0])
        assert np.allclose(out, T.L_kind(qv, 2, kind) * wave[0], atol=1e-13)
    with pytest.raises(ValueError):
        O.laplacian(2, 2, wave[0])


def test_laplacian_symbols_limit():
    # every admissible stencil tends to -q^2 (Sec. III); the SO one to O(q^4)
    for qv in ([1e-3, 0, 0], [1e-3, 2e-3, -1e-3], [7e-4, 7e-4, 7e-4]):
        q2 = float(np.dot(qv, qv))
        for L in (T.L_cd, T.L_pk, T.L_so, T.L_lb):
            assert abs(L(np.array(qv)) + q2) < 1e-6 * q2
        q2d = qv[0] ** 2 + qv[1] ** 2
        assert abs(T.L_so_2d(np.array(qv)) + q2d) < 1e-6 * max(q2d, 1e-30) + 1e-18


def test_fv_laplacian_matches_printed_d3q15_symbol():
    # the finite-volume gradient + link-averaged divergence on the paper's D3Q15
    # lattice reproduces Eq. (fvlapft) exactly; this fixes the normalisation
    # (1/c_s^2 on the gradient, 2/c_s^2 on the divergence) left garbled in Sec. V.B
    shape = (6, 4, 8)
    for qv, wave in _plane_waves(shape):
        out = O.fv_laplacian(3, 15, wave)
        assert np.allclose(out, T.L_fv_d3q15(qv) * wave, atol=1e-13)


@pytest.mark.parametrize("dim,q", [(3, 19), (2, 9)])
def test_fv_laplacian_symbol_d3q19_d2q9(dim, q):
    c, w = O.lattice(dim, q)
    shape = (4, 6, 8) if dim == 3 else (1, 6, 8)
    for qv, wave in _plane_waves(shape):
        out = O.fv_laplacian(dim, q, wave if dim == 3 else wave[0])
        expect = T.L_fv(qv, c, w) * (wave if dim == 3 else wave[0])
        assert np.allclose(out, expect, atol=1e-13)
    # closed forms: D3Q19 -(1/9) sum s_a^2 (1 + c_b + c_g)^2 ; D2Q9 -(1/9) sum s_a^2 (2 + c_b)^2
    rng = np.random.default_rng(3)
    for _ in range(20):
        qv = rng.uniform(-np.pi, np.pi, 3)
        cx, cy, cz = np.cos(qv)
        sx, sy, sz = np.sin(qv)
        if dim == 3:
            closed = -((sx * (1 + cy + cz)) ** 2 + (sy * (1 + cx + cz)) ** 2 + (sz * (1 + cx + cy)) ** 2) / 9
        else:
            closed = -((sx * (2 + cy)) ** 2 + (sy * (2 + cx)) ** 2) / 9
        assert abs(T.L_fv(qv, c, w) - closed) < 1e-14
    # and -> -q^2 as q -> 0
    qv = np.array([1e-3, -2e-3, 5e-4]) if dim == 3 else np.array([1e-3, -2e-3, 0.0])
    assert abs(T.L_fv(qv, c, w) + np.dot(qv, qv)) < 1e-5 * np.dot(qv, qv)


@pytest.mark.parametrize("dim,kind", [(2, 0), (3, 0), (2, 1), (3, 1), (3, 2), (3, 3)])
def test_fd_noise_covariance(dim, kind):
    # <|eta~(q)|^2> = -2 kT M L(q)   (Eq. etafdt with the chosen App. A stencil),
    # estimated over 400 steps; each mode's estimator has relative s.d.
    # 1/sqrt(400) (real-field pairs aside)
    p = O.Params(dim=dim, q=19 if dim == 3 else 9, nx=8, ny=6, nz=4, kT=0.7, M=0.3, laplacian=kind)
    acc = np.zeros(p.shape)
    nsamp = 400
    for step in range(nsamp):
        eta = O.fd_noise(p, step).reshape(p.shape)
        acc += np.abs(np.fft.fftn(eta)) ** 2 / p.n
        assert abs(eta.sum()) < 1e-12 * np.abs(eta).sum()     # conservative by construction
    acc /= nsamp
    qg = T.q_grid(p.shape)
    L = T.L_kind(qg, dim, kind)
    expect = -2 * p.kT * p.M * L
    mask = np.abs(L) > 1e-12
    ratio = acc[mask] / expect[mask]
    assert abs(ratio.mean() - 1) < 4 / np.sqrt(nsamp * mask.sum() / 2)
    assert np.all(np.abs(ratio - 1) < 6 / np.sqrt(nsamp / 2))
    assert acc[0, 0, 0] < 1e-20


@pytest.mark.parametrize("dim,nz", [(2, 4), (3, 4), (3, 5)])
def test_contrast_scheme_noise_covariance(dim, nz):
    # the naive scheme of Sec. III: node noise through the central-difference
    # divergence, Gamma(q) = i sin q, so <|eta~(q)|^2> = 2 kT M sum_a sin^2 q_a
    # (Eq. FTorderpara) -- not -2 kT M L(q); it vanishes where every q_a is 0 or pi.
    # A normal shared between two nodes (a counter or word index gone wrong)
    # would modulate the spectrum; an odd depth checks the periodic wrap.
    p = O.Params(dim=dim, q=19 if dim == 3 else 9, nx=8, ny=6, nz=nz, kT=0.7, M=0.3, scheme=2, laplacian=1,
                 A=0.0, K=0.0, coupling=0)
    acc = np.zeros(p.shape)
    nsamp = 400
    zero = np.zeros(p.n)
    u = np.zeros((3, p.n))
    for step in range(nsamp):
        eta = O.psi_rhs(p, zero, u, step=step, with_noise=True).reshape(p.shape)
        acc += np.abs(np.fft.fftn(eta)) ** 2 / p.n
        assert abs(eta.sum()) < 1e-12 * np.abs(eta).sum()
    acc /= nsamp
    qg = T.q_grid(p.shape)
    expect = 2 * p.kT * p.M * T.cd_divergence_power(qg, dim)
    mask = expect > 1e-12
    ratio = acc[mask] / expect[mask]
    assert abs(ratio.mean() - 1) < 4 / np.sqrt(nsamp * mask.sum() / 2)
    assert np.all(np.abs(ratio - 1) < 6 / np.sqrt(nsamp / 2))
    assert np.all(acc[~mask] < 1e-20)


def test_mu_and_force():
    # mu = A psi + B psi^3 - K lap_SO psi and F = -psi grad_CD mu at a few sites, brute force
    p = O.Params(dim=3, q=19, nx=5, ny=4, nz=3, A=-0.06, B=0.07, K=0.04, force_grad=1)
    rng = np.random.default_rng(0)
    psi = rng.normal(size=p.shape)
    mu = O.mu(p, psi).reshape(p.shape)
    F = O.force(p, psi).reshape(3, *p.shape)
    nz, ny, nx = p.shape
    for (z, y, x) in [(0, 0, 0), (2, 3, 4), (1, 2, 0)]:
        lap = 0.0
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    k = abs(dx) + abs(dy) + abs(dz)
                    wgt = {0: -80 / 22, 1: 6 / 22, 2: 3 / 22, 3: 1 / 22}[k]
                    lap += wgt * psi[(z + dz) % nz, (y + dy) % ny, (x + dx) % nx]
        m = p.A * psi[z, y, x] + p.B * psi[z, y, x] ** 3 - p.K * lap
        assert abs(mu[z, y, x] - m) < 1e-12
        gx = 0.5 * (mu[z, y, (x + 1) % nx] - mu[z, y, (x - 1) % nx])
        gy = 0.5 * (mu[z, (y + 1) % ny, x] - mu[z, (y - 1) % ny, x])
        gz = 0.5 * (mu[(z + 1) % nz, y, x] - mu[(z - 1) % nz, y, x])
        assert np.allclose(F[:, z, y, x], -psi[z, y, x] * np.array([gx, gy, gz]), atol=1e-12)


@pytest.mark.parametrize("dim,q", [(2, 9), (3, 19), (3, 15)])
def test_fv_force_gradient_symbol(dim, q):
    # force_grad 2: F = -psi G mu with G the FV gradient of Eq. (fvgrad), whose
    # Fourier symbol is i (1/c_s^2) sum_i w_i c_i sin(q.c_i) (Eq. fvft); the
    # gradient is applied here spectrally, independently of the stencil
    shape = (5, 6, 7) if dim == 3 else (1, 6, 7)
    p = O.Params(dim=dim, q=q, nx=shape[2], ny=shape[1], nz=shape[0], A=-0.06, B=0.07, K=0.04, force_grad=2)
    rng = np.random.default_rng(3)
    psi = rng.normal(size=shape)
    mu = O.mu(p, psi).reshape(shape)
    F = O.force(p, psi).reshape(3, *shape)
    c, w = O.lattice(dim, q)
    G = T.fv_gradient_symbol(T.q_grid(shape), c, w)
    mk = np.fft.fftn(mu)
    for a in range(3):
        grad = np.fft.ifftn(1j * G[..., a] * mk).real
        assert np.allclose(F[a], -psi * grad, atol=1e-12)
    # force_grad 0 follows the psi scheme: FV -> FV gradient, FD -> central difference
    Fm = O.force(O.Params(**{**p.__dict__, "force_grad": 0, "scheme": 1}), psi)
    assert np.array_equal(Fm, F.reshape(3, -1))
    Fd = O.force(O.Params(**{**p.__dict__, "force_grad": 0, "scheme": 0}), psi)
    assert np.array_equal(Fd, O.force(O.Params(**{**p.__dict__, "force_grad": 1}), psi))


@pytest.mark.parametrize("dim,q", [(2, 9), (3, 19), (3, 15)])
@pytest.mark.parametrize("scheme", [0, 1])
def test_force_advection_energy_exchange(dim, q, scheme):
    # Work done by the force on the fluid, sum u.F, equals the free energy the
    # advection of psi removes, sum mu div(u psi), exactly on the lattice when
    # the force gradient is the negative adjoint of the advecting divergence
    # (Sec. II.B energy balance; central difference for FD, Sec. V.A; FV
    # gradient of Eq. (fvgrad) for the link-averaged flux of Eq. (fvflux)).
    # The unmatched pair leaves a residue of the order of the terms themselves.
    shape = (5, 6, 7) if dim == 3 else (1, 9, 8)
    p = O.Params(dim=dim, q=q, nx=shape[2], ny=shape[1], nz=shape[0], A=-0.06, B=0.07, K=0.04, M=0.0,
                 kT=0.0, scheme=scheme, coupling=3)
    rng = np.random.default_rng(5 + scheme)
    psi = rng.normal(size=p.n)
    u = np.zeros((3, p.n))
    u[:dim] = 0.05 * rng.normal(size=(dim, p.n))
    mu = O.mu(p, psi)
    R = O.psi_rhs(p, psi, u)                       # = -div(u psi) with M = 0, no noise
    work = np.sum(u * O.force(p, psi))
    dfree = np.sum(mu * R)
    scale = np.sum(np.abs(mu * R))
    assert scale > 0.1
    assert abs(work + dfree) < 1e-13 * scale
    other = O.Params(**{**p.__dict__, "force_grad": 2 if scheme == 0 else 1})
    assert abs(np.sum(u * O.force(other, psi)) + dfree) > 1e-2 * scale


@pytest.mark.parametrize("dim,q,scheme", [(2, 9, 0), (3, 19, 1)])
def test_dynamic_structure_factor_exact_decay(dim, q, scheme):
    # Without noise, with B = 0 and diffusion alone, each Fourier mode is multiplied
    # every step by the integrator's amplification g(q) (Eq. strf's decay, discrete
    # time), so S(q, l m) = g(q)^(l m) <|psi~(q, t - l m)|^2> exactly: this fixes the
    # lag direction, the conjugate and the 1/N of the estimator.
    shape = (1, 16, 12) if dim == 2 else (6, 5, 8)
    p = O.Params(dim=dim, q=q, nx=shape[2], ny=shape[1], nz=shape[0], kT=0.0, A=0.05, B=0.0, K=0.04, M=0.1,
                 scheme=scheme, integrator=2, coupling=0)
    rng = np.random.default_rng(7)
    s = O.State.rest(p, psi=rng.normal(size=p.n))
    m, nsamp, nlags = 3, 7, 4
    psis = []
    for _ in range(nsamp):
        psis.append(s.psi.copy())
        s.advance(m)
    S = O.dynamic_structure_factor(p, psis, nlags)
    qg = T.q_grid(shape)
    c, w = O.lattice(dim, q)
    Lmob = (T.L_so_2d(qg) if dim == 2 else T.L_so(qg)) if scheme == 0 else T.L_fv(qg, c, w)
    g = T.amplification(-T.lam(qg, p, Lmob), 2)
    P = [np.abs(np.fft.fftn(x.reshape(shape))) ** 2 / p.n for x in psis]
    for l in range(nlags):
        expect = g ** (l * m) * np.mean(P[:nsamp - l], axis=0)
        assert np.allclose(S[l], expect, rtol=1e-10, atol=1e-14 * np.max(P[0]))
    assert np.allclose(S[0], np.mean(P, axis=0), rtol=1e-13)


@pytest.mark.parametrize("dim,q", [(2, 9), (3, 19), (3, 15)])
def test_stress_force_sums_to_zero(dim, q):
    # force_grad 3: F = -div sigma (Sec. IV, Eq. muf) with a central-difference
    # divergence telescopes to sum_r F = 0 for any psi, also for B != 0, where
    # -psi grad mu leaves a net force (reading P)
    shape = (1, 11, 9) if dim == 2 else (7, 6, 5)
    p = O.Params(dim=dim, q=q, nx=shape[2], ny=shape[1], nz=shape[0], A=-0.06, B=0.3, K=0.04, force_grad=3)
    rng = np.random.default_rng(11)
    psi = rng.normal(size=p.n)
    F = O.force(p, psi)
    assert np.abs(F[:dim].sum(axis=1)).max() < 1e-13 * np.abs(F).sum()
    assert dim == 3 or np.abs(F[dim:]).max() == 0.0
    Fc = O.force(O.Params(**{**p.__dict__, "force_grad": 1}), psi)
    assert np.abs(Fc[:dim].sum(axis=1)).max() > 1e-3 * np.abs(Fc).sum() / p.n


def test_stress_force_second_order_consistency():
    # The divergence of sigma equals psi grad mu in the continuum, so on a smooth
    # field the two lattice forces differ by O(h^2): doubling the wavelength (and
    # the box) divides their difference, relative to the force, by about 4.  A
    # wrong coefficient in sigma leaves an O(1) difference instead.
    errs = []
    for n in (16, 32):
        p = O.Params(dim=3, q=19, nx=n, ny=n, nz=n, A=-0.05, B=0.3, K=0.04, force_grad=3)
        z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        k = 2 * np.pi / n
        psi = (0.6 * np.sin(k * x + 0.3) + 0.4 * np.cos(k * y) * np.sin(k * z + 1.0)).ravel()
        Fs = O.force(p, psi)
        Fc = O.force(O.Params(**{**p.__dict__, "force_grad": 1}), psi)
        errs.append(np.abs(Fs - Fc).max() / np.abs(Fc).max())
    assert errs[0] < 0.2 and 3.0 < errs[0] / errs[1] < 5.0, errs


def test_advected_variance_factor_reduces_and_matches_iteration():
    # theta = 0 is the plain discrete factor
    lmb = np.linspace(0.001, 0.5, 40)
    for integ in (1, 2, 4):
        assert np.allclose(T.advected_variance_factor(lmb, 0.0, integ), T.discrete_variance_factor(lmb, integ),
                           rtol=1e-12)
    # brute force: iterate E|psi|^2 <- |R|^2 E|psi|^2 + |S|^2 for psi <- R psi + S eta
    # with unit-variance eta, R and S from the stage formulas written out directly
    for integ in (1, 2, 4):
        for lm, th in ((0.05, 0.2), (0.02, 0.3), (0.3, 0.6), (0.01, 0.05)):
            z = -lm - 1j * th
            if integ == 1:
                R, S = 1 + z, 1.0
            elif integ == 2:
                R, S = 1 + z + z * z / 2, 1 + z / 2
            else:
                R, S = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24, 1 + z / 2 + z * z / 6 + z ** 3 / 24
            if abs(R) >= 1:        # Euler amplifies advected modes: no stationary state
                assert integ == 1
                continue
            v = 0.0
            for _ in range(20000):
                v = abs(R) ** 2 * v + abs(S) ** 2
            assert abs(v * 2 * lm - T.advected_variance_factor(lm, th, integ)) < 1e-9
    # Heun: for small lambda the phase first lowers the factor, then theta^4/4 in
    # |R|^2 raises it above one
    f = T.advected_variance_factor(0.02, np.array([0.0, 0.1, 0.3]), 2)
    assert f[1] < f[0] < 1.0 < f[2]


def test_discrete_variance_factor_general_form():
    # The general stationary factor 2 lambda S^2 / (1 - R^2) (R the amplification,
    # S = (R - 1)/z the noise gain) reduces to the hand-derived Euler and Heun forms
    lmb = np.linspace(0.01, 1.2, 25)
    z = -lmb
    for integ, S in ((1, np.ones_like(z)), (2, 1 + z / 2)):
        R = T.amplification(z, integ)
        assert np.allclose(2 * lmb * S ** 2 / (1 - R ** 2), T.discrete_variance_factor(lmb, integ), rtol=1e-13)
    R4 = T.amplification(z, 4)
    assert np.allclose((R4 - 1) / z, 1 + z / 2 + z ** 2 / 6 + z ** 3 / 24, rtol=1e-13)
    f4 = T.discrete_variance_factor(lmb, 4)
    assert np.all(np.abs(f4 - 1) < np.abs(T.discrete_variance_factor(lmb, 2) - 1) + 1e-15)
